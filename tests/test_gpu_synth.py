"""The seeded generators give the same bits on the GPU as on the CPU.

They are exact integer constructions; device math-library routines (a pow
behind torch.ldexp, say) must not enter them.
"""
import pytest

from synth import exact_row_sums, prescribed_cond_expansions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,c,nc", [(40, 5.0, 3), (90, 30.0, 3), (64, 45.0, 4), (33, 20.0, 2)])
def test_prescribed_and_row_sums_device_equal_cpu(n, c, nc):
    Mc = prescribed_cond_expansions(n, c, 11, nc)
    Mg = prescribed_cond_expansions(n, c, 11, nc, device="cuda")
    assert torch.equal(Mc, Mg.cpu())
    assert torch.equal(exact_row_sums(Mc, nc), exact_row_sums(Mg, nc).cpu())
