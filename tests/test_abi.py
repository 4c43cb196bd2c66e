"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/ozlu.h declares, and its planners (expansion and p-bit) agree with the
oracle's plan and with the counts the paper prints."""
import os
import re

import pytest

from oracle.plan import make_plan
from paper_2609_29554_gb300 import build, ozlu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return ozlu.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ozlu.h")).read()
    return sorted(set(re.findall(r"\b(ozlu_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert "ozlu_gemm" in names and "ozlu_getrf" in names and "ozlu_getrs" in names
    for name in names:
        assert hasattr(L, name), name
        assert name in ozlu.SIGNATURES, name


@pytest.mark.parametrize("p,k,be,S,extra,gex", [
    (106, 512, "int8", 0, 0, 0), (159, 512, "int8", 0, 0, 0), (212, 512, "int8", 0, 0, 0),
    (212, 256, "int8", 0, 0, 0), (106, 32, "int8", 0, 0, 0), (212, 4096, "int8", 0, 0, 0),
    (159, 64, "int8", 0, 0, 0), (212, 100, "int8", 3, 0, 0), (212, 256, "int8", 0, 1, 0),
    (212, 1024, "int8", 0, 0, 64), (212, 256, "fp8", 0, 0, 0), (106, 512, "fp64", 0, 0, 0),
    (212, 512, "fp64", 2, 0, 0)])
def test_plan_matches_oracle(L, p, k, be, S, extra, gex):
    info = ozlu.ozlu_plan(p, k, ozlu.make_opts(be, S, extra, gex))
    ref = make_plan(p, k, backend=be, S=S or None, extra_groups=extra, g_ex=gex)
    assert (info.S, info.w, info.Q, info.n_mod, info.g0) == (ref.S, ref.w, ref.Q, ref.N, ref.g0)
    assert list(info.moduli)[:info.n_mod] == list(ref.moduli)
    assert info.pair_terms == ref.pair_terms


def _golden_int8_rows():
    path = os.path.join(ROOT, "tests", "golden", "paper_counts.txt")
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line and not line.startswith("mismatch"):
            be, p, K, S, N, ng = line.split()
            if be == "int8" and S == "-":
                yield int(p), int(K), None if N == "-" else int(N), None if ng == "-" else int(ng)


@pytest.mark.parametrize("p,k,N,ng", list(_golden_int8_rows()) + [
    (64, 1, None, None), (1100, 77, None, None), (3136, 256, None, None),
    (6272, 256, None, None), (12544, 256, None, None)])
def test_mp_plan_matches_oracle_and_paper(L, p, k, N, ng):
    # the p-bit planner (ozlu_mp_gemm) on the paper's printed INT8 counts
    # (Table gemmcount, the Sec. 4.2.6 table, Table backend_hp, the p = 8192
    # text) and on the bench's Lotkin precisions
    info = ozlu.ozlu_mp_plan(p, k)
    ref = make_plan(p, k, backend="int8")
    assert (info.S, info.w, info.Q, info.n_mod, info.g0) == (ref.S, ref.w, ref.Q, ref.N, ref.g0)
    assert list(info.moduli)[:info.n_mod] == list(ref.moduli)
    assert info.pair_terms == ref.pair_terms
    if N is not None:
        assert info.n_mod == N
    if ng is not None:
        assert info.pair_terms * info.n_mod == ng


def test_bad_arguments_rejected(L):
    # argument checks happen before any device work
    rc = L.ozlu_gemm(None, 4, 0, 1, 1, 1, 1, None, 1, None, 1, 0, None, 1, None)
    assert rc == -1
    with pytest.raises(ozlu.OzluError):
        ozlu.ozlu_plan(0, 16)
    with pytest.raises(ozlu.OzluError):
        ozlu.ozlu_mp_plan(0, 16)
    with pytest.raises(ozlu.OzluError):
        ozlu.ozlu_mp_plan(128, 0)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ozlu, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ozlu, "_lib", None)
    with pytest.raises(RuntimeError):
        ozlu.lib()


@pytest.mark.parametrize("p,k,S", [(64, 1, 0), (300, 9, 0), (600, 19, 2), (1100, 77, 0), (3136, 256, 0),
                                   (6272, 256, 2), (12544, 256, 2), (12544, 1, 0), (11560, 512, 1)])
def test_mp_ext_plan_matches_oracle(L, p, k, S):
    # the extended-table planner of the p-bit GEMM (Sec. 4.2.4) against the
    # oracle's rule: slice count, width, modulus count and the moduli
    info = ozlu.ozlu_mp_plan_opts(p, k, ozlu.make_opts(modset="ext", nslice=S))
    ref = make_plan(p, k, modset="ext", S=S or None)
    assert (info.S, info.w, info.Q, info.n_mod, info.g0, info.pair_terms) == \
        (ref.S, ref.w, ref.Q, ref.N, ref.g0, ref.pair_terms)
    assert list(info.moduli)[:min(64, info.n_mod)] == list(ref.moduli)[:64]


def test_mp_plan_opts_rejects_bad_options(L):
    with pytest.raises(ozlu.OzluError):
        ozlu.ozlu_mp_plan_opts(300, 9, ozlu.make_opts(modset=7))
    with pytest.raises(ozlu.OzluError):
        ozlu.ozlu_mp_plan_opts(11600, 512, ozlu.make_opts(modset="ext", nslice=1))   # beyond 23226 bits
    # default options are the INT8 route
    a = ozlu.ozlu_mp_plan_opts(3136, 256)
    b = ozlu.ozlu_mp_plan(3136, 256)
    assert (a.S, a.n_mod) == (b.S, b.n_mod)
