"""Modulus sets, CRT constants and the (S, w, N_mod) rule of Ozaki scheme II.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
  * Sec. 3.2, first paragraph: at most 54 pairwise-coprime moduli not
    exceeding 255, the largest power of each prime, about 362.8 bits.
  * Sec. 3.2, "Determining w and N": slack = ceil(log2 2K) + 16 + g_ex;
    for S = 1, 2, ...: w = ceil((p + slack)/S),
    need = 2w + log2 K + log2 S + 5, N = the number of moduli whose
    cumulative log2 first exceeds need; the INT32 condition
    K_pad * S * 127^2 < 2^31.
  * Sec. 3.2, "CRT reconstruction per digit group": M_l = P/m_l,
    y_l = M_l^-1 mod m_l.
  * Sec. 3.2, "Truncation under cancellation": extra retained digit groups.
  * Sec. 4.2.6, Eq. (17): binary64 residues need K (m/2)^2 < 2^53.
  * Sec. 4.2.3, Eq. (15): FP8 balanced base-17 digits keep the INT8 set.
  * Sec. 4.2.3, Eq. (14): binary16 residues (|r| <= 127) with an fp32
    accumulator need K_pad S 127^2 < 2^24; the INT8 modulus set is kept.
  * Sec. 4.2.4 "Precision ceiling of the INT8 back-end": moduli above 255
    (up to 16257, Eq. (int8lim)) with the centered residue split into two
    balanced base-128 digits r = 128 q + r0 and the product formed by
    Karatsuba from the three int8 planes r0, r0 + q, q; the table holds about
    1880 pairwise-coprime moduli not exceeding 16191, 23226 bits.
  * Sec. 3.2 "Choosing S: a cost model", Eq. (Lhint):
    S* = ceil(sqrt(r n_d (M + N) / (M N))), n_d = ceil(t / 16).

Readings where the paper is silent or garbled:
  * the modulus order is descending (largest first); ascending order does not
    reproduce the printed GEMM counts, descending reproduces all of them;
  * the INT8 set uses 2^7 = 128 (|r| <= 127 for every modulus); the printed
    "362.8 bits" equals the set with 2^8, which gives the same counts;
  * "take the smallest S that satisfies the INT32 condition" is read as: the
    smallest S whose modulus set has enough capacity, subject to the
    accumulator condition;
  * K_pad is K rounded up to a multiple of 128.
  * The extended table is the 54 INT8 moduli together with the primes in
    (255, 16191]: 1882 moduli and 23226.2 bits, the two figures the paper
    prints; it is taken in descending order like the INT8 set, and every
    modulus above 255 costs three int8 GEMMs (its Karatsuba planes).
  * In Eq. (Lhint), t is the width of one unsplit pass, p + slack.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


def primes_upto(n: int) -> list[int]:
    """All primes <= n by the sieve of Eratosthenes."""
    if n < 2:
        return []
    sieve = bytearray([1]) * (n + 1)
    sieve[0] = sieve[1] = 0
    for i in range(2, math.isqrt(n) + 1):
        if sieve[i]:
            sieve[i * i :: i] = bytearray(len(sieve[i * i :: i]))
    return [i for i in range(n + 1) if sieve[i]]


def int8_moduli(use_256: bool = False) -> list[int]:
    """The 54 pairwise-coprime prime powers <= 255, largest first (Sec. 3.2)."""
    ms = []
    for q in primes_upto(255):
        v = q
        while v * q <= 255:
            v *= q
        ms.append(v)
    if use_256:
        ms = [256 if m == 128 else m for m in ms]
    return sorted(ms, reverse=True)


def fp64_moduli(K: int) -> list[int]:
    """Primes m with K (m/2)^2 < 2^53, largest first (Sec. 4.2.6, Eq. (17)).

    Eq. (17) bounds one exact binary64 accumulation of length K, so the
    binary64 back-end reduces every pair-term product modulo m before adding
    the pair terms of a digit group (a reading: with this bound the printed
    binary64 counts, 16 moduli at p = 8192 and 13 for DD at K = 512, are
    reproduced; a K*S bound does not reproduce them).
    """
    # K m^2 < 2^55  <=>  m < sqrt(2^55 / K)
    bound = math.isqrt(((1 << 55) - 1) // K)
    while bound > 1 and K * bound * bound >= (1 << 55):
        bound -= 1
    return primes_upto(bound)[::-1]


EXT_LIMIT = 16191      # Sec. 4.2.4: the extended table's largest entry bound
EXT_MAX_MODULUS = 16257  # Eq. (int8lim): |r| <= 63 * 128 + 64 = 8128


def ext_moduli() -> list[int]:
    """Extended INT8 table (Sec. 4.2.4): the 54 INT8 moduli and the primes in
    (255, 16191], pairwise coprime, largest first."""
    big = [q for q in primes_upto(EXT_LIMIT) if q > 255]
    return sorted(int8_moduli() + big, reverse=True)


def base128_digits(r: int) -> tuple[int, int]:
    """r = 128 q + r0 with |r0| <= 64 (Sec. 4.2.4); q is the nearest integer to
    r / 128, ties toward zero (so r0 = +-64 keeps the sign of r).  For
    |r| <= 8128, |q| <= 63 and |r0 + q| <= 127, so all three Karatsuba planes
    are int8."""
    q = (abs(r) + 63) // 128
    if r < 0:
        q = -q
    return r - 128 * q, q


def residue_planes(m: int) -> int:
    """int8 GEMMs per modulus: 1 up to 255, 3 (Karatsuba) above."""
    return 1 if m <= 255 else 3


def lhint_S(r: float, t: int, M: int, N: int) -> int:
    """Eq. (Lhint): the cost-model estimate S* = ceil(sqrt(r n_d (M+N)/(MN))),
    n_d = ceil(t/16); r = 30 (INT8) or 17.9 (binary64) as calibrated in the
    paper, t the width of one unsplit pass."""
    n_d = -(-t // 16)
    return max(1, math.ceil(math.sqrt(r * n_d * (M + N) / (M * N))))


def pairs_in_group(g: int, S: int) -> int:
    """Number of (ta, tb) with ta + tb = g, 0 <= ta, tb < S (Sec. 3.2)."""
    return min(g, 2 * S - 2 - g) + 1


def k_pad(K: int) -> int:
    return -(-K // 128) * 128


@dataclass(frozen=True)
class Plan:
    p: int
    K: int
    backend: str
    g_ex: int
    extra_groups: int
    slack: int
    S: int
    w: int
    Q: int
    need: float
    N: int
    moduli: tuple
    P: int
    M: tuple = field(repr=False)
    y: tuple = field(repr=False)
    g0: int = 0
    modset: str = "int8"

    @property
    def groups(self) -> range:
        """Retained digit groups g0 .. 2S-2 (Sec. 3.2, slice splitting)."""
        return range(self.g0, 2 * self.S - 1)

    @property
    def pair_terms(self) -> int:
        return sum(pairs_in_group(g, self.S) for g in self.groups)

    @property
    def n_gemm(self) -> int:
        """#GEMM = S(S+1)/2 * N_mod with no extra groups (Eq. (8)); a modulus
        of the extended table above 255 counts its three Karatsuba planes."""
        if self.modset != "ext":
            return self.pair_terms * self.N
        return self.pair_terms * sum(residue_planes(m) for m in self.moduli)


def _accumulator_ok(backend: str, K: int, S: int) -> bool:
    if backend == "int8":
        return k_pad(K) * S * 127 * 127 < (1 << 31)
    if backend == "fp8":
        # Karatsuba planes of base-17 digits: |d0|,|d1|,|d0+d1| <= 15, FP32 sum
        return k_pad(K) * S * 15 * 15 < (1 << 24)
    if backend == "fp16":
        # Eq. (14): K_pad S 127^2 < 2^24 for binary16 residues, fp32 accumulator
        return k_pad(K) * S * 127 * 127 < (1 << 24)
    if backend == "fp64":
        return True  # folded into the modulus bound of fp64_moduli
    raise ValueError(backend)


def make_plan(p: int, K: int, backend: str = "int8", g_ex: int = 0,
              extra_groups: int = 0, S: int | None = None,
              use_256: bool = False, modset: str = "int8") -> Plan:
    """The (S, w, Q, N_mod) rule of Sec. 3.2 "Determining w and N".

    modset "ext" (INT8 back-end only) takes the moduli from the extended
    table of Sec. 4.2.4 instead of the 54 moduli up to 255."""
    if p < 1 or K < 1:
        raise ValueError("p and K must be positive")
    if modset not in ("int8", "ext") or (modset == "ext" and backend != "int8"):
        raise ValueError("the extended table is an INT8 route")
    slack = math.ceil(math.log2(2 * K)) + 16 + g_ex
    s_range = [S] if S is not None else range(1, 4097)
    for s in s_range:
        if backend == "fp64":
            mods = fp64_moduli(K)
        elif modset == "ext":
            mods = ext_moduli()
        else:
            mods = int8_moduli(use_256)
        if not _accumulator_ok(backend, K, s):
            continue
        w = -(-(p + slack) // s)
        need = 2 * w + math.log2(K) + math.log2(s) + 5
        cum = 0.0
        n_mod = None
        for i, m in enumerate(mods):
            cum += math.log2(m)
            if cum > need:
                n_mod = i + 1
                break
        if n_mod is None:
            continue
        chosen = tuple(mods[:n_mod])
        P = math.prod(chosen)
        M = tuple(P // m for m in chosen)
        y = tuple(pow(Ml % m, -1, m) for Ml, m in zip(M, chosen))
        g0 = max(0, s - 1 - extra_groups)
        return Plan(p=p, K=K, backend=backend, g_ex=g_ex,
                    extra_groups=extra_groups, slack=slack, S=s, w=w,
                    Q=w * s, need=need, N=n_mod, moduli=chosen, P=P, M=M,
                    y=y, g0=g0, modset=modset)
    raise ValueError(f"no plan for p={p} K={K} backend={backend}")


def single_pass_pmax(K: int, g: int, capacity_bits: float = 362.8) -> float:
    """Proposition 1: Q_max = (C - log2 2K - 2)/2, p_max = Q_max - log2 2K - g."""
    qmax = (capacity_bits - math.log2(2 * K) - 2) / 2
    return qmax - math.log2(2 * K) - g
