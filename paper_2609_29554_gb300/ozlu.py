"""Python binding of the ozlu C ABI (include/ozlu.h): argument marshalling only.

Every entry point of the shared library has a function of the same name here.
Matrices are passed as torch tensors (device memory, used in place) or numpy
arrays (host memory, staged by the library).  An expansion matrix with
leading dimension ld and c columns is a float64 array of shape (c, ld, nc),
contiguous: column-major storage with nc components per element.

The library is required: importing a function that needs it raises
RuntimeError when libozlu.so has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libozlu.so")

OZLU_OK = 0
OZLU_ERR_CUDA = 1001
OZLU_ERR_NOMEM = 1002
OZLU_ERR_CAPACITY = 1003
OZLU_ERR_TIMEOUT = 1004
OZLU_ERR_UNSUPPORTED = 1005
OZLU_MODSET_INT8 = 0
OZLU_MODSET_EXT = 1
BACKENDS = {"auto": 0, "int8": 1, "fp8": 2, "fp64": 3, "fp16": 4}

_lib = None


class ozlu_opts(ctypes.Structure):
    _fields_ = [("backend", ctypes.c_int), ("nslice", ctypes.c_int),
                ("extra_groups", ctypes.c_int), ("g_ex", ctypes.c_int),
                ("native", ctypes.c_int), ("graph", ctypes.c_int),
                ("panel_width", ctypes.c_int), ("modset", ctypes.c_int),
                ("reserved", ctypes.c_int * 8)]


class ozlu_plan_info(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in ("p", "K", "backend", "S", "w", "Q", "n_mod",
                                             "g0", "n_groups", "pair_terms")] + \
               [("moduli", ctypes.c_int * 64)]


class ozlu_stats(ctypes.Structure):
    _fields_ = [("convert_ms", ctypes.c_double), ("gemm_ms", ctypes.c_double),
                ("crt_ms", ctypes.c_double), ("panel_ms", ctypes.c_double),
                ("other_ms", ctypes.c_double), ("gemm_launches", ctypes.c_longlong),
                ("crt_launches", ctypes.c_longlong), ("panel_launches", ctypes.c_longlong),
                ("launches", ctypes.c_longlong), ("gemm_ops", ctypes.c_double),
                ("crt_bytes", ctypes.c_double), ("convert_bytes", ctypes.c_double),
                ("last_backend", ctypes.c_int), ("graph_status", ctypes.c_int),
                ("trsm_ms", ctypes.c_double), ("last_nslice", ctypes.c_int),
                ("tuned_nb", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_longlong
class ozlu_mp_matrix(ctypes.Structure):
    _fields_ = [("limbs", ctypes.c_void_p), ("exps", ctypes.c_void_p), ("signs", ctypes.c_void_p),
                ("ld", ctypes.c_longlong), ("plane", ctypes.c_longlong), ("L", ctypes.c_int),
                ("pad_", ctypes.c_int)]


SIGNATURES = {
    "ozlu_version": (ctypes.c_char_p, []),
    "ozlu_create": (_I, [ctypes.POINTER(_P), _P]),
    "ozlu_destroy": (_I, [_P]),
    "ozlu_set_stream": (_I, [_P, _P]),
    "ozlu_plan": (_I, [_I, _I, ctypes.POINTER(ozlu_opts), ctypes.POINTER(ozlu_plan_info)]),
    "ozlu_mp_plan": (_I, [_I, _I, ctypes.POINTER(ozlu_plan_info)]),
    "ozlu_gemm": (_I, [_P, _I, _I, _I, _I, _I, _I, _P, _L, _P, _L, _I, _P, _L,
                       ctypes.POINTER(ozlu_opts)]),
    "ozlu_getrf": (_I, [_P, _I, _I, _I, _P, _L, _P, _I, _P, ctypes.POINTER(ozlu_opts)]),
    "ozlu_getrs": (_I, [_P, _I, _I, _I, _I, _P, _L, _P, _P, _L, ctypes.POINTER(ozlu_opts)]),
    "ozlu_debug_fetch": (_I, [_P, _I, _P, ctypes.c_size_t]),
    "ozlu_set_timing": (_I, [_P, _I]),
    "ozlu_get_stats": (_I, [_P, ctypes.POINTER(ozlu_stats)]),
    "ozlu_gemm_noalloc": (_I, [_I, _I, _I, _I, _I, _I, _P, _L, _P, _L, _I, _P, _L, _P]),
    "ozlu_getrf_batched": (_I, [_P, _I, _I, _I, _P, _P, _P, _P, _P, _I, ctypes.POINTER(ozlu_opts)]),
    "ozlu_getrs_batched": (_I, [_P, _I, _I, _I, _P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(ozlu_opts)]),
    "ozlu_mp_gemm": (_I, [_P, _I, _I, _I, _I, _I, ctypes.POINTER(ozlu_mp_matrix),
                          ctypes.POINTER(ozlu_mp_matrix), _I, ctypes.POINTER(ozlu_mp_matrix)]),
    "ozlu_mp_getrf": (_I, [_P, _I, _I, ctypes.POINTER(ozlu_mp_matrix), _P, _I, _P]),
    "ozlu_mp_getrs": (_I, [_P, _I, _I, _I, ctypes.POINTER(ozlu_mp_matrix), _P,
                           ctypes.POINTER(ozlu_mp_matrix)]),
    "ozlu_mp_set_opts": (_I, [_P, ctypes.POINTER(ozlu_opts)]),
    "ozlu_mp_plan_opts": (_I, [_I, _I, ctypes.POINTER(ozlu_opts), ctypes.POINTER(ozlu_plan_info)]),
    "ozlu_debug_fail_alloc": (_I, [_I]),
    "ozlu_debug_wait_expiry": (_I, [_P, _I, _L, _P]),
}


def lib():
    """The loaded libozlu.so; raises RuntimeError when it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libozlu.so is not built: run paper_2609_29554_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class OzluError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {code}")
        self.code = code


def _check(fn, code):
    if code != OZLU_OK:
        raise OzluError(fn, code)


def make_opts(backend="int8", nslice=0, extra_groups=0, g_ex=0, native=0, graph=0, panel_width=0,
              modset=0):
    o = ozlu_opts()
    o.backend = BACKENDS[backend] if isinstance(backend, str) else int(backend)
    o.nslice, o.extra_groups, o.g_ex, o.native, o.graph = nslice, extra_groups, g_ex, native, graph
    o.panel_width = panel_width
    o.modset = {"int8": OZLU_MODSET_INT8, "ext": OZLU_MODSET_EXT}.get(modset, modset)
    return o


def _ptr(x):
    """Device pointer of a torch tensor, host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def ozlu_version():
    return lib().ozlu_version().decode()


def ozlu_create(stream=None):
    h = _P()
    _check("ozlu_create", lib().ozlu_create(ctypes.byref(h), _stream_ptr(stream)))
    return h


def ozlu_destroy(h):
    _check("ozlu_destroy", lib().ozlu_destroy(h))


def ozlu_set_stream(h, stream):
    _check("ozlu_set_stream", lib().ozlu_set_stream(h, _stream_ptr(stream)))


def ozlu_plan(p, k, opts=None):
    info = ozlu_plan_info()
    _check("ozlu_plan", lib().ozlu_plan(p, k, ctypes.byref(opts) if opts else None,
                                        ctypes.byref(info)))
    return info


def ozlu_mp_plan(p, k):
    info = ozlu_plan_info()
    _check("ozlu_mp_plan", lib().ozlu_mp_plan(p, k, ctypes.byref(info)))
    return info


def ozlu_mp_plan_opts(p, k, opts=None):
    info = ozlu_plan_info()
    _check("ozlu_mp_plan_opts", lib().ozlu_mp_plan_opts(p, k, ctypes.byref(opts) if opts else None,
                                                        ctypes.byref(info)))
    return info


def ozlu_mp_set_opts(h, opts=None):
    _check("ozlu_mp_set_opts", lib().ozlu_mp_set_opts(h, ctypes.byref(opts) if opts else None))


def ozlu_gemm(h, nc, p, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, opts=None):
    _check("ozlu_gemm", lib().ozlu_gemm(h, nc, p, m, n, k, alpha, _ptr(A), lda, _ptr(B), ldb,
                                        beta, _ptr(C), ldc,
                                        ctypes.byref(opts) if opts else None))


def ozlu_getrf(h, nc, p, n, A, lda, ipiv, nb, info, opts=None):
    _check("ozlu_getrf", lib().ozlu_getrf(h, nc, p, n, _ptr(A), lda, _ptr(ipiv), nb, _ptr(info),
                                          ctypes.byref(opts) if opts else None))


def ozlu_getrs(h, nc, p, n, nrhs, LU, lda, ipiv, B, ldb, opts=None):
    _check("ozlu_getrs", lib().ozlu_getrs(h, nc, p, n, nrhs, _ptr(LU), lda, _ptr(ipiv), _ptr(B),
                                          ldb, ctypes.byref(opts) if opts else None))


def ozlu_gemm_noalloc(nc, p, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """The allocation-free GEMM (device tensors only; see include/ozlu.h)."""
    _check("ozlu_gemm_noalloc", lib().ozlu_gemm_noalloc(nc, p, m, n, k, alpha, _ptr(A), lda, _ptr(B),
                                                        ldb, beta, _ptr(C), ldc,
                                                        _stream_ptr(stream)))


def _arrays(ns, mats, lds, pivs):
    cnt = len(ns)
    n_arr = (ctypes.c_int * cnt)(*[int(v) for v in ns])
    a_arr = (ctypes.c_void_p * cnt)(*[_ptr(x) for x in mats])
    l_arr = (ctypes.c_longlong * cnt)(*[int(v) for v in lds])
    p_arr = (ctypes.c_void_p * cnt)(*[_ptr(x) for x in pivs])
    return n_arr, a_arr, l_arr, p_arr


def ozlu_getrf_batched(h, nc, p, ns, mats, lds, pivs, info, nb=0, opts=None):
    """Batched LU: ns sizes, mats/pivs device tensors, info a device int32 tensor."""
    n_arr, a_arr, l_arr, p_arr = _arrays(ns, mats, lds, pivs)
    _check("ozlu_getrf_batched", lib().ozlu_getrf_batched(
        h, nc, p, len(ns), n_arr, a_arr, l_arr, p_arr, _ptr(info), nb,
        ctypes.byref(opts) if opts else None))


def ozlu_getrs_batched(h, nc, p, ns, nrhs, lus, lds, pivs, bs, ldbs, opts=None):
    n_arr, a_arr, l_arr, p_arr = _arrays(ns, lus, lds, pivs)
    cnt = len(ns)
    b_arr = (ctypes.c_void_p * cnt)(*[_ptr(x) for x in bs])
    lb_arr = (ctypes.c_longlong * cnt)(*[int(v) for v in ldbs])
    _check("ozlu_getrs_batched", lib().ozlu_getrs_batched(
        h, nc, p, cnt, n_arr, nrhs, a_arr, l_arr, p_arr, b_arr, lb_arr,
        ctypes.byref(opts) if opts else None))


def ozlu_debug_fetch(h, what, out: np.ndarray):
    _check("ozlu_debug_fetch", lib().ozlu_debug_fetch(h, what, out.ctypes.data, out.nbytes))
    return out


def ozlu_debug_fail_alloc(count):
    _check("ozlu_debug_fail_alloc", lib().ozlu_debug_fail_alloc(int(count)))


def ozlu_debug_wait_expiry(h, which, limit):
    """Return code and (gave_up, error_word, info) of one bounded-wait self-test."""
    out = np.zeros(3, dtype=np.int32)
    rc = lib().ozlu_debug_wait_expiry(h, which, int(limit), out.ctypes.data)
    return rc, tuple(int(v) for v in out)


def ozlu_set_timing(h, enable):
    _check("ozlu_set_timing", lib().ozlu_set_timing(h, int(enable)))


def ozlu_get_stats(h):
    st = ozlu_stats()
    _check("ozlu_get_stats", lib().ozlu_get_stats(h, ctypes.byref(st)))
    return st


# ----------------------------------------------------------- layouts -----
def to_colmajor(X: np.ndarray) -> np.ndarray:
    """(rows, cols, nc) -> contiguous (cols, rows, nc): column-major, ld = rows."""
    return np.ascontiguousarray(np.transpose(X, (1, 0, 2)))


def from_colmajor(Y: np.ndarray, rows: int) -> np.ndarray:
    """(cols, ld, nc) column-major -> (rows, cols, nc)."""
    return np.ascontiguousarray(np.transpose(Y[:, :rows, :], (1, 0, 2)))


# ------------------------------------------------------------ p-bit matrices
class MPMatrix:
    """A rows x cols p-bit matrix in device memory, the layout of ozlu_mp_matrix.

    Limb k of element (i, j) is limbs[k, i + j * rows] (int32 storage of the
    32-bit words), with exps[i + j * rows] and signs[i + j * rows]; value =
    (-1)^sign * mant * 2^(exp - 32 L) with mant normalised to its top bit.
    """

    def __init__(self, rows, cols, L, device="cuda"):
        import torch
        self.rows, self.cols, self.L = rows, cols, L
        size = max(rows * cols, 1)
        self.limbs = torch.zeros((L, size), dtype=torch.int32, device=device)
        self.exps = torch.zeros(size, dtype=torch.int32, device=device)
        self.signs = torch.zeros(size, dtype=torch.int32, device=device)

    def desc(self, i0=0, j0=0):
        """ozlu_mp_matrix of the submatrix with top-left (i0, j0)."""
        off = i0 + j0 * self.rows
        return ozlu_mp_matrix(self.limbs.data_ptr() + 4 * off, self.exps.data_ptr() + 4 * off,
                              self.signs.data_ptr() + 4 * off, max(self.rows, 1),
                              self.limbs.shape[1], self.L, 0)

    @classmethod
    def from_pairs(cls, pairs, L, device="cuda"):
        """From rows of exact (N, E) pairs (value N 2^E, |N| < 2^(32 L))."""
        import torch
        rows, cols = len(pairs), len(pairs[0]) if pairs else 0
        M = cls(rows, cols, L, device)
        limbs = np.zeros((L, max(rows * cols, 1)), dtype=np.uint32)
        exps = np.zeros(max(rows * cols, 1), dtype=np.int32)
        signs = np.zeros(max(rows * cols, 1), dtype=np.int32)
        for i in range(rows):
            for j in range(cols):
                N, E = pairs[i][j]
                x = i + j * rows
                if N == 0:
                    continue
                a = abs(int(N))
                b = a.bit_length()
                if b > 32 * L:
                    raise ValueError("significand wider than 32 L bits")
                mant = a << (32 * L - b)
                for k in range(L):
                    limbs[k, x] = (mant >> (32 * k)) & 0xffffffff
                exps[x] = b + E
                signs[x] = 1 if N < 0 else 0
        M.limbs.copy_(torch.from_numpy(limbs.view(np.int32)))
        M.exps.copy_(torch.from_numpy(exps))
        M.signs.copy_(torch.from_numpy(signs))
        return M

    def to_pairs(self):
        """Rows of exact (N, E) pairs (E = exp - 32 L)."""
        limbs = self.limbs.cpu().numpy().view(np.uint32)
        exps = self.exps.cpu().numpy()
        signs = self.signs.cpu().numpy()
        out = []
        for i in range(self.rows):
            row = []
            for j in range(self.cols):
                x = i + j * self.rows
                mant = 0
                for k in range(self.L - 1, -1, -1):
                    mant = (mant << 32) | int(limbs[k, x])
                if mant == 0:
                    row.append((0, 0))
                    continue
                row.append((-mant if signs[x] else mant, int(exps[x]) - 32 * self.L))
            out.append(row)
        return out


def ozlu_mp_gemm(h, p, m, n, k, alpha, A, B, beta, C):
    """A, B, C: ozlu_mp_matrix descriptors (MPMatrix.desc())."""
    _check("ozlu_mp_gemm", lib().ozlu_mp_gemm(h, p, m, n, k, alpha, ctypes.byref(A), ctypes.byref(B), beta,
                                              ctypes.byref(C)))


def ozlu_mp_getrf(h, p, n, A, ipiv, nb, info):
    _check("ozlu_mp_getrf", lib().ozlu_mp_getrf(h, p, n, ctypes.byref(A), _ptr(ipiv), nb, _ptr(info)))


def ozlu_mp_getrs(h, p, n, nrhs, LU, ipiv, B):
    _check("ozlu_mp_getrs", lib().ozlu_mp_getrs(h, p, n, nrhs, ctypes.byref(LU), _ptr(ipiv), ctypes.byref(B)))
