"""ctypes wrapper around the C oracle (hb_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.  The oracle is a plain FP64/exact CPU implementation of the
Householder-aligned permutation test (Algorithm 1 of the paper) and shares no
code with the CUDA path.

Every function takes and returns numpy arrays.  FP32 data travel as
``np.float32``; BF16 data travel as their ``np.uint16`` bit patterns.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhb_oracle.so")
_lock = threading.Lock()
_lib = None

F32, BF16 = 0, 1
STAT_LOGVOL_VMF, STAT_ONE_MINUS_R2, STAT_MEAN_COSDIST = 0, 1, 2
ALT_TWO_SIDED, ALT_GREATER, ALT_LESS = 0, 1, 2
OK, ERR_INVALID_ARG, ERR_DEGENERATE = 0, 1, 2


class Opts(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("stream", C.c_uint32),
        ("B", C.c_int64),
        ("stat", C.c_int32),
        ("alt", C.c_int32),
        ("align", C.c_int32),
        ("reflect_side", C.c_int32),
        ("exhaustive", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("p", C.c_double),
        ("count", C.c_int64),
        ("B_eff", C.c_int64),
        ("T_obs", C.c_double),
        ("r_x", C.c_double),
        ("r_y", C.c_double),
        ("reflection_skipped", C.c_int32),
        ("status", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FP contraction, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        vp, i64, u64, u32, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32
        L.hbo_philox4x32_10.argtypes = [vp, vp, vp]
        L.hbo_labels.argtypes = [u64, u32, i64, i64, i64, i64, vp]
        L.hbo_binomial.argtypes = [i64, i64]
        L.hbo_binomial.restype = i64
        L.hbo_labels_exhaustive.argtypes = [i64, i64, vp]
        L.hbo_align.argtypes = [vp, i64, vp, i64, i64, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
        L.hbo_align.restype = C.c_int
        L.hbo_perm_test.argtypes = [vp, i64, vp, i64, i64, C.c_int, C.POINTER(Opts), C.POINTER(Result), vp, vp]
        L.hbo_perm_test.restype = C.c_int
        L.hbo_perm_stats.argtypes = [vp, i64, vp, i64, i64, C.c_int, C.POINTER(Opts), vp, i64,
                                     C.POINTER(Result), vp, vp, vp]
        L.hbo_perm_stats.restype = C.c_int
        L.hbo_perm_test_batched.argtypes = [i64, vp, vp, vp, i64, C.c_int, C.POINTER(Opts), C.POINTER(Result)]
        L.hbo_perm_test_batched.restype = C.c_int
        L.hbo_fixed_from_f32bits.argtypes = [u32, C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]
        L.hbo_round_to_bf16.argtypes = [C.c_double]
        L.hbo_round_to_bf16.restype = C.c_double
        L.hbo_round_to_f32.argtypes = [C.c_double]
        L.hbo_round_to_f32.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.float32:
        return F32
    if a.dtype == np.uint16:
        return BF16
    raise TypeError("oracle inputs are float32 arrays or uint16 BF16 bit patterns")


def opts(seed=0, stream=0, B=999, stat=STAT_LOGVOL_VMF, alt=ALT_TWO_SIDED, align=1, reflect_side=0, exhaustive=0):
    return Opts(seed, stream, B, stat, alt, align, reflect_side, exhaustive)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().hbo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def labels(seed, stream, n, N, b0, count):
    """HB-LABEL-v1 label rows [count][ceil(N/32)] (uint32, LSB-first)."""
    W = (N + 31) // 32
    out = np.zeros((count, W), dtype=np.uint32)
    lib().hbo_labels(seed, stream, n, N, b0, count, _ptr(out))
    return out


def binomial(N, n):
    return int(lib().hbo_binomial(N, n))


def labels_exhaustive(n, N):
    C_ = binomial(N, n)
    out = np.zeros((C_, 1), dtype=np.uint32)
    lib().hbo_labels_exhaustive(n, N, _ptr(out))
    return out


def align(X: np.ndarray, Y: np.ndarray, align=1, reflect_side=0):
    """Returns (status, Z storage array [N][d], u [d] FP64, zf64 [N][d], skipped)."""
    X = np.ascontiguousarray(X)
    Y = np.ascontiguousarray(Y)
    dt = _dtype_code(X)
    assert Y.dtype == X.dtype and X.shape[1] == Y.shape[1]
    n, d = X.shape
    m = Y.shape[0]
    Z = np.zeros((n + m, d), dtype=X.dtype)
    u = np.zeros(d, dtype=np.float64)
    zf = np.zeros((n + m, d), dtype=np.float64)
    sk = C.c_int32(0)
    st = lib().hbo_align(_ptr(X), n, _ptr(Y), m, d, dt, align, reflect_side, _ptr(Z), _ptr(u), _ptr(zf),
                         C.cast(C.pointer(sk), C.c_void_p))
    return st, Z, u, zf, int(sk.value)


def perm_test(X: np.ndarray, Y: np.ndarray, o: Opts, want_T=False):
    """Full test of one pair.  Returns (result dict, T_b array or None, decisions or None)."""
    X = np.ascontiguousarray(X)
    Y = np.ascontiguousarray(Y)
    dt = _dtype_code(X)
    n, d = X.shape
    m = Y.shape[0]
    res = Result()
    T = dec = None
    Tp = dp = None
    if want_T:
        Beff = binomial(n + m, n) if o.exhaustive else o.B
        T = np.zeros(Beff, dtype=np.float64)
        dec = np.zeros(Beff, dtype=np.uint8)
        Tp, dp = _ptr(T), _ptr(dec)
    lib().hbo_perm_test(_ptr(X), n, _ptr(Y), m, d, dt, C.byref(o), C.byref(res), Tp, dp)
    return res.as_dict(), T, dec


def perm_stats(X: np.ndarray, Y: np.ndarray, o: Opts, b_list):
    """T_b, decisions and (q1, q2) for the listed permutation indices."""
    X = np.ascontiguousarray(X)
    Y = np.ascontiguousarray(Y)
    dt = _dtype_code(X)
    n, d = X.shape
    m = Y.shape[0]
    bl = np.ascontiguousarray(np.asarray(b_list, dtype=np.int64))
    T = np.zeros(len(bl), dtype=np.float64)
    dec = np.zeros(len(bl), dtype=np.uint8)
    q = np.zeros((len(bl), 2), dtype=np.float64)
    res = Result()
    lib().hbo_perm_stats(_ptr(X), n, _ptr(Y), m, d, dt, C.byref(o), _ptr(bl), len(bl), C.byref(res), _ptr(T),
                         _ptr(dec), _ptr(q))
    return res.as_dict(), T, dec, q


def perm_test_batched(XY: np.ndarray, n, m, o: Opts):
    XY = np.ascontiguousarray(XY)
    dt = _dtype_code(XY)
    d = XY.shape[1]
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int64))
    m = np.ascontiguousarray(np.asarray(m, dtype=np.int64))
    P = len(n)
    out = (Result * P)()
    lib().hbo_perm_test_batched(P, _ptr(XY), _ptr(n), _ptr(m), d, dt, C.byref(o), out)
    return [r.as_dict() for r in out]


def fixed_from_f32bits(bits: int) -> int:
    hi = C.c_int64(0)
    lo = C.c_uint64(0)
    lib().hbo_fixed_from_f32bits(bits, C.byref(hi), C.byref(lo))
    return (hi.value << 64) + lo.value


def round_to_bf16(x: float) -> float:
    return lib().hbo_round_to_bf16(x)


def round_to_f32(x: float) -> float:
    return lib().hbo_round_to_f32(x)
