"""Thin ctypes binding of libhbperm.so (include/hbperm.h).

Argument marshalling only: every step of the test runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  The binding refuses to
run when the compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import collections.abc
import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhbperm.so")

HB_OK, HB_ERR_INVALID_ARG, HB_ERR_DEGENERATE, HB_ERR_CUDA, HB_ERR_OOM, HB_ERR_TIMEOUT, HB_ERR_UNSUPPORTED = range(7)
HB_F32, HB_BF16 = 0, 1
HB_STAT_LOGVOL_VMF, HB_STAT_ONE_MINUS_R2, HB_STAT_MEAN_COSDIST = 0, 1, 2
HB_ALT_TWO_SIDED, HB_ALT_GREATER, HB_ALT_LESS = 0, 1, 2
HB_PATH_MIXED, HB_PATH_FP32_PLAIN, HB_PATH_AUTO, HB_PATH_MIXED_NARROW, HB_PATH_MIXED_2SM = 0, 1, 2, 3, 4
ROUTE_PATHS = (HB_PATH_MIXED, HB_PATH_MIXED_NARROW, HB_PATH_FP32_PLAIN, HB_PATH_MIXED_2SM)  # hb_autotune's order
ROUTE_BUCKETS = 15  # size buckets of the route table (hb_autotune)


class HbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hbperm status {status}: {msg}")
        self.status = status


class hb_opts(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("stream", C.c_uint32),
        ("B", C.c_int64),
        ("stat", C.c_int32),
        ("alt", C.c_int32),
        ("align", C.c_int32),
        ("reflect_side", C.c_int32),
        ("exhaustive", C.c_int32),
        ("path", C.c_int32),
    ]


class hb_result(C.Structure):
    _fields_ = [
        ("p", C.c_double),
        ("count", C.c_int64),
        ("B_eff", C.c_int64),
        ("T_obs", C.c_double),
        ("r_x", C.c_double),
        ("r_y", C.c_double),
        ("reflection_skipped", C.c_int32),
        ("status", C.c_int32),
        ("n_rechecked", C.c_int64),
        ("band_max", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# hb_result as a numpy structured type with the same field offsets
_RESULT_KEYS = [k for k, _ in hb_result._fields_]
RESULT_DTYPE = np.dtype({
    "names": _RESULT_KEYS,
    "formats": [np.float64 if t is C.c_double else (np.int64 if t is C.c_int64 else np.int32)
                for _, t in hb_result._fields_],
    "offsets": [getattr(hb_result, k).offset for k in _RESULT_KEYS],
    "itemsize": C.sizeof(hb_result),
})


class Results(collections.abc.Sequence):
    """Per-pair results of a batched call in one structured numpy array
    (`array`, fields as hb_result); element i is the same dict that
    hb_result.as_dict gives, built when it is read."""

    __slots__ = ("array",)

    def __init__(self, array: np.ndarray):
        self.array = array

    def __len__(self):
        return len(self.array)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[k] for k in range(*i.indices(len(self)))]
        row = self.array[i]
        return {k: row[k].item() for k in _RESULT_KEYS}

    def column(self, key: str) -> np.ndarray:
        return self.array[key]

    def __eq__(self, other):  # as the list of dicts
        if isinstance(other, Results):
            return list(self) == list(other)
        if isinstance(other, list):
            return list(self) == other
        return NotImplemented

    __hash__ = None


def _sizes(v) -> np.ndarray:
    """Pair sizes as a contiguous int64 array (passed to the library by address)."""
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64))


def _packed(XY: torch.Tensor, na: np.ndarray, ma: np.ndarray) -> None:
    """The library reads sum(n + m) rows of d values from the XY pointer it is
    given, so the tensor must hold exactly that many rows, contiguously, and n
    and m must give one size per pair."""
    if XY.dim() != 2 or not XY.is_contiguous():
        raise ValueError("XY must be a contiguous 2-D tensor")
    if na.ndim != 1 or na.shape != ma.shape:
        raise ValueError("n and m must be 1-D with one entry per pair")
    rows = int(na.sum()) + int(ma.sum())
    if rows != XY.shape[0]:
        raise ValueError(f"XY has {XY.shape[0]} rows but the pair sizes add up to {rows}")


def _pair(X: torch.Tensor, Y: torch.Tensor) -> None:
    """X and Y of one pair: 2-D, one dtype, one embedding dimension."""
    if X.dim() != 2 or Y.dim() != 2:
        raise ValueError("X and Y must be 2-D (rows = embeddings)")
    if X.dtype != Y.dtype or X.shape[1] != Y.shape[1]:
        raise ValueError("X and Y must have the same dtype and embedding dimension")


def _results(P: int):
    arr = np.zeros(P, dtype=RESULT_DTYPE)
    return arr, arr.ctypes.data_as(C.POINTER(hb_result))


_lib = None


def lib():
    """Loads libhbperm.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhbperm.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, u64, u32 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_uint32
        L.hb_ctx_create.argtypes = [C.POINTER(vp), C.c_int]
        L.hb_ctx_create.restype = C.c_int
        L.hb_ctx_destroy.argtypes = [vp]
        L.hb_ctx_destroy.restype = None
        L.hb_align.argtypes = [vp, vp, i64, vp, i64, i64, i32, i32, i32, vp, vp, C.POINTER(i32), vp]
        L.hb_align.restype = C.c_int
        L.hb_perm_test.argtypes = [vp, vp, i64, vp, i64, i64, i32, C.POINTER(hb_opts), C.POINTER(hb_result), vp, vp]
        L.hb_perm_test.restype = C.c_int
        L.hb_perm_test_batched.argtypes = [vp, i64, vp, vp, vp, i64, i32, C.POINTER(hb_opts), C.POINTER(hb_result), vp]
        L.hb_perm_test_batched.restype = C.c_int
        L.hb_perm_labels.argtypes = [u64, u32, i64, i64, i64, i64, vp, vp]
        L.hb_perm_labels.restype = C.c_int
        L.hb_plan_create.argtypes = [vp, i64, vp, vp, i64, i32, C.POINTER(hb_opts), C.POINTER(vp)]
        L.hb_plan_create.restype = C.c_int
        L.hb_plan_execute.argtypes = [vp, vp, C.POINTER(hb_result), vp]
        L.hb_plan_execute.restype = C.c_int
        L.hb_plan_destroy.argtypes = [vp]
        L.hb_plan_destroy.restype = None
        L.hb_autotune.argtypes = [vp, i64, i32, C.POINTER(hb_opts), i64, C.POINTER(C.c_float)]
        L.hb_autotune.restype = C.c_int
        L.hb_route.argtypes = [vp, i64, C.POINTER(i32)]
        L.hb_route.restype = C.c_int
        L.hb_last_error.argtypes = []
        L.hb_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st: int):
    if st != HB_OK:
        raise HbError(st, lib().hb_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return HB_F32
    if t.dtype == torch.bfloat16:
        return HB_BF16
    raise TypeError("embeddings must be torch.float32 or torch.bfloat16")


def _dev(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def make_opts(B=9999, seed=0, stream=0, stat=HB_STAT_LOGVOL_VMF, alt=HB_ALT_TWO_SIDED, align=1, reflect_side=0,
              exhaustive=0, path=HB_PATH_MIXED) -> hb_opts:
    return hb_opts(seed, stream, B, stat, alt, align, reflect_side, exhaustive, path)


class Context:
    """Owns an hb_ctx (device workspace, pinned staging)."""

    def __init__(self, device: int | None = None):
        dev = torch.cuda.current_device() if device is None else device
        self.device = dev
        h = C.c_void_p()
        _check(lib().hb_ctx_create(C.byref(h), dev))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().hb_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hb_align(ctx: Context, X: torch.Tensor, Y: torch.Tensor, align=1, reflect_side=0, stream=None):
    """Returns (Z [n+m][d] same dtype, u [d] float64, skipped)."""
    _pair(X, Y)
    dt = _dtype_code(X)
    n, d = X.shape
    m = Y.shape[0]
    Z = torch.empty((n + m, d), dtype=X.dtype, device=X.device)
    u = torch.empty(d, dtype=torch.float64, device=X.device)
    sk = C.c_int32(0)
    _check(lib().hb_align(ctx.handle, _dev(X), n, _dev(Y), m, d, dt, align, reflect_side, _dev(Z), _dev(u),
                          C.byref(sk), _stream(stream)))
    return Z, u, int(sk.value)


def hb_align_noalloc(X: torch.Tensor, Y: torch.Tensor, align=1, reflect_side=0, stream=None):
    """hb_align for callers that cannot allocate device memory: the library
    takes its scratch from a fixed 2 MiB device array (d <= 1024, n + m <= 8192)
    instead of a context workspace.  The caller provides the output buffers;
    here they are allocated by torch only because this is a Python test
    harness.  Returns (Z, u, skipped)."""
    _pair(X, Y)
    L = lib()
    L.hb_align_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]
    L.hb_align_noalloc.restype = C.c_int
    dt = _dtype_code(X)
    n, d = X.shape
    m = Y.shape[0]
    Z = torch.empty((n + m, d), dtype=X.dtype, device=X.device)
    u = torch.empty(d, dtype=torch.float64, device=X.device)
    sk = C.c_int32(0)
    _check(L.hb_align_noalloc(_dev(X), n, _dev(Y), m, d, dt, align, reflect_side, _dev(Z), _dev(u), C.byref(sk),
                              _stream(stream)))
    return Z, u, int(sk.value)


def hb_perm_test(ctx: Context, X: torch.Tensor, Y: torch.Tensor, opts: hb_opts, want_T=False, stream=None,
                 check=True):
    """Returns (result dict, T_b float32 tensor or None)."""
    _pair(X, Y)
    dt = _dtype_code(X)
    n, d = X.shape
    m = Y.shape[0]
    res = hb_result()
    T = None
    Tp = C.c_void_p(None)
    if want_T:
        from math import comb
        Beff = comb(n + m, n) if opts.exhaustive else opts.B
        T = torch.full((Beff,), float("nan"), dtype=torch.float32, device=X.device)
        Tp = _dev(T)
    st = lib().hb_perm_test(ctx.handle, _dev(X), n, _dev(Y), m, d, dt, C.byref(opts), C.byref(res), Tp,
                            _stream(stream))
    if check:
        _check(st)
    return res.as_dict(), T


def hb_perm_test_batched(ctx: Context, XY: torch.Tensor, n, m, opts: hb_opts, stream=None, check=True):
    """XY packs, per pair, n[p] rows of X then m[p] rows of Y (device or host
    tensor).  Returns a Results sequence: one result dict per pair."""
    dt = _dtype_code(XY)
    na, ma = _sizes(n), _sizes(m)
    _packed(XY, na, ma)
    d = XY.shape[1]
    P = len(na)
    arr, res = _results(P)
    st = lib().hb_perm_test_batched(ctx.handle, P, C.c_void_p(XY.data_ptr()), na.ctypes.data, ma.ctypes.data, d, dt,
                                    C.byref(opts), res, _stream(stream))
    if check:
        _check(st)
    return Results(arr)


class Plan:
    """hb_plan: a batch shape (sizes n, m, d, dtype, opts) planned once; each
    execute() replays the captured CUDA graph of the whole test on new data."""

    def __init__(self, ctx: Context, n, m, d: int, dtype, opts: hb_opts):
        self.P = len(n)
        self.d = int(d)
        self.dtype = dtype if isinstance(dtype, int) else _dtype_code(torch.empty(0, dtype=dtype))
        na, ma = _sizes(n), _sizes(m)
        if na.ndim != 1 or na.shape != ma.shape:
            raise ValueError("n and m must be 1-D with one entry per pair")
        self.rows = int(na.sum()) + int(ma.sum())
        h = C.c_void_p()
        _check(lib().hb_plan_create(ctx.handle, self.P, na.ctypes.data, ma.ctypes.data, self.d, self.dtype, C.byref(opts), C.byref(h)))
        self._h = h
        self._ctx = ctx  # the plan keeps the context alive

    def execute(self, XY: torch.Tensor, stream=None, check=True):
        if XY.dim() != 2 or not XY.is_contiguous():
            raise ValueError("XY must be a contiguous 2-D tensor")
        if XY.shape != (self.rows, self.d) or _dtype_code(XY) != self.dtype:
            raise ValueError("XY does not match the plan's rows / d / dtype")
        arr, res = _results(self.P)
        st = lib().hb_plan_execute(self._h, C.c_void_p(XY.data_ptr()), res, _stream(stream))
        if check:
            _check(st)
        return Results(arr)

    def close(self):
        if getattr(self, "_h", None):
            lib().hb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class hb_layout_counts(C.Structure):
    _fields_ = [("n_chunks", C.c_int32), ("n_pieces", C.c_int32), ("n_label_chunks", C.c_int32),
                ("n_items", C.c_int32)]


def plan_layout(n, m, d: int, dtype, opts: hb_opts) -> dict:
    """hb_plan_layout: the launch layout of a batched call for these sizes
    (host computation, no GPU): row chunks [k][pair, side, row0, rows], input
    pieces [k][p0, p1, c0, c1], label/GEMM chunk cuts [k][order position, first
    item], work items [k][pair, tile group, mode] and the pair order, as int32
    numpy arrays."""
    L = lib()
    vp = C.c_void_p
    L.hb_plan_layout.argtypes = [C.c_int64, vp, vp, C.c_int64, C.c_int32, C.POINTER(hb_opts),
                                 C.POINTER(hb_layout_counts), vp, vp, vp, vp, vp]
    L.hb_plan_layout.restype = C.c_int
    na, ma = _sizes(n), _sizes(m)
    if na.ndim != 1 or na.shape != ma.shape:
        raise ValueError("n and m must be 1-D with one entry per pair")
    code = dtype if isinstance(dtype, int) else _dtype_code(torch.empty(0, dtype=dtype))
    P = len(na)
    cnt = hb_layout_counts()
    args = (P, na.ctypes.data, ma.ctypes.data, int(d), code, C.byref(opts), C.byref(cnt))
    _check(L.hb_plan_layout(*args, None, None, None, None, None))
    out = {"chunks": np.zeros((cnt.n_chunks, 4), np.int32), "pieces": np.zeros((cnt.n_pieces, 4), np.int32),
           "label_chunks": np.zeros((cnt.n_label_chunks + 1, 2), np.int32),
           "items": np.zeros((cnt.n_items, 3), np.int32),
           "order": np.zeros(P if opts.path != HB_PATH_FP32_PLAIN else 0, np.int32)}
    _check(L.hb_plan_layout(*args, *(out[k].ctypes.data if out[k].size else None
                                     for k in ("chunks", "pieces", "label_chunks", "items", "order"))))
    return out


def autotune(ctx: Context, d: int, dtype, opts: hb_opts, max_N: int = 65536):
    """Times the routes per size bucket and fills the context's route table;
    returns the [ROUTE_BUCKETS][len(ROUTE_PATHS)] wall-clock ms (in
    ROUTE_PATHS order; -1 = not timed) as a numpy array."""
    import numpy as np

    code = dtype if isinstance(dtype, int) else _dtype_code(torch.empty(0, dtype=dtype))
    ms = (C.c_float * (ROUTE_BUCKETS * len(ROUTE_PATHS)))()
    _check(lib().hb_autotune(ctx.handle, int(d), code, C.byref(opts), int(max_N), ms))
    return np.array(ms[:], dtype=np.float32).reshape(ROUTE_BUCKETS, len(ROUTE_PATHS))


def route(ctx: Context, N: int) -> int:
    """The path HB_PATH_AUTO takes for a pair of size N."""
    r = C.c_int32()
    _check(lib().hb_route(ctx.handle, int(N), C.byref(r)))
    return r.value


def hb_perm_labels(seed: int, stream_id: int, n: int, N: int, b0: int, count: int, device=None, stream=None):
    """HB-LABEL-v1 rows [count][ceil(N/32)] as an int32 tensor (bit patterns)."""
    W = (N + 31) // 32
    out = torch.zeros((count, W), dtype=torch.int32, device=device or torch.cuda.current_device())
    _check(lib().hb_perm_labels(seed, stream_id, n, N, b0, count, _dev(out), _stream(stream)))
    return out


def declared_symbols(header: str | None = None):
    """Function names declared in include/hbperm.h."""
    import re
    header = header or os.path.join(os.path.dirname(_HERE), "include", "hbperm.h")
    src = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:hb_status|void|int64_t|const char \*)\s*(hb_\w+)\s*\(", src, re.M)))


HB_OPT_WAIT_LIMIT_NS, HB_OPT_SINGLE_SLICE_MAX_N, HB_OPT_TEST_WITHHOLD_ARRIVAL, HB_OPT_A_OPERAND_TMEM = 1, 2, 4, 8


def set_option(ctx: Context, option: int, value: int):
    """hb_ctx_set_option: wait limit, single-slice pair limit, test hook."""
    L = lib()
    L.hb_ctx_set_option.argtypes = [C.c_void_p, C.c_int32, C.c_int64]
    L.hb_ctx_set_option.restype = C.c_int
    _check(L.hb_ctx_set_option(ctx.handle, int(option), int(value)))


def set_timing(ctx: Context, enable: bool = True):
    L = lib()
    L.hb_ctx_set_timing.argtypes = [C.c_void_p, C.c_int32]
    L.hb_ctx_set_timing.restype = C.c_int
    _check(L.hb_ctx_set_timing(ctx.handle, 1 if enable else 0))


STAGES = ("align", "zstats_tobs", "labels", "gemm_epilogue", "recheck", "finalize_copy", "gemm_kernels")


def stage_times(ctx: Context):
    """(dict stage -> ms, kernel launches) of the last test call on ctx."""
    L = lib()
    L.hb_ctx_stage_times.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]
    L.hb_ctx_stage_times.restype = C.c_int
    ms = (C.c_float * len(STAGES))()
    nl = C.c_int32(0)
    _check(L.hb_ctx_stage_times(ctx.handle, ms, C.byref(nl)))
    return dict(zip(STAGES, [float(v) for v in ms])), int(nl.value)


# --------------------------------------------------------------------------
# learned triage
# --------------------------------------------------------------------------
TRIAGE_NFEAT, TRIAGE_NQ = 19, 9
TRIAGE_LEVELS = (0.5, 0.8, 0.9, 0.95, 0.975, 0.99, 0.995, 0.998, 0.999)


class hb_mlp(C.Structure):
    _fields_ = [("params", C.c_void_p), ("params_bf16", C.c_void_p), ("grad", C.c_void_p), ("adam_m", C.c_void_p),
                ("adam_v", C.c_void_p)]


def _batched_args(XY, n, m):
    na, ma = _sizes(n), _sizes(m)
    _packed(XY, na, ma)
    return len(na), (C.c_int64 * len(na)).from_buffer(na), (C.c_int64 * len(ma)).from_buffer(ma)


def triage_features(ctx: Context, XY: torch.Tensor, n, m, opts: hb_opts, stream=None):
    """(features [P][19] float32, T_obs [P] float64, results) of packed pairs."""
    L = lib()
    vp = C.c_void_p
    L.hb_triage_features.argtypes = [vp, C.c_int64, vp, vp, vp, C.c_int64, C.c_int32, C.POINTER(hb_opts), vp, vp,
                                     C.POINTER(hb_result), vp]
    L.hb_triage_features.restype = C.c_int
    P, na, ma = _batched_args(XY, n, m)
    feat = torch.empty((P, TRIAGE_NFEAT), dtype=torch.float32, device=XY.device)
    tobs = torch.empty(P, dtype=torch.float64, device=XY.device)
    res = (hb_result * P)()
    _check(L.hb_triage_features(ctx.handle, P, _dev(XY), na, ma, XY.shape[1], _dtype_code(XY), C.byref(opts),
                                _dev(feat), _dev(tobs), res, _stream(stream)))
    return feat, tobs, [r.as_dict() for r in res]


def null_quantiles(ctx: Context, XY: torch.Tensor, n, m, opts: hb_opts, stream=None):
    """(quantiles of |T_b| x100 [P][9] float32, results) from the full test."""
    L = lib()
    vp = C.c_void_p
    L.hb_null_quantiles.argtypes = [vp, C.c_int64, vp, vp, vp, C.c_int64, C.c_int32, C.POINTER(hb_opts), vp,
                                    C.POINTER(hb_result), vp]
    L.hb_null_quantiles.restype = C.c_int
    P, na, ma = _batched_args(XY, n, m)
    q = torch.empty((P, TRIAGE_NQ), dtype=torch.float32, device=XY.device)
    res = (hb_result * P)()
    _check(L.hb_null_quantiles(ctx.handle, P, _dev(XY), na, ma, XY.shape[1], _dtype_code(XY), C.byref(opts),
                               _dev(q), res, _stream(stream)))
    return q, [r.as_dict() for r in res]


def mlp_param_count() -> int:
    L = lib()
    L.hb_mlp_param_count.argtypes = []
    L.hb_mlp_param_count.restype = C.c_int64
    return int(L.hb_mlp_param_count())


class MLP:
    """Device buffers of the triage network (the library's kernels do all math)."""

    def __init__(self, params: torch.Tensor):
        n = mlp_param_count()
        assert params.numel() == n and params.dtype == torch.float32 and params.is_cuda
        dev = params.device
        self.params = params.contiguous()
        self.params_bf16 = torch.empty(n, dtype=torch.int16, device=dev)
        self.grad = torch.zeros(n, dtype=torch.float32, device=dev)
        self.adam_m = torch.zeros(n, dtype=torch.float32, device=dev)
        self.adam_v = torch.zeros(n, dtype=torch.float32, device=dev)
        self.step = 0
        self._net = hb_mlp(self.params.data_ptr(), self.params_bf16.data_ptr(), self.grad.data_ptr(),
                           self.adam_m.data_ptr(), self.adam_v.data_ptr())
        L = lib()
        L.hb_mlp_sync.argtypes = [C.POINTER(hb_mlp), C.c_void_p]
        L.hb_mlp_sync.restype = C.c_int
        _check(L.hb_mlp_sync(C.byref(self._net), _stream()))

    def forward(self, ctx: Context, feat: torch.Tensor, stream=None) -> torch.Tensor:
        L = lib()
        L.hb_mlp_forward.argtypes = [C.c_void_p, C.POINTER(hb_mlp), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.hb_mlp_forward.restype = C.c_int
        out = torch.empty((feat.shape[0], TRIAGE_NQ), dtype=torch.float32, device=feat.device)
        _check(L.hb_mlp_forward(ctx.handle, C.byref(self._net), feat.shape[0], _dev(feat), _dev(out), _stream(stream)))
        return out

    def grad_step(self, ctx: Context, feat: torch.Tensor, target: torch.Tensor, stream=None) -> torch.Tensor:
        """Fills self.grad with the gradient of the mean pinball loss; returns the loss (device)."""
        L = lib()
        L.hb_mlp_grad.argtypes = [C.c_void_p, C.POINTER(hb_mlp), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]
        L.hb_mlp_grad.restype = C.c_int
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        _check(L.hb_mlp_grad(ctx.handle, C.byref(self._net), feat.shape[0], _dev(feat), _dev(target), _dev(loss),
                             _stream(stream)))
        return loss

    def adam(self, lr: float, stream=None):
        L = lib()
        L.hb_mlp_adam.argtypes = [C.POINTER(hb_mlp), C.c_float, C.c_int64, C.c_void_p]
        L.hb_mlp_adam.restype = C.c_int
        self.step += 1
        _check(L.hb_mlp_adam(C.byref(self._net), lr, self.step, _stream(stream)))


def triage_predict_p(quant: torch.Tensor, tobs: torch.Tensor, stream=None) -> torch.Tensor:
    L = lib()
    L.hb_triage_predict_p.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.hb_triage_predict_p.restype = C.c_int
    p = torch.empty(quant.shape[0], dtype=torch.float32, device=quant.device)
    _check(L.hb_triage_predict_p(quant.shape[0], _dev(quant), _dev(tobs), _dev(p), _stream(stream)))
    return p
