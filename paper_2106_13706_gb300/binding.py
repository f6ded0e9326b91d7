"""Thin ctypes binding over libddks.so (C ABI in include/ddks.h).

Argument marshalling only: every step of the statistic runs in the library's
CUDA kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they
must be 2-D, C-contiguous, float32 or float64.  The binding never computes on
the host and raises if the CUDA library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libddks.so")

DDKS_OK = 0
DDKS_PENDING = 1
DDKS_F32, DDKS_F64 = 0, 1
PATH_AUTO, PATH_REGISTER, PATH_LANE, PATH_WARP, PATH_SORT, PATH_DOMINANCE, PATH_BYTE = 0, 1, 2, 3, 4, 5, 6
MAX_D = 30
VDKS_MAX_D = 10
RDKS_MAX_D = 4096

_lib = None
_lock = threading.Lock()


class DdksError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = f"ddks error {code}: {ddks_strerror(code)}"
        if what:
            msg += f" ({what})"
        super().__init__(msg)
        self.code = code


class ddks_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("path", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_int32),
                ("wait_limit_ms", ctypes.c_int32), ("tune_cache", ctypes.c_char_p),
                ("graphs", ctypes.c_int32), ("radix_min_n", ctypes.c_int64),
                ("register_variant", ctypes.c_int32), ("rank_kernel", ctypes.c_int32)]


class ddks_result(ctypes.Structure):
    _fields_ = [("num_max", ctypes.c_uint64), ("denom", ctypes.c_uint64), ("D", ctypes.c_double),
                ("argmax_origin", ctypes.c_int64), ("argmax_orthant", ctypes.c_int32),
                ("status", ctypes.c_int32)]

    def as_dict(self):
        return dict(num_max=int(self.num_max), denom=int(self.denom), D=float(self.D),
                    argmax_origin=int(self.argmax_origin), argmax_orthant=int(self.argmax_orthant),
                    status=int(self.status))


class ddks_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("submitted", "admitted", "completed", "rejected", "batches", "bytes_resident",
                 "bytes_resident_peak", "kernel_launches", "graph_captures", "graph_replays")]


def load():
    """Load libddks.so (built by paper_2106_13706_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"the CUDA library {LIB_PATH} is not built; run "
                               "paper_2106_13706_gb300.build.build() (there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        R = ctypes.POINTER(ddks_result)
        sig = {
            "ddks_config_default": (None, [ctypes.POINTER(ddks_config)]),
            "ddks_ctx_create": (i32, [ctypes.POINTER(ddks_config), ctypes.POINTER(vp)]),
            "ddks_ctx_destroy": (i32, [vp]),
            "ddks_distance": (i32, [vp, vp, i64, vp, i64, i32, i32, vp, R]),
            "ddks_distance_range": (i32, [vp, vp, i64, vp, i64, i32, i32, i64, i64, vp, vp, R]),
            "ddks_permutation_test": (i32, [vp, vp, i64, vp, i64, i32, i32, i32, u64, vp, R, vp,
                                            ctypes.POINTER(ctypes.c_double)]),
            "ddks_permutation_test_range": (i32, [vp, vp, i64, vp, i64, i32, i32, i64, i64, u64, vp, R, vp,
                                                  ctypes.POINTER(u64)]),
            "ddks_significance": (i32, [vp, vp, i64, vp, i64, i32, i32, u64, i32, i32, vp,
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
            "ddks_batch_distance": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp, R]),
            "ddks_autotune_batch": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp, vp]),
            "ddks_set_batch_shape": (i32, [vp, i32, i32, i32]),
            "ddks_submit": (i32, [vp, vp, i64, vp, i64, i32, i32, ctypes.POINTER(u64)]),
            "ddks_poll": (i32, [vp, u64, i32, R]),
            "ddks_ctx_stats": (i32, [vp, ctypes.POINTER(ddks_stats)]),
            "ddks_strerror": (ctypes.c_char_p, [i32]),
            "ddks_last_cuda_error": (ctypes.c_char_p, [vp]),
            "ddks_version": (ctypes.c_char_p, []),
            "ddks_classify_pointer": (i32, [i32, i32, i32]),
            "ddks_set_device_wait_limit": (i32, [vp, u64]),
            "ddks_wait_selftest": (i32, [vp, vp, ctypes.POINTER(u64)]),
            "ddks_distance_noalloc": (i32, [vp, i64, vp, i64, i32, i32, vp, R]),
            "ddks_vdks": (i32, [vp, vp, i64, vp, i64, i32, i32, i32, vp, R]),
            "ddks_rdks": (i32, [vp, vp, i64, vp, i64, i32, i32, vp, R, vp]),
            "ddks_rescale": (i32, [vp, vp, i64, ctypes.c_double, ctypes.c_double, vp, vp]),
            "ddks_autotune": (i32, [vp, vp, i64, vp, i64, i32, i32, vp, ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_float)]),
            "ddks_set_stage_timing": (i32, [vp, i32]),
            "ddks_stage_times": (i32, [vp, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def declared_symbols():
    """Names of the functions include/ddks.h declares (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(_PKG), "include", "ddks.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ddks_\w+)\s*\(", text, re.M)))


def ddks_strerror(code: int) -> str:
    try:
        return load().ddks_strerror(code).decode()
    except RuntimeError:
        return str(code)


# ------------------------------------------------------------------ marshalling
def _arr(x):
    """(pointer, rows, cols, dtype code, keepalive) of a 2-D float array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dim() == 1:
                x = x.unsqueeze(1)
            if x.dim() != 2 or not x.is_contiguous():
                raise ValueError("expected a contiguous 2-D tensor")
            if x.dtype == torch.float32:
                dt = DDKS_F32
            elif x.dtype == torch.float64:
                dt = DDKS_F64
            else:
                raise ValueError("expected float32 or float64")
            return x.data_ptr(), x.shape[0], x.shape[1], dt, x
    except ImportError:
        pass
    a = np.asarray(x)
    if a.ndim == 1:
        a = a[:, None]
    if a.dtype not in (np.float32, np.float64):
        raise ValueError("expected float32 or float64")
    a = np.ascontiguousarray(a)
    return a.ctypes.data, a.shape[0], a.shape[1], DDKS_F64 if a.dtype == np.float64 else DDKS_F32, a


def _stream(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _check(rc, ctx=None, what=""):
    if rc < 0:
        if rc == -5 and ctx is not None:
            what = (what + " " + load().ddks_last_cuda_error(ctx).decode()).strip()
        raise DdksError(rc, what)
    return rc


def _pair(P, T):
    p, np_, dp, tp, kp = _arr(P)
    t, nt, dt, tt, kt = _arr(T)
    if dp != dt:
        raise ValueError("P and T must have the same dimension")
    if tp != tt:
        raise ValueError("P and T must have the same dtype")
    return p, np_, t, nt, dp, tp, (kp, kt)


# ------------------------------------------------------------------ entry points
def ddks_ctx_create(device=-1, path=PATH_AUTO, hbm_budget_bytes=0, max_batch=0, wait_limit_ms=0,
                    tune_cache=None, graphs=True, radix_min_n=0, register_variant=0, rank_kernel=0):
    lib = load()
    cfg = ddks_config()
    lib.ddks_config_default(ctypes.byref(cfg))
    cfg.device, cfg.path = device, path
    cfg.hbm_budget_bytes, cfg.max_batch, cfg.wait_limit_ms = hbm_budget_bytes, max_batch, wait_limit_ms
    cfg.tune_cache = tune_cache.encode() if tune_cache else None
    cfg.graphs = 1 if graphs else 0
    cfg.radix_min_n = radix_min_n
    cfg.register_variant = register_variant
    cfg.rank_kernel = rank_kernel
    h = ctypes.c_void_p()
    _check(lib.ddks_ctx_create(ctypes.byref(cfg), ctypes.byref(h)), what="ddks_ctx_create")
    return h


def ddks_ctx_destroy(ctx):
    _check(load().ddks_ctx_destroy(ctx))


def ddks_distance(ctx, P, T, stream=None):
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    _check(load().ddks_distance(ctx, p, NP, t, NT, d, dt, _stream(stream), ctypes.byref(r)), ctx)
    return r.as_dict()


def ddks_distance_noalloc(P, T, stream=None):
    """Exact distance without any device allocation (device inputs, N <= 16384, d <= 8)."""
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    _check(load().ddks_distance_noalloc(p, NP, t, NT, d, dt, _stream(stream), ctypes.byref(r)))
    return r.as_dict()


def ddks_distance_range(ctx, P, T, o_begin, o_end, per_origin=False, stream=None):
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    po = np.zeros(max(o_end - o_begin, 1), dtype=np.uint64) if per_origin else None
    _check(load().ddks_distance_range(ctx, p, NP, t, NT, d, dt, o_begin, o_end,
                                      po.ctypes.data if po is not None else None,
                                      _stream(stream), ctypes.byref(r)), ctx)
    out = r.as_dict()
    if per_origin:
        out["per_origin"] = po[: o_end - o_begin]
    return out


def ddks_vdks(ctx, P, T, voxels_per_dim, stream=None):
    """Voxel approximation (Alg. vdKS): dict with num_max, denom, D, the
    arg-max voxel (argmax_origin) and orthant."""
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    _check(load().ddks_vdks(ctx, p, NP, t, NT, d, dt, int(voxels_per_dim), _stream(stream),
                            ctypes.byref(r)), ctx)
    return r.as_dict()


def ddks_rdks(ctx, P, T, stream=None):
    """Radial approximation (Alg. rdKS): dict with num_max, denom, D, the
    arg-max corner (argmax_origin) and per_corner numerators (d + 1)."""
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    pc = np.zeros(d + 1, dtype=np.uint64)
    _check(load().ddks_rdks(ctx, p, NP, t, NT, d, dt, _stream(stream), ctypes.byref(r),
                            pc.ctypes.data), ctx)
    out = r.as_dict()
    out["per_corner"] = pc
    return out


def ddks_rescale(ctx, v, lo, span, stream=None):
    """NormalizeData of one dimension, (v - lo) / span in IEEE double, on the
    device: v a float64 torch tensor (device; the result is a new device
    tensor) or array-like (host; the result is a numpy array)."""
    p, n, cols, dt, keep = _arr(v)
    if dt != DDKS_F64 or cols != 1:
        raise ValueError("expected a 1-D float64 array")
    try:
        import torch
        if isinstance(keep, torch.Tensor):
            out = torch.empty(n, dtype=torch.float64, device=keep.device)
            _check(load().ddks_rescale(ctx, p, n, float(lo), float(span), out.data_ptr(), _stream(stream)), ctx)
            return out
    except ImportError:
        pass
    out = np.empty(n, dtype=np.float64)
    _check(load().ddks_rescale(ctx, p, n, float(lo), float(span), out.ctypes.data, _stream(stream)), ctx)
    return out


def ddks_permutation_test(ctx, P, T, B, seed, stream=None, want_perm=True):
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    pm = np.zeros(max(B, 1), dtype=np.uint64) if want_perm else None
    pv = ctypes.c_double(0)
    _check(load().ddks_permutation_test(ctx, p, NP, t, NT, d, dt, B, seed, _stream(stream),
                                        ctypes.byref(r), pm.ctypes.data if pm is not None else None,
                                        ctypes.byref(pv)), ctx)
    out = dict(observed=r.as_dict(), p_value=float(pv.value))
    if want_perm:
        out["perm_num_max"] = pm[:B]
    return out


def ddks_permutation_test_range(ctx, P, T, b_begin, b_end, seed, stream=None, want_perm=True):
    """Relabellings [b_begin, b_end) of one permutation test: observed result,
    their numerators and the count with num_b >= num_obs (merge: sum the counts)."""
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    r = ddks_result()
    n = int(b_end) - int(b_begin)
    pm = np.zeros(max(n, 1), dtype=np.uint64) if want_perm else None
    ge = ctypes.c_uint64(0)
    _check(load().ddks_permutation_test_range(ctx, p, NP, t, NT, d, dt, int(b_begin), int(b_end), seed,
                                              _stream(stream), ctypes.byref(r),
                                              pm.ctypes.data if pm is not None else None, ctypes.byref(ge)), ctx)
    out = dict(observed=r.as_dict(), count_ge=int(ge.value))
    if want_perm:
        out["perm_num_max"] = pm[:n]
    return out


def ddks_significance(ctx, P, T, num_max, estimator=1, model=0, stream=None):
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    S = ctypes.c_double(0)
    lp = ctypes.c_double(0)
    _check(load().ddks_significance(ctx, p, NP, t, NT, d, dt, int(num_max), estimator, model,
                                    _stream(stream), ctypes.byref(S), ctypes.byref(lp)), ctx)
    return float(S.value), float(lp.value)


def _batch_arrays(problems):
    n = len(problems)
    ps = (ctypes.c_void_p * n)()
    ts = (ctypes.c_void_p * n)()
    nps = (ctypes.c_int64 * n)()
    nts = (ctypes.c_int64 * n)()
    ds = (ctypes.c_int32 * n)()
    keep = []
    dtype = None
    for i, (P, T) in enumerate(problems):
        p, NP, t, NT, d, dt, k = _pair(P, T)
        if dtype is None:
            dtype = dt
        elif dtype != dt:
            raise ValueError("all problems of a batch must share one dtype")
        ps[i], ts[i], nps[i], nts[i], ds[i] = p, t, NP, NT, d
        keep.append(k)
    return n, ps, nps, ts, nts, ds, dtype or 0, keep


def ddks_autotune_batch(ctx, problems, stream=None):
    """Tile shape per dimension ({d: (origins per unit, points per tile)}) chosen for this batch."""
    n, ps, nps, ts, nts, ds, dtype, keep = _batch_arrays(problems)
    shapes = (ctypes.c_int32 * 24)()
    _check(load().ddks_autotune_batch(ctx, n, ps, nps, ts, nts, ds, dtype, _stream(stream), shapes), ctx)
    return {k: (int(shapes[2 * k]), int(shapes[2 * k + 1])) for k in range(1, 12)}


def ddks_set_batch_shape(ctx, d, origins_per_unit, points_per_tile):
    _check(load().ddks_set_batch_shape(ctx, int(d), int(origins_per_unit), int(points_per_tile)), ctx)


def ddks_batch_distance(ctx, problems, stream=None):
    n = len(problems)
    ps = (ctypes.c_void_p * n)()
    ts = (ctypes.c_void_p * n)()
    nps = (ctypes.c_int64 * n)()
    nts = (ctypes.c_int64 * n)()
    ds = (ctypes.c_int32 * n)()
    keep = []
    dtype = None
    for i, (P, T) in enumerate(problems):
        p, NP, t, NT, d, dt, k = _pair(P, T)
        if dtype is None:
            dtype = dt
        elif dtype != dt:
            raise ValueError("all problems of a batch must share one dtype")
        ps[i], ts[i], nps[i], nts[i], ds[i] = p, t, NP, NT, d
        keep.append(k)
    res = (ddks_result * max(n, 1))()
    _check(load().ddks_batch_distance(ctx, n, ps, nps, ts, nts, ds, dtype or 0, _stream(stream),
                                      res), ctx)
    return [res[i].as_dict() for i in range(n)]


def ddks_submit(ctx, P, T):
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    tk = ctypes.c_uint64(0)
    _check(load().ddks_submit(ctx, p, NP, t, NT, d, dt, ctypes.byref(tk)), ctx)
    return int(tk.value)


def ddks_poll(ctx, ticket, timeout_us=0):
    """Returns (DDKS_OK, result dict) or (DDKS_PENDING, None); raises on errors."""
    r = ddks_result()
    rc = _check(load().ddks_poll(ctx, ticket, int(timeout_us), ctypes.byref(r)), ctx)
    return (rc, r.as_dict() if rc == DDKS_OK else None)


def ddks_ctx_stats(ctx):
    s = ddks_stats()
    _check(load().ddks_ctx_stats(ctx, ctypes.byref(s)))
    return {n: int(getattr(s, n)) for n, _ in ddks_stats._fields_}


def ddks_autotune(ctx, P, T, stream=None):
    """Time every kernel configuration on these inputs; returns (path, ms)."""
    p, NP, t, NT, d, dt, keep = _pair(P, T)
    path = ctypes.c_int32(0)
    ms = ctypes.c_float(0)
    _check(load().ddks_autotune(ctx, p, NP, t, NT, d, dt, _stream(stream), ctypes.byref(path),
                                ctypes.byref(ms)), ctx)
    return int(path.value), float(ms.value)


def ddks_set_stage_timing(ctx, enable=True):
    _check(load().ddks_set_stage_timing(ctx, 1 if enable else 0), ctx)


def ddks_stage_times(ctx):
    """(encode_ms, count_ms, reduce_ms) of the last distance call with stage timing on."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(load().ddks_stage_times(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return float(a.value), float(b.value), float(c.value)


def ddks_version():
    return load().ddks_version().decode()


def ddks_set_device_wait_limit(ctx, limit_ns):
    """Bound (ns) on each device-side wait for an asynchronous copy; 0 = the default."""
    _check(load().ddks_set_device_wait_limit(ctx, int(limit_ns)), ctx, "ddks_set_device_wait_limit")


def ddks_wait_selftest(ctx, stream=None):
    """(return code, waited ns) of one wait on a phase that never completes."""
    w = ctypes.c_uint64()
    rc = load().ddks_wait_selftest(ctx, _stream(stream), ctypes.byref(w))
    if rc != -6:  # DDKS_ETIMEOUT is the expected outcome
        _check(rc, ctx, "ddks_wait_selftest")
    return rc, int(w.value)


class Context:
    """Owns a ddks_ctx; `with Context() as c: c.distance(P, T)`."""

    def __init__(self, **cfg):
        self.h = ddks_ctx_create(**cfg)

    def close(self):
        if self.h is not None:
            ddks_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def distance(self, P, T, stream=None):
        return ddks_distance(self.h, P, T, stream)

    def distance_range(self, P, T, o_begin, o_end, per_origin=False, stream=None):
        return ddks_distance_range(self.h, P, T, o_begin, o_end, per_origin, stream)

    def vdks(self, P, T, voxels_per_dim, stream=None):
        return ddks_vdks(self.h, P, T, voxels_per_dim, stream)

    def rescale(self, v, lo, span, stream=None):
        return ddks_rescale(self.h, v, lo, span, stream)

    def rdks(self, P, T, stream=None):
        return ddks_rdks(self.h, P, T, stream)

    def permutation_test(self, P, T, B, seed, stream=None, want_perm=True):
        return ddks_permutation_test(self.h, P, T, B, seed, stream, want_perm)

    def permutation_test_range(self, P, T, b_begin, b_end, seed, stream=None, want_perm=True):
        return ddks_permutation_test_range(self.h, P, T, b_begin, b_end, seed, stream, want_perm)

    def significance(self, P, T, num_max, estimator=1, model=0, stream=None):
        return ddks_significance(self.h, P, T, num_max, estimator, model, stream)

    def batch_distance(self, problems, stream=None):
        return ddks_batch_distance(self.h, problems, stream)

    def autotune_batch(self, problems, stream=None):
        return ddks_autotune_batch(self.h, problems, stream)

    def set_batch_shape(self, d, origins_per_unit, points_per_tile):
        ddks_set_batch_shape(self.h, d, origins_per_unit, points_per_tile)

    def submit(self, P, T):
        return ddks_submit(self.h, P, T)

    def poll(self, ticket, timeout_us=0):
        return ddks_poll(self.h, ticket, timeout_us)

    def stats(self):
        return ddks_ctx_stats(self.h)

    def autotune(self, P, T, stream=None):
        return ddks_autotune(self.h, P, T, stream)

    def set_stage_timing(self, enable=True):
        ddks_set_stage_timing(self.h, enable)

    def stage_times(self):
        return ddks_stage_times(self.h)

    def set_device_wait_limit(self, limit_ns):
        ddks_set_device_wait_limit(self.h, limit_ns)

    def wait_selftest(self, stream=None):
        return ddks_wait_selftest(self.h, stream)
