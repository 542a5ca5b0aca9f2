"""Thin ctypes binding of ``include/lcs_bound.h`` (argument marshalling only).

Every function keeps the C name and raises :class:`LcsError` when the C call
returns a status other than ``LCS_OK``.  Vectors may be numpy arrays (host
memory) or torch tensors (host or CUDA memory); nothing here computes on
them.  The library is loaded from the package's ``_build`` directory and
built there with nvcc when missing; if that is impossible the import fails
loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LCS_OK, LCS_EINVAL, LCS_ENOMEM, LCS_ECUDA, LCS_ETIMEOUT, LCS_ENOBOUND, LCS_EOVERFLOW, LCS_EUNSUPPORTED, LCS_EIO = range(9)

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lcs_bound_opts(ctypes.Structure):
    _fields_ = [
        ("check_every", ctypes.c_int),
        ("r_mode", ctypes.c_int),
        ("f_mode", ctypes.c_int),
        ("frac_bits", ctypes.c_int),
        ("keep_u", ctypes.c_int),
        ("symmetry", ctypes.c_int),
        ("timing", ctypes.c_int),
        ("alloc", _ALLOC),
        ("free", _FREE),
        ("alloc_ctx", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("storage", ctypes.c_int),
        ("host_slots", ctypes.c_int),
    ]


class lcs_bound_report(ctypes.Structure):
    _fields_ = [
        ("iters_done", ctypes.c_int64),
        ("R", ctypes.c_int64),
        ("argmin", ctypes.c_uint64),
        ("E", ctypes.c_int64),
        ("r", ctypes.c_int64),
        ("eps", ctypes.c_int64),
        ("kept_iter", ctypes.c_int64),
        ("have_check", ctypes.c_int64),
        ("frac_bits", ctypes.c_int),
        ("status", ctypes.c_int),
    ]


class lcs_bound_stats_t(ctypes.Structure):
    _fields_ = [
        ("sweep_launches", ctypes.c_int64),
        ("sweep_ms", ctypes.c_double),
        ("check_launches", ctypes.c_int64),
        ("check_ms", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("sweep_bytes", ctypes.c_uint64),
        ("check_bytes", ctypes.c_uint64),
        ("h2d_ms", ctypes.c_double),
        ("h2d_bytes", ctypes.c_uint64),
        ("d2h_ms", ctypes.c_double),
        ("d2h_bytes", ctypes.c_uint64),
        ("xfer_kernel_ms", ctypes.c_double),
    ]


class lcs_bound_check_record(ctypes.Structure):
    _fields_ = [
        ("iter", ctypes.c_int64),
        ("R", ctypes.c_int64),
        ("argmin", ctypes.c_uint64),
        ("E", ctypes.c_int64),
        ("kept", ctypes.c_int64),
        ("r", ctypes.c_int64),
        ("eps", ctypes.c_int64),
        ("kept_iter", ctypes.c_int64),
    ]


class lcs_bound_batch_info_t(ctypes.Structure):
    _fields_ = [
        ("n_instances", ctypes.c_int),
        ("grid", ctypes.c_int),
        ("units_per_item", ctypes.c_int),
        ("graph", ctypes.c_int),
        ("tuned_ms_per_iter", ctypes.c_double),
        ("launches", ctypes.c_int64),
        ("mode", ctypes.c_int),
        ("persistent_ms_per_iter", ctypes.c_double),
        ("concurrent_ms_per_iter", ctypes.c_double),
        ("graph_captured", ctypes.c_int),
        ("min_ctas_per_sm", ctypes.c_int),
        ("graph_replays", ctypes.c_int64),
    ]


class LcsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded CUDA library (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_build.build())
            vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            P = ctypes.POINTER
            sig = {
                "lcs_bound_default_opts": [P(lcs_bound_opts)],
                "lcs_bound_create": [i32, i32, i32, P(lcs_bound_opts), P(vp)],
                "lcs_bound_size": [vp, P(u64), P(u64)],
                "lcs_bound_shape": [vp, P(i32), P(i32), P(i32)],
                "lcs_bound_iterate": [vp, i64],
                "lcs_bound_read": [vp, P(dbl), P(u64), P(dbl), P(dbl), P(i64)],
                "lcs_bound_read_report": [vp, P(lcs_bound_report)],
                "lcs_bound_set_start": [vp, vp, i32],
                "lcs_bound_set_start_fx": [vp, vp, i32],
                "lcs_bound_set_start_stored_fx": [vp, vp, i32],
                "lcs_bound_set_start_lift_fx": [vp, i32, vp, i32, i64],
                "lcs_bound_export_stored_fx": [vp, i32, vp, i32],
                "lcs_bound_orbit_size": [vp, P(u64)],
                "lcs_bound_set_start_orbit_fx": [vp, vp, i32],
                "lcs_bound_export_orbit_fx": [vp, i32, vp, i32],
                "lcs_bound_save": [vp, ctypes.c_char_p],
                "lcs_bound_history": [vp, vp, i64, vp],
                "lcs_bound_restore": [vp, ctypes.c_char_p],
                "lcs_bound_export": [vp, i32, vp, i32],
                "lcs_bound_export_fx": [vp, i32, vp, i32],
                "lcs_bound_check_vector": [vp, vp, i64, P(i64)],
                "lcs_bound_stats": [vp, P(lcs_bound_stats_t), i32],
                "lcs_bound_synchronize": [vp],
                "lcs_bound_batch_create": [i32, vp, P(lcs_bound_opts), P(vp)],
                "lcs_bound_batch_read": [vp, i32, P(dbl), P(u64), P(dbl), P(dbl), P(i64)],
                "lcs_bound_batch_report": [vp, i32, P(lcs_bound_report)],
                "lcs_bound_batch_export_fx": [vp, i32, i32, vp, i32],
                "lcs_bound_batch_info": [vp, P(lcs_bound_batch_info_t)],
                "lcs_bound_batch_set_mode": [vp, i32],
                "lcs_bound_batch_set_spin_budget": [vp, i64],
                "lcs_mlp_create": [u64, P(vp)],
                "lcs_mlp_create_with_allocator": [u64, _ALLOC, _FREE, vp, P(vp)],
                "lcs_mlp_get_params": [vp, vp],
                "lcs_mlp_set_params": [vp, vp],
                "lcs_mlp_gradient": [vp, i32, vp, vp, vp, P(ctypes.c_float), vp],
                "lcs_mlp_train": [vp, i32, vp, vp, i64, i32, ctypes.c_float, u64, i32, P(ctypes.c_float)],
                "lcs_mlp_predict": [vp, i32, i64, vp, vp],
                "lcs_mlp_start_vectors": [vp, i32, dbl, vp, vp],
                "lcs_mlp_start_vectors_stored_fx": [vp, i32, dbl, i32, vp, vp],
                "lcs_mlp_predict_bf16": [vp, i32, u64, i64, vp],
                "lcs_lift_prefix": [i32, i32, vp, i32, dbl, vp, vp],
                "lcs_fp32_experiment": [i32, i32, i32, i64, dbl, vp, P(dbl)],
                "lcs_sweep_fx": [i32, i32, i32, i32, i32, vp, vp, vp],
                "lcs_host_alloc": [ctypes.c_size_t, P(vp)],
                "lcs_host_free": [vp],
                "lcs_sweep_incr_fx_noalloc": [i32, i32, i32, i32, i32, vp, vp, vp, vp, vp],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.lcs_mlp_param_count.argtypes = []
            L.lcs_mlp_param_count.restype = i64
            L.lcs_mlp_destroy.argtypes = [vp]
            L.lcs_mlp_destroy.restype = None
            L.lcs_bound_destroy.argtypes = [vp]
            L.lcs_bound_destroy.restype = None
            L.lcs_bound_errstr.argtypes = [ctypes.c_int]
            L.lcs_bound_errstr.restype = ctypes.c_char_p
            L.lcs_bound_last_error.argtypes = []
            L.lcs_bound_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def lcs_bound_errstr(status: int) -> str:
    return lib().lcs_bound_errstr(status).decode()


def lcs_bound_last_error() -> str:
    return lib().lcs_bound_last_error().decode()


def _check(status: int, what: str):
    if status != LCS_OK:
        raise LcsError(status, f"{what}: {lcs_bound_errstr(status)}: {lcs_bound_last_error()}")


# ---------------------------------------------------------------------------
# pointers of numpy arrays / torch tensors


def _ptr_and_kind(a, dtype):
    """(address, on_device) of a contiguous vector of the given numpy dtype."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float64 if dtype == np.float64 else torch.int64
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        if a.is_cuda:
            # the library reads and writes on its own stream: let the work
            # that produced (or still reads) this tensor on torch's stream end
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a contiguous numpy {np.dtype(dtype)} array")
    return a.ctypes.data, 0


def _numel(a) -> int:
    """number of values of a numpy array or torch tensor"""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        return int(a.numel())
    if isinstance(a, np.ndarray):
        return int(a.size)
    raise TypeError("expected a numpy array or a torch tensor")


def _require_vectors(vs, count: int, n: int, what: str):
    """The C side reads `count` pointers and n values behind each: check both before the call."""
    if len(vs) != count:
        raise ValueError(f"{what}: {len(vs)} vectors given, {count} expected")
    for k, v in enumerate(vs):
        m = _numel(v)
        if m != n:
            raise ValueError(f"{what}: vector {k} holds {m} values, {n} expected")


def _require_len(a, n: int, what: str, at_least: bool = False):
    m = _numel(a)
    if (m < n) if at_least else (m != n):
        raise ValueError(f"{what} holds {m} values, {'at least ' if at_least else ''}{n} expected")


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device=None):
        import torch

        self._torch = torch
        self._device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._live = {}
        self.alloc = _ALLOC(self._alloc)
        self.free = _FREE(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes) + 256, dtype=self._torch.uint8, device=self._device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        p = (p + 255) // 256 * 256
        self._live[p] = t
        return p

    def _free(self, ptr, ctx):
        self._live.pop(ptr, None)


# ---------------------------------------------------------------------------
# C functions, same names


def lcs_bound_default_opts() -> lcs_bound_opts:
    o = lcs_bound_opts()
    _check(lib().lcs_bound_default_opts(ctypes.byref(o)), "lcs_bound_default_opts")
    return o


def lcs_bound_create(sigma: int, d: int, h: int, opts: lcs_bound_opts | None = None) -> ctypes.c_void_p:
    hnd = ctypes.c_void_p()
    _check(lib().lcs_bound_create(sigma, d, h, ctypes.byref(opts) if opts is not None else None, ctypes.byref(hnd)),
           "lcs_bound_create")
    return hnd


def lcs_bound_size(hnd):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().lcs_bound_size(hnd, ctypes.byref(a), ctypes.byref(b)), "lcs_bound_size")
    return a.value, b.value


def lcs_bound_shape(hnd):
    """(sigma, d, h) of a single-instance handle."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().lcs_bound_shape(hnd, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "lcs_bound_shape")
    return a.value, b.value, c.value


def _vectors_for(hnd, form: str):
    """(d, values per vector) of the handle for a form: 'full', 'stored' or 'orbit'"""
    _, d, _ = lcs_bound_shape(hnd)
    if form == "orbit":
        return d, lcs_bound_orbit_size(hnd)
    n, n_stored = lcs_bound_size(hnd)
    return d, n if form == "full" else n_stored


def lcs_bound_iterate(hnd, n_iters: int):
    _check(lib().lcs_bound_iterate(hnd, int(n_iters)), "lcs_bound_iterate")


def lcs_bound_read(hnd):
    """(bound_rd, argmin_state, r, eps, at_iter)."""
    b, a, r, e, it = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().lcs_bound_read(hnd, ctypes.byref(b), ctypes.byref(a), ctypes.byref(r), ctypes.byref(e),
                                ctypes.byref(it)), "lcs_bound_read")
    return b.value, a.value, r.value, e.value, it.value


def lcs_bound_read_report(hnd) -> dict:
    rep = lcs_bound_report()
    _check(lib().lcs_bound_read_report(hnd, ctypes.byref(rep)), "lcs_bound_read_report")
    return {f: getattr(rep, f) for f, _ in lcs_bound_report._fields_}


def _vec_array(vs, dtype):
    ptrs, kinds = zip(*[_ptr_and_kind(v, dtype) for v in vs])
    if len(set(kinds)) != 1:
        raise TypeError("start vectors must all be on the host or all on the device")
    return (ctypes.c_void_p * len(ptrs))(*ptrs), kinds[0]


def lcs_bound_set_start(hnd, vs):
    """vs[k]: the iterate k steps older than the newest (float64, every state)."""
    _require_vectors(vs, *_vectors_for(hnd, "full"), "lcs_bound_set_start")
    arr, on_dev = _vec_array(vs, np.float64)
    _check(lib().lcs_bound_set_start(hnd, arr, on_dev), "lcs_bound_set_start")


def lcs_bound_set_start_fx(hnd, vs):
    _require_vectors(vs, *_vectors_for(hnd, "full"), "lcs_bound_set_start_fx")
    arr, on_dev = _vec_array(vs, np.int64)
    _check(lib().lcs_bound_set_start_fx(hnd, arr, on_dev), "lcs_bound_set_start_fx")


def lcs_bound_set_start_stored_fx(hnd, vs):
    """vs[k]: the stored form (lcs_bound_size's n_stored values) of the iterate k steps older than the newest."""
    _require_vectors(vs, *_vectors_for(hnd, "stored"), "lcs_bound_set_start_stored_fx")
    arr, on_dev = _vec_array(vs, np.int64)
    _check(lib().lcs_bound_set_start_stored_fx(hnd, arr, on_dev), "lcs_bound_set_start_stored_fx")


def lcs_bound_set_start_lift_fx(hnd, h_from: int, src, r_hat: int):
    """Start from the stored form of a shorter shape's iterate (sigma = d = 2): v[x] = src[x >> 2 (h - h_from)]."""
    _require_len(src, 4 ** h_from // 2, "lcs_bound_set_start_lift_fx: src")
    p, on_dev = _ptr_and_kind(src, np.int64)
    _check(lib().lcs_bound_set_start_lift_fx(hnd, h_from, p, on_dev, int(r_hat)), "lcs_bound_set_start_lift_fx")


def lcs_bound_export_stored_fx(hnd, k: int, out):
    _require_len(out, _vectors_for(hnd, "stored")[1], "lcs_bound_export_stored_fx: out")
    p, on_dev = _ptr_and_kind(out, np.int64)
    _check(lib().lcs_bound_export_stored_fx(hnd, k, p, on_dev), "lcs_bound_export_stored_fx")
    if on_dev:
        lcs_bound_synchronize(hnd)
    return out


def lcs_bound_orbit_size(hnd) -> int:
    """values of the orbit form (sigma = d = 2 with the complement and the swap)."""
    n = ctypes.c_uint64()
    _check(lib().lcs_bound_orbit_size(hnd, ctypes.byref(n)), "lcs_bound_orbit_size")
    return int(n.value)


def lcs_bound_set_start_orbit_fx(hnd, vs):
    """vs[k]: the orbit form (lcs_bound_orbit_size values) of the iterate k steps older than the newest."""
    _require_vectors(vs, *_vectors_for(hnd, "orbit"), "lcs_bound_set_start_orbit_fx")
    arr, on_dev = _vec_array(vs, np.int64)
    _check(lib().lcs_bound_set_start_orbit_fx(hnd, arr, on_dev), "lcs_bound_set_start_orbit_fx")


def lcs_bound_export_orbit_fx(hnd, k: int, out):
    _require_len(out, _vectors_for(hnd, "orbit")[1], "lcs_bound_export_orbit_fx: out")
    p, on_dev = _ptr_and_kind(out, np.int64)
    _check(lib().lcs_bound_export_orbit_fx(hnd, k, p, on_dev), "lcs_bound_export_orbit_fx")
    if on_dev:
        lcs_bound_synchronize(hnd)
    return out


def lcs_bound_history(hnd, max_records=4096):
    """(records, n_checks): the newest check records, oldest first, as dicts."""
    buf = (lcs_bound_check_record * max(1, max_records))()
    n = ctypes.c_int64()
    _check(lib().lcs_bound_history(hnd, buf, max_records, ctypes.byref(n)), "lcs_bound_history")
    got = min(n.value, 4096, max_records)
    return [{f: getattr(buf[i], f) for f, _ in lcs_bound_check_record._fields_} for i in range(got)], n.value


def lcs_bound_save(hnd, path):
    _check(lib().lcs_bound_save(hnd, os.fsencode(path)), "lcs_bound_save")


def lcs_bound_restore(hnd, path):
    _check(lib().lcs_bound_restore(hnd, os.fsencode(path)), "lcs_bound_restore")


def lcs_bound_synchronize(hnd):
    _check(lib().lcs_bound_synchronize(hnd), "lcs_bound_synchronize")


def lcs_bound_export(hnd, k: int, out):
    _require_len(out, _vectors_for(hnd, "full")[1], "lcs_bound_export: out")
    p, on_dev = _ptr_and_kind(out, np.float64)
    _check(lib().lcs_bound_export(hnd, k, p, on_dev), "lcs_bound_export")
    if on_dev:
        lcs_bound_synchronize(hnd)  # the tensor is complete when this returns
    return out


def lcs_bound_export_fx(hnd, k: int, out):
    _require_len(out, _vectors_for(hnd, "full")[1], "lcs_bound_export_fx: out")
    p, on_dev = _ptr_and_kind(out, np.int64)
    _check(lib().lcs_bound_export_fx(hnd, k, p, on_dev), "lcs_bound_export_fx")
    if on_dev:
        lcs_bound_synchronize(hnd)
    return out


def lcs_bound_check_vector(hnd, u_dev, R: int) -> int:
    _require_len(u_dev, _vectors_for(hnd, "stored")[1], "lcs_bound_check_vector: u", at_least=True)
    p, on_dev = _ptr_and_kind(u_dev, np.int64)
    if not on_dev:
        raise TypeError("u must be a CUDA tensor")
    E = ctypes.c_int64()
    _check(lib().lcs_bound_check_vector(hnd, p, int(R), ctypes.byref(E)), "lcs_bound_check_vector")
    return E.value


def lcs_bound_stats(hnd, reset: bool = False) -> dict:
    s = lcs_bound_stats_t()
    _check(lib().lcs_bound_stats(hnd, ctypes.byref(s), 1 if reset else 0), "lcs_bound_stats")
    return {f: getattr(s, f) for f, _ in lcs_bound_stats_t._fields_}


def lcs_bound_destroy(hnd):
    if hnd:
        lib().lcs_bound_destroy(hnd)


def _shape_states(sigma, d, h) -> int:
    """sigma^(d h), or 0 for a shape the library rejects itself (LCS_EINVAL)"""
    if sigma < 2 or d < 2 or h < 1 or d > 16 or sigma ** (d * h) >= 1 << 40:
        return 0
    return sigma ** (d * h)


def lcs_sweep_fx(sigma, d, h, v_prev, v_out, f_mode=0, frac_bits=44, stream=None):
    """v_out = F(v_prev[0], .., v_prev[d-1]) on the device (CUDA int64 tensors)."""
    n = _shape_states(sigma, d, h)
    if n:  # a bad shape is the library's LCS_EINVAL
        _require_vectors(v_prev, d, n, "lcs_sweep_fx: v_prev")
        _require_len(v_out, n, "lcs_sweep_fx: v_out")
    arr, on_dev = _vec_array(v_prev, np.int64)
    po, od = _ptr_and_kind(v_out, np.int64)
    if not (on_dev and od):
        raise TypeError("lcs_sweep_fx takes CUDA tensors")
    _check(lib().lcs_sweep_fx(sigma, d, h, f_mode, frac_bits, arr, po, stream), "lcs_sweep_fx")


def lcs_sweep_incr_fx_noalloc(sigma, d, h, v_prev, v_out, R_out, argmin_out, frac_bits=44, r_mode=0, stream=None):
    """One sweep fused with the increment reduction, allocating nothing (CUDA tensors only).

    For callers that cannot allocate device memory: the reduction's scratch is
    a fixed array inside the library.  R_out and argmin_out are one-element
    CUDA int64 tensors that receive R and its state index.
    """
    n = _shape_states(sigma, d, h)
    if n:  # a bad shape is the library's LCS_EINVAL
        _require_vectors(v_prev, d, n, "lcs_sweep_incr_fx_noalloc: v_prev")
        _require_len(v_out, n, "lcs_sweep_incr_fx_noalloc: v_out")
    _require_len(R_out, 1, "lcs_sweep_incr_fx_noalloc: R_out", at_least=True)
    _require_len(argmin_out, 1, "lcs_sweep_incr_fx_noalloc: argmin_out", at_least=True)
    arr, on_dev = _vec_array(v_prev, np.int64)
    po, od = _ptr_and_kind(v_out, np.int64)
    pr, rd = _ptr_and_kind(R_out, np.int64)
    pa, ad = _ptr_and_kind(argmin_out, np.int64)
    if not (on_dev and od and rd and ad):
        raise TypeError("lcs_sweep_incr_fx_noalloc takes CUDA tensors")
    _check(lib().lcs_sweep_incr_fx_noalloc(sigma, d, h, frac_bits, r_mode, arr, po, pr, pa, stream),
           "lcs_sweep_incr_fx_noalloc")


def lcs_bound_batch_create(shapes, opts: lcs_bound_opts | None = None):
    arr = (ctypes.c_int * (3 * len(shapes)))(*[int(v) for sh in shapes for v in sh])
    hnd = ctypes.c_void_p()
    _check(lib().lcs_bound_batch_create(len(shapes), arr, ctypes.byref(opts) if opts is not None else None,
                                        ctypes.byref(hnd)), "lcs_bound_batch_create")
    return hnd


def lcs_bound_batch_read(hnd, i: int):
    b, a, r, e, it = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().lcs_bound_batch_read(hnd, i, ctypes.byref(b), ctypes.byref(a), ctypes.byref(r), ctypes.byref(e),
                                      ctypes.byref(it)), "lcs_bound_batch_read")
    return b.value, a.value, r.value, e.value, it.value


def lcs_bound_batch_report(hnd, i: int) -> dict:
    rep = lcs_bound_report()
    _check(lib().lcs_bound_batch_report(hnd, i, ctypes.byref(rep)), "lcs_bound_batch_report")
    return {f: getattr(rep, f) for f, _ in lcs_bound_report._fields_}


def lcs_bound_batch_export_fx(hnd, i: int, k: int, out):
    p, on_dev = _ptr_and_kind(out, np.int64)
    _check(lib().lcs_bound_batch_export_fx(hnd, i, k, p, on_dev), "lcs_bound_batch_export_fx")
    if on_dev:
        lcs_bound_synchronize(hnd)
    return out


def lcs_bound_batch_set_mode(hnd, mode):
    _check(lib().lcs_bound_batch_set_mode(hnd, mode), "lcs_bound_batch_set_mode")


def lcs_bound_batch_info(hnd) -> dict:
    info = lcs_bound_batch_info_t()
    _check(lib().lcs_bound_batch_info(hnd, ctypes.byref(info)), "lcs_bound_batch_info")
    return {f: getattr(info, f) for f, _ in lcs_bound_batch_info_t._fields_}


def lcs_bound_batch_set_spin_budget(hnd, cycles: int):
    _check(lib().lcs_bound_batch_set_spin_budget(hnd, int(cycles)), "lcs_bound_batch_set_spin_budget")


class LcsBatch:
    """Owns one batch handle (lcs_bound_batch_create); instances are indexed 0..n-1."""

    def __init__(self, shapes, *, check_every=0, r_mode=0, frac_bits=44, symmetry=1, stream=None):
        self.shapes = [tuple(s) for s in shapes]
        o = lcs_bound_default_opts()
        o.check_every, o.r_mode, o.frac_bits, o.symmetry = check_every, r_mode, frac_bits, symmetry
        if stream is not None:
            if not stream:
                raise ValueError("stream 0 means 'library-owned stream'; pass a non-default stream handle")
            o.stream = stream
        self.hnd = lcs_bound_batch_create(self.shapes, o)

    def close(self):
        if self.hnd:
            lcs_bound_destroy(self.hnd)
            self.hnd = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, n):
        lcs_bound_iterate(self.hnd, n)

    def read(self, i):
        return lcs_bound_batch_read(self.hnd, i)

    def report(self, i):
        return lcs_bound_batch_report(self.hnd, i)

    def export_fx(self, i, k=0, out=None):
        s, d, h = self.shapes[i]
        if out is None:
            out = np.empty(s ** (d * h), dtype=np.int64)
        _require_len(out, s ** (d * h), "LcsBatch.export_fx: out")
        return lcs_bound_batch_export_fx(self.hnd, i, k, out)

    def info(self):
        return lcs_bound_batch_info(self.hnd)

    def set_spin_budget(self, cycles):
        lcs_bound_batch_set_spin_budget(self.hnd, cycles)

    def set_mode(self, mode):
        """0: the persistent launch, 1: concurrent single-instance kernels with repeated call
        schedules replayed from CUDA graphs, 2: the same kernels never captured (before the
        first iteration)."""
        lcs_bound_batch_set_mode(self.hnd, mode)


class HostBuffer:
    """n int64 values of host memory from lcs_host_alloc (pinned, mapped, huge-page advised) as a numpy array.

    Keep this object alive while the array is in use; close() (or the end of
    a with-block) frees the memory.
    """

    def __init__(self, n, dtype=np.int64):
        self.ptr = ctypes.c_void_p()
        nbytes = int(n) * np.dtype(dtype).itemsize
        _check(lib().lcs_host_alloc(nbytes, ctypes.byref(self.ptr)), "lcs_host_alloc")
        buf = (ctypes.c_char * nbytes).from_address(self.ptr.value)
        self.array = np.frombuffer(buf, dtype=dtype, count=int(n))

    def close(self):
        if self.ptr:
            self.array = None
            _check(lib().lcs_host_free(self.ptr), "lcs_host_free")
            self.ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lcs_fp32_experiment(sigma, d, h, n_iters, rho, newest_dev):
    """Float32-stored iteration from the zero start (an experiment, no bound); returns ms per sweep."""
    _require_len(newest_dev, sigma ** (d * h), "lcs_fp32_experiment: newest")
    p, on = _ptr_and_kind(newest_dev, np.float64)
    if not on:
        raise TypeError("lcs_fp32_experiment writes a CUDA tensor")
    ms = ctypes.c_double()
    _check(lib().lcs_fp32_experiment(sigma, d, h, n_iters, float(rho), p, ctypes.byref(ms)), "lcs_fp32_experiment")
    return ms.value


def lcs_lift_prefix(h_from, h_to, src_dev, r_hat, newest_dev, older_dev, frac_bits=44):
    """Prefix-truncation start: every tuple of length h_to takes the value of its first h_from letters."""
    _require_len(src_dev, 4 ** h_from, "lcs_lift_prefix: src")
    _require_len(newest_dev, 4 ** h_to, "lcs_lift_prefix: newest")
    _require_len(older_dev, 4 ** h_to, "lcs_lift_prefix: older")
    ps, a = _ptr_and_kind(src_dev, np.int64)
    pn, b = _ptr_and_kind(newest_dev, np.float64)
    po, c = _ptr_and_kind(older_dev, np.float64)
    if not (a and b and c):
        raise TypeError("lcs_lift_prefix takes CUDA tensors")
    _check(lib().lcs_lift_prefix(h_from, h_to, ps, frac_bits, float(r_hat), pn, po), "lcs_lift_prefix")


def lcs_mlp_param_count() -> int:
    return int(lib().lcs_mlp_param_count())


class LcsMlp:
    """The warm-start network (lcs_mlp_*); every computation runs in the library's kernels."""

    def __init__(self, seed=1, allocator=None):
        """allocator: an object with ctypes callbacks .alloc and .free (e.g. TorchAllocator), or None"""
        self.hnd = ctypes.c_void_p()
        self._allocator = allocator  # the callbacks must outlive the handle
        if allocator is None:
            _check(lib().lcs_mlp_create(seed, ctypes.byref(self.hnd)), "lcs_mlp_create")
        else:
            _check(lib().lcs_mlp_create_with_allocator(seed, allocator.alloc, allocator.free, None,
                                                       ctypes.byref(self.hnd)), "lcs_mlp_create_with_allocator")
        self.n_params = lcs_mlp_param_count()

    def close(self):
        if self.hnd:
            lib().lcs_mlp_destroy(self.hnd)
            self.hnd = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().lcs_mlp_get_params(self.hnd, out.ctypes.data), "lcs_mlp_get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib().lcs_mlp_set_params(self.hnd, flat.ctypes.data), "lcs_mlp_set_params")

    def gradient(self, states, hs, targets):
        states = np.ascontiguousarray(states, dtype=np.int64)
        hs = np.ascontiguousarray(hs, dtype=np.int32)
        targets = np.ascontiguousarray(targets, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().lcs_mlp_gradient(self.hnd, states.size, states.ctypes.data, hs.ctypes.data, targets.ctypes.data,
                                      ctypes.byref(loss), g.ctypes.data), "lcs_mlp_gradient")
        return loss.value, g

    def train(self, vectors, hs, steps, batch=4096, lr=1e-3, seed=7, frac_bits=44):
        arr, on_dev = _vec_array(vectors, np.int64)
        if not on_dev:
            raise TypeError("training vectors must be CUDA tensors")
        hs_arr = (ctypes.c_int * len(hs))(*hs)
        loss = ctypes.c_float()
        _check(lib().lcs_mlp_train(self.hnd, len(hs), arr, hs_arr, steps, batch, lr, seed, frac_bits,
                                   ctypes.byref(loss)), "lcs_mlp_train")
        return loss.value

    def predict(self, h, states_dev, out_dev):
        _require_len(out_dev, _numel(states_dev), "LcsMlp.predict: out", at_least=True)
        ps, sd = _ptr_and_kind(states_dev, np.int64)
        if not sd or not out_dev.is_cuda:
            raise TypeError("predict takes CUDA tensors")
        import torch

        torch.cuda.current_stream().synchronize()
        _check(lib().lcs_mlp_predict(self.hnd, h, states_dev.numel(), ps, out_dev.data_ptr()), "lcs_mlp_predict")
        return out_dev

    def predict_bf16(self, h, base, n, out_dev):
        if not out_dev.is_cuda:
            raise TypeError("predict_bf16 writes a CUDA tensor")
        _require_len(out_dev, n, "LcsMlp.predict_bf16: out", at_least=True)
        _check(lib().lcs_mlp_predict_bf16(self.hnd, h, base, n, out_dev.data_ptr()), "lcs_mlp_predict_bf16")
        return out_dev

    def start_vectors(self, h, r_hat, newest_dev, older_dev):
        _require_vectors([newest_dev, older_dev], 2, 4 ** h, "LcsMlp.start_vectors")
        pn, dn = _ptr_and_kind(newest_dev, np.float64)
        po, do = _ptr_and_kind(older_dev, np.float64)
        if not (dn and do):
            raise TypeError("start vectors must be CUDA tensors")
        _check(lib().lcs_mlp_start_vectors(self.hnd, h, float(r_hat), pn, po), "lcs_mlp_start_vectors")

    def start_vectors_stored_fx(self, h, r_hat, newest_dev, older_dev, frac_bits=44):
        """The start in a complement-symmetric handle's stored form, fixed point (int64 CUDA tensors of 4^h / 2)."""
        _require_vectors([newest_dev, older_dev], 2, 4 ** h // 2, "LcsMlp.start_vectors_stored_fx")
        pn, a = _ptr_and_kind(newest_dev, np.int64)
        po, b = _ptr_and_kind(older_dev, np.int64)
        if not (a and b):
            raise TypeError("start_vectors_stored_fx writes CUDA tensors")
        _check(lib().lcs_mlp_start_vectors_stored_fx(self.hnd, h, float(r_hat), frac_bits, pn, po),
               "lcs_mlp_start_vectors_stored_fx")


# ---------------------------------------------------------------------------
# convenience object


class LcsBound:
    """Owns one handle; see ``include/lcs_bound.h`` for the semantics."""

    def __init__(self, sigma, d, h, *, check_every=0, r_mode=0, f_mode=0, frac_bits=44, keep_u=0, symmetry=1,
                 timing=0, stream=None, torch_alloc=False, storage=0, host_slots=0):
        self.sigma, self.d, self.h = sigma, d, h
        o = lcs_bound_default_opts()
        o.check_every, o.r_mode, o.f_mode, o.frac_bits = check_every, r_mode, f_mode, frac_bits
        o.keep_u, o.symmetry, o.timing = keep_u, symmetry, timing
        o.storage, o.host_slots = storage, host_slots
        self._alloc = None
        if torch_alloc:
            self._alloc = TorchAllocator()
            o.alloc, o.free = self._alloc.alloc, self._alloc.free
        if stream is not None:
            if not stream:
                raise ValueError("stream 0 means 'library-owned stream'; pass a non-default stream handle")
            o.stream = stream
        self.opts = o
        self.frac_bits = frac_bits
        self.hnd = lcs_bound_create(sigma, d, h, o)
        self.n_states, self.n_stored = lcs_bound_size(self.hnd)

    def close(self):
        if self.hnd:
            lcs_bound_destroy(self.hnd)
            self.hnd = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, n):
        lcs_bound_iterate(self.hnd, n)

    def read(self):
        return lcs_bound_read(self.hnd)

    def report(self):
        return lcs_bound_read_report(self.hnd)

    def set_start(self, vs):
        lcs_bound_set_start(self.hnd, vs)

    def set_start_fx(self, vs):
        lcs_bound_set_start_fx(self.hnd, vs)

    def export(self, k=0, out=None):
        if out is None:
            out = np.empty(self.n_states, dtype=np.float64)
        return lcs_bound_export(self.hnd, k, out)

    def export_fx(self, k=0, out=None):
        if out is None:
            out = np.empty(self.n_states, dtype=np.int64)
        return lcs_bound_export_fx(self.hnd, k, out)

    def set_start_stored_fx(self, vs):
        lcs_bound_set_start_stored_fx(self.hnd, vs)

    def set_start_lift_fx(self, h_from, src, r_hat):
        lcs_bound_set_start_lift_fx(self.hnd, h_from, src, r_hat)

    def export_stored_fx(self, k=0, out=None):
        if out is None:
            out = np.empty(self.n_stored, dtype=np.int64)
        return lcs_bound_export_stored_fx(self.hnd, k, out)

    @property
    def n_orbit(self):
        return lcs_bound_orbit_size(self.hnd)

    def set_start_orbit_fx(self, vs):
        lcs_bound_set_start_orbit_fx(self.hnd, vs)

    def export_orbit_fx(self, k=0, out=None):
        if out is None:
            out = np.empty(self.n_orbit, dtype=np.int64)
        return lcs_bound_export_orbit_fx(self.hnd, k, out)

    def history(self, max_records=4096):
        return lcs_bound_history(self.hnd, max_records)

    def save(self, path):
        lcs_bound_save(self.hnd, path)

    def restore(self, path):
        lcs_bound_restore(self.hnd, path)

    def check_vector(self, u_dev, R):
        return lcs_bound_check_vector(self.hnd, u_dev, R)

    def stats(self, reset=False):
        return lcs_bound_stats(self.hnd, reset)
