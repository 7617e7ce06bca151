"""Direct search (Cannizzo, arXiv 1506.08620) as a GB300-native CUDA library.

Thin Python binding over the C ABI of ``include/ds.h`` (``libds.so``): the
functions below carry the C names and only marshal arguments (torch tensors
to device pointers, the current torch stream to a cudaStream_t).  Every step
of the lookup runs in the library's CUDA kernels; there is no CPU fallback,
and calls fail loudly when ``libds.so`` is not built.
"""
import ctypes

import torch

from . import _abi
from ._abi import (DS_CACHE_LAYOUT, DS_CHECKED, DS_F32, DS_F64, DS_FMA, DS_LEARNED_FORCE,  # noqa: F401
                   DS_GAP2, DS_LEARNED_LINEAR, DS_LS_CLASSIC, DS_LS_CLASSICMOD, DS_LS_EYTZINGER,
                   DS_LS_LEADBIT, DS_LS_LEADBIT_NOPAD, DS_LS_NAMES, DS_LS_OFFSET, DS_NO_FINGERPRINT, DS_NO_SMEM, DS_OK,
                   DS_REFINE_H, DS_STRICT, DS_E_NOMEM, DsError, check, lib)

__all__ = [
    "ds_build", "ds_search", "ds_search_host", "ds_index_export", "ds_batch_build", "ds_batch_search",
    "ds_batch_autotune", "ds_batch_set_tune", "ds_batch_get_tune", "ds_batch_array", "ds_learned_build",
    "ds_learned_search", "ds_learned_autotune", "ds_learned_set_tune", "ds_learned_get_tune", "ds_learned_array",
    "ds_learned_cfg_default", "ds_learned_build_xy", "ds_learned_cells", "ds_learned_export_cells",
    "ds_learned_search_host", "ds_mlp_forward", "ds_mlp_loss_grad",
    "ds_adam_step", "ds_info", "ds_free", "DsError", "ds_debug_fail_alloc", "ds_debug_alloc_stats",
]


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dtype(t):
    if t.dtype == torch.float32:
        return DS_F32
    if t.dtype == torch.float64:
        return DS_F64
    raise TypeError("knots and queries must be float32 or float64, got %s" % t.dtype)


def _dev(t, name, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _host(t, name, dtype=None):
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
        raise TypeError("%s must be a contiguous host tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (name, dtype))
    return ctypes.c_void_p(t.data_ptr())


class _Handle:
    kind = "handle"

    def __init__(self, ptr, dtype):
        self._ptr = ptr
        self.dtype = dtype

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("%s has been freed" % self.kind)
        return self._ptr

    def info(self):
        return ds_info(self)

    def free(self):
        if self._ptr:
            lib().ds_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Index(_Handle):
    """One knot array with its direct-search table (``ds_index``)."""
    kind = "ds_index"

    def search(self, Z, out=None, stream=None):
        return ds_search(self, Z, out, stream)


class Batch(_Handle):
    """Many independent knot arrays in CSR form (``ds_batch``)."""
    kind = "ds_batch"

    def search(self, Zcat, z_off, out=None, stream=None):
        return ds_batch_search(self, Zcat, z_off, out, stream)


class LSearch(_Handle):
    """One array laid out for a logarithmic search (``ds_lsearch``)."""
    kind = "ds_lsearch"

    def search(self, Z, out=None, stream=None):
        return ds_lsearch_search(self, Z, out, stream)


class Learned(_Handle):
    """Learned-index form (``ds_learned``); ``xy``: the handle holds its knot values."""
    kind = "ds_learned"
    xy = False

    def search(self, Z, z_off=None, Y=None, out=None, y_out=None, stream=None):
        return ds_learned_search(self, Z, z_off, Y, out, y_out, stream)


# ---------------------------------------------------------------- single array
def ds_build(X, flags=0, stream=None):
    """Build the direct-search table of knot array X (CUDA tensor); returns an Index."""
    out = ctypes.c_void_p()
    check(lib().ds_build(_dev(X, "X"), X.numel(), _dtype(X), int(flags), _stream(stream), ctypes.byref(out)),
          "ds_build")
    return Index(out.value, X.dtype)


def ds_build_q(X, q, budget_bytes=0, flags=0, q_max=64, stream=None):
    """Gap-q table of X (q >= 1), or with q = 0 the smallest q in 1..q_max whose table fits budget_bytes."""
    out = ctypes.c_void_p()
    check(lib().ds_build_q(_dev(X, "X"), X.numel(), _dtype(X), int(flags), int(q), int(q_max), int(budget_bytes),
                           _stream(stream), ctypes.byref(out)), "ds_build_q")
    return Index(out.value, X.dtype)


def ds_search(idx, Z, out=None, stream=None):
    """int32 interval index of every query in Z (CUDA tensor of the index's dtype)."""
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32, device=Z.device)
    check(lib().ds_search(idx.ptr, _dev(Z, "Z", idx.dtype), Z.numel(), _dev(out, "out", torch.int32),
                          _stream(stream)), "ds_search")
    return out


def ds_search_sorted(X, Z, out=None, stream=None):
    """Answers for non-decreasing queries Z by merging them into X (CUDA tensors, same dtype)."""
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32, device=Z.device)
    check(lib().ds_search_sorted(_dev(X, "X"), X.numel(), _dtype(X), _dev(Z, "Z", X.dtype), Z.numel(),
                                 _dev(out, "out", torch.int32), _stream(stream)), "ds_search_sorted")
    return out


def ds_histogram(idx, Z, counts=None, stream=None):
    """Counts (int64, N+2 bins: below X_0, each interval, at or above X_N) of the queries Z."""
    if counts is None:
        counts = torch.zeros(int(ds_info(idx)["n_knots"]) + 1, dtype=torch.int64, device=Z.device)
    check(lib().ds_histogram(idx.ptr, _dev(Z, "Z", idx.dtype), Z.numel(), _dev(counts, "counts", torch.int64),
                             _stream(stream)), "ds_histogram")
    return counts


def ds_search_host(idx, Z, out=None, stream=None):
    """Search with host buffers (pinned CPU tensors); copies run inside the call."""
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32, pin_memory=True)
    check(lib().ds_search_host(idx.ptr, _host(Z, "Z", idx.dtype), Z.numel(), _host(out, "out", torch.int32),
                               _stream(stream)), "ds_search_host")
    return out


def ds_index_export(idx, stream=None):
    """Copies of the index's tables: (K int32[R+1], X[N+1], pairs or None).  Pairs
    come back as raw bytes reshaped to (R+1, 8) or (R+1, 16) uint8."""
    info = ds_info(idx)
    R = int(info["R"])
    dev = torch.device("cuda", torch.cuda.current_device())
    K = torch.empty(R + 1, dtype=torch.int32, device=dev)
    X = torch.empty(int(info["n_knots"]), dtype=idx.dtype, device=dev)
    pairs = None
    pp = None
    if info["flags"] & DS_CACHE_LAYOUT:
        pairs = torch.empty((R + 1, 8 if idx.dtype == torch.float32 else 16), dtype=torch.uint8, device=dev)
        pp = _dev(pairs, "pairs")
    check(lib().ds_index_export(idx.ptr, _dev(K, "K"), _dev(X, "X"), pp, _stream(stream)), "ds_index_export")
    return K, X, pairs


# ---------------------------------------------------------------- logarithmic searches
def ds_lsearch_constants(method, n_knots):
    """(consts[4], layout_len) of a logarithmic method (host only)."""
    c = (_abi.I64 * 4)()
    n = _abi.I64()
    check(lib().ds_lsearch_constants(int(method), int(n_knots), c, ctypes.byref(n)), "ds_lsearch_constants")
    return list(c), n.value


def ds_lsearch_build(X, method, flags=0, stream=None):
    """Lay out knot array X (CUDA tensor) for a logarithmic method (DS_LS_*)."""
    out = ctypes.c_void_p()
    check(lib().ds_lsearch_build(_dev(X, "X"), X.numel(), _dtype(X), int(method), int(flags), _stream(stream),
                                 ctypes.byref(out)), "ds_lsearch_build")
    return LSearch(out.value, X.dtype)


def ds_lsearch_search(h, Z, out=None, stream=None):
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32, device=Z.device)
    check(lib().ds_lsearch_search(h.ptr, _dev(Z, "Z", h.dtype), Z.numel(), _dev(out, "out", torch.int32),
                                  _stream(stream)), "ds_lsearch_search")
    return out


# ---------------------------------------------------------------- batched
def ds_batch_build(Xcat, x_off, flags=0, stream=None):
    """Build per-array tables for knots Xcat with device CSR offsets x_off (int64)."""
    out = ctypes.c_void_p()
    check(lib().ds_batch_build(_dev(Xcat, "Xcat"), _dev(x_off, "x_off", torch.int64), x_off.numel() - 1,
                               _dtype(Xcat), int(flags), _stream(stream), ctypes.byref(out)), "ds_batch_build")
    return Batch(out.value, Xcat.dtype)


def ds_batch_search(b, Zcat, z_off, out=None, stream=None):
    if out is None:
        out = torch.empty(Zcat.numel(), dtype=torch.int32, device=Zcat.device)
    check(lib().ds_batch_search(b.ptr, _dev(Zcat, "Zcat", b.dtype), _dev(z_off, "z_off", torch.int64),
                                _dev(out, "out", torch.int32), _stream(stream)), "ds_batch_search")
    return out


def ds_batch_autotune(b, Zcat, z_off, out=None, stream=None):
    if out is None:
        out = torch.empty(Zcat.numel(), dtype=torch.int32, device=Zcat.device)
    best = _abi.ds_tune_t()
    check(lib().ds_batch_autotune(b.ptr, _dev(Zcat, "Zcat", b.dtype), _dev(z_off, "z_off", torch.int64),
                                  _dev(out, "out", torch.int32), _stream(stream), ctypes.byref(best)),
          "ds_batch_autotune")
    return best.as_dict()


def ds_batch_set_tune(b, block, items, smem_limit, blocks_per_sm=0):
    t = _abi.ds_tune_t(block, items, smem_limit, blocks_per_sm, 0.0)
    check(lib().ds_batch_set_tune(b.ptr, ctypes.byref(t)), "ds_batch_set_tune")


def ds_batch_get_tune(b):
    t = _abi.ds_tune_t()
    check(lib().ds_batch_get_tune(b.ptr, ctypes.byref(t)), "ds_batch_get_tune")
    return t.as_dict()


def ds_batch_array(b, a):
    H = ctypes.c_double(); W = ctypes.c_double(); R = ctypes.c_uint64(); mode = ctypes.c_int32()
    check(lib().ds_batch_array(b.ptr, int(a), ctypes.byref(H), ctypes.byref(W), ctypes.byref(R),
                               ctypes.byref(mode)), "ds_batch_array")
    return dict(H=H.value, W=W.value, R=R.value, mode=mode.value)


# ---------------------------------------------------------------- learned
def ds_learned_cfg_default(**overrides):
    cfg = _abi.ds_learned_cfg()
    lib().ds_learned_cfg_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def ds_learned_build(X, x_off=None, cfg=None, stream=None):
    """Learned form of one array (x_off None) or of many arrays (device CSR x_off)."""
    return ds_learned_build_xy(X, None, x_off, cfg, stream)


def ds_learned_build_xy(X, Y, x_off=None, cfg=None, stream=None):
    """Learned form holding the knot values Y as (X_i, Y_i) pairs (Y None: ds_learned_build)."""
    cfg = cfg if cfg is not None else ds_learned_cfg_default()
    out = ctypes.c_void_p()
    yp = None if Y is None else _dev(Y, "Y", X.dtype)
    if Y is not None and Y.numel() != X.numel():
        raise ValueError("Y must have one value per knot")
    if x_off is None:
        rc = lib().ds_learned_build_xy(_dev(X, "X"), yp, None, 1, X.numel(), _dtype(X), ctypes.byref(cfg),
                                       _stream(stream), ctypes.byref(out))
    else:
        rc = lib().ds_learned_build_xy(_dev(X, "Xcat"), yp, _dev(x_off, "x_off", torch.int64), x_off.numel() - 1, 0,
                                       _dtype(X), ctypes.byref(cfg), _stream(stream), ctypes.byref(out))
    check(rc, "ds_learned_build_xy" if Y is not None else "ds_learned_build")
    L = Learned(out.value, X.dtype)
    L.xy = Y is not None
    return L


def _interp_args(L, Z, Y, y_out):
    """(Ycat pointer, y_out pointer, y_out tensor) of a learned search: interpolation when the
    handle holds its values and y_out is given, or when the caller passes Y."""
    if L.xy:
        if Y is not None:
            raise ValueError("this learned handle holds its knot values: pass y_out, not Y")
        if y_out is None:
            return None, None, None
        return None, _dev(y_out, "y_out", L.dtype), y_out
    if Y is None:
        return None, None, None
    if y_out is None:
        y_out = torch.empty(Z.numel(), dtype=L.dtype, device=Z.device)
    return _dev(Y, "Y", L.dtype), _dev(y_out, "y_out", L.dtype), y_out


def ds_learned_search(L, Z, z_off=None, Y=None, out=None, y_out=None, stream=None):
    """Indices (and, with Y or with y_out on a handle that holds its values, the interpolant)."""
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32, device=Z.device)
    yp, yo, y_out = _interp_args(L, Z, Y, y_out)
    zo = None if z_off is None else _dev(z_off, "z_off", torch.int64)
    check(lib().ds_learned_search(L.ptr, _dev(Z, "Z", L.dtype), zo, Z.numel(), yp, yo, _dev(out, "out", torch.int32),
                                  _stream(stream)), "ds_learned_search")
    return (out, y_out) if yo is not None else out


def ds_learned_search_host(L, Z, z_off=None, out=None, y_out=None, stream=None):
    """The search on host tensors (pinned ones used in place, others registered
    for the call); z_off a host int64 tensor or None.  Returns when the results
    are in host memory."""
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32)
    zo = None if z_off is None else _host(z_off, "z_off", torch.int64)
    yo = None if y_out is None else _host(y_out, "y_out", L.dtype)
    check(lib().ds_learned_search_host(L.ptr, _host(Z, "Z", L.dtype), zo, Z.numel(), yo, _host(out, "out", torch.int32),
                                       _stream(stream)), "ds_learned_search_host")
    return (out, y_out) if y_out is not None else out


def ds_learned_autotune(L, Z, z_off=None, out=None, stream=None, Y=None, y_out=None):
    """Autotune the learned handle's launch configuration on these queries (with the
    interpolation when Y, or y_out on a handle that holds its values, is given); returns it."""
    if out is None:
        out = torch.empty(Z.numel(), dtype=torch.int32, device=Z.device)
    best = _abi.ds_tune_t()
    yp, yo, _ = _interp_args(L, Z, Y, y_out)
    zo = _dev(z_off, "z_off", torch.int64) if z_off is not None else None
    check(lib().ds_learned_autotune(L.ptr, _dev(Z, "Z", L.dtype), zo, Z.numel(), yp, yo,
                                    _dev(out, "out", torch.int32), _stream(stream), ctypes.byref(best)),
          "ds_learned_autotune")
    return best.as_dict()


def ds_learned_cells(L, a=0):
    """Cell table of learned array a: cells, max_pop, nonempty, escaped, mean_pop, from_network."""
    C = ctypes.c_uint64(); mp = ctypes.c_int32(); ne = ctypes.c_int64(); esc = ctypes.c_int64()
    mean = ctypes.c_double(); net = ctypes.c_int32()
    check(lib().ds_learned_cells(L.ptr, int(a), ctypes.byref(C), ctypes.byref(mp), ctypes.byref(ne),
                                 ctypes.byref(esc), ctypes.byref(mean), ctypes.byref(net)), "ds_learned_cells")
    return dict(cells=C.value, max_pop=mp.value, nonempty=ne.value, escaped=esc.value, mean_pop=mean.value,
                from_network=net.value)


def ds_learned_export_cells(L, a=0, stream=None):
    """K_0 .. K_C of learned array a (int32 tensor on the current device)."""
    C = ds_learned_cells(L, a)["cells"]
    K = torch.empty(C + 1, dtype=torch.int32, device="cuda")
    check(lib().ds_learned_export_cells(L.ptr, int(a), _dev(K, "K"), _stream(stream)), "ds_learned_export_cells")
    return K


def ds_learned_set_tune(L, block, items, smem_limit, blocks_per_sm=0):
    t = _abi.ds_tune_t(block, items, smem_limit, blocks_per_sm, 0.0)
    check(lib().ds_learned_set_tune(L.ptr, ctypes.byref(t)), "ds_learned_set_tune")


def ds_learned_get_tune(L):
    t = _abi.ds_tune_t()
    check(lib().ds_learned_get_tune(L.ptr, ctypes.byref(t)), "ds_learned_get_tune")
    return t.as_dict()


def ds_learned_array(L, a):
    theta = torch.empty(1153, dtype=torch.float32)
    e_lo = ctypes.c_int32(); e_hi = ctypes.c_int32(); mode = ctypes.c_int32()
    check(lib().ds_learned_array(L.ptr, int(a), ctypes.c_void_p(theta.data_ptr()), ctypes.byref(e_lo),
                                 ctypes.byref(e_hi), ctypes.byref(mode)), "ds_learned_array")
    return dict(theta=theta, e_lo=e_lo.value, e_hi=e_hi.value, mode=mode.value)


def ds_mlp_forward(theta, u, out=None, stream=None):
    if out is None:
        out = torch.empty(u.numel(), dtype=torch.float32, device=u.device)
    check(lib().ds_mlp_forward(_dev(theta, "theta", torch.float32), _dev(u, "u", torch.float32), u.numel(),
                               _dev(out, "out", torch.float32), _stream(stream)), "ds_mlp_forward")
    return out


def ds_mlp_loss_grad(theta, u, y, stream=None):
    grad = torch.empty(1153, dtype=torch.float32, device=u.device)
    loss = torch.empty(1, dtype=torch.float32, device=u.device)
    check(lib().ds_mlp_loss_grad(_dev(theta, "theta", torch.float32), _dev(u, "u", torch.float32),
                                 _dev(y, "y", torch.float32), u.numel(), _dev(grad, "grad"), _dev(loss, "loss"),
                                 _stream(stream)), "ds_mlp_loss_grad")
    return loss, grad


def ds_adam_step(theta, m, v, grad, t, lr, stream=None):
    check(lib().ds_adam_step(_dev(theta, "theta", torch.float32), _dev(m, "m", torch.float32),
                             _dev(v, "v", torch.float32), _dev(grad, "grad", torch.float32), int(t), float(lr),
                             _stream(stream)), "ds_adam_step")


# ---------------------------------------------------------------- handles
def ds_info(h):
    info = _abi.ds_info_t()
    check(lib().ds_info(h.ptr, ctypes.byref(info)), "ds_info")
    return info.as_dict()


def ds_free(h):
    h.free()


# ---------------------------------------------------------------- test aids
def ds_debug_fail_alloc(nth):
    """Make the library's device allocation nth + 1 from now fail (nth < 0: off)."""
    check(lib().ds_debug_fail_alloc(int(nth)), "ds_debug_fail_alloc")


def ds_debug_alloc_stats():
    """The library's live device allocations: (count, bytes)."""
    n, b = ctypes.c_int64(), ctypes.c_int64()
    check(lib().ds_debug_alloc_stats(ctypes.byref(n), ctypes.byref(b)), "ds_debug_alloc_stats")
    return n.value, b.value
