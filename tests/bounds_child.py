"""Runs in a child process with DS_LIBRARY=bounds (the range-checking build
of the library): every search form on valid inputs, each result compared
with the oracle and each handle's device error word read back; then one
single-array table with an entry moved one knot past the end (inside the
padding of the table's own allocation) to see the knot-gather check fire.
Prints one JSON object: {case: [mismatches, device_error], ...}."""
import ctypes
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_1506_08620_gb300 as ds  # noqa: E402
from paper_1506_08620_gb300 import _abi  # noqa: E402
from paper_1506_08620_gb300 import workloads as W  # noqa: E402

assert os.path.realpath(_abi.lib()._name) == os.path.realpath(_abi.BOUNDS_LIB_PATH), _abi.lib()._name
out = {}


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def record(name, got, ref, h):
    torch.cuda.synchronize()
    out[name] = [int(np.count_nonzero(np.asarray(got) != np.asarray(ref))), int(h.info()["device_error"])]


def queries(g, X, m, dtype):
    Z = W.uniform_queries(g, X[0], X[-1], m, dtype)
    edge = np.array([X[0], X[-1], X[0] - 1, X[-1] + 1, X[len(X) // 2]], dtype=dtype)
    return np.concatenate([Z, edge, X[:: max(1, len(X) // 97)]]).astype(dtype)


g = np.random.default_rng(7)
# single array, both precisions, every table form, shared-memory and global paths, vector and scalar paths
for dtype, n in ((np.float32, 1025), (np.float32, 40_001), (np.float64, 1025), (np.float64, 70_001)):
    X = W.knots_from_gaps(0.0, g.uniform(1, 5, n - 1), dtype)
    Z = queries(g, X, 50_001, dtype)
    ref = oracle.upper_bound(X, Z)
    for name, flags in (("plain", 0), ("fma", ds.DS_FMA), ("cache", ds.DS_CACHE_LAYOUT), ("gap2", ds.DS_GAP2),
                        ("global", ds.DS_NO_SMEM)):
        idx = ds.ds_build(cuda(X), flags=flags)
        record("single_%s_%d_%s" % (np.dtype(dtype).name, n, name), idx.search(cuda(Z)).cpu().numpy(), ref, idx)
        zb = torch.zeros(Z.size + 1, dtype=torch.float32 if dtype == np.float32 else torch.float64, device="cuda")
        zb[1:] = cuda(Z)
        ob = torch.zeros(Z.size + 1, dtype=torch.int32, device="cuda")
        idx.search(zb[1:], out=ob[1:])
        record("single_%s_%d_%s_scalar" % (np.dtype(dtype).name, n, name), ob[1:].cpu().numpy(), ref, idx)
        if name == "plain":
            counts = ds.ds_histogram(idx, cuda(Z)).cpu().numpy()
            hist = np.bincount(ref + 1, minlength=n + 1)
            record("histogram_%s_%d" % (np.dtype(dtype).name, n), counts, hist, idx)
        idx.free()
    idx = ds.ds_build_q(cuda(X), 4)
    record("single_%s_%d_gap4" % (np.dtype(dtype).name, n), idx.search(cuda(Z)).cpu().numpy(), ref, idx)
    idx.free()

# batched direct search: staged and global images, vector and scalar paths
w = W.workload3(n_arrays=96, total_queries=1 << 18)
Xc, xo, Zc, zo = (w[k] for k in ("Xcat", "x_off", "Zcat", "z_off"))
ref = np.concatenate([oracle.upper_bound(Xc[xo[a]:xo[a + 1]], Zc[zo[a]:zo[a + 1]]) for a in range(len(xo) - 1)])
for name, flags in (("staged", 0), ("global", ds.DS_NO_SMEM), ("nofp", ds.DS_NO_FINGERPRINT)):
    b = ds.ds_batch_build(cuda(Xc), cuda(xo), flags=flags)
    record("batched_%s" % name, ds.ds_batch_search(b, cuda(Zc), cuda(zo)).cpu().numpy(), ref, b)
    b.free()

# learned form: direct and learned arrays (two launches), knot values stored or the caller's,
# every array learned, and cell tables with escaped blocks
w = W.workload5(n_arrays=10, size_lo=1 << 10, size_hi=1 << 15, total_queries=1 << 18)
Xc, Yc, xo, Zc, zo = (w[k] for k in ("Xcat", "Ycat", "x_off", "Zcat", "z_off"))
Iref, yref = oracle.interp_batch(Xc, Yc, xo, Zc, zo)
for name, with_y, flags, cpk in (("xy", True, 0, 0.0), ("caller_y", False, 0, 0.0),
                                 ("xy_all_learned", True, ds.DS_LEARNED_FORCE, 0.0),
                                 ("escaped", False, ds.DS_LEARNED_FORCE, 0.0004)):
    cfg = ds.ds_learned_cfg_default(steps=100, flags=flags, cells_per_knot=cpk)
    L = ds.ds_learned_build_xy(cuda(Xc), cuda(Yc) if with_y else None, cuda(xo), cfg=cfg)
    y = torch.empty(Zc.size, dtype=torch.float32, device="cuda")
    I, _ = ds.ds_learned_search(L, cuda(Zc), cuda(zo), Y=None if with_y else cuda(Yc), y_out=y)
    record("learned_%s" % name, I.cpu().numpy(), Iref, L)
    L.free()

# the logarithmic searches
for dtype in (np.float32, np.float64):
    X = W.knots_from_gaps(0.0, g.uniform(1, 5, 3000), dtype)
    Z = queries(g, X, 20_001, dtype)
    ref = oracle.upper_bound(X, Z)
    for method in range(6):
        h = ds.ds_lsearch_build(cuda(X), method)
        record("lsearch_%s_%s" % (np.dtype(dtype).name, ds.DS_LS_NAMES[method]), h.search(cuda(Z)).cpu().numpy(),
               ref, h)
        h.free()

# a table entry moved one knot past the end: N + 1 = 1001 float64 knots fill
# 8008 bytes, padded to 8016, so X_{N+1} lies inside the table's allocation
# (and inside the staged image), and the moved entry's read stays in memory
# the table owns whether or not the check is compiled in
class DeviceView:
    """A device buffer of the library as a torch tensor (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False), "version": 2,
                                         "strides": None}


os.environ["DS_PACKED"] = "0"  # the global path reads K itself, not its packed copy
X = W.knots_from_gaps(0.0, g.uniform(1, 5, 1000), np.float64)
assert X.size % 2 == 1
t = X.size // 2
for name, flags in (("smem", 0), ("global", ds.DS_NO_SMEM)):
    idx = ds.ds_build(cuda(X), flags=flags)
    assert idx.info()["device_error"] == 0
    kp = ctypes.c_void_p()
    ds.check(_abi.lib().ds_index_tables(idx.ptr, ctypes.byref(kp), None, None), "ds_index_tables")
    R = int(idx.info()["R"])
    Kd = torch.as_tensor(DeviceView(kp.value, R + 1), device="cuda")
    K = Kd.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    flag = 1 << 31
    js = np.nonzero(((K & flag) != 0) & ((K & ~flag) == t))[0]
    assert js.size == 1, js
    Kd[int(js[0])] = int(np.array([X.size | flag], dtype=np.uint32).view(np.int32)[0])
    torch.cuda.synchronize()
    idx.search(cuda(np.array([X[t], X[t], X[1], X[2]], dtype=np.float64)))
    torch.cuda.synchronize()
    out["moved_entry_%s" % name] = [0, int(idx.info()["device_error"])]
    idx.free()

print(json.dumps(out))
