"""The allocation-free table build (ds_build_table_static).

It serves callers that may not allocate device memory when they build a
table (a host framework that owns every device allocation, real-time loops
that cannot afford cudaMalloc's implicit synchronisation, plug-ins barred
from allocating after start-up).  This test calls it through the C ABI and
checks, on two calls in a row that share its static scratch, that it returns
exactly the H, W, R and K table of ds_build.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_1506_08620_gb300 import build
    build.build()
    from paper_1506_08620_gb300 import _abi
    _abi.lib()
    return _abi


def _reference(X, flags):
    import paper_1506_08620_gb300 as ds
    idx = ds.ds_build(X, flags)
    info = idx.info()
    K, _, _ = ds.ds_index_export(idx)
    torch.cuda.synchronize()
    idx.free()
    return info, K.cpu().numpy()


def _static(abi, X, flags, capacity):
    L = abi.lib()
    K = torch.full((capacity,), -9, dtype=torch.int32, device="cuda")
    H, W, R = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    dtype = abi.DS_F32 if X.dtype == torch.float32 else abi.DS_F64
    rc = L.ds_build_table_static(ctypes.c_void_p(X.data_ptr()), X.numel(), dtype, flags, ctypes.c_void_p(K.data_ptr()),
                                 capacity, ctypes.byref(H), ctypes.byref(W), ctypes.byref(R),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, H.value, W.value, R.value, K.cpu().numpy()


def _arrays():
    g = np.random.default_rng(2024)
    big = np.cumsum(g.lognormal(0.0, 0.5, 200_000))
    small = -50.0 + np.cumsum(g.uniform(0.5, 1.5, 3000))
    return [(torch.from_numpy(np.concatenate([[0.0], big])).cuda(), 1),                  # float64, FMA form
            (torch.from_numpy(small.astype(np.float32)).cuda(), 0)]                     # float32, plain form


def test_two_calls_match_ds_build(abi):
    for X, flags in _arrays():  # two calls in a row on the shared scratch
        info, K_ref = _reference(X, flags)
        cap = int(info["R"]) + 1 + 17
        rc, H, W, R, K = _static(abi, X, flags, cap)
        assert rc == abi.DS_OK, abi.lib().ds_last_error()
        assert H == info["H"] and R == info["R"]
        if flags & abi.DS_FMA:
            assert W == info["W"]
        assert np.array_equal(K[: R + 1], K_ref)
        assert np.all(K[R + 1:] == -9)


def test_limits_are_rejected(abi):
    X = torch.linspace(0.0, 1.0, abi.DS_STATIC_MAX_KNOTS + 1, dtype=torch.float64, device="cuda")
    rc, *_ = _static(abi, X, 0, 16)
    assert rc == abi.DS_E_ARG
    assert b"static scratch limit" in abi.lib().ds_last_error()
    X = torch.linspace(0.0, 1.0, 1000, dtype=torch.float64, device="cuda")
    rc, H, W, R, _ = _static(abi, X, 0, 10)
    assert rc == abi.DS_E_ARG and R + 1 > 10
