"""The allocation-free table build (ds_build_table_static).

It serves callers that may not allocate device memory when they build a
table (a host framework that owns every device allocation, real-time loops
that cannot afford cudaMalloc's implicit synchronisation, plug-ins barred
from allocating after start-up).  This test calls it through the C ABI on two
calls in a row that share its static scratch and checks that:
  - H, W, R and K equal the CPU oracle's ComputeHR (Section 4.4) and Eq.
    indexdef, and the same values from ds_build;
  - a warm call leaves the device's free memory unchanged (nothing allocated).
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

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


def _static(abi, X, flags, capacity, K=None):
    L = abi.lib()
    if K is None:
        K = torch.full((capacity,), -9, dtype=torch.int32, device="cuda")
    H, W, R = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    dtype = abi.DS_F32 if X.dtype == torch.float32 else abi.DS_F64
    rc = L.ds_build_table_static(ctypes.c_void_p(X.data_ptr()), X.numel(), dtype, flags, ctypes.c_void_p(K.data_ptr()),
                                 capacity, ctypes.byref(H), ctypes.byref(W), ctypes.byref(R),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, H.value, W.value, R.value, K


def _arrays():
    g = np.random.default_rng(2024)
    big = np.concatenate([[0.0], np.cumsum(g.lognormal(0.0, 0.5, 200_000))])
    small = (-50.0 + np.cumsum(g.uniform(0.5, 1.5, 3000))).astype(np.float32)
    return [(big, 1),      # float64, FMA form
            (small, 0),    # float32, plain form
            (big, 0),      # float64, plain form
            (small, 1)]    # float32, FMA form


def test_two_calls_match_oracle_and_ds_build(abi):
    for Xh, flags in _arrays():  # calls in a row on the shared scratch
        fma = bool(flags & abi.DS_FMA)
        hr = oracle.compute_hr(Xh, fma=fma)
        assert hr["status"] == oracle.OR_OK
        st, K_or, _ = oracle.fill_k(Xh, hr["H"], hr["W"], hr["R"], fma=fma)
        assert st == oracle.OR_OK
        X = torch.from_numpy(Xh).cuda()
        info, K_ref = _reference(X, flags)
        cap = int(hr["R"]) + 1 + 17
        rc, H, W, R, Kd = _static(abi, X, flags, cap)
        assert rc == abi.DS_OK, abi.lib().ds_last_error()
        K = Kd.cpu().numpy()
        # the oracle first, then ds_build: H, W and R bit for bit in both forms
        assert (H, W, R) == (hr["H"], hr["W"], hr["R"])
        assert (H, W, R) == (info["H"], info["W"], info["R"])
        assert np.array_equal(K[: R + 1], K_or)
        assert np.array_equal(K[: R + 1], K_ref)
        assert np.all(K[R + 1:] == -9)


def test_warm_call_allocates_nothing(abi):
    Xh, flags = _arrays()[0]
    X = torch.from_numpy(Xh).cuda()
    hr = oracle.compute_hr(Xh, fma=True)
    cap = int(hr["R"]) + 1
    K = torch.empty(cap, dtype=torch.int32, device="cuda")
    rc, *_ = _static(abi, X, flags, cap, K)  # warm: the library's module is loaded
    assert rc == abi.DS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        rc, *_ = _static(abi, X, flags, cap, K)
        assert rc == abi.DS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_limits_and_infeasible_are_rejected(abi):
    X = torch.linspace(0.0, 1.0, abi.DS_STATIC_MAX_KNOTS + 1, dtype=torch.float64, device="cuda")
    rc, *_ = _static(abi, X, 0, 16)
    assert rc == abi.DS_E_ARG
    assert b"static scratch limit" in abi.lib().ds_last_error()
    X = torch.linspace(0.0, 1.0, 1000, dtype=torch.float64, device="cuda")
    rc, H, W, R, _ = _static(abi, X, 0, 10)
    assert rc == abi.DS_E_ARG and R + 1 > 10
    # the first counter-example of Section 4.4: indistinguishable knots, named by index
    X = torch.tensor([-1e9, 0.0, 1.0], dtype=torch.float32, device="cuda")
    rc, *_ = _static(abi, X, 0, 16)
    assert rc == abi.DS_E_INDISTINGUISHABLE
    assert b"(knot 2)" in abi.lib().ds_last_error()
