"""GPU parity of the logarithmic searches (Section 3) with the definition of
the answer: every method, both precisions, the paper's sizes (N+1 = 2^h - 1)
and ragged ones, shared-memory and L2 layouts, aligned and misaligned
buffers.  Bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_08620_gb300 import workloads as W

pytestmark = pytest.mark.gpu

METHODS = list(range(6))


@pytest.fixture(scope="module")
def ds():
    from paper_1506_08620_gb300 import build
    build.build()
    import paper_1506_08620_gb300 as ds
    return ds


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _queries(X, g, n=5000):
    dt = X.dtype.type
    inf = dt(np.inf)
    return np.concatenate([
        W.adversarial_queries(X), W.midpoints(X), W.uniform_queries(g, X[0], X[-1], n, X.dtype),
        np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, float(X[0]) - 1e6, float(X[-1]) * 2 + 1, 0.0, -0.0],
                 dtype=X.dtype)])


def _arrays(dtype):
    g = np.random.default_rng(55)
    out = [("two", np.array([-3.0, 7.0]).astype(dtype)), ("three", np.array([1.0, 1.5, 4.0]).astype(dtype))]
    for n in (15, 255, 4095, 65535, 16, 17, 100, 1000, 3001):
        out.append(("paper%d" % n, W.paper_layout(n, 10, dtype)["X"]))
    for k in range(4):
        n = int(g.integers(2, 5000))
        out.append(("random%d" % k, W.knots_from_gaps(g.uniform(-1e4, 1e4),
                                                     g.lognormal(0, 1.5, n - 1) * 10.0 ** g.uniform(-3, 3), dtype)))
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("flags", [0, 8], ids=["smem", "l2"])
def test_lsearch_matches_definition(ds, dtype, method, flags):
    g = np.random.default_rng(method)
    for name, X in _arrays(dtype):
        Z = _queries(X, g)
        h = ds.ds_lsearch_build(_cuda(X), method, flags)
        got = ds.ds_lsearch_search(h, _cuda(Z)).cpu().numpy()
        ref = oracle.upper_bound(X, Z)
        nan_free = ~np.isnan(Z)
        assert np.array_equal(got[nan_free], ref[nan_free]), (name, ds.DS_LS_NAMES[method],
                                                              int(np.count_nonzero(got != ref)))
        h.free()


@pytest.mark.parametrize("method", METHODS)
def test_lsearch_large_and_nan(ds, method):
    # 2^20 + 1 float64 knots in L2, a million queries; NaN answers -1
    w = W.workload2(n_knots=(1 << 20) + 1, m=1 << 20)
    X, Z = w["X"], w["Z"]
    Z = Z.copy()
    Z[::1000] = np.nan
    h = ds.ds_lsearch_build(_cuda(X), method)
    assert h.info()["smem_resident"] == 0
    got = ds.ds_lsearch_search(h, _cuda(Z)).cpu().numpy()
    ref = oracle.upper_bound(X, Z)
    assert np.array_equal(got, ref)  # the oracle also answers -1 for NaN
    h.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("method", [0, 2, 5])
def test_lsearch_ragged_and_misaligned(ds, dtype, method):
    g = np.random.default_rng(9)
    X = W.knots_from_gaps(0.0, g.uniform(0.5, 1.5, 2000), dtype)
    Zall = W.uniform_queries(g, X[0], X[-1], (1 << 18) + 40, dtype)
    h = ds.ds_lsearch_build(_cuda(X), method)
    Zd = _cuda(Zall)
    for m in (0, 1, 3, 5, 31, 1023, 4099, (1 << 18) + 3):
        for zoff, ioff in ((0, 0), (1, 0), (0, 1), (3, 5)):
            out = torch.full((m + ioff,), -7, dtype=torch.int32, device="cuda")
            ds.ds_lsearch_search(h, Zd[zoff:zoff + m], out[ioff:])
            o = out.cpu().numpy()
            assert np.array_equal(o[ioff:], oracle.upper_bound(X, Zall[zoff:zoff + m])), (m, zoff, ioff)
            assert np.all(o[:ioff] == -7)
    h.free()


def test_lsearch_layout_sizes(ds):
    X = W.paper_layout(4095, 10, np.float64)["X"]
    for method in METHODS:
        c, length = ds.ds_lsearch_constants(method, X.size)
        h = ds.ds_lsearch_build(_cuda(X), method)
        assert h.info()["table_bytes"] == (length * 8 + 15) // 16 * 16
        h.free()
