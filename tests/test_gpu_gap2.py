"""GPU parity of DirectGap2 (Section 4.7) with the oracle.

Bit-exact: H, W, R, the growth counts, the table of Eq. kgeneral and every
returned index must equal the oracle's DirectGap2 ComputeHR, its K and the
definition of the answer."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_08620_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    from paper_1506_08620_gb300 import build
    build.build()
    import paper_1506_08620_gb300 as ds
    return ds


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _shared_cells(X, fma):
    hr = oracle.compute_hr(X, fma, gap2=True)
    _, _, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma, gap2=True)
    return int(np.count_nonzero(F[1:] == F[:-1]))


def _arrays(dtype):
    g = np.random.default_rng(41)
    out = [
        ("section44_counterexample", np.array([-1e9, 0.0, 1.0]).astype(dtype)),
        ("directmap", np.array([0, 6, 15, 23, 31, 37, 50]).astype(dtype)),
        ("workload1", W.workload1(n_uniform=10)["X"].astype(dtype)),
        ("workload2_small", W.workload2(n_knots=4097, m=10)["X"].astype(dtype)),
        ("paper_U15", W.paper_layout(4095, 10, dtype)["X"]),
        ("two_knots", np.array([-3.0, 7.0]).astype(dtype)),
        ("three_knots", np.array([1.0, 1.5, 4.0]).astype(dtype)),
    ]
    # alternating short/long gaps: many cells hold two knots
    for k in range(3):
        n = int(g.integers(100, 3000))
        gaps = np.where(np.arange(n - 1) % 2 == 0, g.uniform(0.001, 0.01, n - 1), g.uniform(0.5, 1.5, n - 1))
        out.append(("pairs%d" % k, W.knots_from_gaps(g.uniform(-100, 100), gaps, dtype)))
    for k in range(6):
        n = int(g.integers(2, 3000))
        X0 = g.uniform(-1e4, 1e4)
        out.append(("random%d" % k, W.knots_from_gaps(X0, g.lognormal(0, 1, n - 1) * 10.0 ** g.uniform(-3, 3),
                                                     dtype)))
    return out


def _queries(X, g, n=4000):
    dt = X.dtype.type
    inf = dt(np.inf)
    return np.concatenate([
        W.adversarial_queries(X), W.midpoints(X), W.uniform_queries(g, X[0], X[-1], n, X.dtype),
        np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, float(X[0]) - 1e6, float(X[-1]) * 2 + 1, 0.0, -0.0],
                 dtype=X.dtype)])


def test_some_cells_hold_two_knots():
    # the parity cases below exercise the second comparison of Algorithm direct-2
    for dtype in (np.float32, np.float64):
        total = sum(_shared_cells(X, False) for _, X in _arrays(dtype))
        assert total > 100


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_gap2_tables_bit_identical(ds, dtype, fma):
    flags = ds.DS_GAP2 | (ds.DS_FMA if fma else 0)
    for name, X in _arrays(dtype):
        hr = oracle.compute_hr(X, fma, gap2=True)
        assert hr["status"] == oracle.OR_OK, name
        st, K_ref, _ = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma, gap2=True)
        assert st == oracle.OR_OK
        idx = ds.ds_build(_cuda(X), flags)
        info = idx.info()
        assert info["H"] == hr["H"] and info["R"] == hr["R"], name
        if fma:
            assert info["W"] == hr["W"], name
        assert info["h_updates"] == hr["updates"] and info["hr_passes"] == hr["passes"], name
        K, Xc, _ = ds.ds_index_export(idx)
        torch.cuda.synchronize()
        assert np.array_equal(K.cpu().numpy(), K_ref), name
        assert np.array_equal(Xc.cpu().numpy(), X), name
        idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("flags", [0, 1, 8, 9], ids=["smem", "smem_fma", "l2", "l2_fma"])
@pytest.mark.parametrize("variant", ["bits_packed", "bits", "float"])
def test_gap2_search_matches_definition(ds, dtype, flags, variant, monkeypatch):
    if dtype == np.float32 and variant != "float":
        pytest.skip("integer-arithmetic variants exist for float64 only")
    monkeypatch.setenv("DS_F64_INTOPS", "0" if variant == "float" else "1")
    monkeypatch.setenv("DS_PACKED", "1" if variant == "bits_packed" else "0")
    g = np.random.default_rng(13)
    for name, X in _arrays(dtype):
        Z = _queries(X, g)
        idx = ds.ds_build(_cuda(X), flags | ds.DS_GAP2)
        got = ds.ds_search(idx, _cuda(Z)).cpu().numpy()
        ref = oracle.upper_bound(X, Z)
        assert np.array_equal(got, ref), (name, int(np.count_nonzero(got != ref)))
        # and Algorithm direct-2 on the oracle's own table gives the same
        hr, K = oracle.build_table(X, bool(flags & 1), gap2=True)
        assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, bool(flags & 1), gap2=True), ref)
        idx.free()


@pytest.mark.parametrize("vpt", ["2", "4"])
def test_gap2_vectors_per_thread(ds, vpt, monkeypatch):
    monkeypatch.setenv("DS_F64_VPT", vpt)
    g = np.random.default_rng(19)
    X = W.workload2(n_knots=70_001, m=10)["X"]
    Z = W.uniform_queries(g, X[0], X[-1], 3_000_017, np.float64)
    idx = ds.ds_build(_cuda(X), ds.DS_GAP2 | ds.DS_NO_SMEM)
    assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    idx.free()


@pytest.mark.parametrize("sort", [False, True], ids=["unsorted", "sorted"])
def test_gap2_workload2_full_size_sampled(ds, sort):
    w = W.workload2(sort=sort)
    X, Z = w["X"], w["Z"]
    hr = oracle.compute_hr(X, gap2=True)
    hr1 = oracle.compute_hr(X)
    idx = ds.ds_build(_cuda(X), ds.DS_GAP2)
    info = idx.info()
    assert info["H"] == hr["H"] and info["R"] == hr["R"]
    assert info["R"] <= hr1["R"]
    Zd = _cuda(Z)
    got = ds.ds_search(idx, Zd)
    g = np.random.default_rng(9)
    pos = np.concatenate([g.integers(0, Z.size, 1 << 20), np.arange(4096), np.arange(Z.size - 4096, Z.size)])
    ref = oracle.upper_bound(X, Z[pos])
    assert np.array_equal(got[_cuda(pos)].cpu().numpy(), ref)
    Xd = _cuda(X)
    gl = got.long()
    assert bool((gl >= 0).all()) and bool((gl <= X.size - 2).all())
    assert bool((Xd[gl] <= Zd).all()) and bool((Zd < Xd[gl + 1]).all())
    idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_gap2_ragged_sizes_and_misaligned_pointers(ds, dtype):
    g = np.random.default_rng(5)
    gaps = np.where(np.arange(1999) % 2 == 0, g.uniform(0.001, 0.01, 1999), g.uniform(0.5, 1.5, 1999))
    X = W.knots_from_gaps(0.0, gaps, dtype)
    Zall = W.uniform_queries(g, X[0], X[-1], (1 << 20) + 40, dtype)
    for flags in (ds.DS_GAP2, ds.DS_GAP2 | ds.DS_NO_SMEM):
        idx = ds.ds_build(_cuda(X), flags)
        Zd = _cuda(Zall)
        for m in (0, 1, 2, 3, 5, 7, 31, 1023, 4099, (1 << 20) + 3):
            for zoff, ioff in ((0, 0), (1, 0), (0, 1), (3, 5)):
                z = Zd[zoff:zoff + m]
                out = torch.full((m + ioff,), -7, dtype=torch.int32, device="cuda")
                ds.ds_search(idx, z, out[ioff:])
                ref = oracle.upper_bound(X, Zall[zoff:zoff + m])
                o = out.cpu().numpy()
                assert np.array_equal(o[ioff:], ref), (flags, m, zoff, ioff)
                assert np.all(o[:ioff] == -7)
        idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_gap2_checked_nan(ds, dtype):
    X = np.linspace(-1, 1, 101).astype(dtype)
    Z = np.array([np.nan, -np.nan, 0.0, np.nan, 2.0, -3.0], dtype=dtype)
    idx = ds.ds_build(_cuda(X), ds.DS_CHECKED | ds.DS_GAP2)
    assert list(ds.ds_search(idx, _cuda(Z)).cpu().numpy()) == [-1, -1, 50, -1, 100, -1]
    idx.free()


def test_gap2_statuses(ds):
    from paper_1506_08620_gb300 import _abi

    def status(X, flags):
        try:
            ds.ds_build(_cuda(X), flags).free()
            return _abi.DS_OK
        except ds.DsError as e:
            return e.status

    G = ds.DS_GAP2
    # Section 4.4's first counter-example is infeasible for Direct, feasible for DirectGap2
    X = np.array([-1e9, 0, 1], dtype=np.float32)
    assert status(X, 0) == _abi.DS_E_INDISTINGUISHABLE and status(X, G) == _abi.DS_OK
    # m(X_{i+2} - X_0) == m(X_i - X_0): infeasible for both
    assert status(np.array([-1e9, 0, 1, 2], dtype=np.float32), G) == _abi.DS_E_INDISTINGUISHABLE
    assert status(np.array([0.0, 1.0, 1.0]), G) == _abi.DS_E_NOT_INCREASING
    assert status(np.array([0.0, np.nan, 1.0]), G) == _abi.DS_E_NOT_INCREASING
    assert status(np.array([0.0, 1.0, 2.0]), G | ds.DS_CACHE_LAYOUT) == _abi.DS_E_ARG
    # the oracle agrees on the statuses
    assert oracle.compute_hr(np.array([-1e9, 0, 1, 2], dtype=np.float32), gap2=True)["status"] == \
        oracle.OR_E_INDISTINGUISHABLE
