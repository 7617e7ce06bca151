"""GPU parity of the Gap-q tables (Section 4.7, Eq. f-monotonic-n) and of the
memory-budget choice of q with the oracle.

Bit-exact: H, W, R, the growth counts, the table of Eq. kgeneral, the chosen
q and every returned index."""
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


def _arrays(dtype, seed=43):
    g = np.random.default_rng(seed)
    out = [
        ("directmap", np.array([0, 6, 15, 23, 31, 37, 50]).astype(dtype)),
        ("workload1", W.workload1(n_uniform=10)["X"].astype(dtype)),
        ("workload2_small", W.workload2(n_knots=4097, m=10)["X"].astype(dtype)),
        ("two_knots", np.array([-3.0, 7.0]).astype(dtype)),
        ("three_knots", np.array([1.0, 1.5, 4.0]).astype(dtype)),
    ]
    for k in range(3):  # clusters of close knots: cells hold up to q knots
        n = int(g.integers(200, 3000))
        gaps = np.where(g.random(n - 1) < 0.7, g.uniform(0.001, 0.01, n - 1), g.uniform(0.5, 1.5, n - 1))
        out.append(("clustered%d" % k, W.knots_from_gaps(g.uniform(-100, 100), gaps, dtype)))
    for k in range(5):
        n = int(g.integers(2, 3000))
        out.append(("random%d" % k, W.knots_from_gaps(g.uniform(-1e4, 1e4),
                                                     g.lognormal(0, 1.5, n - 1) * 10.0 ** g.uniform(-3, 3), dtype)))
    return out


def _queries(X, g, n=3000):
    dt = X.dtype.type
    inf = dt(np.inf)
    return np.concatenate([
        W.adversarial_queries(X), W.midpoints(X), W.uniform_queries(g, X[0], X[-1], n, X.dtype),
        np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, float(X[0]) - 1e6, float(X[-1]) * 2 + 1, 0.0, -0.0],
                 dtype=X.dtype)])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [1, 3, 4, 8, 15, 40])
def test_gapq_tables_bit_identical(ds, dtype, q):
    for fma in (False, True):
        for name, X in _arrays(dtype):
            hr = oracle.compute_hr(X, fma, q=q)
            assert hr["status"] == oracle.OR_OK, name
            st, K_ref, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma, q=q)
            idx = ds.ds_build_q(_cuda(X), q, flags=ds.DS_FMA if fma else 0)
            info = idx.info()
            assert info["gap_q"] == q
            assert info["H"] == hr["H"] and info["R"] == hr["R"], name
            if fma:
                assert info["W"] == hr["W"], name
            assert info["h_updates"] == hr["updates"] and info["hr_passes"] == hr["passes"], name
            K, Xc, _ = ds.ds_index_export(idx)
            assert np.array_equal(K.cpu().numpy(), K_ref), name
            idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [3, 5, 11, 12, 40])
@pytest.mark.parametrize("flags", [0, 1, 8, 9], ids=["smem", "smem_fma", "l2", "l2_fma"])
@pytest.mark.parametrize("variant", ["bits_packed", "bits", "float"])
def test_gapq_search_matches_definition(ds, dtype, q, flags, variant, monkeypatch):
    if dtype == np.float32 and variant != "float":
        pytest.skip("integer-arithmetic variants exist for float64 only")
    monkeypatch.setenv("DS_F64_INTOPS", "0" if variant == "float" else "1")
    monkeypatch.setenv("DS_PACKED", "1" if variant == "bits_packed" else "0")
    g = np.random.default_rng(q + 100)
    for name, X in _arrays(dtype, seed=q):
        Z = _queries(X, g)
        idx = ds.ds_build_q(_cuda(X), q, flags=flags)
        got = ds.ds_search(idx, _cuda(Z)).cpu().numpy()
        ref = oracle.upper_bound(X, Z)
        assert np.array_equal(got, ref), (name, int(np.count_nonzero(got != ref)))
        idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_budget_choice_of_q_matches_oracle(ds, dtype):
    g = np.random.default_rng(8)
    chosen = set()
    for k in range(12):
        n = int(g.integers(300, 6000))
        X = W.knots_from_gaps(0.0 if k % 2 else g.uniform(-50, 50), g.lognormal(0, 1.5, n - 1), dtype)
        x_bytes = (X.nbytes + 15) // 16 * 16
        for fma in (False, True):
            for budget in (x_bytes + 4 * n, x_bytes + 16 * n, x_bytes + 64 * n):
                q_ref, hr = oracle.choose_q(X, fma, budget, 24)
                if q_ref == 0:
                    with pytest.raises(ds.DsError):
                        ds.ds_build_q(_cuda(X), 0, budget, flags=ds.DS_FMA if fma else 0, q_max=24)
                    continue
                chosen.add(q_ref)
                idx = ds.ds_build_q(_cuda(X), 0, budget, flags=ds.DS_FMA if fma else 0, q_max=24)
                info = idx.info()
                assert info["gap_q"] == q_ref and info["R"] == hr["R"] and info["H"] == hr["H"]
                Z = _queries(X, g, 2000)
                assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
                idx.free()
    assert len(chosen) >= 3


def test_default_budget_is_the_shared_memory_stage(ds):
    # an array whose Direct table is too large for shared memory, staged with a larger q
    g = np.random.default_rng(12)
    X = W.knots_from_gaps(0.0, g.lognormal(0, 1.5, 12000), np.float32)
    direct = ds.ds_build(_cuda(X))
    assert direct.info()["smem_resident"] == 0
    idx = ds.ds_build_q(_cuda(X), 0)
    info = idx.info()
    assert info["gap_q"] > 1 and info["smem_resident"] == 1
    Z = W.uniform_queries(g, X[0], X[-1], 1 << 20, np.float32)
    assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    direct.free()
    idx.free()


def test_gapq_statuses(ds):
    from paper_1506_08620_gb300 import _abi

    def status(X, q, budget=0, flags=0, q_max=64):
        try:
            ds.ds_build_q(_cuda(X), q, budget, flags, q_max).free()
            return _abi.DS_OK
        except ds.DsError as e:
            return e.status

    X = np.linspace(0, 1, 1000).astype(np.float32)
    assert status(X, 1000) == _abi.DS_OK  # q above N: pair distance N
    assert status(X, -1) == _abi.DS_E_ARG
    assert status(X, 3, flags=ds.DS_CACHE_LAYOUT) == _abi.DS_E_ARG
    assert status(X, 1, flags=ds.DS_CACHE_LAYOUT) == _abi.DS_OK
    assert status(X, 0, budget=100) == _abi.DS_E_TABLE_TOO_LARGE
    assert status(X, 0, q_max=0) == _abi.DS_E_ARG
    assert status(np.array([0.0, 2.0, 1.0]), 0) == _abi.DS_E_NOT_INCREASING
    # infeasible for Direct and DirectGap2 (m(X_3 - X_0) == m(X_1 - X_0)), feasible for q = 3
    Y = np.array([-1e9, 0, 1, 2], dtype=np.float32)
    assert status(Y, 1) == _abi.DS_E_INDISTINGUISHABLE and status(Y, 2) == _abi.DS_E_INDISTINGUISHABLE
    assert oracle.compute_hr(Y, q=3)["status"] == oracle.OR_OK and status(Y, 3) == _abi.DS_OK
    idx = ds.ds_build_q(_cuda(Y), 0, 1 << 20)
    assert idx.info()["gap_q"] == 3
    idx.free()


def test_large_q_makes_the_two_scale_gap_law_feasible(ds):
    # workload 4's gap law (99% U[1e-3,1e-2], 1% U[1e3,1e4]) on 2^18 + 1 knots:
    # Direct overflows (R >= 2^32); a large q gives a feasible table
    w = W.workload4(n_knots=(1 << 18) + 1, m=1 << 20, seed=1)
    X, Z = w["X"], w["Z"]
    assert oracle.compute_hr(X)["status"] == oracle.OR_E_OVERFLOW
    q_ref, hr = oracle.choose_q(X, False, 1 << 30, 256)
    assert q_ref > 1
    idx = ds.ds_build_q(_cuda(X), 0, 1 << 30, q_max=256)
    info = idx.info()
    assert info["gap_q"] == q_ref and info["R"] == hr["R"] and info["H"] == hr["H"]
    st, K_ref, _ = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], q=q_ref)
    K, _, _ = ds.ds_index_export(idx)
    assert np.array_equal(K.cpu().numpy(), K_ref)
    # uniform queries (mostly in the wide gaps) and queries inside the dense clusters
    g = np.random.default_rng(2)
    Zc = np.concatenate([Z, W.adversarial_queries(X), W.midpoints(X)])
    got = ds.ds_search(idx, _cuda(Zc)).cpu().numpy()
    assert np.array_equal(got, oracle.upper_bound(X, Zc))
    idx.free()
