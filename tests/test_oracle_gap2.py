"""Pins for the oracle's DirectGap2 (Section 4.7): the relaxed property
f(X_{i+2}) > f(X_i), the table of Eq. kgeneral, Algorithm direct-2 and the
proof's case structure t in {i, i+1, i+2}."""
import numpy as np
import pytest

import oracle
from paper_1506_08620_gb300 import workloads as W
from tests import exact


def _arrays(dtype, seed=7):
    g = np.random.default_rng(seed)
    yield W.workload1(n_uniform=10)["X"].astype(dtype)
    yield W.paper_layout(255, 10, dtype)["X"]
    yield W.workload2(n_knots=4097, m=10)["X"].astype(dtype)
    yield np.array([-3.0, 7.0]).astype(dtype)
    yield np.array([0.0, 6.0, 15.0, 23.0, 31.0, 37.0, 50.0]).astype(dtype)
    for _ in range(30):
        n = int(g.integers(3, 400))
        X0 = g.uniform(-1e3, 1e3)
        yield W.knots_from_gaps(X0, g.lognormal(0, 1, n - 1) * 10.0 ** g.uniform(-2, 2), dtype)


def test_section_4_7_mitigates_the_section_4_4_counterexample():
    # {-1e9, 0, 1} in single precision: D_1 == D_2, so Direct is infeasible,
    # but D_0 < D_2 and DirectGap2 only needs f(X_{i+2}) > f(X_i).
    X = np.array([-1e9, 0.0, 1.0], dtype=np.float32)
    assert oracle.compute_hr(X)["status"] == oracle.OR_E_INDISTINGUISHABLE
    hr, K = oracle.build_table(X, gap2=True)
    assert hr["R"] == 1 and list(K) == [0, 2]
    inf = np.float32(np.inf)
    Z = np.concatenate([np.linspace(-1e9, 1.0, 20001, dtype=np.float32), W.adversarial_queries(X),
                        np.array([-inf, inf, 1.0, 0.5, -2e9], dtype=np.float32)])
    assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, gap2=True), oracle.upper_bound(X, Z))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_gap2_equals_definition_and_case_structure(dtype, fma):
    g = np.random.default_rng(3)
    for X in _arrays(dtype):
        hr = oracle.compute_hr(X, fma, gap2=True)
        assert hr["status"] == oracle.OR_OK
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma, gap2=True)
        assert st == oracle.OR_OK
        inf = dtype(np.inf)
        Z = np.concatenate([W.adversarial_queries(X), W.midpoints(X),
                            W.uniform_queries(g, X[0], X[-1], 3000, dtype),
                            np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf], dtype=dtype)])
        ref = oracle.upper_bound(X, Z)
        assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, fma, gap2=True), ref)
        # the proof: for z in [X_i, X_{i+1}), t = K_{f(z)} is one of i, i+1, i+2
        inside = (Z >= X[0]) & (Z < X[-1])
        j = np.minimum(oracle.fvals(hr["H"], hr["W"], X[0], Z[inside], fma), hr["R"]).astype(np.int64)
        t = K[j].astype(np.int64)
        d = t - ref[inside]
        assert np.all((d >= 0) & (d <= 2))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_kgeneral_is_the_count_of_cells_at_or_below(dtype):
    for X in _arrays(dtype, seed=11):
        hr = oracle.compute_hr(X, gap2=True)
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], gap2=True)
        j = np.arange(hr["R"] + 1, dtype=np.int64)
        ref = np.maximum(np.searchsorted(F.astype(np.int64), j, side="right") - 1, 0)  # max{i : F_i <= j}
        assert np.array_equal(K, ref)
        # properties (kgeneralprop): F_i < F_{i+1} -> K_{F_i} = i ; F_i = F_{i+1} -> K_{F_i} = i+1
        for i in range(F.size - 1):
            if F[i] < F[i + 1]:
                assert K[F[i]] == i
            else:
                assert K[F[i]] == i + 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_gap2_table_is_never_larger(dtype):
    # Eq. fcond11: H > 1/min(X_{i+2} - X_i) is a smaller bound than Eq. minh
    smaller = 0
    for X in _arrays(dtype, seed=13):
        a, b = oracle.compute_hr(X), oracle.compute_hr(X, gap2=True)
        if a["status"] != oracle.OR_OK:
            continue
        assert b["R"] <= a["R"]
        smaller += b["R"] < a["R"]
    assert smaller > 10


def test_exhaustive_float32_gap2():
    g = np.random.default_rng(17)
    b0 = np.array([2.0], dtype=np.float32).view(np.int32)[0]
    bits = (b0 + np.concatenate([[0], np.cumsum(g.integers(1, 30, 40))])).astype(np.int32)
    X = bits.view(np.float32)
    for fma in (False, True):
        hr, K = oracle.build_table(X, fma, gap2=True)
        Z = np.arange(bits[0] - 2, bits[-1] + 3, dtype=np.int32).view(np.float32)
        assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, fma, gap2=True), oracle.scan(X, Z))


def _feasible_gap2_exact(X, H, dtype, fma):
    Wv = exact.mul(H, X[0], dtype)
    F = [exact.f_fma(H, Wv, x, dtype) if fma else exact.f_plain(H, X[0], x, dtype) for x in X]
    return all(F[i] < F[i + 2] for i in range(len(F) - 2))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_gap2_growth_finds_first_feasible_h(dtype):
    g = np.random.default_rng(23)
    found = 0
    while found < 6:
        n = int(g.integers(5, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if not np.all(np.diff(X) > 0):
            continue
        hr = oracle.compute_hr(X, True, gap2=True)
        if hr["status"] != oracle.OR_OK or hr["updates"] == 0:
            continue
        found += 1
        D = (X - X[0]).astype(dtype)
        dmin = np.min(D[2:] - D[:-2])
        H0 = np.nextafter(exact.round_nearest(1 / exact.Fraction(float(dmin)), dtype), dtype(np.inf))
        P0 = np.nextafter(H0, dtype(np.inf)) - H0
        H, P, k = H0, P0, 0
        while not _feasible_gap2_exact(X, H, dtype, True):
            H, P, k = exact.add(H, P, dtype), dtype(2) * P, k + 1
            assert k < 64
        assert k == hr["updates"] and H == dtype(hr["H"])
