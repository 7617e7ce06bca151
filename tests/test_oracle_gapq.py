"""Pins for the oracle's Gap-q generalisation of DirectGap2 (Section 4.7,
Eq. f-monotonic-n): ComputeHR over the pairs (i, i+q), the table of Eq.
kgeneral, the search with q comparisons, and the memory-budget choice of the
smallest q."""
import numpy as np
import pytest

import oracle
from paper_1506_08620_gb300 import workloads as W
from tests import exact


def _arrays(dtype, seed=5, count=25):
    g = np.random.default_rng(seed)
    yield W.workload1(n_uniform=10)["X"].astype(dtype)
    yield W.workload2(n_knots=2049, m=10)["X"].astype(dtype)
    yield np.array([-3.0, 7.0]).astype(dtype)
    yield np.array([1.0, 1.5, 4.0]).astype(dtype)
    for _ in range(count):
        n = int(g.integers(2, 500))
        X0 = g.uniform(-1e3, 1e3)
        yield W.knots_from_gaps(X0, g.lognormal(0, 1.5, n - 1) * 10.0 ** g.uniform(-2, 2), dtype)


def _growth_arrays(dtype, fma, count, seed):
    g = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(g.integers(4, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if np.all(np.diff(X) > 0) and oracle.compute_hr(X, fma)["updates"] > 0:
            out.append(X)
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_q1_general_is_computehr(dtype, fma):
    # the generalised routine at q = 1 is the separately written ComputeHR of Section 4.4
    arrays = list(_arrays(dtype)) + _growth_arrays(dtype, True, 5, 8 + (dtype == np.float64))
    grew = 0
    for X in arrays:
        a, b = oracle.compute_hr(X, fma), oracle.compute_hr(X, fma, q=1, general=True)
        assert a == b
        grew += a["updates"] > 0
    if fma:
        assert grew >= 5


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [1, 2, 3, 5, 8])
def test_gapq_search_is_the_definition(dtype, q):
    g = np.random.default_rng(31 + q)
    for fma in (False, True):
        for X in _arrays(dtype, seed=q):
            hr, K = oracle.build_table(X, fma, q=q, general=True)
            inf = dtype(np.inf)
            Z = np.concatenate([W.adversarial_queries(X), W.midpoints(X),
                                W.uniform_queries(g, X[0], X[-1], 2000, dtype),
                                np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, X[0] - abs(X[0]) - 1],
                                         dtype=dtype)])
            ref = oracle.upper_bound(X, Z)
            got = oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, fma, q=q, general=True)
            assert np.array_equal(got, ref)
            # the case structure: for z in [X_i, X_{i+1}), t = K_{f(z)} lies in i .. i+q
            inside = (Z >= X[0]) & (Z < X[-1])
            j = np.minimum(oracle.fvals(hr["H"], hr["W"], X[0], Z[inside], fma), hr["R"]).astype(np.int64)
            d = K[j].astype(np.int64) - ref[inside]
            assert np.all((d >= 0) & (d <= q))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [2, 3, 4, 7])
def test_gapq_cells_hold_at_most_q_knots(dtype, q):
    runs = 0
    for X in _arrays(dtype, seed=40 + q):
        hr = oracle.compute_hr(X, q=q)
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], q=q)
        assert st == oracle.OR_OK
        qe = min(q, X.size - 1)
        assert np.all(F[qe:] > F[:-qe])                     # Eq. f-monotonic-n
        _, counts = np.unique(F, return_counts=True)
        assert counts.max() <= q
        runs += int(np.count_nonzero(counts == q))
        # K_j = max{i : F_i <= j} (Eq. kgeneral), 0 below F_0
        j = np.arange(hr["R"] + 1, dtype=np.int64)
        assert np.array_equal(K, np.maximum(np.searchsorted(F.astype(np.int64), j, side="right") - 1, 0))
    assert runs > 0  # some cells hold q knots, so every comparison is exercised


def test_exhaustive_float32_gapq():
    g = np.random.default_rng(71)
    b0 = np.array([3.0], dtype=np.float32).view(np.int32)[0]
    bits = (b0 + np.concatenate([[0], np.cumsum(g.integers(1, 25, 60))])).astype(np.int32)
    X = bits.view(np.float32)
    Z = np.arange(bits[0] - 3, bits[-1] + 4, dtype=np.int32).view(np.float32)
    for q in (3, 4, 6):
        for fma in (False, True):
            hr, K = oracle.build_table(X, fma, q=q)
            assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, fma, q=q), oracle.scan(X, Z))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_table_shrinks_with_q(dtype):
    total = {q: 0 for q in (1, 2, 4, 8)}
    for X in _arrays(dtype, seed=17, count=40):
        for q in total:
            hr = oracle.compute_hr(X, q=q)
            assert hr["status"] == oracle.OR_OK
            total[q] += hr["R"]
    assert total[1] > total[2] > total[4] > total[8]


def _feasible_gapq_exact(X, H, q, dtype):
    Wv = exact.mul(H, X[0], dtype)
    F = [exact.f_fma(H, Wv, x, dtype) for x in X]
    return all(F[i] < F[i + q] for i in range(len(F) - q))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [3, 4])
def test_gapq_growth_finds_first_feasible_h(dtype, q):
    g = np.random.default_rng(29 + q)
    found = tries = 0
    while found < 4:
        tries += 1
        assert tries < 200000
        n = int(g.integers(q + 3, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if not np.all(np.diff(X) > 0):
            continue
        hr = oracle.compute_hr(X, True, q=q)
        if hr["status"] != oracle.OR_OK or hr["updates"] == 0:
            continue
        found += 1
        D = (X - X[0]).astype(dtype)
        dmin = np.min(D[q:] - D[:-q])
        H0 = np.nextafter(exact.round_nearest(1 / exact.Fraction(float(dmin)), dtype), dtype(np.inf))
        P0 = np.nextafter(H0, dtype(np.inf)) - H0
        H, P, k = H0, P0, 0
        while not _feasible_gapq_exact(X, H, q, dtype):
            H, P, k = exact.add(H, P, dtype), dtype(2) * P, k + 1
            assert k < 64
        assert k == hr["updates"] and H == dtype(hr["H"])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_choose_q_is_the_smallest_that_fits(dtype):
    g = np.random.default_rng(3)
    chosen = set()
    for _ in range(30):
        n = int(g.integers(200, 3000))
        X = W.knots_from_gaps(0.0, g.lognormal(0, 1.5, n - 1), dtype)
        x_bytes = (X.nbytes + 15) // 16 * 16
        for budget in (x_bytes + 64, x_bytes + 4 * n, x_bytes + 16 * n, 10 ** 9):
            q, hr = oracle.choose_q(X, False, budget, 16)
            if q == 0:
                # then no q up to 16 fits
                for qq in range(1, 17):
                    h = oracle.compute_hr(X, q=qq)
                    assert h["status"] != oracle.OR_OK or oracle.table_bytes(X, h["R"]) > budget
                continue
            chosen.add(q)
            assert oracle.table_bytes(X, hr["R"]) <= budget
            for qq in range(1, q):
                h = oracle.compute_hr(X, q=qq)
                assert h["status"] != oracle.OR_OK or oracle.table_bytes(X, h["R"]) > budget
            # a larger budget never needs a larger q
            q2, _ = oracle.choose_q(X, False, budget * 2, 16)
            assert 1 <= q2 <= q
    assert len(chosen) >= 3
