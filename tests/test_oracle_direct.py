"""Pins for the oracle's direct-search construction: ComputeHR (Section 4.4),
the index table of Eq. indexdef and Algorithm "direct", against the paper's
worked examples, its rounding counter-examples, the feasibility family of
Eq. feasibility, exact rational arithmetic and the problem's definition."""
import numpy as np
import pytest

import oracle
from paper_1506_08620_gb300 import workloads as W
from tests import exact


# ---------------------------------------------------------------- worked examples
def test_section_4_1_example_h3_is_admissible():
    # Section 4.1: X = {0, 0.5, 0.7, 1.1} admits H = 3 although Eq. minh gives ~6.36.
    X = np.array([0.0, 0.5, 0.7, 1.1])
    R = exact.trunc_u32(exact.mul(3.0, 1.1, np.float64))
    assert R == 3
    st, K, F = oracle.fill_k(X, 3.0, 0.0, R)
    assert st == oracle.OR_OK
    assert list(F) == [0, 1, 2, 3] and list(K) == [0, 1, 2, 3]
    Z = np.concatenate([np.linspace(0.0, 1.1, 2001)[:-1], W.adversarial_queries(X)])
    assert np.array_equal(oracle.direct(X, K, 3.0, 0.0, R, Z), oracle.upper_bound(X, Z))


def test_section_4_1_example_compute_hr():
    # min m(D_{i+1}-D_i) = m(0.7-0.5) = 0.19999999999999996; m(1/that) = 5.000000000000001;
    # H = phi(.) = 5.000000000000002; R = trunc(m(H*1.1)) = trunc(5.500000000000002) = 5.
    X = np.array([0.0, 0.5, 0.7, 1.1])
    for fma in (False, True):
        hr = oracle.compute_hr(X, fma)
        assert hr["status"] == oracle.OR_OK
        assert hr["H"] == 5.000000000000002 and hr["R"] == 5 and hr["updates"] == 0
    dmin = exact.round_nearest(exact.Fraction(0.7) - exact.Fraction(0.5), np.float64)
    hbar = exact.round_nearest(1 / exact.Fraction(float(dmin)), np.float64)
    assert np.nextafter(hbar, np.inf) == 5.000000000000002


def test_figure_directmap_tables():
    # Figure "directmap": knots 0,6,15,23,31,37,50 and grid cells of width 5 (H = 0.2).
    X = np.array([0.0, 6.0, 15.0, 23.0, 31.0, 37.0, 50.0])
    H = 0.2
    R = exact.trunc_u32(exact.mul(H, 50.0, np.float64))
    assert R == 10
    st, K, F = oracle.fill_k(X, H, 0.0, R)
    assert st == oracle.OR_OK
    assert list(F) == [0, 1, 3, 4, 6, 7, 10]
    assert list(K) == [0, 1, 2, 2, 3, 4, 4, 5, 6, 6, 6]  # Eq. indexdef
    # the figure's arrows: K_j = max{i : X_i <= Y_{j+1}}, Y_j = 5 j (Section 4.3)
    geo = [0, 1, 2, 2, 3, 3, 4, 5, 5, 6]
    assert geo == [int(np.max(np.nonzero(X <= 5 * (j + 1))[0])) for j in range(10)]
    Kg = np.array(geo + [6], dtype=np.int32)
    Z = np.concatenate([np.linspace(0, 50, 5001)[:-1], W.adversarial_queries(X)])
    ref = oracle.upper_bound(X, Z)
    assert np.array_equal(oracle.direct(X, K, H, 0.0, R, Z), ref)
    assert np.array_equal(oracle.direct(X, Kg, H, 0.0, R, Z), ref)


# ---------------------------------------------------------------- rounding failures
def test_section_4_4_counterexamples():
    # {-1e9, 0, 1} in single precision: X_2 - X_0 rounds to X_1 - X_0.
    hr = oracle.compute_hr(np.array([-1e9, 0.0, 1.0], dtype=np.float32))
    assert hr["status"] == oracle.OR_E_INDISTINGUISHABLE and hr["bad"] == 2
    # {0, 1.42e-45, 1} in single precision: 1 / min gap overflows to +inf.
    X = np.array([0.0, 1.42e-45, 1.0], dtype=np.float32)
    assert X[1] > 0
    hr = oracle.compute_hr(X)
    assert hr["status"] == oracle.OR_E_OVERFLOW and np.isinf(hr["H"])


def test_invalid_arrays():
    assert oracle.compute_hr(np.array([1.0]))["status"] == oracle.OR_E_ARG
    assert oracle.compute_hr(np.array([0.0, 1.0, 1.0]))["status"] == oracle.OR_E_NOT_INCREASING
    assert oracle.compute_hr(np.array([0.0, 2.0, 1.0]))["status"] == oracle.OR_E_NOT_INCREASING
    assert oracle.compute_hr(np.array([0.0, np.nan, 1.0]))["status"] == oracle.OR_E_NOT_INCREASING
    assert oracle.compute_hr(np.array([0.0, 1.0, np.inf]))["status"] == oracle.OR_E_NOT_INCREASING


def test_feasibility_family_clear_margins():
    # Eq. feasibility: min gap / (X_N - X_0) > max(2^-Q, 2 eps); checked 4x away on each side.
    f32 = np.float32
    ok = np.array([-1.0, 0.0, 2.0 ** -20, 1.0], dtype=f32)  # ratio 2^-21 = 4 * 2^-23
    assert oracle.compute_hr(ok)["status"] == oracle.OR_OK
    bad = np.array([-1.0, 0.0, 2.0 ** -25, 1.0], dtype=f32)  # ratio 2^-26: D_1 == D_2
    assert oracle.compute_hr(bad)["status"] == oracle.OR_E_INDISTINGUISHABLE
    ok64 = np.array([0.0, 2.0 ** -30, 1.0])  # ratio 2^-30 = 4 * 2^-32 (Q = 32)
    hr = oracle.compute_hr(ok64)
    assert hr["status"] == oracle.OR_OK and hr["R"] < 2 ** 32
    bad64 = np.array([0.0, 2.0 ** -34, 1.0])  # ratio 2^-34: R would exceed 2^32
    assert oracle.compute_hr(bad64)["status"] == oracle.OR_E_OVERFLOW


# ---------------------------------------------------------------- f's rounding
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_f_matches_exact_rational_rounding(dtype, fma):
    g = np.random.default_rng(21)
    for _ in range(60):
        X0 = dtype(g.uniform(-50, 50))
        H = dtype(g.uniform(0.5, 40))
        Wv = exact.mul(H, X0, dtype)
        Z = (float(X0) + g.uniform(-1, 60, 40)).astype(dtype)
        got = oracle.fvals(H, Wv, X0, Z, fma)
        if fma:
            ref = [exact.f_fma(H, Wv, z, dtype) for z in Z]
        else:
            ref = [exact.f_plain(H, X0, z, dtype) for z in Z]
        assert list(got) == ref


# ---------------------------------------------------------------- growth of H
def _growth_arrays(dtype, count, seed):
    """Arrays with X_0 != 0 on which the FMA form needs H to grow: the plain
    form's H is computed from the rounded D_i, which can overestimate a gap."""
    g = np.random.default_rng(seed)
    found = []
    while len(found) < count:
        n = int(g.integers(4, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if not np.all(np.diff(X) > 0):
            continue
        hr = oracle.compute_hr(X, fma=True)
        if hr["status"] == oracle.OR_OK and hr["updates"] > 0:
            found.append((X, hr))
    return found


def _feasible_exact(X, H, dtype):
    """Eq. cond2 in FMA form evaluated with exact rational rounding."""
    Wv = exact.mul(H, X[0], dtype)
    F = [exact.f_fma(H, Wv, x, dtype) for x in X]
    return all(F[i] < F[i + 1] for i in range(len(F) - 1))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_growth_finds_first_feasible_h_of_the_sequence(dtype):
    # The growth rule H += P, P *= 2 visits H_k = H_0 + (2^k - 1) P_0 while the
    # additions stay exact; the result must be the first feasible H_k, checked
    # with exact rational arithmetic on all pairs at once.
    for X, hr in _growth_arrays(dtype, 12, 31 if dtype == np.float32 else 32):
        D = (X - X[0]).astype(dtype)
        dmin = np.min(np.diff(D))
        H0 = np.nextafter(exact.round_nearest(1 / exact.Fraction(float(dmin)), dtype), dtype(np.inf))
        P0 = np.nextafter(H0, dtype(np.inf)) - H0
        H, P, k = H0, P0, 0
        while not _feasible_exact(X, H, dtype):
            H, P, k = exact.add(H, P, dtype), dtype(2) * P, k + 1
            assert k < 64
        assert k == hr["updates"] and H == dtype(hr["H"])
        assert not _feasible_exact(X, H0, dtype)
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma=True)
        assert st == oracle.OR_OK


# ---------------------------------------------------------------- method exactness
def _feasible_arrays(dtype):
    g = np.random.default_rng(41)
    yield W.workload1(n_uniform=1000)["X"].astype(dtype)
    yield W.paper_layout(255, 10, dtype)["X"]
    yield W.workload2(n_knots=4097, m=10)["X"].astype(dtype)
    for _ in range(40):
        n = int(g.integers(2, 300))
        X0 = g.uniform(-1e3, 1e3)
        X = W.knots_from_gaps(X0, g.uniform(0.01, 2.0, n - 1) * 10.0 ** g.uniform(-3, 3), dtype)
        yield X


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_direct_equals_definition(dtype, fma):
    g = np.random.default_rng(51)
    for X in _feasible_arrays(dtype):
        hr = oracle.compute_hr(X, fma)
        if hr["status"] != oracle.OR_OK:
            continue
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma)
        assert st == oracle.OR_OK
        inf = dtype(np.inf)
        Z = np.concatenate([
            W.adversarial_queries(X), W.midpoints(X),
            W.uniform_queries(g, X[0], X[-1], 2000, dtype),
            # outside the domain the table answers like the definition too
            np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, float(X[0]) - 1e6], dtype=dtype)])
        assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, fma),
                              oracle.upper_bound(X, Z))


@pytest.mark.parametrize("fma", [False, True])
def test_table_properties(fma):
    for X in _feasible_arrays(np.float64):
        hr = oracle.compute_hr(X, fma)
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma)
        N = X.size - 1
        assert K[0] == 0 and K[-1] == N and K.size == hr["R"] + 1
        assert np.all(np.diff(K) >= 0)
        assert F[-1] == hr["R"]
        assert np.array_equal(K[F.astype(np.int64)], np.arange(N + 1))  # Eq. kidentity


def test_exhaustive_float32_direct():
    # every float32 between the first and last knot of small arrays with close knots
    g = np.random.default_rng(61)
    for base in (1.0, 3.0e3):
        b0 = np.array([base], dtype=np.float32).view(np.int32)[0]
        bits = (b0 + np.concatenate([[0], np.cumsum(g.integers(1, 40, 30))])).astype(np.int32)
        X = bits.view(np.float32)
        for fma in (False, True):
            hr = oracle.compute_hr(X, fma)
            assert hr["status"] == oracle.OR_OK
            st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma)
            Z = np.arange(bits[0] - 2, bits[-1] + 3, dtype=np.int32).view(np.float32)
            assert np.array_equal(oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z, fma),
                                  oracle.scan(X, Z))
