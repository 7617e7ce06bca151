"""Pins for the oracle's refinement of H by bisection (end of Section 4.4):
when ComputeHR had to grow H, the refined H is feasible and the float just
below it is not, both checked in exact rational arithmetic; it never exceeds
ComputeHR's H; and the table it gives answers every query correctly."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1506_08620_gb300 import workloads as W
from tests import exact


def _feasible_exact(X, H, q, dtype, fma):
    H = dtype(H)
    Wv = exact.mul(H, X[0], dtype)
    if fma:
        top = exact.round_nearest(Fraction(float(H)) * Fraction(float(X[-1])) - Fraction(float(Wv)), dtype)
        F = [exact.f_fma(H, Wv, x, dtype) for x in X]
    else:
        D = exact.round_nearest(Fraction(float(X[-1])) - Fraction(float(X[0])), dtype)
        top = exact.round_nearest(Fraction(float(H)) * Fraction(float(D)), dtype)
        F = [exact.f_plain(H, X[0], x, dtype) for x in X]
    if not float(top) < 4294967296.0:
        return False
    qe = min(q, len(X) - 1)
    return all(F[i] < F[i + qe] for i in range(len(F) - qe))


def _growth_arrays(dtype, q, count, seed):
    g = np.random.default_rng(seed)
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        assert tries < 200000
        n = int(g.integers(q + 3, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if np.all(np.diff(X) > 0) and oracle.compute_hr(X, True, q=q)["updates"] > 0:
            out.append(X)
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [1, 2])
def test_refined_h_is_a_boundary(dtype, q):
    # with one growth step the interval is two adjacent floats and nothing is
    # bisected; with more, H usually comes down (R rarely: the overshoot is a
    # few dozen ulps, "negligible in relative terms" as the section says)
    smaller = 0
    for X in _growth_arrays(dtype, q, 12, 40 + q + (dtype == np.float64)):
        a = oracle.compute_hr(X, True, q=q, general=q > 1)
        b = oracle.compute_hr_refined(X, True, q=q)
        assert b["status"] == oracle.OR_OK and b["updates"] == a["updates"]
        if a["updates"] == 1:  # H grew by one ulp: [last infeasible, final] has nothing inside
            assert b["probes"] == 0 and b["H"] == a["H"]
        H = dtype(b["H"])
        assert H <= dtype(a["H"]) and b["R"] <= a["R"]
        assert _feasible_exact(X, H, q, dtype, True)
        assert not _feasible_exact(X, np.nextafter(H, dtype(0)), q, dtype, True)
        assert b["W"] == float(exact.mul(H, X[0], dtype))
        smaller += H < dtype(a["H"])
        # the refined table is a correct table
        st, K, _ = oracle.fill_k(X, b["H"], b["W"], b["R"], True, q=q, general=q > 1)
        assert st == oracle.OR_OK
        g = np.random.default_rng(1)
        Z = np.concatenate([W.adversarial_queries(X), W.uniform_queries(g, X[0], X[-1], 500, dtype)])
        assert np.array_equal(oracle.direct(X, K, b["H"], b["W"], b["R"], Z, True, q=q, general=q > 1),
                              oracle.upper_bound(X, Z))
    assert smaller >= 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_no_growth_no_refinement(dtype):
    g = np.random.default_rng(2)
    for _ in range(20):
        X = W.knots_from_gaps(0.0, g.uniform(0.5, 1.5, int(g.integers(2, 300))), dtype)
        a, b = oracle.compute_hr(X), oracle.compute_hr_refined(X)
        if a["updates"] == 0:
            assert b["probes"] == 0 and (a["H"], a["W"], a["R"]) == (b["H"], b["W"], b["R"])
