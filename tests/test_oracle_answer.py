"""Pins for the oracle's answer (problem statement, Section 2): the index of the
largest X_i <= z.  Checked against a brute-force scan, numpy's searchsorted,
exhaustive float enumeration between knots and the defining invariant."""
import numpy as np
import pytest

import oracle


def _tiny_cases(dtype, count, seed):
    g = np.random.default_rng(seed)
    for _ in range(count):
        n = int(g.integers(2, 17))
        x0 = g.uniform(-10, 10)
        X = (x0 + np.concatenate([[0.0], np.cumsum(g.uniform(0.01, 3.0, n - 1))])).astype(dtype)
        X = np.unique(X)
        if X.size < 2:
            continue
        inf = dtype(np.inf)
        q = [X, np.nextafter(X, inf), np.nextafter(X, -inf),
             g.uniform(float(X[0]) - 2, float(X[-1]) + 2, 16).astype(dtype),
             np.array([np.inf, -np.inf, np.nan, 0.0, -0.0], dtype=dtype)]
        yield X, np.concatenate(q).astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_upper_bound_equals_brute_force_on_tiny_arrays(dtype):
    for X, Z in _tiny_cases(dtype, 10000, 11 if dtype == np.float32 else 12):
        assert np.array_equal(oracle.upper_bound(X, Z), oracle.scan(X, Z))


def test_exhaustive_float32_between_knots():
    # knots a few ulps apart: every float32 between (and just outside) them
    g = np.random.default_rng(5)
    for base in (1.0, -3.5, 1e-40, 7.0e6):
        b0 = np.array([base], dtype=np.float32).view(np.int32)[0]
        steps = g.integers(1, 6, 12)
        bits = (b0 + np.concatenate([[0], np.cumsum(steps)])).astype(np.int32)
        X = bits.view(np.float32)
        if base < 0:  # negative floats: larger bit pattern = smaller value
            X = np.sort(X)
        assert np.all(np.diff(X) > 0)
        lo = np.array([X[0]], dtype=np.float32).view(np.int32)[0]
        hi = np.array([X[-1]], dtype=np.float32).view(np.int32)[0]
        a, b = min(lo, hi) - 3, max(lo, hi) + 3
        Z = np.arange(a, b + 1, dtype=np.int32).view(np.float32)
        assert np.array_equal(oracle.upper_bound(X, Z), oracle.scan(X, Z))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_upper_bound_equals_searchsorted(dtype):
    g = np.random.default_rng(3)
    X = np.unique(g.normal(size=200000).astype(dtype))
    Z = np.concatenate([g.normal(size=200000), X[::7], [-1e30, 1e30]]).astype(dtype)
    ref = np.searchsorted(X, Z, side="right") - 1
    assert np.array_equal(oracle.upper_bound(X, Z), ref)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_defining_invariant(dtype):
    g = np.random.default_rng(4)
    X = np.unique(g.uniform(-5, 5, 5000).astype(dtype))
    Z = g.uniform(float(X[0]), float(X[-1]), 100000).astype(dtype)
    Z = Z[(Z >= X[0]) & (Z < X[-1])]
    I = oracle.upper_bound(X, Z).astype(np.int64)
    assert I.min() >= 0 and I.max() <= X.size - 2
    assert np.all(X[I] <= Z) and np.all(Z < X[I + 1])


def test_edge_cases():
    X = np.array([0.0, 1.0], dtype=np.float64)
    assert oracle.upper_bound(X, np.zeros(0)).shape == (0,)
    Z = np.array([0.0, -0.0, 0.5, np.nextafter(1.0, 0.0), 1.0, -1e-300, np.nan])
    assert list(oracle.upper_bound(X, Z)) == [0, 0, 0, 0, 1, -1, -1]


def test_batch_is_per_array():
    g = np.random.default_rng(8)
    sizes = [2, 5, 17, 3]
    Xs = [np.sort(g.uniform(-1, 1, s)).astype(np.float32) for s in sizes]
    Zs = [g.uniform(-1.2, 1.2, k).astype(np.float32) for k in (0, 9, 40, 5)]
    x_off = np.concatenate([[0], np.cumsum(sizes)])
    z_off = np.concatenate([[0], np.cumsum([len(z) for z in Zs])])
    I = oracle.upper_bound_batch(np.concatenate(Xs), x_off, np.concatenate(Zs), z_off)
    ref = np.concatenate([oracle.scan(X, Z) for X, Z in zip(Xs, Zs)])
    assert np.array_equal(I, ref)
