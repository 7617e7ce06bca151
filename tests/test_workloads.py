"""The seeded input generators: strictly increasing knots, in-domain queries,
deterministic seeds, CSR bookkeeping (host only, small sizes)."""
import numpy as np
import pytest

from paper_1506_08620_gb300 import workloads as W


def test_strictly_increasing_bump():
    x = np.array([-1.0, -1.0, -0.0, 0.0, 0.0, 1.0, 1.0], dtype=np.float32)
    y = W.strictly_increasing(x)
    assert np.all(np.diff(y) > 0)
    assert y[0] == -1.0 and y[1] == np.nextafter(np.float32(-1.0), np.float32(1))
    x64 = np.array([5.0, 5.0, 5.0, 7.0])
    y64 = W.strictly_increasing(x64)
    assert np.all(np.diff(y64) > 0) and y64[-1] == 7.0


@pytest.mark.parametrize("gen,kw", [
    (W.workload1, dict(n_uniform=1000)),
    (W.workload2, dict(n_knots=1025, m=5000)),
    (W.workload4, dict(n_knots=20001, m=5000)),
    (W.paper_layout, dict(n_knots=255, m=100)),
])
def test_single_array_workloads(gen, kw):
    a = gen(**kw)
    b = gen(**kw)
    X, Z = a["X"], a["Z"]
    assert np.all(np.diff(X) > 0)
    assert np.all(Z >= X[0]) and np.all(Z < X[-1])
    assert np.array_equal(X, b["X"]) and np.array_equal(Z, b["Z"])


def test_workload1_shape():
    a = W.workload1()
    assert a["X"].size == 1025 and a["Z"].size == 1_002_048 and a["X"].dtype == np.float32


@pytest.mark.parametrize("gen,kw", [
    (W.workload3, dict(n_arrays=64, size_hi=2048, total_queries=100000)),
    (W.workload5, dict(n_arrays=12, size_lo=1024, size_hi=8192, total_queries=50000)),
])
def test_batched_workloads(gen, kw):
    a = gen(**kw)
    x_off, z_off = a["x_off"], a["z_off"]
    assert x_off[0] == 0 and z_off[0] == 0 and z_off[-1] == kw["total_queries"]
    sizes = np.diff(x_off)
    q = np.diff(z_off)
    assert np.all(sizes >= 2)
    # queries proportional to size (largest remainder: within one of exact)
    exact = kw["total_queries"] * sizes / sizes.sum()
    assert np.all(np.abs(q - exact) < 1.0 + 1e-9)
    for k in range(len(sizes)):
        Xa = a["Xcat"][x_off[k]:x_off[k + 1]]
        Za = a["Zcat"][z_off[k]:z_off[k + 1]]
        assert np.all(np.diff(Xa) > 0)
        assert np.all(Za >= Xa[0]) and np.all(Za < Xa[-1])
