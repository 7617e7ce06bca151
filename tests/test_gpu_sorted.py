"""GPU parity of the sorted-query merge (ds_search_sorted) and of the fused
histogram (ds_histogram) with the definition of the answer."""
import numpy as np
import pytest
import torch

import oracle
from paper_1506_08620_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILE = 256 * 11  # elements of the merged sequence per block tile


@pytest.fixture(scope="module")
def ds():
    from paper_1506_08620_gb300 import build
    build.build()
    import paper_1506_08620_gb300 as ds
    return ds


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sorted_queries(X, g, n):
    dt = X.dtype.type
    inf = dt(np.inf)
    Z = np.concatenate([W.adversarial_queries(X), W.uniform_queries(g, X[0], X[-1], n, X.dtype),
                        np.repeat(X[g.integers(0, X.size, 7)], 50),  # runs of equal queries on knots
                        np.array([-inf, inf, X[0] - abs(X[0]) - 1, X[-1] + abs(X[-1]) + 1], dtype=X.dtype)])
    return np.sort(Z)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_merge_matches_definition(ds, dtype):
    g = np.random.default_rng(4)
    sizes = [1, 2, 3, 17, TILE - 1, TILE, TILE + 1, 5000, 100_000]
    for n in sizes:
        X = W.knots_from_gaps(g.uniform(-10, 10), g.lognormal(0, 1, max(n - 1, 0)), dtype) if n > 1 else \
            np.array([1.5], dtype=dtype)
        for m in (0, 1, 7, TILE - 3, 3 * TILE + 5, 200_003):
            Zall = _sorted_queries(X, g, m)
            Z = np.sort(g.choice(Zall, m, replace=False)) if m else np.empty(0, dtype=dtype)
            got = ds.ds_search_sorted(_cuda(X), _cuda(Z)).cpu().numpy()
            assert np.array_equal(got, oracle.upper_bound(X, Z)), (n, m)


def test_merge_full_size_workload2(ds):
    w = W.workload2(sort=True)
    X, Z = w["X"], w["Z"]
    Zd = _cuda(Z)
    got = ds.ds_search_sorted(_cuda(X), Zd)
    g = np.random.default_rng(1)
    pos = np.concatenate([g.integers(0, Z.size, 1 << 20), np.arange(4096), np.arange(Z.size - 4096, Z.size)])
    assert np.array_equal(got[_cuda(pos)].cpu().numpy(), oracle.upper_bound(X, Z[pos]))
    Xd, gl = _cuda(X), got.long()
    assert bool((gl >= 0).all()) and bool((gl <= X.size - 2).all())
    assert bool((Xd[gl] <= Zd).all()) and bool((Zd < Xd[gl + 1]).all())
    # the same answers as direct search
    idx = ds.ds_build(Xd)
    assert torch.equal(ds.ds_search(idx, Zd), got)
    idx.free()


def test_merge_unsorted_input_stays_in_bounds(ds):
    # not sorted: the answers are unspecified, but nothing is written outside I
    g = np.random.default_rng(6)
    X = W.knots_from_gaps(0.0, g.uniform(0.5, 1.5, 10_000), np.float32)
    Z = W.uniform_queries(g, X[0], X[-1], 50_000, np.float32)
    guard = 4096
    buf = torch.full((Z.size + 2 * guard,), -7, dtype=torch.int32, device="cuda")
    ds.ds_search_sorted(_cuda(X), _cuda(Z), buf[guard:guard + Z.size])
    o = buf.cpu().numpy()
    assert np.all(o[:guard] == -7) and np.all(o[guard + Z.size:] == -7)
    # the context is still usable
    Zs = np.sort(Z)
    assert np.array_equal(ds.ds_search_sorted(_cuda(X), _cuda(Zs)).cpu().numpy(), oracle.upper_bound(X, Zs))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["direct", "fma", "gap2", "gapq7"])
def test_histogram_matches_counts(ds, dtype, kind):
    g = np.random.default_rng(12)
    for n in (3, 1000, 30_000, 200_000):  # shared-memory counters up to ~24k bins, global above
        X = W.knots_from_gaps(g.uniform(-5, 5), g.lognormal(0, 0.7, n - 1), dtype)
        Z = np.concatenate([W.uniform_queries(g, X[0] - 1, X[-1] + 1, 500_000, dtype), W.adversarial_queries(X),
                            np.array([np.nan, -np.inf, np.inf], dtype=dtype)])
        if kind == "gapq7":
            idx = ds.ds_build_q(_cuda(X), 7)
        else:
            idx = ds.ds_build(_cuda(X), {"direct": 0, "fma": ds.DS_FMA, "gap2": ds.DS_GAP2}[kind])
        counts = ds.ds_histogram(idx, _cuda(Z))
        ref = np.bincount(oracle.upper_bound(X, Z).astype(np.int64) + 1, minlength=n + 1)
        assert np.array_equal(counts.cpu().numpy(), ref), (n, kind)
        # counts are added to
        ds.ds_histogram(idx, _cuda(Z), counts)
        assert np.array_equal(counts.cpu().numpy(), 2 * ref)
        idx.free()
