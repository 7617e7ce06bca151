"""Every device allocation of every build can fail: the build then returns
DS_E_NOMEM and leaves no allocation behind, and the next build succeeds.  The
failures are injected on the host (ds_debug_fail_alloc: the chosen allocation
reports cudaErrorMemoryAllocation without allocating), so nothing faults on
the device."""
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


def _each_failure(ds, build, check):
    """Fail allocation 0, 1, 2, ... of `build` until it makes no more; each
    failure must give DS_E_NOMEM and leave the live allocations as they were.
    Returns the number of allocations the build makes."""
    torch.cuda.synchronize()
    base = ds.ds_debug_alloc_stats()
    for nth in range(400):
        ds.ds_debug_fail_alloc(nth)
        try:
            h = build()
        except ds.DsError as e:
            assert e.status == ds.DS_E_NOMEM, "allocation %d: %s" % (nth, e)
            torch.cuda.synchronize()
            assert ds.ds_debug_alloc_stats() == base, "allocation %d failed and left memory behind" % nth
            continue
        finally:
            ds.ds_debug_fail_alloc(-1)
        check(h)
        h.free()
        torch.cuda.synchronize()
        assert ds.ds_debug_alloc_stats() == base
        assert nth > 0  # every build allocates
        return nth
    raise AssertionError("the build still failed after 400 injected failures")


@pytest.mark.parametrize("flags", ["plain", "cache", "gap2"])
def test_single_array_build(ds, flags):
    g = np.random.default_rng(1)
    X = W.knots_from_gaps(0.0, g.uniform(1, 5, 20_000), np.float64)
    Z = W.uniform_queries(g, X[0], X[-1], 10_000, np.float64)
    f = {"plain": 0, "cache": ds.DS_CACHE_LAYOUT, "gap2": ds.DS_GAP2}[flags]
    ref = oracle.upper_bound(X, Z)
    n = _each_failure(ds, lambda: ds.ds_build(_cuda(X), flags=f),
                      lambda h: np.testing.assert_array_equal(h.search(_cuda(Z)).cpu().numpy(), ref))
    assert n >= 2


def test_gap_q_build(ds):
    g = np.random.default_rng(2)
    gaps = g.uniform(1, 5, 5000)
    gaps[100] = 1e-6  # one narrow gap: a plain table would be large
    X = W.knots_from_gaps(0.0, gaps, np.float64)
    Z = W.uniform_queries(g, X[0], X[-1], 10_000, np.float64)
    ref = oracle.upper_bound(X, Z)
    _each_failure(ds, lambda: ds.ds_build_q(_cuda(X), 8),
                  lambda h: np.testing.assert_array_equal(h.search(_cuda(Z)).cpu().numpy(), ref))


def test_batched_build(ds):
    w = W.workload3(n_arrays=64, total_queries=1 << 16)
    Xc, xo, Zc, zo = (w[k] for k in ("Xcat", "x_off", "Zcat", "z_off"))
    Xd, xod, Zd, zod = _cuda(Xc), _cuda(xo), _cuda(Zc), _cuda(zo)
    arr = np.searchsorted(zo, np.arange(Zc.size), side="right") - 1
    ref = np.array([oracle.upper_bound(Xc[xo[a]:xo[a + 1]], Zc[zo[a]:zo[a + 1]]) for a in range(len(xo) - 1)],
                   dtype=object)
    ref = np.concatenate(list(ref))
    assert ref.size == arr.size

    def check(b):
        np.testing.assert_array_equal(ds.ds_batch_search(b, Zd, zod).cpu().numpy(), ref)

    _each_failure(ds, lambda: ds.ds_batch_build(Xd, xod), check)


@pytest.mark.parametrize("with_y", [False, True])
def test_learned_build(ds, with_y):
    # several arrays, direct and learned (with training), one handle
    w = W.workload5(n_arrays=6, size_lo=1 << 10, size_hi=1 << 13, total_queries=1 << 15)
    Xc, Yc, xo, Zc, zo = (w[k] for k in ("Xcat", "Ycat", "x_off", "Zcat", "z_off"))
    Xd, Yd, xod, Zd, zod = _cuda(Xc), _cuda(Yc), _cuda(xo), _cuda(Zc), _cuda(zo)
    Iref, _ = oracle.interp_batch(Xc, Yc, xo, Zc, zo)
    cfg = ds.ds_learned_cfg_default(steps=20)

    def build():
        return ds.ds_learned_build_xy(Xd, Yd if with_y else None, xod, cfg=cfg)

    def check(L):
        np.testing.assert_array_equal(ds.ds_learned_search(L, Zd, zod).cpu().numpy(), Iref)

    _each_failure(ds, build, check)


def test_learned_search_host(ds):
    # the host-buffer search allocates its device copy of the query offsets on
    # first use: a failure there leaves the handle usable
    w = W.workload5(n_arrays=4, size_lo=1 << 10, size_hi=1 << 12, total_queries=1 << 14)
    Xc, Yc, xo, Zc, zo = (w[k] for k in ("Xcat", "Ycat", "x_off", "Zcat", "z_off"))
    Iref, _ = oracle.interp_batch(Xc, Yc, xo, Zc, zo)
    L = ds.ds_learned_build_xy(_cuda(Xc), _cuda(Yc), _cuda(xo), cfg=ds.ds_learned_cfg_default(steps=20))
    torch.cuda.synchronize()
    base = ds.ds_debug_alloc_stats()
    Zh, zoh = torch.from_numpy(Zc).pin_memory(), torch.from_numpy(zo)
    out = torch.empty(Zc.size, dtype=torch.int32).pin_memory()
    ds.ds_debug_fail_alloc(0)
    try:
        with pytest.raises(ds.DsError) as e:
            ds.ds_learned_search_host(L, Zh, zoh, out=out)
        assert e.value.status == ds.DS_E_NOMEM
    finally:
        ds.ds_debug_fail_alloc(-1)
    assert ds.ds_debug_alloc_stats() == base
    ds.ds_learned_search_host(L, Zh, zoh, out=out)
    np.testing.assert_array_equal(out.numpy(), Iref)
    L.free()


@pytest.mark.parametrize("method", [0, 3])
def test_log_search_build(ds, method):
    g = np.random.default_rng(3)
    X = W.knots_from_gaps(0.0, g.uniform(1, 5, 3000), np.float32)
    Z = W.uniform_queries(g, X[0], X[-1], 5000, np.float32)
    ref = oracle.upper_bound(X, Z)
    _each_failure(ds, lambda: ds.ds_lsearch_build(_cuda(X), method),
                  lambda h: np.testing.assert_array_equal(h.search(_cuda(Z)).cpu().numpy(), ref))
