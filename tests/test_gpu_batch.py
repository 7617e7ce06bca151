"""GPU parity of the batched ragged path (ds_batch_build / ds_batch_search).

Every array's H, W, R must equal the oracle's ComputeHR on that array alone,
and every local index the definition, bit-exactly, for every launch
configuration the autotuner can pick."""
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


def _small(seed=None, n_arrays=64, size_hi=4096, total=1 << 20):
    return W.workload3(n_arrays=n_arrays, size_hi=size_hi, total_queries=total, seed=seed)


def _check_params(ds, b, w, fma):
    x_off = w["x_off"]
    for a in range(len(x_off) - 1):
        X = w["Xcat"][x_off[a]:x_off[a + 1]]
        hr = oracle.compute_hr(X, fma)
        p = ds.ds_batch_array(b, a)
        if hr["status"] == oracle.OR_OK:
            assert p["mode"] == 0 and p["H"] == hr["H"] and p["R"] == hr["R"], a
            if fma:
                assert p["W"] == hr["W"], a
        else:
            assert p["mode"] == 2, a


@pytest.mark.parametrize("fma", [False, True])
def test_small_batch_all_tunings(ds, fma):
    w = _small()
    Xd, xo, Zd, zo = _cuda(w["Xcat"]), _cuda(w["x_off"]), _cuda(w["Zcat"]), _cuda(w["z_off"])
    b = ds.ds_batch_build(Xd, xo, ds.DS_FMA if fma else 0)
    _check_params(ds, b, w, fma)
    ref = oracle.upper_bound_batch(w["Xcat"], w["x_off"], w["Zcat"], w["z_off"])
    for block in (128, 256, 512, 1024):
        for items in (1, 2, 4):
            for smem in (-1, 0, 24 * 1024, 96 * 1024):
                ds.ds_batch_set_tune(b, block, items, smem)
                out = ds.ds_batch_search(b, Zd, zo)
                got = out.cpu().numpy()
                assert np.array_equal(got, ref), (block, items, smem, int(np.count_nonzero(got != ref)))
    b.free()


def test_infeasible_arrays_fall_back_and_strict_fails(ds):
    g = np.random.default_rng(4)
    arrays = [np.array([-1e9, 0.0, 1.0], dtype=np.float32),            # indistinguishable
              np.array([0.0, 1.42e-45, 1.0], dtype=np.float32),         # overflow
              W.knots_from_gaps(3.0, g.uniform(0.5, 1.5, 500), np.float32),
              np.array([-2.0, 5.0], dtype=np.float32)]
    x_off = W.csr([a.size for a in arrays])
    Xcat = np.concatenate(arrays)
    Zs = []
    for a in arrays:
        inf = np.float32(np.inf)
        Zs.append(np.concatenate([W.adversarial_queries(a), W.uniform_queries(g, a[0], a[-1], 999, np.float32),
                                  np.array([a[-1], -inf, inf, np.nextafter(a[0], -inf)], dtype=np.float32)]))
    z_off = W.csr([z.size for z in Zs])
    Zcat = np.concatenate(Zs)
    b = ds.ds_batch_build(_cuda(Xcat), _cuda(x_off))
    info = b.info()
    assert info["n_fallback"] == 2 and info["n_direct"] == 2
    assert [ds.ds_batch_array(b, a)["mode"] for a in range(4)] == [2, 2, 0, 0]
    got = ds.ds_batch_search(b, _cuda(Zcat), _cuda(z_off)).cpu().numpy()
    assert np.array_equal(got, oracle.upper_bound_batch(Xcat, x_off, Zcat, z_off))
    b.free()
    with pytest.raises(ds.DsError):
        ds.ds_batch_build(_cuda(Xcat), _cuda(x_off), ds.DS_STRICT)


def test_empty_arrays_of_queries_and_misalignment(ds):
    w = _small(n_arrays=40, size_hi=3000, total=100_003)
    q = np.diff(w["z_off"])
    q[::3] = 0  # arrays without queries
    z_off = W.csr(q)
    Zcat = np.concatenate([w["Zcat"][w["z_off"][a]:w["z_off"][a] + q[a]] for a in range(len(q))])
    ref = oracle.upper_bound_batch(w["Xcat"], w["x_off"], Zcat, z_off)
    b = ds.ds_batch_build(_cuda(w["Xcat"]), _cuda(w["x_off"]))
    Zsrc = _cuda(Zcat)
    for zo_, io_ in ((0, 0), (1, 0), (0, 3), (3, 1)):
        buf = torch.zeros(Zcat.size + 4, dtype=torch.float32, device="cuda")
        buf[zo_:zo_ + Zcat.size] = Zsrc
        z = buf[zo_:zo_ + Zcat.size]  # data pointer offset by zo_ elements
        outb = torch.full((Zcat.size + io_,), -9, dtype=torch.int32, device="cuda")
        ds.ds_batch_search(b, z, _cuda(z_off), outb[io_:])
        o = outb.cpu().numpy()
        assert np.array_equal(o[io_:], ref), (zo_, io_)
        assert np.all(o[:io_] == -9)
    b.free()


def test_checked_nan_batched(ds):
    X = np.linspace(-1, 1, 101).astype(np.float32)
    Xcat = np.concatenate([X, X * 2])
    x_off = np.array([0, 101, 202])
    Zcat = np.array([np.nan, 0.0, 3.0, np.nan, -5.0], dtype=np.float32)
    z_off = np.array([0, 3, 5])
    b = ds.ds_batch_build(_cuda(Xcat), _cuda(x_off), ds.DS_CHECKED)
    assert list(ds.ds_batch_search(b, _cuda(Zcat), _cuda(z_off)).cpu().numpy()) == [-1, 50, 100, -1, -1]
    b.free()


def test_repeated_calls_and_graph_reuse(ds):
    w = _small(n_arrays=32, size_hi=2048, total=300_000)
    ref = oracle.upper_bound_batch(w["Xcat"], w["x_off"], w["Zcat"], w["z_off"])
    b = ds.ds_batch_build(_cuda(w["Xcat"]), _cuda(w["x_off"]))
    Zd, zo = _cuda(w["Zcat"]), _cuda(w["z_off"])
    out = torch.empty(Zd.numel(), dtype=torch.int32, device="cuda")
    for _ in range(3):
        out.fill_(-3)
        ds.ds_batch_search(b, Zd, zo, out)
        assert np.array_equal(out.cpu().numpy(), ref)
    # captured inside the caller's own graph
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ds.ds_batch_search(b, Zd, zo, out)
    out.fill_(-3)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
    b.free()


@pytest.mark.slow
def test_workload3_full_size_autotuned(ds):
    w = W.workload3()
    Xd, xo, Zd, zo = _cuda(w["Xcat"]), _cuda(w["x_off"]), _cuda(w["Zcat"]), _cuda(w["z_off"])
    b = ds.ds_batch_build(Xd, xo)
    info = b.info()
    assert info["n_direct"] == 4096 and info["n_fallback"] == 0
    best = ds.ds_batch_autotune(b, Zd, zo)
    assert best["ms"] > 0 and best["block"] in (128, 256, 512, 1024)
    out = ds.ds_batch_search(b, Zd, zo)
    # sampled exact check against the oracle, one by one per array
    g = np.random.default_rng(12)
    pos = np.sort(np.concatenate([g.integers(0, w["Zcat"].size, 1 << 20), w["z_off"][1:-1] - 1, w["z_off"][:-1]]))
    arr = np.searchsorted(w["z_off"], pos, side="right") - 1
    got = out[_cuda(pos)].cpu().numpy()
    for a in np.unique(arr):
        sel = arr == a
        X = w["Xcat"][w["x_off"][a]:w["x_off"][a + 1]]
        assert np.array_equal(got[sel], oracle.upper_bound(X, w["Zcat"][pos[sel]])), a
    # the defining invariant at every position, on the device
    arr_all = torch.searchsorted(zo, torch.arange(Zd.numel(), device="cuda"), right=True) - 1
    base = xo[arr_all]
    gi = base + out.long()
    assert bool((out >= 0).all())
    assert bool((gi + 1 < xo[arr_all + 1]).all())
    assert bool((Xd[gi] <= Zd).all()) and bool((Zd < Xd[gi + 1]).all())
    b.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_fingerprints_across_cell_ranges(ds, dtype, fma):
    # arrays whose largest cell R spans every exponent range of f(z): fractional
    # bits below 2^17 cells, fewer of them up to 2^24, none above (float32)
    g = np.random.default_rng(21)
    arrays = []
    for cells_per_knot, n in ((3, 100), (40, 2000), (200, 3000), (2000, 4000), (20000, 2000), (2e5, 1000)):
        X0 = 0.0 if len(arrays) % 2 == 0 else g.uniform(-1e3, 1e3)
        gaps = g.uniform(0.5, 1.5, n - 1)
        gaps[g.integers(0, n - 1)] = 1.0 / cells_per_knot  # one narrow gap sets H
        arrays.append(W.knots_from_gaps(X0, gaps, dtype))
    x_off = W.csr([a.size for a in arrays])
    Xcat = np.concatenate(arrays)
    Zs = []
    for a in arrays:
        inf = dtype(np.inf)
        Zs.append(np.concatenate([W.adversarial_queries(a), W.midpoints(a), W.uniform_queries(g, a[0], a[-1], 20000, dtype),
                                  np.array([a[-1], -inf, inf, np.nextafter(a[0], -inf), a[-1] * 2 + 1], dtype=dtype)]))
    z_off = W.csr([z.size for z in Zs])
    Zcat = np.concatenate(Zs)
    ref = oracle.upper_bound_batch(Xcat, x_off, Zcat, z_off)
    flags = ds.DS_FMA if fma else 0
    Rs = []
    for extra in (0, ds.DS_NO_FINGERPRINT):
        b = ds.ds_batch_build(_cuda(Xcat), _cuda(x_off), flags | extra)
        Rs = [ds.ds_batch_array(b, a)["R"] for a in range(len(arrays))]
        for smem in (-1, 0, 96 * 1024):
            ds.ds_batch_set_tune(b, 256, 4, smem)
            got = ds.ds_batch_search(b, _cuda(Zcat), _cuda(z_off)).cpu().numpy()
            assert np.array_equal(got, ref), (extra, smem, int(np.count_nonzero(got != ref)))
        b.free()
    assert max(Rs) > (1 << 24) and min(Rs) < (1 << 10)


def test_many_arrays_claim_order_and_long_chunks(ds):
    # more arrays than the planner's register rounds (8 x 1024), sizes spanning
    # three decades so the claim order (most knots first) differs from the CSR
    # order, a few arrays without queries, and staged images long enough that
    # their chunks are several base chunks long
    g = np.random.default_rng(31)
    n_arrays = 9000
    sizes = np.maximum(2, np.exp(g.uniform(np.log(2), np.log(3000), n_arrays))).astype(np.int64)
    sizes[g.integers(0, n_arrays, 3)] = 60000
    arrays = [W.knots_from_gaps(g.uniform(-5, 5), g.uniform(0.5, 1.5, int(n) - 1), np.float32) for n in sizes]
    x_off = W.csr(sizes)
    Xcat = np.concatenate(arrays)
    q = (sizes * 3).astype(np.int64)
    q[g.integers(0, n_arrays, 50)] = 0
    Zs = [W.uniform_queries(g, a[0], a[-1], int(k), np.float32) for a, k in zip(arrays, q)]
    z_off = W.csr(q)
    Zcat = np.concatenate(Zs)
    ref = oracle.upper_bound_batch(Xcat, x_off, Zcat, z_off)
    b = ds.ds_batch_build(_cuda(Xcat), _cuda(x_off))
    for block, items, smem in ((512, 1, 96 * 1024), (1024, 1, 136 * 1024), (256, 2, 0), (512, 1, -1)):
        ds.ds_batch_set_tune(b, block, items, smem)
        got = ds.ds_batch_search(b, _cuda(Zcat), _cuda(z_off)).cpu().numpy()
        assert np.array_equal(got, ref), (block, items, smem, int(np.count_nonzero(got != ref)))
    b.free()


def test_array_near_the_32_bit_cell_limit(ds):
    # one narrow gap among unit gaps sets R = trunc(H D_N) close to 2^32: about
    # 1 GB of rank words, built by warps whose cell spans hold millions of
    # groups, and searched through L1 (no shared-memory limit holds it)
    g = np.random.default_rng(41)
    gaps = np.ones(999)
    gaps[500] = 2.6e-7
    big = W.knots_from_gaps(-3.0, gaps, np.float64)
    small = W.knots_from_gaps(5.0, g.uniform(0.5, 1.5, 300), np.float64)
    hr = oracle.compute_hr(big)
    assert hr["status"] == oracle.OR_OK and 3.0e9 < hr["R"] < 2 ** 32
    x_off = W.csr([big.size, small.size])
    Xcat = np.concatenate([big, small])
    Zs = []
    for a in (big, small):
        Zs.append(np.concatenate([W.adversarial_queries(a), W.midpoints(a), W.uniform_queries(g, a[0], a[-1], 200_000, np.float64),
                                  np.array([np.nextafter(a[0], -np.inf), a[-1], a[-1] + 1.0])]))
    z_off = W.csr([z.size for z in Zs])
    Zcat = np.concatenate(Zs)
    ref = oracle.upper_bound_batch(Xcat, x_off, Zcat, z_off)
    b = ds.ds_batch_build(_cuda(Xcat), _cuda(x_off))
    p = ds.ds_batch_array(b, 0)
    assert p["mode"] == 0 and p["R"] == hr["R"] and p["H"] == hr["H"]
    for block, items, smem in ((512, 1, 96 * 1024), (256, 2, 0)):
        ds.ds_batch_set_tune(b, block, items, smem)
        got = ds.ds_batch_search(b, _cuda(Zcat), _cuda(z_off)).cpu().numpy()
        assert np.array_equal(got, ref), (block, items, smem, int(np.count_nonzero(got != ref)))
    b.free()
