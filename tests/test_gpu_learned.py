"""GPU tests of the learned form: training kernels against the float64
oracle, exactness of direct search on the learned cell map (every map, every
table format), the recorded bounds, the gain of the trained network over the
network-free map, and the fused interpolation (caller's values and stored
(X, Y) pairs) against its float64 reference."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
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


def _theta(g):
    return (g.normal(0, 0.5, mlp.N_PARAMS)).astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


# ---------------------------------------------------------------- training kernels
@pytest.mark.parametrize("n", [1, 127, 4096, 50_000])
def test_gradient_matches_float64_oracle(ds, n):
    g = np.random.default_rng(n)
    th = _theta(g)
    u = g.uniform(-0.2, 1.2, n).astype(np.float32)
    y = g.uniform(0, 1, n).astype(np.float32)
    loss, grad = ds.ds_mlp_loss_grad(_cuda(th), _cuda(u), _cuda(y))
    loss, grad = float(loss.cpu()[0]), grad.cpu().numpy().astype(np.float64)
    ref_loss, ref_grad = mlp.loss_and_grad(th.astype(np.float64), u.astype(np.float64), y.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-5 * max(abs(ref_loss), 1e-12)
    sl = [(0, 32), (32, 64), (64, 1088), (1088, 1120), (1120, 1152), (1152, 1153)]
    for a, b in sl:  # per tensor, relative L2 error
        if np.linalg.norm(ref_grad[a:b]) > 0:
            assert _rel(grad[a:b], ref_grad[a:b]) <= 1e-4, (n, a, b)


def test_forward_matches_float64_oracle(ds):
    g = np.random.default_rng(5)
    th = _theta(g)
    u = g.uniform(-0.5, 1.5, 100_000).astype(np.float32)
    out = ds.ds_mlp_forward(_cuda(th), _cuda(u)).cpu().numpy()
    ref = mlp.forward(th.astype(np.float64), u.astype(np.float64))
    assert np.max(np.abs(out - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_adam_steps_match_float64_oracle(ds):
    g = np.random.default_rng(6)
    th = _theta(g)
    grads = [g.normal(size=th.size).astype(np.float32) for _ in range(3)]
    tht, m, v = _cuda(th), torch.zeros(th.size, device="cuda"), torch.zeros(th.size, device="cuda")
    rt, rm, rv = th.astype(np.float64), np.zeros(th.size), np.zeros(th.size)
    for t, gr in enumerate(grads, start=1):
        ds.ds_adam_step(tht, m, v, _cuda(gr), t, 1e-3)
        rt, rm, rv = mlp.adam_step(rt, rm, rv, gr.astype(np.float64), t, 1e-3)
    assert np.max(np.abs(tht.cpu().numpy() - rt)) <= 1e-6


# ---------------------------------------------------------------- learned search
def _cfg(ds, **kw):
    base = dict(steps=300, batch=8192, n_queries=1 << 16)
    base.update(kw)
    return ds.ds_learned_cfg_default(**base)


def _learned_small(n_knots=(1 << 18) + 1, m=1 << 20, seed=None):
    # at 2^18+1 knots the two-scale gaps already make R exceed 2^32
    return W.workload4(n_knots=n_knots, m=m, seed=seed)


def _queries(X, Z, dtype):
    inf = dtype(np.inf)
    extra = np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, float(X[0]) - 1.0, float(X[-1]) * 2.0], dtype=dtype)
    return np.concatenate([Z, W.adversarial_queries(X), W.midpoints(X), extra]).astype(dtype)


def _check_cells(ds, L, a, n_knots):
    """The exported table is Eq. indexdef's over some monotone map: K_0 = 0,
    K_C = N + 1, non-decreasing; its largest step and its non-empty cells are
    the recorded statistics, and max_window is the largest step plus one."""
    c = ds.ds_learned_cells(L, a)
    K = ds.ds_learned_export_cells(L, a).cpu().numpy().astype(np.int64)
    assert K.size == c["cells"] + 1
    assert K[0] == 0 and K[-1] == n_knots
    d = np.diff(K)
    assert np.all(d >= 0)
    assert int(d.max()) == c["max_pop"] and int((d > 0).sum()) == c["nonempty"]
    assert c["mean_pop"] == pytest.approx(float((d * d).sum()) / n_knots, rel=1e-12)
    blocks = np.add.reduceat(d, np.arange(0, d.size, 8))  # knots per block of 8 cells
    assert c["escaped"] == int((blocks > 4095).sum())
    return c, K


def test_learned_single_array_is_exact(ds):
    w = _learned_small()
    X = w["X"]
    assert oracle.compute_hr(X)["status"] == oracle.OR_E_OVERFLOW  # plain direct search infeasible
    Z = _queries(X, w["Z"], np.float64)
    L = ds.ds_learned_build(_cuda(X), cfg=_cfg(ds))
    info = L.info()
    assert info["n_learned"] == 1 and info["n_direct"] == 0
    arr = ds.ds_learned_array(L, 0)
    assert arr["mode"] == 1 and arr["e_lo"] >= 0 and arr["e_hi"] >= 0
    got = L.search(_cuda(Z)).cpu().numpy()
    assert np.array_equal(got, oracle.upper_bound(X, Z))
    c, _ = _check_cells(ds, L, 0, X.size)
    assert info["max_window"] == c["max_pop"] + 1 and info["fallback_queries"] == 0
    assert c["cells"] == X.size  # the default: one cell per knot
    L.free()


def test_default_cells_per_knot(ds):
    # the default map has one cell per knot, two on a handle that holds the
    # knot values (ds_learned_build_xy with Y); an explicit value is kept
    g = np.random.default_rng(33)
    X = W.knots_from_gaps(0.0, g.lognormal(0, 1, 3000), np.float32)
    Y = g.standard_normal(X.size).astype(np.float32)
    Z = W.uniform_queries(g, X[0], X[-1], 20_000, np.float32)
    Ir, yr = oracle.interp(X, Y, Z)
    for with_y, cpk, want in ((False, 0.0, X.size), (True, 0.0, 2 * X.size), (True, 1.0, X.size)):
        cfg = _cfg(ds, steps=100, flags=ds.DS_LEARNED_FORCE, cells_per_knot=cpk)
        L = (ds.ds_learned_build_xy(_cuda(X), _cuda(Y), cfg=cfg) if with_y
             else ds.ds_learned_build(_cuda(X), cfg=cfg))
        c, _ = _check_cells(ds, L, 0, X.size)
        assert c["cells"] == want
        if with_y:
            I, y = L.search(_cuda(Z), y_out=torch.empty(Z.size, dtype=torch.float32, device="cuda"))
            I, y = I.cpu().numpy(), y.cpu().numpy()
            ok = (Ir >= 0) & (Ir < X.size - 1)
            assert np.array_equal(I, Ir) and np.all(_interp_tol(y[ok], yr[ok], Y[Ir[ok]], Y[Ir[ok] + 1]))
        else:
            assert np.array_equal(L.search(_cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
        L.free()


@pytest.mark.parametrize("cpk,linear,steps", [(1.0, True, 300), (0.01, False, 0), (0.0004, True, 0), (4.0, False, 300)])
def test_every_cell_map_is_exact(ds, cpk, linear, steps):
    # any non-decreasing map gives exact answers: the linear map, the untrained
    # network, cells holding thousands of knots (escaped blocks: more than 4095
    # knots in 8 cells), and four cells per knot
    w = _learned_small(n_knots=200_001, m=300_000, seed=77)
    X = w["X"]
    Z = _queries(X, w["Z"], np.float64)
    flags = ds.DS_LEARNED_FORCE | (ds.DS_LEARNED_LINEAR if linear else 0)
    L = ds.ds_learned_build(_cuda(X), cfg=_cfg(ds, steps=steps, flags=flags, cells_per_knot=cpk))
    c, _ = _check_cells(ds, L, 0, X.size)
    assert (c["escaped"] > 0) == (cpk < 0.001)
    assert np.array_equal(L.search(_cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    L.free()


def _bumps(n, seed):
    """Knots whose density varies at scales the network can follow: eight
    narrow bumps of different widths over a sparse background (float64)."""
    g = np.random.default_rng(seed)
    parts = [g.uniform(0.0, 1.0, n // 5)]
    for k in range(8):
        parts.append(g.normal(0.06 + 0.12 * k, 10.0 ** g.uniform(-3, -2), (n - n // 5) // 8))
    X = np.unique(np.concatenate(parts))
    return W.strictly_increasing(X)


def _time(fn, reps=20):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(3):
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / reps)
    return best


def test_trained_network_beats_the_model_without_it(ds):
    # on knots whose density varies at scales the network follows, cells of
    # equal predicted rank hold fewer knots than cells of equal width, so
    # fewer lookups compare and bisect: the same exact answers, a smaller mean
    # cell population, less time
    X = _bumps(1 << 20, 3)
    g = np.random.default_rng(4)
    mids = W.midpoints(X)
    Z = mids[g.integers(0, mids.size, 1 << 24)]  # queries distributed like the knots (the paper's harness)
    Xd, Zd = _cuda(X), _cuda(Z)
    trained = ds.ds_learned_build(Xd, cfg=_cfg(ds, steps=6000, flags=ds.DS_LEARNED_FORCE))
    linear = ds.ds_learned_build(Xd, cfg=_cfg(ds, flags=ds.DS_LEARNED_LINEAR | ds.DS_LEARNED_FORCE))
    ct = _check_cells(ds, trained, 0, X.size)[0]
    cl = _check_cells(ds, linear, 0, X.size)[0]
    assert ct["from_network"] == 1 and cl["from_network"] == 0
    assert ct["mean_pop"] * 2 < cl["mean_pop"], (ct, cl)
    ref = oracle.upper_bound(X, Z[: 1 << 20])
    out_t, out_l = trained.search(Zd), linear.search(Zd)
    assert np.array_equal(out_t[: 1 << 20].cpu().numpy(), ref)
    assert torch.equal(out_t, out_l)
    ds.ds_learned_autotune(trained, Zd)
    ds.ds_learned_autotune(linear, Zd)
    t_t = _time(lambda: trained.search(Zd, out=out_t))
    t_l = _time(lambda: linear.search(Zd, out=out_l))
    assert t_t * 1.15 < t_l, (t_t, t_l, ct, cl)
    trained.free()
    linear.free()


def test_map_choice_never_worse_than_linear(ds):
    # the build keeps the network's map only where its cells are better balanced
    w = _learned_small(n_knots=(1 << 20) + 1, m=1 << 16, seed=5)
    Xd = _cuda(w["X"])
    trained = ds.ds_learned_build(Xd, cfg=_cfg(ds, flags=ds.DS_LEARNED_FORCE))
    linear = ds.ds_learned_build(Xd, cfg=_cfg(ds, flags=ds.DS_LEARNED_LINEAR | ds.DS_LEARNED_FORCE))
    ct, cl = ds.ds_learned_cells(trained, 0), ds.ds_learned_cells(linear, 0)
    assert ct["mean_pop"] <= cl["mean_pop"]
    assert (ct["from_network"] == 1) == (ct["mean_pop"] < cl["mean_pop"])
    trained.free()
    linear.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_forced_learned_on_feasible_arrays(ds, dtype):
    g = np.random.default_rng(8)
    X = W.knots_from_gaps(-5.0, g.lognormal(0, 1, 30_000), dtype)
    Z = _queries(X, W.uniform_queries(g, X[0], X[-1], 100_000, dtype), dtype)
    L = ds.ds_learned_build(_cuda(X), cfg=_cfg(ds, flags=ds.DS_LEARNED_FORCE))
    assert L.info()["n_learned"] == 1
    assert np.array_equal(L.search(_cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    L.free()


# ---------------------------------------------------------------- batched learned + interpolation
def _interp_tol(y, y64, Y0, Y1):
    scale = np.maximum(np.abs(y64), np.maximum(np.abs(Y0), np.abs(Y1)))
    return np.abs(y.astype(np.float64) - y64) <= 1e-6 * scale


def test_batched_learned_with_interpolation(ds):
    w = W.workload5(n_arrays=24, size_lo=1 << 10, size_hi=1 << 17, total_queries=1 << 21)
    Xcat, Ycat, x_off, Zcat, z_off = w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"], w["z_off"]
    # default selector: direct search exactly where ComputeHR succeeds with at
    # most max_cells_per_knot cells per knot
    cfg = _cfg(ds, steps=50)
    Ld = ds.ds_learned_build(_cuda(Xcat), _cuda(x_off), cfg=cfg)
    modes = []
    for a in range(24):
        Xa = Xcat[x_off[a]:x_off[a + 1]]
        hr = oracle.compute_hr(Xa)
        direct = hr["status"] == oracle.OR_OK and hr["R"] + 1 <= cfg.max_cells_per_knot * Xa.size
        modes.append(ds.ds_learned_array(Ld, a)["mode"])
        assert modes[-1] == (0 if direct else 1), a
    assert 0 in modes and 1 in modes
    Id, yd = Ld.search(_cuda(Zcat), _cuda(z_off), Y=_cuda(Ycat))
    Ld.free()
    Iref, yref = oracle.interp_batch(Xcat, Ycat, x_off, Zcat, z_off)
    arr = np.searchsorted(z_off, np.arange(Zcat.size), side="right") - 1
    gi = x_off[arr] + Iref
    for flags, cpk in ((ds.DS_LEARNED_FORCE, 1.0), (0, 1.0), (0, 0.05), (ds.DS_LEARNED_FORCE, 0.05)):
        # every array through the learned map, then the default selector, and
        # with about 20 knots per learned cell (queries past a cell's second
        # knot bisect it); the handle holds its values as intervals
        L = ds.ds_learned_build_xy(_cuda(Xcat), _cuda(Ycat), _cuda(x_off),
                                   cfg=_cfg(ds, steps=50, flags=flags, cells_per_knot=cpk))
        if flags & ds.DS_LEARNED_FORCE:
            assert L.info()["n_learned"] == 24
        y = torch.empty(Zcat.size, dtype=torch.float32, device="cuda")
        I, _ = L.search(_cuda(Zcat), _cuda(z_off), y_out=y)
        I, y = I.cpu().numpy(), y.cpu().numpy()
        assert np.array_equal(I, Iref)
        assert np.array_equal(Id.cpu().numpy(), Iref)
        # the same rounding steps whichever way the values are read
        assert np.array_equal(yd.cpu().numpy(), y, equal_nan=True)
        assert np.all(_interp_tol(y, yref, Ycat[gi], Ycat[gi + 1]))
        # at a knot the interpolant is the knot value exactly
        Zk = np.concatenate([Xcat[x_off[a]:x_off[a + 1] - 1] for a in range(24)])
        zk_off = W.csr(np.diff(x_off) - 1)
        yk = torch.empty(Zk.size, dtype=torch.float32, device="cuda")
        Ik, _ = L.search(_cuda(Zk), _cuda(zk_off), y_out=yk)
        assert np.array_equal(Ik.cpu().numpy(), np.concatenate([np.arange(n - 1) for n in np.diff(x_off)]))
        ref_yk = np.concatenate([Ycat[x_off[a]:x_off[a + 1] - 1] for a in range(24)])
        assert np.array_equal(yk.cpu().numpy(), ref_yk)
        # a handle that holds its values refuses the caller's
        with pytest.raises((ds.DsError, ValueError)):
            L.search(_cuda(Zcat), _cuda(z_off), Y=_cuda(Ycat))
        L.free()


@pytest.mark.parametrize("cpk", [1.0, 0.02])
def test_interpolation_misaligned_and_out_of_domain(ds, cpk):
    # the scalar path (buffers off 16-byte alignment) and queries outside
    # [X_0, X_N): NaN values, indices -1 and N
    g = np.random.default_rng(21)
    X = W.knots_from_gaps(0.0, g.lognormal(0, 1, 5000), np.float32)
    Y = g.standard_normal(X.size).astype(np.float32)
    Z = np.concatenate([W.uniform_queries(g, X[0], X[-1], 10_001, np.float32),
                        np.array([X[0] - 1, X[-1], X[-1] + 1, X[0]], dtype=np.float32)])
    L = ds.ds_learned_build_xy(_cuda(X), _cuda(Y), cfg=_cfg(ds, flags=ds.DS_LEARNED_FORCE, cells_per_knot=cpk))
    zb = torch.zeros(Z.size + 1, dtype=torch.float32, device="cuda")
    zb[1:] = _cuda(Z)
    ob = torch.zeros(Z.size + 1, dtype=torch.int32, device="cuda")
    yb = torch.zeros(Z.size + 1, dtype=torch.float32, device="cuda")
    L.search(zb[1:], out=ob[1:], y_out=yb[1:])
    Ir, yr = oracle.interp(X, Y, Z)
    I, y = ob[1:].cpu().numpy(), yb[1:].cpu().numpy()
    assert np.array_equal(I, Ir)
    ok = (Ir >= 0) & (Ir < X.size - 1)
    assert np.all(np.isnan(y[~ok])) and np.all(~np.isnan(y[ok]))
    assert np.all(_interp_tol(y[ok], yr[ok], Y[Ir[ok]], Y[Ir[ok] + 1]))
    L.free()


@pytest.mark.parametrize("pinned", [True, False])
def test_search_host_buffers(ds, pinned):
    # the end-to-end call: queries, indices and interpolated values in host
    # memory (page-locked used in place, pageable registered for the call),
    # the same results as the device search
    w = W.workload5(n_arrays=16, size_lo=1 << 10, size_hi=1 << 16, total_queries=1 << 20)
    Xcat, Ycat, x_off, Zcat, z_off = w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"], w["z_off"]
    L = ds.ds_learned_build_xy(_cuda(Xcat), _cuda(Ycat), _cuda(x_off), cfg=_cfg(ds, steps=50))
    yd = torch.empty(Zcat.size, dtype=torch.float32, device="cuda")
    Id, _ = L.search(_cuda(Zcat), _cuda(z_off), y_out=yd)
    Zh = torch.from_numpy(Zcat)
    Ih = torch.full((Zcat.size,), -7, dtype=torch.int32)
    yh = torch.full((Zcat.size,), -7.0, dtype=torch.float32)
    if pinned:
        Zh, Ih, yh = Zh.pin_memory(), Ih.pin_memory(), yh.pin_memory()
    for _ in range(2):
        ds.ds_learned_search_host(L, Zh, torch.from_numpy(z_off), out=Ih, y_out=yh)
        assert torch.equal(Ih, Id.cpu())
        assert torch.equal(yh, yd.cpu())
    # index only, one array
    w4 = _learned_small(n_knots=20_001, m=100_003)
    L4 = ds.ds_learned_build(_cuda(w4["X"]), cfg=_cfg(ds, flags=ds.DS_LEARNED_FORCE))
    I4 = ds.ds_learned_search_host(L4, torch.from_numpy(w4["Z"]))
    assert np.array_equal(I4.numpy(), oracle.upper_bound(w4["X"], w4["Z"]))
    with pytest.raises(ds.DsError):  # interpolation needs a handle that holds its values
        ds.ds_learned_search_host(L4, torch.from_numpy(w4["Z"]), y_out=torch.empty(w4["Z"].size, dtype=torch.float64))
    L.free()
    L4.free()


@pytest.mark.slow
def test_workload4_full_size(ds):
    w = W.workload4()
    X, Z = w["X"], w["Z"]
    Xd, Zd = _cuda(X), _cuda(Z)
    L = ds.ds_learned_build(Xd, cfg=ds.ds_learned_cfg_default(n_queries=1 << 20))
    out = L.search(Zd)
    g = np.random.default_rng(13)
    pos = np.concatenate([g.integers(0, Z.size, 1 << 20), np.arange(1000)])
    assert np.array_equal(out[_cuda(pos)].cpu().numpy(), oracle.upper_bound(X, Z[pos]))
    gl = out.long()
    assert bool((gl >= 0).all()) and bool((gl <= X.size - 2).all())
    assert bool((Xd[gl] <= Zd).all()) and bool((Zd < Xd[gl + 1]).all())
    _check_cells(ds, L, 0, X.size)
    L.free()


@pytest.mark.slow
def test_workload5_full_size(ds):
    w = W.workload5()
    Xcat, Ycat, x_off, Zcat, z_off = w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"], w["z_off"]
    Xd, Yd, xo, Zd, zo = _cuda(Xcat), _cuda(Ycat), _cuda(x_off), _cuda(Zcat), _cuda(z_off)
    L = ds.ds_learned_build_xy(Xd, Yd, xo)
    y = torch.empty_like(Zd)
    I, _ = L.search(Zd, zo, y_out=y)
    g = np.random.default_rng(14)
    pos = np.sort(g.integers(0, Zcat.size, 1 << 20))
    arr = np.searchsorted(z_off, pos, side="right") - 1
    Is, ys = I[_cuda(pos)].cpu().numpy(), y[_cuda(pos)].cpu().numpy()
    for a in np.unique(arr):
        sel = arr == a
        Xa, Ya = Xcat[x_off[a]:x_off[a + 1]], Ycat[x_off[a]:x_off[a + 1]]
        Ir, yr = oracle.interp(Xa, Ya, Zcat[pos[sel]])
        assert np.array_equal(Is[sel], Ir), a
        assert np.all(_interp_tol(ys[sel], yr, Ya[Ir], Ya[Ir + 1])), a
    # every position: the index by the defining invariant X_I <= z < X_{I+1},
    # then y against the interpolant restated in float64 on those exact indices
    arr_all = torch.searchsorted(zo, torch.arange(Zd.numel(), device="cuda"), right=True) - 1
    gi = xo[arr_all] + I.long()
    del arr_all
    assert bool((Xd[gi] <= Zd).all()) and bool((Zd < Xd[gi + 1]).all())
    x0, x1 = Xd[gi].double(), Xd[gi + 1].double()
    y0, y1 = Yd[gi].double(), Yd[gi + 1].double()
    y64 = y0 + (y1 - y0) * ((Zd.double() - x0) / (x1 - x0))
    scale = torch.maximum(y64.abs(), torch.maximum(y0.abs(), y1.abs()))
    assert bool(((y.double() - y64).abs() <= 1e-6 * scale).all())
    L.free()


def test_autotuned_learned_stays_exact(ds):
    # the autotuner tries every launch configuration (block and warp claims,
    # staging limits) on these queries; the answers of the one it keeps, and of
    # the batched interpolating form after its own tuning, stay exact
    w = _learned_small(n_knots=50_001, m=400_000)
    X, Z = w["X"], _queries(w["X"], w["Z"], np.float64)
    L = ds.ds_learned_build(_cuda(X), cfg=_cfg(ds, flags=ds.DS_LEARNED_FORCE))
    tune = ds.ds_learned_autotune(L, _cuda(Z))
    assert tune["block"] in (128, 256, 512) and tune["ms"] > 0
    assert np.array_equal(L.search(_cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    L.free()
    w5 = W.workload5(n_arrays=24, size_lo=1 << 10, size_hi=1 << 16, total_queries=1 << 20)
    Xcat, Ycat, x_off, Zcat, z_off = w5["Xcat"], w5["Ycat"], w5["x_off"], w5["Zcat"], w5["z_off"]
    L5 = ds.ds_learned_build_xy(_cuda(Xcat), _cuda(Ycat), _cuda(x_off), cfg=_cfg(ds, steps=50))
    y = torch.empty(Zcat.size, dtype=torch.float32, device="cuda")
    ds.ds_learned_autotune(L5, _cuda(Zcat), _cuda(z_off), y_out=y)
    I, _ = L5.search(_cuda(Zcat), _cuda(z_off), y_out=y)
    Iref, yref = oracle.interp_batch(Xcat, Ycat, x_off, Zcat, z_off)
    assert np.array_equal(I.cpu().numpy(), Iref)
    arr = np.searchsorted(z_off, np.arange(Zcat.size), side="right") - 1
    gi = x_off[arr] + Iref
    assert np.all(_interp_tol(y.cpu().numpy(), yref, Ycat[gi], Ycat[gi + 1]))
    L5.free()


def test_learned_set_tune_every_configuration_exact(ds):
    w = _learned_small(n_knots=50_001, m=100_000)
    X, Z = w["X"], _queries(w["X"], w["Z"], np.float64)
    ref = oracle.upper_bound(X, Z)
    L = ds.ds_learned_build(_cuda(X), cfg=_cfg(ds))
    for block, items, smem in ((512, 1, 0), (256, 2, -1), (128, 4, 48 * 1024), (1024, 1, 0)):
        ds.ds_learned_set_tune(L, block, items, smem)
        t = ds.ds_learned_get_tune(L)
        assert (t["items"], t["smem_limit"]) == (items, smem)
        assert np.array_equal(L.search(_cuda(Z)).cpu().numpy(), ref), (block, items, smem)
    with pytest.raises(ds.DsError):
        ds.ds_learned_set_tune(L, 256, 1, -2)
    L.free()


def test_split_handle_every_configuration_exact(ds):
    # a handle with direct and learned arrays searches each group with its own
    # launch: every configuration, set for both launches, and the autotuner's
    # own pair of configurations, stay exact, with and without the interpolation
    w5 = W.workload5(n_arrays=20, size_lo=1 << 10, size_hi=1 << 15, total_queries=1 << 19)
    Xcat, Ycat, x_off, Zcat, z_off = w5["Xcat"], w5["Ycat"], w5["x_off"], w5["Zcat"], w5["z_off"]
    L = ds.ds_learned_build_xy(_cuda(Xcat), _cuda(Ycat), _cuda(x_off), cfg=_cfg(ds, steps=50))
    info = L.info()
    assert info["n_direct"] > 0 and info["n_learned"] > 0 and info["search_launches"] == 3
    Iref, yref = oracle.interp_batch(Xcat, Ycat, x_off, Zcat, z_off)
    arr = np.searchsorted(z_off, np.arange(Zcat.size), side="right") - 1
    gi = x_off[arr] + Iref
    Zd, zod = _cuda(Zcat), _cuda(z_off)
    y = torch.empty(Zcat.size, dtype=torch.float32, device="cuda")
    for block, items, smem in ((512, 1, 0), (256, 2, -1), (128, 4, 48 * 1024), (1024, 1, 96 * 1024)):
        ds.ds_learned_set_tune(L, block, items, smem)
        I, _ = L.search(Zd, zod, y_out=y)
        assert np.array_equal(I.cpu().numpy(), Iref), (block, items, smem)
        assert np.all(_interp_tol(y.cpu().numpy(), yref, Ycat[gi], Ycat[gi + 1])), (block, items, smem)
        assert np.array_equal(L.search(Zd, zod).cpu().numpy(), Iref), (block, items, smem)
    tune = ds.ds_learned_autotune(L, Zd, zod, y_out=y)
    assert tune["ms"] > 0
    I, _ = L.search(Zd, zod, y_out=y)
    assert np.array_equal(I.cpu().numpy(), Iref)
    assert np.all(_interp_tol(y.cpu().numpy(), yref, Ycat[gi], Ycat[gi + 1]))
    L.free()
