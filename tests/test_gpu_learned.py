"""GPU tests of the learned form: training kernels against the float64
oracle, exactness of the learned search (window + certificate + fall-back),
the recorded error bound, the gain over the network-free model, and the
fused interpolation against its float64 reference."""
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


def test_learned_single_array_is_exact_and_bound_holds(ds):
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
    # the recorded bound covers every knot and the top of every interval: no
    # certificate may fail on those queries
    f0 = L.info()["fallback_queries"]
    probes = np.concatenate([X[:-1], np.nextafter(X[1:], -np.inf)])
    got = L.search(_cuda(probes)).cpu().numpy()
    assert np.array_equal(got, oracle.upper_bound(X, probes))
    assert L.info()["fallback_queries"] == f0
    L.free()


def test_zero_bound_forces_the_certificate_and_stays_exact(ds):
    w = _learned_small(n_knots=20_001, m=200_000)
    X, Z = w["X"], _queries(w["X"], w["Z"], np.float64)
    L = ds.ds_learned_build(_cuda(X), cfg=_cfg(ds, flags=ds.DS_LEARNED_ZERO_BOUND | ds.DS_LEARNED_FORCE))
    got = L.search(_cuda(Z)).cpu().numpy()
    assert np.array_equal(got, oracle.upper_bound(X, Z))
    assert L.info()["fallback_queries"] > 0
    L.free()


def test_trained_network_beats_the_model_without_it(ds):
    w = _learned_small()
    X = w["X"]
    Xd = _cuda(X)
    trained = ds.ds_learned_build(Xd, cfg=_cfg(ds, steps=600))
    linear = ds.ds_learned_build(Xd, cfg=_cfg(ds, flags=ds.DS_LEARNED_LINEAR))
    ti, li = trained.info(), linear.info()
    # the recorded window (max error over all knots) shrinks
    assert ti["max_window"] < li["max_window"], (ti["max_window"], li["max_window"])
    Z = _cuda(w["Z"])
    assert torch.equal(trained.search(Z), linear.search(Z))
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
    # every array through the learned predictor
    L = ds.ds_learned_build(_cuda(Xcat), _cuda(x_off), cfg=_cfg(ds, flags=ds.DS_LEARNED_FORCE))
    info = L.info()
    assert info["n_learned"] == 24
    I, y = L.search(_cuda(Zcat), _cuda(z_off), Y=_cuda(Ycat))
    I, y = I.cpu().numpy(), y.cpu().numpy()
    Iref, yref = oracle.interp_batch(Xcat, Ycat, x_off, Zcat, z_off)
    assert np.array_equal(I, Iref)
    assert np.array_equal(Id.cpu().numpy(), Iref)
    assert np.array_equal(yd.cpu().numpy(), y)
    arr = np.searchsorted(z_off, np.arange(Zcat.size), side="right") - 1
    gi = x_off[arr] + I
    assert np.all(_interp_tol(y, yref, Ycat[gi], Ycat[gi + 1]))
    # at a knot the interpolant is the knot value exactly
    Zk = np.concatenate([Xcat[x_off[a]:x_off[a + 1] - 1] for a in range(24)])
    zk_off = W.csr(np.diff(x_off) - 1)
    Ik, yk = L.search(_cuda(Zk), _cuda(zk_off), Y=_cuda(Ycat))
    Ik = Ik.cpu().numpy()
    assert np.array_equal(Ik, np.concatenate([np.arange(n - 1) for n in np.diff(x_off)]))
    ref_yk = np.concatenate([Ycat[x_off[a]:x_off[a + 1] - 1] for a in range(24)])
    assert np.array_equal(yk.cpu().numpy(), ref_yk)
    L.free()


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
    L.free()


@pytest.mark.slow
def test_workload5_full_size(ds):
    w = W.workload5()
    Xcat, Ycat, x_off, Zcat, z_off = w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"], w["z_off"]
    Xd, Yd, xo, Zd, zo = _cuda(Xcat), _cuda(Ycat), _cuda(x_off), _cuda(Zcat), _cuda(z_off)
    L = ds.ds_learned_build(Xd, xo)
    I, y = L.search(Zd, zo, Y=Yd)
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
    arr_all = torch.searchsorted(zo, torch.arange(Zd.numel(), device="cuda"), right=True) - 1
    gi = xo[arr_all] + I.long()
    assert bool((Xd[gi] <= Zd).all()) and bool((Zd < Xd[gi + 1]).all())
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
    L5 = ds.ds_learned_build(_cuda(Xcat), _cuda(x_off), cfg=_cfg(ds, steps=50))
    ds.ds_learned_autotune(L5, _cuda(Zcat), _cuda(z_off))
    I, _ = L5.search(_cuda(Zcat), _cuda(z_off), Y=_cuda(Ycat))
    assert np.array_equal(I.cpu().numpy(), oracle.interp_batch(Xcat, Ycat, x_off, Zcat, z_off)[0])
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
