"""GPU parity of the single-array path (ds_build / ds_search) with the oracle.

Bit-exact: H, W, R, the K table, the pair table and every returned index
must equal the oracle's ComputeHR, Eq. indexdef table and the definition of
the answer."""
import os

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


def _growth_arrays(dtype, count, seed):
    g = np.random.default_rng(seed)
    found = []
    while len(found) < count:
        n = int(g.integers(4, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if np.all(np.diff(X) > 0) and oracle.compute_hr(X, fma=True)["updates"] > 0:
            found.append(X)
    return found


def _arrays(dtype):
    g = np.random.default_rng(77)
    out = [
        ("section42", np.array([0.0, 0.5, 0.7, 1.1]).astype(dtype)),
        ("directmap", np.array([0, 6, 15, 23, 31, 37, 50]).astype(dtype)),
        ("workload1", W.workload1(n_uniform=10)["X"].astype(dtype)),
        ("workload2_small", W.workload2(n_knots=4097, m=10)["X"].astype(dtype)),
        ("paper_U15", W.paper_layout(4095, 10, dtype)["X"]),
        ("two_knots", np.array([-3.0, 7.0]).astype(dtype)),
    ]
    for k, X in enumerate(_growth_arrays(dtype, 6, 5 + (dtype == np.float64))):
        out.append(("growth%d" % k, X))
    for k in range(8):
        n = int(g.integers(2, 3000))
        X0 = g.uniform(-1e4, 1e4)
        out.append(("random%d" % k, W.knots_from_gaps(X0, g.uniform(0.01, 2.0, n - 1) * 10.0 ** g.uniform(-3, 3),
                                                     dtype)))
    return out


def _queries(X, g, n=4000):
    dt = X.dtype.type
    inf = dt(np.inf)
    return np.concatenate([
        W.adversarial_queries(X), W.midpoints(X), W.uniform_queries(g, X[0], X[-1], n, X.dtype),
        np.array([X[-1], np.nextafter(X[0], -inf), -inf, inf, float(X[0]) - 1e6, float(X[-1]) * 2 + 1, 0.0, -0.0],
                 dtype=X.dtype)])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("flags", [0, 1, 2, 3], ids=["plain", "fma", "cache", "fma_cache"])
def test_build_tables_bit_identical(ds, dtype, flags):
    fma = bool(flags & ds.DS_FMA)
    for name, X in _arrays(dtype):
        hr = oracle.compute_hr(X, fma)
        assert hr["status"] == oracle.OR_OK, name
        st, K_ref, _ = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma)
        idx = ds.ds_build(_cuda(X), flags)
        info = idx.info()
        assert info["H"] == hr["H"] and info["R"] == hr["R"], name
        if fma:
            assert info["W"] == hr["W"], name
        assert info["h_updates"] == hr["updates"] and info["hr_passes"] == hr["passes"], name
        K, Xc, pairs = ds.ds_index_export(idx)
        torch.cuda.synchronize()
        assert np.array_equal(K.cpu().numpy(), K_ref), name
        assert np.array_equal(Xc.cpu().numpy(), X), name
        if flags & ds.DS_CACHE_LAYOUT:
            p = pairs.cpu().numpy()
            assert np.array_equal(p[:, :4].copy().view(np.int32).ravel(), K_ref), name
            xoff = 4 if dtype == np.float32 else 8
            assert np.array_equal(p[:, xoff:].copy().view(dtype).ravel(), X[K_ref]), name
        idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("flags", [0, 1, 2, 3, 8, 9, 10, 11],
                         ids=["plain", "fma", "cache", "fma_cache", "l2", "l2_fma", "l2_cache", "l2_fma_cache"])
@pytest.mark.parametrize("intops", ["0", "1"])
def test_search_matches_definition(ds, dtype, flags, intops, monkeypatch):
    if dtype == np.float32 and intops == "0":
        pytest.skip("integer-arithmetic variant exists for float64 only")
    monkeypatch.setenv("DS_F64_INTOPS", intops)
    g = np.random.default_rng(3)
    for name, X in _arrays(dtype):
        Z = _queries(X, g)
        idx = ds.ds_build(_cuda(X), flags)
        got = ds.ds_search(idx, _cuda(Z)).cpu().numpy()
        assert np.array_equal(got, oracle.upper_bound(X, Z)), (name, int(np.count_nonzero(got != oracle.upper_bound(X, Z))))
        idx.free()


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_workload1_full_size(ds, flags):
    w = W.workload1()
    X, Z = w["X"], w["Z"]
    ref = oracle.upper_bound(X, Z)
    idx = ds.ds_build(_cuda(X), flags)
    assert idx.info()["smem_resident"] == 1
    got = ds.ds_search(idx, _cuda(Z)).cpu().numpy()
    assert np.count_nonzero(got != ref) == 0
    # the same stream tiled 64x, as the bandwidth run does (one launch)
    Zt = _cuda(np.tile(Z, 64))
    out = ds.ds_search(idx, Zt)
    assert torch.equal(out.view(64, -1), _cuda(ref).view(1, -1).expand(64, -1))
    idx.free()


@pytest.mark.parametrize("sort", [False, True], ids=["unsorted", "sorted"])
@pytest.mark.parametrize("flags", [0, 1, 2])
def test_workload2_full_size_sampled(ds, sort, flags):
    w = W.workload2(sort=sort)
    X, Z = w["X"], w["Z"]
    hr = oracle.compute_hr(X, bool(flags & 1))
    idx = ds.ds_build(_cuda(X), flags)
    info = idx.info()
    assert info["H"] == hr["H"] and info["R"] == hr["R"]
    Zd = _cuda(Z)
    got = ds.ds_search(idx, Zd)
    g = np.random.default_rng(9)
    pos = np.concatenate([g.integers(0, Z.size, 1 << 20), np.arange(4096), np.arange(Z.size - 4096, Z.size)])
    ref = oracle.upper_bound(X, Z[pos])
    assert np.array_equal(got[_cuda(pos)].cpu().numpy(), ref)
    # properties at every position: X_I <= z < X_{I+1}
    Xd = _cuda(X)
    gl = got.long()
    assert bool((gl >= 0).all()) and bool((gl <= X.size - 2).all())
    assert bool((Xd[gl] <= Zd).all()) and bool((Zd < Xd[gl + 1]).all())
    idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_ragged_sizes_and_misaligned_pointers(ds, dtype):
    g = np.random.default_rng(5)
    X = W.knots_from_gaps(0.0, g.uniform(0.5, 1.5, 2000), dtype)
    Zall = W.uniform_queries(g, X[0], X[-1], (1 << 20) + 40, dtype)
    idx = ds.ds_build(_cuda(X))
    Zd = _cuda(Zall)
    for m in (0, 1, 2, 3, 5, 7, 31, 1023, 4099, (1 << 20) + 3):
        for zoff, ioff in ((0, 0), (1, 0), (0, 1), (3, 5)):
            z = Zd[zoff:zoff + m]
            out = torch.full((m + ioff,), -7, dtype=torch.int32, device="cuda")
            ds.ds_search(idx, z, out[ioff:])
            ref = oracle.upper_bound(X, Zall[zoff:zoff + m])
            o = out.cpu().numpy()
            assert np.array_equal(o[ioff:], ref), (m, zoff, ioff)
            assert np.all(o[:ioff] == -7)
    idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_checked_nan(ds, dtype):
    X = np.linspace(-1, 1, 101).astype(dtype)
    Z = np.array([np.nan, -np.nan, 0.0, np.nan, 2.0], dtype=dtype)
    idx = ds.ds_build(_cuda(X), ds.DS_CHECKED)
    assert list(ds.ds_search(idx, _cuda(Z)).cpu().numpy()) == [-1, -1, 50, -1, 100]
    idx2 = ds.ds_build(_cuda(X))
    got = ds.ds_search(idx2, _cuda(Z)).cpu().numpy()
    assert np.all((got >= -1) & (got <= 100)) and got[2] == 50 and got[4] == 100
    idx.free()
    idx2.free()


def test_error_statuses(ds):
    from paper_1506_08620_gb300 import _abi

    def status(X, flags=0):
        try:
            ds.ds_build(_cuda(X), flags).free()
            return _abi.DS_OK
        except ds.DsError as e:
            return e.status

    assert status(np.array([-1e9, 0, 1], dtype=np.float32)) == _abi.DS_E_INDISTINGUISHABLE
    assert status(np.array([0, 1.42e-45, 1], dtype=np.float32)) == _abi.DS_E_OVERFLOW
    assert status(np.array([0.0, 2.0 ** -34, 1.0])) == _abi.DS_E_OVERFLOW
    assert status(np.array([0.0, 1.0, 1.0])) == _abi.DS_E_NOT_INCREASING
    assert status(np.array([0.0, 2.0, 1.0], dtype=np.float32)) == _abi.DS_E_NOT_INCREASING
    assert status(np.array([0.0, np.nan, 1.0])) == _abi.DS_E_NOT_INCREASING
    assert status(np.array([0.0, 1.0, np.inf])) == _abi.DS_E_NOT_INCREASING
    assert status(np.array([-1.0, 0.0, 2.0 ** -20, 1.0], dtype=np.float32)) == _abi.DS_OK
    assert status(np.array([-1.0, 0.0, 2.0 ** -25, 1.0], dtype=np.float32)) == _abi.DS_E_INDISTINGUISHABLE
    os.environ["DS_TABLE_BUDGET_BYTES"] = "1000"
    try:
        assert status(np.linspace(0, 1, 5000)) == _abi.DS_E_TABLE_TOO_LARGE
    finally:
        del os.environ["DS_TABLE_BUDGET_BYTES"]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("mode", ["direct", "pipeline", "pageable"])
def test_search_host_buffers(ds, dtype, mode, monkeypatch):
    # pinned buffers are read and written by the kernel in place; DS_HOST_PIPE=1
    # and pageable buffers take the chunked copy pipeline
    monkeypatch.setenv("DS_PIPE_CHUNK", str(100_003))
    if mode == "pipeline":
        monkeypatch.setenv("DS_HOST_PIPE", "1")
    g = np.random.default_rng(6)
    X = W.knots_from_gaps(1.0, g.lognormal(0, 0.5, 50_000), dtype)
    Z = W.uniform_queries(g, X[0], X[-1], 1_000_001, dtype)
    idx = ds.ds_build(_cuda(X), ds.DS_FMA)
    if mode == "pageable":
        Zh = torch.from_numpy(Z.copy())
        out = torch.full((Z.size,), -7, dtype=torch.int32)
        ds.ds_search_host(idx, Zh, out)
    else:
        Zh = torch.from_numpy(Z).pin_memory()
        out = ds.ds_search_host(idx, Zh)
    assert np.array_equal(out.numpy(), oracle.upper_bound(X, Z))
    # misaligned views of pinned memory (scalar kernel path)
    if mode == "direct":
        out2 = torch.full((Z.size,), -7, dtype=torch.int32).pin_memory()
        ds.ds_search_host(idx, Zh[1:], out2[1:])
        assert np.array_equal(out2.numpy()[1:], oracle.upper_bound(X, Z[1:])) and out2[0] == -7
    idx.free()


def test_search_in_cuda_graph(ds):
    w = W.workload1(n_uniform=200_000)
    X, Z = w["X"], w["Z"]
    idx = ds.ds_build(_cuda(X))
    Zd = _cuda(Z)
    out = torch.empty(Z.size, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ds.ds_search(idx, Zd, out)  # warm-up outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    out.fill_(-5)
    with torch.cuda.graph(graph, stream=s):
        ds.ds_search(idx, Zd, out)
    out.fill_(-5)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.upper_bound(X, Z))
    idx.free()


@pytest.mark.parametrize("flags", [8, 9], ids=["l2", "l2_fma"])
def test_packed_float64_tables_across_cell_ranges(ds, flags):
    # the packed L2 table on arrays whose cells span small to very large f
    # values (R up to ~1.5e9), X_0 zero and not
    g = np.random.default_rng(33)
    fl = flags
    for k, (cells_per_knot, n) in enumerate(((3, 100), (40, 2000), (700, 3000), (2e4, 3000), (1e6, 1500))):
        X0 = 0.0 if k % 2 == 0 else g.uniform(-1e3, 1e3)
        gaps = g.uniform(0.5, 1.5, n - 1)
        gaps[g.integers(0, n - 1)] = 1.0 / cells_per_knot
        X = W.knots_from_gaps(X0, gaps, np.float64)
        Z = _queries(X, g, 20000)
        idx = ds.ds_build(_cuda(X), fl)
        got = ds.ds_search(idx, _cuda(Z)).cpu().numpy()
        ref = oracle.upper_bound(X, Z)
        assert np.array_equal(got, ref), (k, int(np.count_nonzero(got != ref)))
        idx.free()


@pytest.mark.slow
def test_table_near_the_32_bit_cell_limit(ds):
    # one narrow gap sets H so that R = trunc(m(H D_N)) is close to 2^32 - 1:
    # a 16 GB table; cells and the clamp at R work in the top of the uint32 range
    g = np.random.default_rng(71)
    gaps = g.uniform(0.5, 1.5, 1000)
    gaps[500] = 1.0 / 3.9e6
    X = W.knots_from_gaps(0.0, gaps, np.float64)
    hr = oracle.compute_hr(X)
    assert hr["status"] == oracle.OR_OK and hr["R"] > 3.5e9
    idx = ds.ds_build(_cuda(X))
    info = idx.info()
    assert info["H"] == hr["H"] and info["R"] == hr["R"]
    Z = _queries(X, g, 1_000_000)
    assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    idx.free()


@pytest.mark.slow
def test_array_of_2p28_knots(ds):
    # indices near 2^28 in the int32 results; sampled queries and the array's ends
    g = np.random.default_rng(72)
    X = W.knots_from_gaps(-5.0, g.uniform(0.5, 1.5, 1 << 28), np.float64)
    idx = ds.ds_build(_cuda(X))
    assert idx.info()["R"] == oracle.compute_hr(X)["R"]
    Z = np.concatenate([W.uniform_queries(g, X[0], X[-1], 1 << 20, np.float64), X[-1000:],
                        np.nextafter(X[-1000:], -np.inf), X[:1000], np.array([np.inf, -np.inf, X[-1] + 1.0])])
    assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    idx.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_indices_with_different_staged_tables(ds, dtype):
    # tables staged in shared memory share one kernel: a later index with a
    # smaller table must leave the earlier (larger) one searchable
    g = np.random.default_rng(41)
    arrays = [W.knots_from_gaps(0.0, g.uniform(0.5, 1.5, n), dtype) for n in (5000, 300, 3000, 40)]
    idxs = [ds.ds_build(_cuda(X)) for X in arrays]
    assert all(i.info()["smem_resident"] == 1 for i in idxs)
    for X, idx in zip(arrays, idxs):
        Z = _queries(X, g, 5000)
        assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
    for i in idxs:
        i.free()
