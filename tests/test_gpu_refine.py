"""GPU parity of the refinement of H (DS_REFINE_H, end of Section 4.4) with
the oracle: the same H, W and R bit for bit, the same table, exact answers."""
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


def _growth_arrays(dtype, q, count, seed, min_updates=2):
    g = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(g.integers(q + 3, 40))
        X0 = -g.uniform(0.1, 10) * n
        X = (X0 + np.concatenate([[0], np.cumsum(g.uniform(0.5, 1.5, n))])).astype(dtype)
        if np.all(np.diff(X) > 0) and oracle.compute_hr(X, True, q=q, general=q > 1)["updates"] >= min_updates:
            out.append(X)
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_refined_h_matches_oracle(ds, dtype, q):
    moved = 0
    for X in _growth_arrays(dtype, q, 10, 7 + q + (dtype == np.float64)):
        ref = oracle.compute_hr_refined(X, True, q=q)
        plain = oracle.compute_hr(X, True, q=q, general=q > 1)
        flags = ds.DS_FMA | ds.DS_REFINE_H
        idx = ds.ds_build(_cuda(X), flags) if q == 1 else ds.ds_build_q(_cuda(X), q, flags=flags)
        info = idx.info()
        assert (info["H"], info["W"], info["R"]) == (ref["H"], ref["W"], ref["R"])
        assert info["h_updates"] == ref["updates"]
        moved += ref["H"] != plain["H"]
        st, K_ref, _ = oracle.fill_k(X, ref["H"], ref["W"], ref["R"], True, q=q, general=q > 1)
        K, _, _ = ds.ds_index_export(idx)
        assert np.array_equal(K.cpu().numpy(), K_ref)
        g = np.random.default_rng(3)
        Z = np.concatenate([W.adversarial_queries(X), W.uniform_queries(g, X[0], X[-1], 3000, dtype)])
        assert np.array_equal(ds.ds_search(idx, _cuda(Z)).cpu().numpy(), oracle.upper_bound(X, Z))
        idx.free()
    assert moved >= 1


def test_no_growth_is_unchanged(ds):
    X = W.workload2(n_knots=4097, m=10)["X"]
    a, b = ds.ds_build(_cuda(X)), ds.ds_build(_cuda(X), ds.DS_REFINE_H)
    ia, ib = a.info(), b.info()
    assert ia["h_updates"] == 0 and (ia["H"], ia["R"]) == (ib["H"], ib["R"])
    a.free()
    b.free()
