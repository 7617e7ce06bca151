"""Pins, on the oracle's own tables, for the two facts the batched rank table
rests on (Section 4, Eq. indexdef):

* with pairs (i, i+1) ComputeHR makes F strictly increasing, so a cell holds at
  most one knot and K_j = min{i : F_i >= j} is the rank #{i : F_i < j}; a
  word per 32 cells (K at the group's first cell and a mask of the cells that
  hold a knot) then gives K_j = K_{32 g} + popc(mask below j mod 32);
* the knot fingerprint floor(256 (v - trunc v)) is computed exactly in float
  arithmetic (v - trunc v is exact, and so is the product by 256), and within
  one cell it is a non-decreasing function of v;

and, for the float32 one-conversion cell form, that trunc(m(256 H y + 256 c))
equals 256 j + g; and, for the learned form, that the certificate tested on
the answer is the window certificate."""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
from paper_1506_08620_gb300 import workloads as W


def _arrays(dtype, count, seed):
    g = np.random.default_rng(seed)
    for _ in range(count):
        n = int(g.integers(2, 400))
        law = g.integers(0, 3)
        gaps = (g.uniform(0.5, 1.5, n - 1) if law == 0 else
                g.lognormal(0.0, 1.0, n - 1) if law == 1 else
                np.where(g.random(n - 1) < 0.05, g.uniform(50, 100, n - 1), g.uniform(0.5, 1.5, n - 1)))
        yield W.knots_from_gaps(float(g.uniform(-50, 50)), gaps, dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fma", [False, True])
def test_k_is_the_rank_of_the_knot_cells(dtype, fma):
    checked = 0
    for X in _arrays(dtype, 150, 5 + fma + 2 * (dtype == np.float64)):
        hr = oracle.compute_hr(X, fma)
        if hr["status"] != oracle.OR_OK:
            continue
        st, K, F = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], fma)
        assert st == oracle.OR_OK
        F = F.astype(np.int64)
        assert np.all(np.diff(F) > 0)  # strictly increasing: at most one knot per cell
        R = int(hr["R"])
        j = np.arange(R + 1)
        assert np.array_equal(K, np.searchsorted(F, j, side="left"))  # K_j = #{i : F_i < j}
        assert set(np.unique(np.diff(K))) <= {0, 1}
        # the 32-cell words: K at each group's first cell and the knot mask
        holds = np.zeros(R + 1, dtype=bool)
        holds[F] = True
        G = R // 32 + 1
        base = K[np.arange(G) * 32]
        mask = np.zeros(G, dtype=np.uint64)
        for c in np.nonzero(holds)[0]:
            mask[c // 32] |= np.uint64(1) << np.uint64(c % 32)
        for jj in j:
            below = int(mask[jj // 32]) & ((1 << (jj % 32)) - 1)
            assert base[jj // 32] + bin(below).count("1") == K[jj]
            assert bool((int(mask[jj // 32]) >> (jj % 32)) & 1) == holds[jj]
        checked += 1
    assert checked > 100


def _exact_fp(v):
    fv = Fraction(float(v))
    if fv < 0:
        return 0
    return math.floor(256 * (fv - math.floor(fv)))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_fingerprint_is_exact_and_monotone_within_a_cell(dtype):
    g = np.random.default_rng(17)
    # values across the exponent range of the cells a table can have
    v = np.concatenate([g.uniform(0, 1, 4000), g.uniform(0, 2 ** 12, 4000), g.uniform(0, 2 ** 23, 4000),
                        2.0 ** g.uniform(-10, 31, 4000)]).astype(dtype)
    j = np.trunc(v)
    frac = (v - j).astype(dtype)  # one rounding of the array's precision
    fp = np.floor(frac * dtype(256)).astype(np.int64)
    exact = np.array([_exact_fp(x) for x in v])
    assert np.array_equal(fp, exact)
    # monotone within a cell: sort, and compare neighbours in the same cell
    order = np.argsort(v, kind="stable")
    vs, js, fs = v[order], j[order], fp[order]
    same = js[1:] == js[:-1]
    assert np.all(fs[1:][same] >= fs[:-1][same])
    assert np.all((fs >= 0) & (fs < 256))


def test_answer_side_certificate_equals_the_window_certificate():
    # learned form: for every window [lo, hi] and query z, some i in [lo, hi]
    # passes X_i <= z < X_{i+1} exactly when X_lo <= z < X_{hi+1}, and then
    # that i is the definition's answer (the knots are sorted)
    g = np.random.default_rng(23)
    for _ in range(40):
        X = W.knots_from_gaps(float(g.uniform(-5, 5)), g.uniform(0.5, 1.5, int(g.integers(2, 24))), np.float64)
        N = X.size - 1
        Z = np.concatenate([X, np.nextafter(X, -np.inf), np.nextafter(X, np.inf), g.uniform(X[0] - 2, X[-1] + 2, 50)])
        truth = oracle.upper_bound(X, Z)
        for lo in range(N):
            for hi in range(lo, N):
                win = (X[lo] <= Z) & (Z < X[hi + 1])
                for k, z in enumerate(Z):
                    passing = [i for i in range(lo, hi + 1) if X[i] <= z < X[i + 1]]
                    assert bool(passing) == bool(win[k])
                    if passing:
                        assert passing == [truth[k]]


def test_one_conversion_cell_form_of_float32():
    # q = trunc(m(256 H y + 256 c)) gives the cell and the fingerprint at once:
    # scaling by 256 commutes with the single rounding of the fused multiply-add
    # (where the result is a normal float; below 2^-126 both give cell 0 and
    # fingerprint 0), and trunc(256 v) = 256 trunc(v) + floor(256 frac(v))
    from tests import exact
    g = np.random.default_rng(29)
    f32 = np.float32
    checked = 0
    for _ in range(4000):
        H = f32(2.0 ** g.uniform(-12, 16))
        if g.random() < 0.5:  # Eq. function: y = m(z - X0), c = 0
            X0 = f32(g.uniform(-1e4, 1e4))
            z = f32(float(X0) + g.uniform(-10, 2 ** 24 / float(H)))
            y = exact.add(z, -X0, f32)
            c = f32(0.0)
        else:  # Eq. fma: y = z, c = -W with W = m(H X0)
            X0 = f32(g.uniform(-1e4, 1e4))
            y = f32(float(X0) + g.uniform(-10, 2 ** 24 / float(H)))
            c = -exact.mul(H, X0, f32)
        v = exact.round_nearest(Fraction(float(H)) * Fraction(float(y)) + Fraction(float(c)), f32)
        v256 = exact.round_nearest(Fraction(float(f32(256) * H)) * Fraction(float(y)) + Fraction(float(f32(256) * c)), f32)
        if abs(float(v)) >= 2.0 ** -126:
            assert float(v256) == 256.0 * float(v)
        elif float(v) >= 0:
            assert 0 <= float(v256) < 1.0
        if 0 <= float(v) < 2 ** 24 - 1:
            q = exact.trunc_u32(v256)
            fv = Fraction(float(v))
            assert q == 256 * math.floor(fv) + math.floor(256 * (fv - math.floor(fv)))
            checked += 1
    assert checked > 1500


@pytest.mark.parametrize("q", [1, 2, 3, 5])
def test_packed_cell_differences_fit_six_bits(q):
    # the float64 single-array path packs K in blocks of 12 cells as a base and
    # 12 differences of 6 bits: a cell holds at most q knots (pairs (i, i+q)
    # are separated), so within a block K grows by at most 11 q <= 55 < 64
    g = np.random.default_rng(31 + q)
    checked = 0
    for X in _arrays(np.float64, 120, 40 + q):
        hr = oracle.compute_hr(X, False, q=q, general=q > 1)
        if hr["status"] != oracle.OR_OK:
            continue
        st, K, _ = oracle.fill_k(X, hr["H"], hr["W"], hr["R"], False, q=q, general=q > 1)
        assert st == oracle.OR_OK
        K = K.astype(np.int64) & 0x3FFFFFFF
        d = np.diff(K)
        assert d.min() >= 0 and d.max() <= q
        nb = (K.size + 11) // 12
        Kp = np.concatenate([K, np.full(nb * 12 - K.size, K[-1])]).reshape(nb, 12)
        assert (Kp - Kp[:, :1]).max() <= 11 * q < 64
        checked += 1
    assert checked > 60
