"""Seeded synthetic inputs for interval lookup.

This module holds data recipes only -- no step of the search method.  The
same arrays feed the CUDA library and the CPU oracle.  Every generator draws
from numpy's PCG64 ``default_rng(seed)`` with seed ``1506086200 + workload id``
unless a seed is given; knots are produced in float64 (cumulative sums of
i.i.d. gaps from X_0), rounded to the array dtype, then bumped to the next
representable value wherever rounding made two knots equal, so every array is
strictly increasing as the problem statement requires (Section 2).

Queries are uniform in value over [X_0, X_N): z = X_0 + u (X_N - X_0) with u
uniform in [0, 1) in float64, rounded to the dtype and clamped to
[X_0, nextafter(X_N, -inf)].

Workloads (sizes are the full ones; every generator takes smaller overrides
for tests):
  1  float32, 1025 knots, X_0 = 0, gaps U[0.5, 1.5] / 1024; 10^6 uniform
     queries plus every X_i (i < N) and every nextafter(X_{i+1}, -inf).
  2  float64, 2^20 + 1 knots, X_0 = 0, gaps lognormal(0, 0.5); 2^27 uniform
     queries (and a sorted copy).
  3  float32, 4096 arrays, knots per array floor(exp(U(ln 16, ln 65536))),
     scale s = 10^U(-3, 3), X_0 = s U(-n, n), gaps U[0.5, 1.5] s; queries per
     array proportional to its size, 2^28 in total (largest remainder).
  4  float64, 2^24 + 1 knots, X_0 = 0, gaps U[1e3, 1e4] with probability 0.01
     else U[1e-3, 1e-2]; 2^27 uniform queries.
  5  float32, 256 arrays, knots per array floor(exp(U(ln 2^10, ln 2^22))),
     X_0 = 0, each array's gap law picked uniformly among
     uniform U[0.5, 1.5] s, lognormal(0, 1) s and a two-scale "clustered" law
     (U[1, 10] s with probability 0.99, U[1e3, 1e4] s otherwise);
     Y ~ N(0, 1) float32 per knot; 2^28 queries proportional to size.
  paper  the paper's own layout (Section 6.1): gaps U[1, 5], queries drawn
     uniformly from the interval midpoints (X_i + X_{i+1}) / 2.
"""
import numpy as np

SEED_BASE = 1506086200


def rng(workload_id, seed=None):
    return np.random.default_rng(SEED_BASE + workload_id if seed is None else seed)


# --------------------------------------------------------------------------
# helpers (data generation only)
# --------------------------------------------------------------------------
def _order_key(a):
    """Signed integer key that orders floats like their values (+0 == -0)."""
    if a.dtype == np.float32:
        b = a.view(np.int32).astype(np.int64)
        mag = b & 0x7FFFFFFF
    else:
        b = a.view(np.int64)
        mag = b & 0x7FFFFFFFFFFFFFFF
    return np.where(b < 0, -mag, mag)


def _from_order_key(k, dtype):
    if dtype == np.float32:
        bits = np.where(k < 0, (-k) | 0x80000000, k).astype(np.uint32)
        return bits.view(np.float32)
    bits = np.where(k < 0, (-k).astype(np.uint64) | np.uint64(1 << 63), k.astype(np.uint64))
    return bits.view(np.float64)


def strictly_increasing(x):
    """Make a non-decreasing float array strictly increasing by replacing each
    element with max(x_i, next representable value above x_{i-1})."""
    x = np.asarray(x)
    if x.size < 2:
        return x.copy()
    k = _order_key(x)
    idx = np.arange(k.size, dtype=np.int64)
    k2 = idx + np.maximum.accumulate(k - idx)
    return _from_order_key(k2, x.dtype)


def knots_from_gaps(x0, gaps, dtype):
    x = np.empty(gaps.size + 1, dtype=np.float64)
    x[0] = x0
    np.cumsum(gaps, out=x[1:])
    x[1:] += x0
    return strictly_increasing(x.astype(dtype))


def uniform_queries(g, x_lo, x_hi, m, dtype):
    """m queries uniform in value over [x_lo, x_hi) in the given dtype."""
    u = g.random(m)
    z = (float(x_lo) + u * (float(x_hi) - float(x_lo))).astype(dtype)
    top = np.nextafter(np.array(x_hi, dtype=dtype), np.array(-np.inf, dtype=dtype))
    np.clip(z, np.array(x_lo, dtype=dtype), top, out=z)
    return z


def adversarial_queries(X):
    """Every X_i (i < N), every nextafter(X_{i+1}, -inf), and X_0."""
    X = np.asarray(X)
    below = np.nextafter(X[1:], np.array(-np.inf, dtype=X.dtype))
    return np.concatenate([X[:-1], below, X[:1]]).astype(X.dtype)


def midpoints(X):
    X = np.asarray(X)
    return ((X[:-1].astype(np.float64) + X[1:].astype(np.float64)) * 0.5).astype(X.dtype)


def split_proportional(total, weights):
    """Integer split of ``total`` proportional to ``weights`` (largest remainder)."""
    w = np.asarray(weights, dtype=np.float64)
    exact = total * w / w.sum()
    base = np.floor(exact).astype(np.int64)
    rem = int(total - base.sum())
    if rem > 0:
        order = np.argsort(-(exact - base), kind="stable")
        base[order[:rem]] += 1
    return base


def csr(sizes):
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def workload1(n_knots=1025, n_uniform=1_000_000, seed=None):
    g = rng(1, seed)
    gaps = g.uniform(0.5, 1.5, n_knots - 1) / 1024.0
    X = knots_from_gaps(0.0, gaps, np.float32)
    Zu = uniform_queries(g, X[0], X[-1], n_uniform, np.float32)
    below = np.nextafter(X[1:], np.float32(-np.inf))
    Z = np.concatenate([Zu, X[:-1], below]).astype(np.float32)
    return dict(X=X, Z=Z, name="direct_f32_1025knots")


def workload2(n_knots=(1 << 20) + 1, m=1 << 27, seed=None, sort=False):
    g = rng(2, seed)
    gaps = g.lognormal(0.0, 0.5, n_knots - 1)
    X = knots_from_gaps(0.0, gaps, np.float64)
    Z = uniform_queries(g, X[0], X[-1], m, np.float64)
    if sort:
        Z = np.sort(Z)
    return dict(X=X, Z=Z, name="direct_f64_%dknots_%dq%s" % (n_knots, m, "_sorted" if sort else ""))


def _array_sizes(g, n_arrays, lo, hi):
    return np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), n_arrays))).astype(np.int64)


def workload3(n_arrays=4096, size_lo=16, size_hi=65536, total_queries=1 << 28, seed=None):
    g = rng(3, seed)
    n = _array_sizes(g, n_arrays, size_lo, size_hi)
    n = np.maximum(n, 2)
    s = 10.0 ** g.uniform(-3.0, 3.0, n_arrays)
    x0 = s * g.uniform(-1.0, 1.0, n_arrays) * n
    x_off = csr(n)
    Xcat = np.empty(int(x_off[-1]), dtype=np.float32)
    for a in range(n_arrays):
        gaps = g.uniform(0.5, 1.5, int(n[a]) - 1) * s[a]
        Xcat[x_off[a]:x_off[a + 1]] = knots_from_gaps(x0[a], gaps, np.float32)
    q = split_proportional(total_queries, n)
    z_off = csr(q)
    Zcat = np.empty(int(z_off[-1]), dtype=np.float32)
    for a in range(n_arrays):
        Xa = Xcat[x_off[a]:x_off[a + 1]]
        Zcat[z_off[a]:z_off[a + 1]] = uniform_queries(g, Xa[0], Xa[-1], int(q[a]), np.float32)
    return dict(Xcat=Xcat, x_off=x_off, Zcat=Zcat, z_off=z_off,
                name="batched_f32_%darrays_%dq" % (n_arrays, total_queries))


def workload4(n_knots=(1 << 24) + 1, m=1 << 27, seed=None, p_big=0.01):
    g = rng(4, seed)
    big = g.random(n_knots - 1) < p_big
    gaps = np.where(big, g.uniform(1e3, 1e4, n_knots - 1), g.uniform(1e-3, 1e-2, n_knots - 1))
    X = knots_from_gaps(0.0, gaps, np.float64)
    Z = uniform_queries(g, X[0], X[-1], m, np.float64)
    return dict(X=X, Z=Z, name="learned_f64_%dknots_%dq" % (n_knots, m))


LAW_UNIFORM, LAW_LOGNORMAL, LAW_CLUSTERED = 0, 1, 2


def _gaps(g, law, count, scale):
    if law == LAW_UNIFORM:
        return g.uniform(0.5, 1.5, count) * scale
    if law == LAW_LOGNORMAL:
        return g.lognormal(0.0, 1.0, count) * scale
    big = g.random(count) < 0.01
    return np.where(big, g.uniform(1e3, 1e4, count), g.uniform(1.0, 10.0, count)) * scale


def workload5(n_arrays=256, size_lo=1 << 10, size_hi=1 << 22, total_queries=1 << 28, seed=None,
              laws=None):
    g = rng(5, seed)
    n = np.maximum(_array_sizes(g, n_arrays, size_lo, size_hi), 2)
    s = 10.0 ** g.uniform(-3.0, 3.0, n_arrays)
    law = g.integers(0, 3, n_arrays) if laws is None else np.resize(np.asarray(laws), n_arrays)
    x_off = csr(n)
    Xcat = np.empty(int(x_off[-1]), dtype=np.float32)
    for a in range(n_arrays):
        Xcat[x_off[a]:x_off[a + 1]] = knots_from_gaps(0.0, _gaps(g, int(law[a]), int(n[a]) - 1, s[a]),
                                                      np.float32)
    Ycat = g.standard_normal(Xcat.size).astype(np.float32)
    q = split_proportional(total_queries, n)
    z_off = csr(q)
    Zcat = np.empty(int(z_off[-1]), dtype=np.float32)
    for a in range(n_arrays):
        Xa = Xcat[x_off[a]:x_off[a + 1]]
        Zcat[z_off[a]:z_off[a + 1]] = uniform_queries(g, Xa[0], Xa[-1], int(q[a]), np.float32)
    return dict(Xcat=Xcat, Ycat=Ycat, x_off=x_off, Zcat=Zcat, z_off=z_off, law=law,
                name="learned_interp_f32_%darrays_%dq" % (n_arrays, total_queries))


def paper_layout(n_knots, m, dtype=np.float64, seed=None):
    """The paper's test layout (Section 6.1): gaps U[1, 5], X_0 = 0, queries drawn
    with equal probability from the interval midpoints."""
    g = rng(0, seed)
    X = knots_from_gaps(0.0, g.uniform(1.0, 5.0, n_knots - 1), dtype)
    mids = midpoints(X)
    Z = mids[g.integers(0, mids.size, m)]
    return dict(X=X, Z=Z, name="paper_U15_%dknots" % n_knots)
