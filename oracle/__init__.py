"""CPU oracle for direct search (Cannizzo, arXiv 1506.08620).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library under ``paper_1506_08620_gb300/``: nothing here imports
it, and it imports nothing from here.

* ``ds_oracle.c`` (plain C, loaded with ctypes) holds the definition of the
  answer (Section 2), the brute-force scan it is pinned against, ComputeHR
  (Section 4.4), the index table of Eq. indexdef and Algorithm "direct", and
  their DirectGap2 / Gap-q versions (Section 4.7, Eq. kgeneral).
* ``mlp.py`` holds the float64 reference of the learned predictor (forward,
  loss, backward, Adam) used to check the GPU training kernels' gradients.
* The fused-interpolation reference evaluates the interpolant in float64
  from float32 inputs.
"""
import ctypes
import numpy as np

from . import build as _build

OR_OK = 0
OR_E_ARG = 1
OR_E_NOT_INCREASING = 2
OR_E_INDISTINGUISHABLE = 3
OR_E_OVERFLOW = 4
OR_E_NO_CONVERGENCE = 5
OR_E_BAD_TABLE = 6

_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_U32 = ctypes.c_uint32
_INT = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for nm in ("or_upper_bound_f64", "or_upper_bound_f32", "or_scan_f64", "or_scan_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _P, _I64, _P]
            getattr(L, nm).restype = None
        for nm in ("or_upper_bound_batch_f32", "or_upper_bound_batch_f64"):
            getattr(L, nm).argtypes = [_P, _P, _I32, _P, _P, _P]
            getattr(L, nm).restype = None
        for nm in ("or_compute_hr_f64", "or_compute_hr_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _INT, _P, _P, _P, _P, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_compute_hr_gap2_f64", "or_compute_hr_gap2_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _INT, _P, _P, _P, _P, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_compute_hr_gapq_f64", "or_compute_hr_gapq_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _I32, _INT, _P, _P, _P, _P, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_compute_hr_refined_f64", "or_compute_hr_refined_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _I32, _INT, _P, _P, _P, _P, _P, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_fill_k_gap2_f64", "or_fill_k_gap2_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _D, _D, _U32, _INT, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_fill_k_gapq_f64", "or_fill_k_gapq_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _I32, _D, _D, _U32, _INT, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_direct_gap2_f64", "or_direct_gap2_f32"):
            getattr(L, nm).argtypes = [_P, _P, _D, _D, _U32, _INT, _P, _I64, _P]
            getattr(L, nm).restype = None
        for nm in ("or_direct_gapq_f64", "or_direct_gapq_f32"):
            getattr(L, nm).argtypes = [_P, _P, _I32, _D, _D, _U32, _INT, _P, _I64, _P]
            getattr(L, nm).restype = None
        for nm in ("or_fill_k_f64", "or_fill_k_f32"):
            getattr(L, nm).argtypes = [_P, _I64, _D, _D, _U32, _INT, _P, _P]
            getattr(L, nm).restype = _INT
        for nm in ("or_direct_f64", "or_direct_f32"):
            getattr(L, nm).argtypes = [_P, _P, _D, _D, _U32, _INT, _P, _I64, _P]
            getattr(L, nm).restype = None
        for nm in ("or_fvals_f64", "or_fvals_f32"):
            getattr(L, nm).argtypes = [_D, _D, _D, _INT, _P, _I64, _P]
            getattr(L, nm).restype = None
        L.or_interp_f32.argtypes = [_P, _P, _I64, _P, _I64, _P, _P]
        L.or_interp_f32.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _suffix(a):
    if a.dtype == np.float64:
        return "f64"
    if a.dtype == np.float32:
        return "f32"
    raise TypeError("oracle arrays must be float32 or float64, got %s" % a.dtype)


def upper_bound(X, Z):
    """Index of the largest X_i <= z for every z (Section 2); -1 below X_0 and
    for NaN, N = len(X)-1 at or above X_N."""
    X = np.ascontiguousarray(X)
    Z = np.ascontiguousarray(Z, dtype=X.dtype)
    out = np.empty(Z.shape[0], dtype=np.int32)
    getattr(lib(), "or_upper_bound_" + _suffix(X))(_ptr(X), X.shape[0], _ptr(Z), Z.shape[0], _ptr(out))
    return out


def scan(X, Z):
    """Brute force: count of knots <= z, minus one (linear scan)."""
    X = np.ascontiguousarray(X)
    Z = np.ascontiguousarray(Z, dtype=X.dtype)
    out = np.empty(Z.shape[0], dtype=np.int32)
    getattr(lib(), "or_scan_" + _suffix(X))(_ptr(X), X.shape[0], _ptr(Z), Z.shape[0], _ptr(out))
    return out


def upper_bound_batch(Xcat, x_off, Zcat, z_off):
    """Per-array answers for arrays/queries in CSR form; indices local to each array."""
    Xcat = np.ascontiguousarray(Xcat)
    Zcat = np.ascontiguousarray(Zcat, dtype=Xcat.dtype)
    x_off = np.ascontiguousarray(x_off, dtype=np.int64)
    z_off = np.ascontiguousarray(z_off, dtype=np.int64)
    out = np.empty(Zcat.shape[0], dtype=np.int32)
    getattr(lib(), "or_upper_bound_batch_" + _suffix(Xcat))(
        _ptr(Xcat), _ptr(x_off), x_off.shape[0] - 1, _ptr(Zcat), _ptr(z_off), _ptr(out))
    return out


def _q_of(gap2, q):
    if gap2:
        return 2
    return 1 if q is None else int(q)


def compute_hr(X, fma=False, gap2=False, q=None, general=False):
    """ComputeHR of Section 4.4 in the array's precision.  With q >= 2 (gap2
    is q = 2) its DirectGap2 / Gap-q version of Section 4.7 over the pairs
    (i, i+q); general=True runs that version for q = 1 too.

    Returns a dict with status (OR_*), H, W, R, updates (number of growth
    steps), passes, bad (offending knot index or -1)."""
    X = np.ascontiguousarray(X)
    q = _q_of(gap2, q)
    H = _D(); W = _D(); R = _U32(); upd = _I64(); passes = _I64(); bad = _I64()
    outs = (ctypes.byref(H), ctypes.byref(W), ctypes.byref(R), ctypes.byref(upd), ctypes.byref(passes),
            ctypes.byref(bad))
    if q == 1 and not general:
        st = getattr(lib(), "or_compute_hr_" + _suffix(X))(_ptr(X), X.shape[0], int(bool(fma)), *outs)
    else:
        st = getattr(lib(), "or_compute_hr_gapq_" + _suffix(X))(_ptr(X), X.shape[0], q, int(bool(fma)), *outs)
    return dict(status=st, H=H.value, W=W.value, R=R.value, updates=upd.value,
                passes=passes.value, bad=bad.value)


def compute_hr_refined(X, fma=False, q=1):
    """ComputeHR over the pairs (i, i+q), then, if H had to grow, the bisection
    of [last infeasible H, final H] proposed at the end of Section 4.4.
    Returns the dict of compute_hr plus `probes` (feasibility checks made)."""
    X = np.ascontiguousarray(X)
    H = _D(); W = _D(); R = _U32(); upd = _I64(); passes = _I64(); bad = _I64(); probes = _I64()
    st = getattr(lib(), "or_compute_hr_refined_" + _suffix(X))(
        _ptr(X), X.shape[0], int(q), int(bool(fma)), ctypes.byref(H), ctypes.byref(W), ctypes.byref(R),
        ctypes.byref(upd), ctypes.byref(passes), ctypes.byref(bad), ctypes.byref(probes))
    return dict(status=st, H=H.value, W=W.value, R=R.value, updates=upd.value, passes=passes.value, bad=bad.value,
                probes=probes.value)


def fill_k(X, H, W, R, fma=False, gap2=False, q=None, general=False):
    """Index table of Eq. indexdef (q = 1), or of Eq. kgeneral (q >= 2, or
    general=True), R+1 int32 entries, and F_i = f(X_i).  Returns (status, K, F)."""
    X = np.ascontiguousarray(X)
    q = _q_of(gap2, q)
    K = np.empty(int(R) + 1, dtype=np.int32)
    F = np.empty(X.shape[0], dtype=np.uint32)
    if q == 1 and not general:
        st = getattr(lib(), "or_fill_k_" + _suffix(X))(
            _ptr(X), X.shape[0], float(H), float(W), int(R), int(bool(fma)), _ptr(K), _ptr(F))
    else:
        st = getattr(lib(), "or_fill_k_gapq_" + _suffix(X))(
            _ptr(X), X.shape[0], q, float(H), float(W), int(R), int(bool(fma)), _ptr(K), _ptr(F))
    return st, K, F


def build_table(X, fma=False, gap2=False, q=None, general=False):
    """ComputeHR followed by its table (Eq. indexdef, or Eq. kgeneral for
    q >= 2 or general=True); returns (hr dict, K) or raises."""
    hr = compute_hr(X, fma, gap2, q, general)
    if hr["status"] != OR_OK:
        raise ValueError("array infeasible for direct search: status %d" % hr["status"])
    st, K, _ = fill_k(X, hr["H"], hr["W"], hr["R"], fma, gap2, q, general)
    if st != OR_OK:
        raise ValueError("table construction failed: status %d" % st)
    return hr, K


def direct(X, K, H, W, R, Z, fma=False, gap2=False, q=None, general=False):
    """Algorithm "direct" (q = 1), or Algorithm direct-2 and its q-comparison
    generalisation (q >= 2, or general=True), on the CPU with a given (H, W, R, K)."""
    X = np.ascontiguousarray(X)
    Z = np.ascontiguousarray(Z, dtype=X.dtype)
    K = np.ascontiguousarray(K, dtype=np.int32)
    q = _q_of(gap2, q)
    out = np.empty(Z.shape[0], dtype=np.int32)
    if q == 1 and not general:
        getattr(lib(), "or_direct_" + _suffix(X))(
            _ptr(X), _ptr(K), float(H), float(W), int(R), int(bool(fma)), _ptr(Z), Z.shape[0], _ptr(out))
    else:
        getattr(lib(), "or_direct_gapq_" + _suffix(X))(
            _ptr(X), _ptr(K), q, float(H), float(W), int(R), int(bool(fma)), _ptr(Z), Z.shape[0], _ptr(out))
    return out


def table_bytes(X, R):
    """Bytes of the index's table image: K ((R+1) int32) and X, each padded to 16 bytes."""
    r16 = lambda b: (b + 15) // 16 * 16
    return r16((int(R) + 1) * 4) + r16(X.shape[0] * X.dtype.itemsize)


def choose_q(X, fma, budget_bytes, q_max):
    """The paper's memory-budget use of Eq. f-monotonic-n (Section 4.7): the
    smallest q in 1..q_max for which ComputeHR succeeds and the table fits
    budget_bytes.  Returns (q, hr) or (0, None) if no q qualifies."""
    for q in range(1, q_max + 1):
        hr = compute_hr(X, fma, q=q)
        if hr["status"] == OR_OK and table_bytes(X, hr["R"]) <= budget_bytes:
            return q, hr
    return 0, None


def fvals(H, W, X0, Z, fma=False):
    """j = f(z) truncated to 32 bits (Eq. function / Eq. fma), no clamp to R."""
    Z = np.ascontiguousarray(Z)
    out = np.empty(Z.shape[0], dtype=np.uint32)
    getattr(lib(), "or_fvals_" + _suffix(Z))(float(H), float(W), float(X0), int(bool(fma)),
                                             _ptr(Z), Z.shape[0], _ptr(out))
    return out


def interp(X, Y, Z):
    """Interval index and the float64 linear interpolant from float32 inputs."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    Z = np.ascontiguousarray(Z, dtype=np.float32)
    I = np.empty(Z.shape[0], dtype=np.int32)
    y = np.empty(Z.shape[0], dtype=np.float64)
    lib().or_interp_f32(_ptr(X), _ptr(Y), X.shape[0], _ptr(Z), Z.shape[0], _ptr(I), _ptr(y))
    return I, y


def interp_batch(Xcat, Ycat, x_off, Zcat, z_off):
    """Batched version of :func:`interp` (CSR arrays and queries)."""
    I = np.empty(Zcat.shape[0], dtype=np.int32)
    y = np.empty(Zcat.shape[0], dtype=np.float64)
    for a in range(len(x_off) - 1):
        xs, xe, zs, ze = x_off[a], x_off[a + 1], z_off[a], z_off[a + 1]
        if ze > zs:
            I[zs:ze], y[zs:ze] = interp(Xcat[xs:xe], Ycat[xs:xe], Zcat[zs:ze])
    return I, y
