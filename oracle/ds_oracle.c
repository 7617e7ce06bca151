/*
 * ds_oracle.c -- plain, slow, obviously-correct CPU oracle for direct search
 * (F. Cannizzo, "A Fast and Vectorizable Alternative to Binary Search in O(1)
 * with Wide Applicability to Arrays of Floating Point Numbers", arXiv 1506.08620).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA library: it is written directly from the
 * paper so that the two can be compared.
 *
 * Built with `-O2 -ffp-contract=off` and without -ffast-math, so every float
 * and double operation below is one IEEE-754 operation rounded to nearest
 * (no FMA contraction, no flush-to-zero); fma()/fmaf() are the correctly
 * rounded C99 library functions.
 *
 * Contents
 *   or_upper_bound_*   Section 2 problem statement: I = index of the largest
 *                      X_i <= z  (= #{i : X_i <= z} - 1), plain bisection.
 *   or_scan_*          the same by a linear scan (the brute force it is
 *                      pinned against).
 *   or_compute_hr_*    Section 4.4 "Computation of a feasible H", the
 *                      ComputeHR algorithm, plain (Eq. function) and FMA
 *                      (Eq. fma) forms.
 *   or_fill_k_*        Eq. indexdef: K_0 = 0, K_j = i for f(X_{i-1}) < j <= f(X_i).
 *   or_direct_*        Algorithm "direct": j = f(z), t = K_j, i = t - [z < X_t].
 *   or_compute_hr_refined_*  ComputeHR followed by the bisection of H that the end
 *                      of Section 4.4 proposes (not implemented in the paper).
 *   or_*_gapq_*        DirectGap2 and its q-knot generalisation (Section 4.7):
 *                      ComputeHR over pairs (i, i+q), K of Eq. kgeneral,
 *                      Algorithm direct-2 with q comparisons; or_*_gap2_* are
 *                      the q = 2 case.
 *
 * Readings of the paper this file takes where the text is silent or garbled:
 *   - floor in f is truncation toward zero with negatives clamped to 0 and
 *     values >= 2^32 saturated (Q = 32 bit j), NaN -> 0;
 *   - R = trunc(m(H D_N)) is the largest j, K has R+1 entries;
 *   - the growth loop of ComputeHR is repeated as whole passes until a pass
 *     changes nothing (a later growth step can merge an earlier pair); the
 *     growth term P keeps doubling across passes; at most 64 passes;
 *   - the overflow test "floor(H D_N >= 2^Q)" is read as m(H D_N) >= 2^32
 *     (which also catches H = +inf);
 *   - H, W, D and P are held in the array's own precision;
 *   - in the FMA form W = m(H X_0) is recomputed whenever H changes and the
 *     starting H is the plain form's one.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* status codes of the oracle (its own numbering; tests map them) */
#define OR_OK 0
#define OR_E_ARG 1
#define OR_E_NOT_INCREASING 2
#define OR_E_INDISTINGUISHABLE 3
#define OR_E_OVERFLOW 4
#define OR_E_NO_CONVERGENCE 5
#define OR_E_BAD_TABLE 6

#define OR_MAX_PASSES 64

/* ------------------------------------------------------------------------ */
/* Problem statement (Section 2): the index of the largest X_i <= z.        */
/* Bisection on the count of knots <= z; for z < X_0 (or NaN) the count is 0 */
/* and the result -1; for z >= X_N it is N.                                 */
/* ------------------------------------------------------------------------ */
static int64_t count_le_f64(const double *X, int64_t n_knots, double z)
{
    int64_t lo = 0, hi = n_knots; /* X[k] <= z for k < lo, X[k] > z for k >= hi */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (X[mid] <= z) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int64_t count_le_f32(const float *X, int64_t n_knots, float z)
{
    int64_t lo = 0, hi = n_knots;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (X[mid] <= z) lo = mid + 1; else hi = mid;
    }
    return lo;
}

void or_upper_bound_f64(const double *X, int64_t n_knots, const double *Z, int64_t m, int32_t *I)
{
    for (int64_t q = 0; q < m; ++q) I[q] = (int32_t)(count_le_f64(X, n_knots, Z[q]) - 1);
}

void or_upper_bound_f32(const float *X, int64_t n_knots, const float *Z, int64_t m, int32_t *I)
{
    for (int64_t q = 0; q < m; ++q) I[q] = (int32_t)(count_le_f32(X, n_knots, Z[q]) - 1);
}

/* Many independent arrays in CSR form: array a owns knots x_off[a]..x_off[a+1]-1
 * and queries z_off[a]..z_off[a+1]-1; indices are local to the array. */
void or_upper_bound_batch_f32(const float *Xcat, const int64_t *x_off, int32_t n_arrays,
                              const float *Zcat, const int64_t *z_off, int32_t *Icat)
{
    for (int32_t a = 0; a < n_arrays; ++a)
        or_upper_bound_f32(Xcat + x_off[a], x_off[a + 1] - x_off[a], Zcat + z_off[a],
                           z_off[a + 1] - z_off[a], Icat + z_off[a]);
}

void or_upper_bound_batch_f64(const double *Xcat, const int64_t *x_off, int32_t n_arrays,
                              const double *Zcat, const int64_t *z_off, int32_t *Icat)
{
    for (int32_t a = 0; a < n_arrays; ++a)
        or_upper_bound_f64(Xcat + x_off[a], x_off[a + 1] - x_off[a], Zcat + z_off[a],
                           z_off[a + 1] - z_off[a], Icat + z_off[a]);
}

/* Brute force: count the knots <= z one by one. */
void or_scan_f64(const double *X, int64_t n_knots, const double *Z, int64_t m, int32_t *I)
{
    for (int64_t q = 0; q < m; ++q) {
        int64_t c = 0;
        for (int64_t i = 0; i < n_knots; ++i) c += (X[i] <= Z[q]);
        I[q] = (int32_t)(c - 1);
    }
}

void or_scan_f32(const float *X, int64_t n_knots, const float *Z, int64_t m, int32_t *I)
{
    for (int64_t q = 0; q < m; ++q) {
        int64_t c = 0;
        for (int64_t i = 0; i < n_knots; ++i) c += (X[i] <= Z[q]);
        I[q] = (int32_t)(c - 1);
    }
}

/* ------------------------------------------------------------------------ */
/* The map f (Eq. function, Eq. fma) and its truncation to a 32-bit j.      */
/* ------------------------------------------------------------------------ */
static uint32_t trunc_u32(double v) /* float values widen exactly */
{
    if (!(v > 0.0)) return 0u;                 /* negative, zero or NaN */
    if (v >= 4294967296.0) return 0xFFFFFFFFu; /* saturate at 2^32 - 1 */
    return (uint32_t)v;                        /* C conversion truncates toward zero */
}

/* plain form: m(H * m(z - X0)) */
static double fval_plain_f64(double H, double X0, double z)
{
    double D = z - X0;
    return H * D;
}
static float fval_plain_f32(float H, float X0, float z)
{
    float D = z - X0;
    return H * D;
}
/* FMA form: m(H z - W), one rounding */
static double fval_fma_f64(double H, double W, double z) { return fma(H, z, -W); }
static float fval_fma_f32(float H, float W, float z) { return fmaf(H, z, -W); }

/* ------------------------------------------------------------------------ */
/* ComputeHR (Section 4.4).  out: H, W, R, number of H updates, passes, and */
/* the knot index that made the array infeasible (or -1).                   */
/* ------------------------------------------------------------------------ */
int or_compute_hr_f64(const double *X, int64_t n_knots, int fma_form, double *H_out, double *W_out,
                      uint32_t *R_out, int64_t *updates_out, int64_t *passes_out, int64_t *bad_out)
{
    *H_out = 0; *W_out = 0; *R_out = 0; *updates_out = 0; *passes_out = 0; *bad_out = -1;
    if (n_knots < 2) return OR_E_ARG;
    const int64_t N = n_knots - 1;
    /* the problem statement requires a strictly increasing array of finite numbers */
    for (int64_t i = 0; i <= N; ++i)
        if (!isfinite(X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    for (int64_t i = 1; i <= N; ++i)
        if (!(X[i - 1] < X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    const double X0 = X[0];
    /* Eq. distinguishable-exact: D_i = m(X_i - X_0) strictly increasing */
    for (int64_t i = 1; i <= N; ++i) {
        double Dprev = X[i - 1] - X0, Di = X[i] - X0;
        if (Dprev == Di) { *bad_out = i; return OR_E_INDISTINGUISHABLE; }
    }
    /* Eq. minhnumeric: Hbar = m(1 / min_i m(D_{i+1} - D_i)) */
    double dmin = INFINITY;
    for (int64_t i = 0; i < N; ++i) {
        double Dnext = X[i + 1] - X0, Di = X[i] - X0;
        double g = Dnext - Di;
        if (g < dmin) dmin = g;
    }
    double Hbar = 1.0 / dmin;
    double H = nextafter(Hbar, INFINITY); /* phi(Hbar) */
    double W = H * X0;
#define OR_F64(x) (fma_form ? fval_fma_f64(H, W, (x)) : fval_plain_f64(H, X0, (x)))
    /* Eq. overflowexact */
    if (!(OR_F64(X[N]) < 4294967296.0)) { *bad_out = N; return OR_E_OVERFLOW; }
    double P = nextafter(H, INFINITY) - H; /* growth term */
    int64_t updates = 0, passes = 0;
    int changed;
    do {
        changed = 0;
        ++passes;
        for (int64_t i = 1; i <= N; ++i) {
            /* Eq. cond2 for the pair (i-1, i) */
            while (trunc_u32(OR_F64(X[i - 1])) == trunc_u32(OR_F64(X[i]))) {
                H = H + P;
                W = H * X0;
                if (!(OR_F64(X[N]) < 4294967296.0)) {
                    *bad_out = i; *H_out = H; *updates_out = updates + 1; *passes_out = passes;
                    return OR_E_OVERFLOW;
                }
                P = 2.0 * P;
                ++updates;
                changed = 1;
            }
        }
    } while (changed && passes < OR_MAX_PASSES);
    *H_out = H; *W_out = W; *updates_out = updates; *passes_out = passes;
    if (changed) return OR_E_NO_CONVERGENCE;
    *R_out = trunc_u32(OR_F64(X[N]));
#undef OR_F64
    return OR_OK;
}

int or_compute_hr_f32(const float *X, int64_t n_knots, int fma_form, double *H_out, double *W_out,
                      uint32_t *R_out, int64_t *updates_out, int64_t *passes_out, int64_t *bad_out)
{
    *H_out = 0; *W_out = 0; *R_out = 0; *updates_out = 0; *passes_out = 0; *bad_out = -1;
    if (n_knots < 2) return OR_E_ARG;
    const int64_t N = n_knots - 1;
    for (int64_t i = 0; i <= N; ++i)
        if (!isfinite(X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    for (int64_t i = 1; i <= N; ++i)
        if (!(X[i - 1] < X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    const float X0 = X[0];
    for (int64_t i = 1; i <= N; ++i) {
        float Dprev = X[i - 1] - X0, Di = X[i] - X0;
        if (Dprev == Di) { *bad_out = i; return OR_E_INDISTINGUISHABLE; }
    }
    float dmin = INFINITY;
    for (int64_t i = 0; i < N; ++i) {
        float Dnext = X[i + 1] - X0, Di = X[i] - X0;
        float g = Dnext - Di;
        if (g < dmin) dmin = g;
    }
    float Hbar = 1.0f / dmin;
    float H = nextafterf(Hbar, INFINITY);
    float W = H * X0;
#define OR_F32(x) (fma_form ? fval_fma_f32(H, W, (x)) : fval_plain_f32(H, X0, (x)))
    if (!((double)OR_F32(X[N]) < 4294967296.0)) { *bad_out = N; *H_out = H; return OR_E_OVERFLOW; }
    float P = nextafterf(H, INFINITY) - H;
    int64_t updates = 0, passes = 0;
    int changed;
    do {
        changed = 0;
        ++passes;
        for (int64_t i = 1; i <= N; ++i) {
            while (trunc_u32(OR_F32(X[i - 1])) == trunc_u32(OR_F32(X[i]))) {
                H = H + P;
                W = H * X0;
                if (!((double)OR_F32(X[N]) < 4294967296.0)) {
                    *bad_out = i; *H_out = H; *updates_out = updates + 1; *passes_out = passes;
                    return OR_E_OVERFLOW;
                }
                P = 2.0f * P;
                ++updates;
                changed = 1;
            }
        }
    } while (changed && passes < OR_MAX_PASSES);
    *H_out = H; *W_out = W; *updates_out = updates; *passes_out = passes;
    if (changed) return OR_E_NO_CONVERGENCE;
    *R_out = trunc_u32(OR_F32(X[N]));
#undef OR_F32
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. indexdef, written out: F_i = f(X_i); K starts at 0 and, for each i,   */
/* the cells F_{i-1}+1 .. F_i receive i.  Cells 0..F_0 keep 0.  K has R+1    */
/* entries.  F must be strictly increasing with F_N = R (properties fprop).  */
/* ------------------------------------------------------------------------ */
int or_fill_k_f64(const double *X, int64_t n_knots, double H, double W, uint32_t R, int fma_form,
                  int32_t *K, uint32_t *F)
{
    const int64_t N = n_knots - 1;
    const double X0 = X[0];
    for (int64_t i = 0; i <= N; ++i)
        F[i] = trunc_u32(fma_form ? fval_fma_f64(H, W, X[i]) : fval_plain_f64(H, X0, X[i]));
    for (int64_t i = 1; i <= N; ++i)
        if (!(F[i - 1] < F[i])) return OR_E_BAD_TABLE;
    if (F[N] != R) return OR_E_BAD_TABLE;
    memset(K, 0, sizeof(int32_t) * ((size_t)R + 1));
    for (int64_t i = 1; i <= N; ++i)
        for (uint64_t j = (uint64_t)F[i - 1] + 1; j <= F[i]; ++j) K[j] = (int32_t)i;
    return OR_OK;
}

int or_fill_k_f32(const float *X, int64_t n_knots, double H, double W, uint32_t R, int fma_form,
                  int32_t *K, uint32_t *F)
{
    const int64_t N = n_knots - 1;
    const float X0 = X[0], Hf = (float)H, Wf = (float)W;
    for (int64_t i = 0; i <= N; ++i)
        F[i] = trunc_u32(fma_form ? fval_fma_f32(Hf, Wf, X[i]) : fval_plain_f32(Hf, X0, X[i]));
    for (int64_t i = 1; i <= N; ++i)
        if (!(F[i - 1] < F[i])) return OR_E_BAD_TABLE;
    if (F[N] != R) return OR_E_BAD_TABLE;
    memset(K, 0, sizeof(int32_t) * ((size_t)R + 1));
    for (int64_t i = 1; i <= N; ++i)
        for (uint64_t j = (uint64_t)F[i - 1] + 1; j <= F[i]; ++j) K[j] = (int32_t)i;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm "direct": j = f(z) (clamped to R so that every z is memory-safe),*/
/* t = K_j, i = t - [z < X_t].                                              */
/* ------------------------------------------------------------------------ */
void or_direct_f64(const double *X, const int32_t *K, double H, double W, uint32_t R, int fma_form,
                   const double *Z, int64_t m, int32_t *I)
{
    const double X0 = X[0];
    for (int64_t q = 0; q < m; ++q) {
        double z = Z[q];
        uint32_t j = trunc_u32(fma_form ? fval_fma_f64(H, W, z) : fval_plain_f64(H, X0, z));
        if (j > R) j = R;
        int32_t t = K[j];
        I[q] = t - (z < X[t] ? 1 : 0);
    }
}

void or_direct_f32(const float *X, const int32_t *K, double H, double W, uint32_t R, int fma_form,
                   const float *Z, int64_t m, int32_t *I)
{
    const float X0 = X[0], Hf = (float)H, Wf = (float)W;
    for (int64_t q = 0; q < m; ++q) {
        float z = Z[q];
        uint32_t j = trunc_u32(fma_form ? fval_fma_f32(Hf, Wf, z) : fval_plain_f32(Hf, X0, z));
        if (j > R) j = R;
        int32_t t = K[j];
        I[q] = t - (z < X[t] ? 1 : 0);
    }
}

/* f itself, exposed so tests can pin its rounding against closed forms. */
void or_fvals_f64(double H, double W, double X0, int fma_form, const double *Z, int64_t m, uint32_t *J)
{
    for (int64_t q = 0; q < m; ++q)
        J[q] = trunc_u32(fma_form ? fval_fma_f64(H, W, Z[q]) : fval_plain_f64(H, X0, Z[q]));
}

void or_fvals_f32(double H, double W, double X0, int fma_form, const float *Z, int64_t m, uint32_t *J)
{
    const float Hf = (float)H, Wf = (float)W, X0f = (float)X0;
    for (int64_t q = 0; q < m; ++q)
        J[q] = trunc_u32(fma_form ? fval_fma_f32(Hf, Wf, Z[q]) : fval_plain_f32(Hf, X0f, Z[q]));
}

/* Fused linear interpolation reference (the use case of the Introduction):
 * y = Y_i + (Y_{i+1} - Y_i) * (z - X_i) / (X_{i+1} - X_i) evaluated in double
 * from float inputs (exact widening), i from the definition above. */
void or_interp_f32(const float *X, const float *Y, int64_t n_knots, const float *Z, int64_t m,
                   int32_t *I, double *y)
{
    for (int64_t q = 0; q < m; ++q) {
        int64_t i = count_le_f32(X, n_knots, Z[q]) - 1;
        I[q] = (int32_t)i;
        if (i < 0 || i >= n_knots - 1) { y[q] = NAN; continue; }
        double x0 = X[i], x1 = X[i + 1], y0 = Y[i], y1 = Y[i + 1], z = Z[q];
        y[q] = y0 + (y1 - y0) * ((z - x0) / (x1 - x0));
    }
}

/* ------------------------------------------------------------------------ */
/* DirectGap2 and its generalisation (Section 4.7): f need only satisfy      */
/* f(X_{i+q}) > f(X_i) (Eq. f-monotonic-2 for q = 2, Eq. f-monotonic-n in    */
/* general), so H > 1/min(X_{i+q} - X_i) (Eq. fcond11 for q = 2), taken in   */
/* its rounded form m(1/min m(D_{i+q} - D_i)), and the growth loop of        */
/* ComputeHR runs over the pairs (i, i+q) ("algorithm ComputeHR needs to be  */
/* modified accordingly").  D_i == D_{i+q} is not allowed; closer pairs may  */
/* share a cell.  With fewer than q+1 knots the pair distance is N.  q = 1   */
/* is ComputeHR itself.                                                      */
/* ------------------------------------------------------------------------ */
static int compute_hr_gapq_track_f64(const double *X, int64_t n_knots, int32_t q, int fma_form, double *H_out,
                                       double *W_out, uint32_t *R_out, int64_t *updates_out, int64_t *passes_out,
                                       int64_t *bad_out, double *H_inf_out)
{
    *H_out = 0; *W_out = 0; *R_out = 0; *updates_out = 0; *passes_out = 0; *bad_out = -1;
    if (n_knots < 2 || q < 1) return OR_E_ARG;
    const int64_t N = n_knots - 1;
    const int64_t gap = N >= q ? q : N;
    for (int64_t i = 0; i <= N; ++i)
        if (!isfinite(X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    for (int64_t i = 1; i <= N; ++i)
        if (!(X[i - 1] < X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    const double X0 = X[0];
    for (int64_t i = gap; i <= N; ++i) {
        double Da = X[i - gap] - X0, Db = X[i] - X0;
        if (Da == Db) { *bad_out = i; return OR_E_INDISTINGUISHABLE; }
    }
    double dmin = INFINITY;
    for (int64_t i = gap; i <= N; ++i) {
        double Db = X[i] - X0, Da = X[i - gap] - X0;
        double g = Db - Da;
        if (g < dmin) dmin = g;
    }
    double H = nextafter(1.0 / dmin, INFINITY);
    double W = H * X0;
#define OR_G64(x) (fma_form ? fval_fma_f64(H, W, (x)) : fval_plain_f64(H, X0, (x)))
    if (!(OR_G64(X[N]) < 4294967296.0)) { *bad_out = N; return OR_E_OVERFLOW; }
    double P = nextafter(H, INFINITY) - H;
    int64_t updates = 0, passes = 0;
    int changed;
    do {
        changed = 0;
        ++passes;
        for (int64_t i = gap; i <= N; ++i) {
            while (trunc_u32(OR_G64(X[i - gap])) == trunc_u32(OR_G64(X[i]))) {
                if (H_inf_out) *H_inf_out = H; /* the last H found infeasible */
                H = H + P;
                W = H * X0;
                if (!(OR_G64(X[N]) < 4294967296.0)) { *bad_out = i; *H_out = H; return OR_E_OVERFLOW; }
                P = 2.0 * P;
                ++updates;
                changed = 1;
            }
        }
    } while (changed && passes < OR_MAX_PASSES);
    *H_out = H; *W_out = W; *updates_out = updates; *passes_out = passes;
    if (changed) return OR_E_NO_CONVERGENCE;
    *R_out = trunc_u32(OR_G64(X[N]));
#undef OR_G64
    return OR_OK;
}

static int compute_hr_gapq_track_f32(const float *X, int64_t n_knots, int32_t q, int fma_form, double *H_out,
                                       double *W_out, uint32_t *R_out, int64_t *updates_out, int64_t *passes_out,
                                       int64_t *bad_out, double *H_inf_out)
{
    *H_out = 0; *W_out = 0; *R_out = 0; *updates_out = 0; *passes_out = 0; *bad_out = -1;
    if (n_knots < 2 || q < 1) return OR_E_ARG;
    const int64_t N = n_knots - 1;
    const int64_t gap = N >= q ? q : N;
    for (int64_t i = 0; i <= N; ++i)
        if (!isfinite(X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    for (int64_t i = 1; i <= N; ++i)
        if (!(X[i - 1] < X[i])) { *bad_out = i; return OR_E_NOT_INCREASING; }
    const float X0 = X[0];
    for (int64_t i = gap; i <= N; ++i) {
        float Da = X[i - gap] - X0, Db = X[i] - X0;
        if (Da == Db) { *bad_out = i; return OR_E_INDISTINGUISHABLE; }
    }
    float dmin = INFINITY;
    for (int64_t i = gap; i <= N; ++i) {
        float Db = X[i] - X0, Da = X[i - gap] - X0;
        float g = Db - Da;
        if (g < dmin) dmin = g;
    }
    float H = nextafterf(1.0f / dmin, INFINITY);
    float W = H * X0;
#define OR_G32(x) (fma_form ? fval_fma_f32(H, W, (x)) : fval_plain_f32(H, X0, (x)))
    if (!((double)OR_G32(X[N]) < 4294967296.0)) { *bad_out = N; *H_out = H; return OR_E_OVERFLOW; }
    float P = nextafterf(H, INFINITY) - H;
    int64_t updates = 0, passes = 0;
    int changed;
    do {
        changed = 0;
        ++passes;
        for (int64_t i = gap; i <= N; ++i) {
            while (trunc_u32(OR_G32(X[i - gap])) == trunc_u32(OR_G32(X[i]))) {
                if (H_inf_out) *H_inf_out = H; /* the last H found infeasible */
                H = H + P;
                W = H * X0;
                if (!((double)OR_G32(X[N]) < 4294967296.0)) { *bad_out = i; *H_out = H; return OR_E_OVERFLOW; }
                P = 2.0f * P;
                ++updates;
                changed = 1;
            }
        }
    } while (changed && passes < OR_MAX_PASSES);
    *H_out = H; *W_out = W; *updates_out = updates; *passes_out = passes;
    if (changed) return OR_E_NO_CONVERGENCE;
    *R_out = trunc_u32(OR_G32(X[N]));
#undef OR_G32
    return OR_OK;
}

int or_compute_hr_gapq_f64(const double *X, int64_t n_knots, int32_t q, int fma_form, double *H_out, double *W_out,
                           uint32_t *R_out, int64_t *updates_out, int64_t *passes_out, int64_t *bad_out)
{
    return compute_hr_gapq_track_f64(X, n_knots, q, fma_form, H_out, W_out, R_out, updates_out, passes_out, bad_out,
                                     0);
}

int or_compute_hr_gapq_f32(const float *X, int64_t n_knots, int32_t q, int fma_form, double *H_out, double *W_out,
                           uint32_t *R_out, int64_t *updates_out, int64_t *passes_out, int64_t *bad_out)
{
    return compute_hr_gapq_track_f32(X, n_knots, q, fma_form, H_out, W_out, R_out, updates_out, passes_out, bad_out,
                                     0);
}

/* ------------------------------------------------------------------------ */
/* Refinement of H by bisection (end of Section 4.4): when ComputeHR had to  */
/* grow H, the last value found infeasible and the final, feasible one bound */
/* an interval; bisect it for the smallest feasible H it can reach.  Each    */
/* probe checks the whole array (every pair (i, i+q) and the overflow test). */
/* The midpoint is taken on the bit patterns (positive floats order like     */
/* their patterns), so the steps are exact integer arithmetic.               */
/* ------------------------------------------------------------------------ */
static int feasible_f64(const double *X, int64_t n_knots, int64_t gap, int fma_form, double H)
{
    const int64_t N = n_knots - 1;
    const double X0 = X[0], W = H * X0;
#define OR_P64(x) (fma_form ? fval_fma_f64(H, W, (x)) : fval_plain_f64(H, X0, (x)))
    if (!(OR_P64(X[N]) < 4294967296.0)) return 0;
    for (int64_t i = gap; i <= N; ++i)
        if (trunc_u32(OR_P64(X[i - gap])) == trunc_u32(OR_P64(X[i]))) return 0;
#undef OR_P64
    return 1;
}

static int feasible_f32(const float *X, int64_t n_knots, int64_t gap, int fma_form, float H)
{
    const int64_t N = n_knots - 1;
    const float X0 = X[0], W = H * X0;
#define OR_P32(x) (fma_form ? fval_fma_f32(H, W, (x)) : fval_plain_f32(H, X0, (x)))
    if (!((double)OR_P32(X[N]) < 4294967296.0)) return 0;
    for (int64_t i = gap; i <= N; ++i)
        if (trunc_u32(OR_P32(X[i - gap])) == trunc_u32(OR_P32(X[i]))) return 0;
#undef OR_P32
    return 1;
}

int or_compute_hr_refined_f64(const double *X, int64_t n_knots, int32_t q, int fma_form, double *H_out,
                              double *W_out, uint32_t *R_out, int64_t *updates_out, int64_t *passes_out,
                              int64_t *bad_out, int64_t *probes_out)
{
    double H_inf = 0;
    *probes_out = 0;
    int st = compute_hr_gapq_track_f64(X, n_knots, q, fma_form, H_out, W_out, R_out, updates_out, passes_out, bad_out,
                                       &H_inf);
    if (st != OR_OK || *updates_out == 0) return st;
    const int64_t N = n_knots - 1, gap = N >= q ? q : N;
    uint64_t lo, hi;
    double Hf = *H_out;
    memcpy(&lo, &H_inf, 8);
    memcpy(&hi, &Hf, 8);
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        double Hm;
        memcpy(&Hm, &mid, 8);
        ++*probes_out;
        if (feasible_f64(X, n_knots, gap, fma_form, Hm)) hi = mid;
        else lo = mid;
    }
    memcpy(&Hf, &hi, 8);
    const double X0 = X[0], W = Hf * X0;
    *H_out = Hf;
    *W_out = W;
    *R_out = trunc_u32(fma_form ? fval_fma_f64(Hf, W, X[N]) : fval_plain_f64(Hf, X0, X[N]));
    return OR_OK;
}

int or_compute_hr_refined_f32(const float *X, int64_t n_knots, int32_t q, int fma_form, double *H_out,
                              double *W_out, uint32_t *R_out, int64_t *updates_out, int64_t *passes_out,
                              int64_t *bad_out, int64_t *probes_out)
{
    double H_inf = 0;
    *probes_out = 0;
    int st = compute_hr_gapq_track_f32(X, n_knots, q, fma_form, H_out, W_out, R_out, updates_out, passes_out, bad_out,
                                       &H_inf);
    if (st != OR_OK || *updates_out == 0) return st;
    const int64_t N = n_knots - 1, gap = N >= q ? q : N;
    const float Hi = (float)H_inf, Hfe = (float)*H_out;
    uint32_t lo, hi;
    memcpy(&lo, &Hi, 4);
    memcpy(&hi, &Hfe, 4);
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        float Hm;
        memcpy(&Hm, &mid, 4);
        ++*probes_out;
        if (feasible_f32(X, n_knots, gap, fma_form, Hm)) hi = mid;
        else lo = mid;
    }
    float Hf;
    memcpy(&Hf, &hi, 4);
    const float X0 = X[0], W = Hf * X0;
    *H_out = Hf;
    *W_out = W;
    *R_out = trunc_u32(fma_form ? fval_fma_f32(Hf, W, X[N]) : fval_plain_f32(Hf, X0, X[N]));
    return OR_OK;
}

int or_compute_hr_gap2_f64(const double *X, int64_t n_knots, int fma_form, double *H_out, double *W_out,
                           uint32_t *R_out, int64_t *updates_out, int64_t *passes_out, int64_t *bad_out)
{
    return or_compute_hr_gapq_f64(X, n_knots, 2, fma_form, H_out, W_out, R_out, updates_out, passes_out, bad_out);
}

int or_compute_hr_gap2_f32(const float *X, int64_t n_knots, int fma_form, double *H_out, double *W_out,
                           uint32_t *R_out, int64_t *updates_out, int64_t *passes_out, int64_t *bad_out)
{
    return or_compute_hr_gapq_f32(X, n_knots, 2, fma_form, H_out, W_out, R_out, updates_out, passes_out, bad_out);
}

/* Eq. kgeneral written out: K_j = max{ i : F_i <= j }, j = 0..R (0 where no
 * knot qualifies, which only cells below F_0 can be). */
static void fill_k_general(const uint32_t *F, int64_t n_knots, uint32_t R, int32_t *K)
{
    int64_t i = -1;
    for (uint64_t j = 0; j <= R; ++j) {
        while (i + 1 < n_knots && F[i + 1] <= j) ++i;
        K[j] = (int32_t)(i < 0 ? 0 : i);
    }
}

/* F and the table of Eq. kgeneral for a given (H, W, R); checks that F is
 * non-decreasing, that F_{i+q} > F_i (Eq. f-monotonic-n) and that F_N = R. */
int or_fill_k_gapq_f64(const double *X, int64_t n_knots, int32_t q, double H, double W, uint32_t R, int fma_form,
                       int32_t *K, uint32_t *F)
{
    const int64_t N = n_knots - 1;
    const double X0 = X[0];
    if (q < 1) return OR_E_ARG;
    for (int64_t i = 0; i <= N; ++i)
        F[i] = trunc_u32(fma_form ? fval_fma_f64(H, W, X[i]) : fval_plain_f64(H, X0, X[i]));
    for (int64_t i = 1; i <= N; ++i)
        if (F[i - 1] > F[i]) return OR_E_BAD_TABLE;
    for (int64_t i = q; i <= N; ++i)
        if (!(F[i - q] < F[i])) return OR_E_BAD_TABLE;
    if (F[N] != R) return OR_E_BAD_TABLE;
    fill_k_general(F, n_knots, R, K);
    return OR_OK;
}

int or_fill_k_gapq_f32(const float *X, int64_t n_knots, int32_t q, double H, double W, uint32_t R, int fma_form,
                       int32_t *K, uint32_t *F)
{
    const int64_t N = n_knots - 1;
    const float X0 = X[0], Hf = (float)H, Wf = (float)W;
    if (q < 1) return OR_E_ARG;
    for (int64_t i = 0; i <= N; ++i)
        F[i] = trunc_u32(fma_form ? fval_fma_f32(Hf, Wf, X[i]) : fval_plain_f32(Hf, X0, X[i]));
    for (int64_t i = 1; i <= N; ++i)
        if (F[i - 1] > F[i]) return OR_E_BAD_TABLE;
    for (int64_t i = q; i <= N; ++i)
        if (!(F[i - q] < F[i])) return OR_E_BAD_TABLE;
    if (F[N] != R) return OR_E_BAD_TABLE;
    fill_k_general(F, n_knots, R, K);
    return OR_OK;
}

int or_fill_k_gap2_f64(const double *X, int64_t n_knots, double H, double W, uint32_t R, int fma_form,
                       int32_t *K, uint32_t *F)
{
    return or_fill_k_gapq_f64(X, n_knots, 2, H, W, R, fma_form, K, F);
}

int or_fill_k_gap2_f32(const float *X, int64_t n_knots, double H, double W, uint32_t R, int fma_form,
                       int32_t *K, uint32_t *F)
{
    return or_fill_k_gapq_f32(X, n_knots, 2, H, W, R, fma_form, K, F);
}

/* Algorithm direct-2 and its q-knot generalisation: t = K_j,
 * i = t - [z < X_t] - [z < X_{t-1}] - ... - [z < X_{t-q+1}], with the left
 * padding X_{-1} = X_{-2} = ... = X_0; the result is clamped at -1 so that
 * z < X_0 answers -1 like the definition. */
void or_direct_gapq_f64(const double *X, const int32_t *K, int32_t q, double H, double W, uint32_t R, int fma_form,
                        const double *Z, int64_t m, int32_t *I)
{
    const double X0 = X[0];
    for (int64_t k = 0; k < m; ++k) {
        double z = Z[k];
        uint32_t j = trunc_u32(fma_form ? fval_fma_f64(H, W, z) : fval_plain_f64(H, X0, z));
        if (j > R) j = R;
        int32_t t = K[j];
        int32_t i = t;
        for (int32_t l = 0; l < q; ++l) {
            double x = t - l >= 0 ? X[t - l] : X0;
            if (z < x) --i;
        }
        I[k] = i < -1 ? -1 : i;
    }
}

void or_direct_gapq_f32(const float *X, const int32_t *K, int32_t q, double H, double W, uint32_t R, int fma_form,
                        const float *Z, int64_t m, int32_t *I)
{
    const float X0 = X[0], Hf = (float)H, Wf = (float)W;
    for (int64_t k = 0; k < m; ++k) {
        float z = Z[k];
        uint32_t j = trunc_u32(fma_form ? fval_fma_f32(Hf, Wf, z) : fval_plain_f32(Hf, X0, z));
        if (j > R) j = R;
        int32_t t = K[j];
        int32_t i = t;
        for (int32_t l = 0; l < q; ++l) {
            float x = t - l >= 0 ? X[t - l] : X0;
            if (z < x) --i;
        }
        I[k] = i < -1 ? -1 : i;
    }
}

void or_direct_gap2_f64(const double *X, const int32_t *K, double H, double W, uint32_t R, int fma_form,
                        const double *Z, int64_t m, int32_t *I)
{
    or_direct_gapq_f64(X, K, 2, H, W, R, fma_form, Z, m, I);
}

void or_direct_gap2_f32(const float *X, const int32_t *K, double H, double W, uint32_t R, int fma_form,
                        const float *Z, int64_t m, int32_t *I)
{
    or_direct_gapq_f32(X, K, 2, H, W, R, fma_form, Z, m, I);
}
