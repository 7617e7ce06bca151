// ds_multi.cuh -- many independent knot arrays searched by one persistent
// launch ("vectorial problem" of Section 2 over a ragged CSR batch).
//
// Work is split into chunks of at most `chunk` consecutive queries of one
// array.  A small planning kernel turns the query offsets z_off into chunk
// offsets on the device (so the whole search is stream-ordered and can be
// captured in a CUDA graph); persistent blocks then claim chunks with an
// atomic counter.  A block that claims a chunk of an array whose image (its
// K table and knots, or the learned predictor's tables) fits the shared-memory
// budget stages that image with a bulk asynchronous copy, unless it already
// holds it from its previous chunk; other arrays are read from global memory,
// where the array being worked on stays L2-resident.
//
// Per-array modes:
//   MODE_DIRECT    Algorithm direct with the array's own H, W, R, K.
//   MODE_LEARNED   predicted index, bounded window, certificate, exact
//                  fall-back; the window is searched in two fixed-depth
//                  levels: over every 32nd knot (a small, L2-resident copy),
//                  then over at most 32 knots.
//   MODE_BISECT    fixed-depth bisection over all knots (Algorithm
//                  binaryoptnopad), the log-time fall-back where direct
//                  search is infeasible.
#pragma once

#include "ds_search.cuh"

namespace ds {

enum ArrMode : int32_t { MODE_DIRECT = 0, MODE_LEARNED = 1, MODE_BISECT = 2 };

// Sampling stride of the learned window search: S_k = X_{min(k * SG_STRIDE, N)}.
// 32 measured faster than 8 on the 2^24-knot learned workload (13.5 against
// 11.7 G lookups/s: the 4x larger sample table raised DRAM reads per lookup
// from 146 to 181 bytes).
constexpr int SG_SHIFT = 5;
constexpr int SG_STRIDE = 1 << SG_SHIFT;

// 128 bytes per array.
struct __align__(16) ArrDesc {
    long long img;        // byte offset of the staged image in the blob
    long long xg;         // byte offset of the knots in the blob
    long long yoff;       // element offset of the array's knot values Y in the caller's Ycat
    uint32_t img_bytes;   // bytes of the image (multiple of 16), 0 if nothing to stage
    uint32_t x_in_img;    // byte offset of the knots inside the image (direct mode)
    int32_t n;            // N: the array has N+1 knots
    int32_t mode;         // ArrMode
    uint32_t R;           // direct: largest cell
    int32_t form;         // direct: FForm
    int32_t pbits;        // bisection over all knots: 2^floor(log2 N)
    int32_t aux;          // learned: 2^floor(log2(window width)); direct: 1 if K entries carry
                          // fingerprints (bits 24..30, t in bits 0..23)
    double H, W, X0;      // direct: parameters in the array's precision (held exactly)
    double XN;            // last knot
    float uscale;         // learned: u = (narrow(z) - x0f) * uscale (float32)
    float x0f;            // learned: narrow(X0)
    int32_t e_lo, e_hi;   // learned: recorded error bounds
    int32_t seg_off;      // learned: first predictor segment in the model tables
    int32_t seg_n;        // learned: number of predictor segments
    long long sg;         // learned: byte offset of the sampled knots S_k = X_{min(32 k, N)}, k = 0..N/32+1
};
static_assert(sizeof(ArrDesc) == 128, "ArrDesc layout");

template <typename T> struct BatchArgs {
    const ArrDesc *desc;
    const unsigned char *blob;
    const long long *z_off;     // n_arrays+1 (device), or nullptr for a single array of m queries
    long long m_single;
    int32_t n_arrays;
    const T *Z;
    int32_t *I;
    const T *Y;                 // knot values (interpolation) or nullptr
    T *y_out;
    long long *chunk_off;       // n_arrays+1 chunk offsets (written by the planner)
    unsigned long long *counter;// chunk counter (reset by the planner)
    unsigned long long *fallbacks; // learned: certificate failures
    long long chunk;            // queries per chunk
    uint32_t smem_limit;        // largest image staged in shared memory
    int checked;
    int *err;
    // learned predictor tables (device): breakpoints, slopes, intercepts
    const float *seg_x;
    const float *seg_a;
    const float *seg_b;
};

// Chunk offsets from the query offsets; resets the chunk counter.  One block.
__global__ void k_plan_chunks(const long long *z_off, long long m_single, int n_arrays, long long chunk,
                              long long *chunk_off, unsigned long long *counter);

__device__ __forceinline__ long long q_begin(const long long *z_off, int a) { return z_off ? z_off[a] : 0; }

// ------------------------------------------------------------------ per-query pieces
template <typename T>
__device__ __forceinline__ uint32_t cell_rt(T z, const ArrDesc &d)
{
    using A = Arith<T>;
    const T H = (T)d.H;
    T v;
    if (d.form == F_FMA) v = A::fma(H, z, -(T)d.W);
    else if (d.form == F_PLAIN_X0ZERO) v = A::mul(H, z);
    else v = A::mul(H, A::sub(z, (T)d.X0));
    uint32_t j;
    if constexpr (sizeof(T) == 8) j = trunc_u32_bits((double)v);
    else j = A::trunc_u32(v);
    return min(j, d.R);
}

// Cell and fingerprint of a query (cell_fp_bits); a query past the last
// cell gets FP_ABOVE, larger than any knot's fingerprint in cell R.
template <typename T>
__device__ __forceinline__ uint32_t cell_rt_fp(T z, const ArrDesc &d, uint32_t *g)
{
    using A = Arith<T>;
    const T H = (T)d.H;
    T v;
    if (d.form == F_FMA) v = A::fma(H, z, -(T)d.W);
    else if (d.form == F_PLAIN_X0ZERO) v = A::mul(H, z);
    else v = A::mul(H, A::sub(z, (T)d.X0));
    const uint32_t j = cell_fp_bits(v, g);
    if (j > d.R) {
        *g = FP_ABOVE;
        return d.R;
    }
    return j;
}

constexpr uint32_t FP_T_MASK = 0x00FFFFFFu;  // t of a K entry that carries a fingerprint
constexpr int FP_SHIFT = 24;
constexpr long long FP_MAX_KNOTS = 1ll << 24;

template <typename T> __device__ __forceinline__ bool lt_exact(T a, T b)
{
    if constexpr (sizeof(T) == 8) return okey((double)a) < okey((double)b);
    else return a < b;
}

// Largest i in [lo, lo + n - 1] with X_i <= z, given X_lo <= z and
// z < X_{lo+n} (fixed depth, Algorithm binaryoptnopad on X[lo .. lo+n]);
// `top` = 2^floor(log2 n) (or any larger power of two).
template <typename T>
__device__ __forceinline__ int32_t bisect(const T *X, int32_t lo, int32_t n, int32_t top, T z)
{
    int32_t i = 0;
    for (int32_t k = top; k > 0; k >>= 1) {
        const int32_t r = i | k;
        const int32_t w = r < n ? r : n;
        if (!lt_exact<T>(z, X[lo + w])) i = r;
    }
    return lo + (i < n ? i : n);
}

template <typename T, bool INTERP>
__device__ __forceinline__ void interp_store(const BatchArgs<T> &a, const ArrDesc &d, const T *X, long long q,
                                             T z, int32_t i)
{
    if constexpr (INTERP) {
        using A = Arith<T>;
        T y;
        if (i >= 0 && i < d.n) {
            const T x0 = X[i], x1 = X[i + 1];
            const T y0 = a.Y[d.yoff + i], y1 = a.Y[d.yoff + i + 1];
            // y = Y_i + (Y_{i+1} - Y_i) * ((z - X_i) / (X_{i+1} - X_i)), each step rounded once
            const T t = A::div(A::sub(z, x0), A::sub(x1, x0));
            y = A::fma(A::sub(y1, y0), t, y0);
        } else {
            y = T(NAN);
        }
        a.y_out[q] = y;
    }
}

}  // namespace ds
