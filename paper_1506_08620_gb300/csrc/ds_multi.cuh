// ds_multi.cuh -- many independent knot arrays searched by one persistent
// launch ("vectorial problem" of Section 2 over a ragged CSR batch).
//
// Work is split into chunks of at most `chunk` consecutive queries of one
// array.  A small planning kernel turns the query offsets z_off into chunk
// offsets on the device (so the whole search is stream-ordered and can be
// captured in a CUDA graph); persistent blocks then claim chunks with an
// atomic counter.  A block that claims a chunk of an array whose image (the
// rank table of a direct array, the cell map of a learned one, or the knots
// of a bisected one) fits the shared-memory budget stages that image with a
// bulk asynchronous copy, unless it already holds it from its previous chunk;
// other arrays are read from global memory, where the array being worked on
// stays L2-resident.
//
// Per-array modes:
//   MODE_DIRECT    Algorithm direct with the array's own H, W, R; K is held
//                  as a rank table with knot fingerprints (below).
//   MODE_LEARNED   direct search on a learned cell map: the cell of z is
//                  j = f(z) with f a monotone piecewise-linear map sampled
//                  from the trained network's CDF (uniform in predicted
//                  rank, not in z), K_j = #{i : f(X_i) < j} (Eq. indexdef
//                  with cells that may hold several knots), and the answer is
//                  K_j - 1 plus the number of the cell's knots <= z.
//   MODE_BISECT    fixed-depth bisection over all knots (Algorithm
//                  binaryoptnopad), the log-time fall-back where direct
//                  search is infeasible.
//
// Knots are stored either alone (stride xs = 1) or, when the handle holds
// the knot values Y of the interpolation, as (X_i, Y_i) pairs (stride xs =
// 2), so that one lookup's four operands lie in 16 contiguous bytes.
#pragma once

#include "ds_search.cuh"

namespace ds {

enum ArrMode : int32_t { MODE_DIRECT = 0, MODE_LEARNED = 1, MODE_BISECT = 2 };

// Learned cell maps: G uniform macro cells over u = (z - X_0) / (X_N - X_0)
// in [0, 1), each holding the first cells {J_g, J_{g+1}} of its span (8 bytes).
constexpr int LMAP_MAX = 4096;  // largest G (32 KB, staged in shared memory)
constexpr int LMAP_MIN = 64;
// Learned cell table: a 16-byte block per 8 cells, K_{8b} then the
// differences K_{8b+r} - K_{8b}, r = 1..8, in 12 bits each.  A block whose 8
// cells hold more than LBLK_MAXSPAN knots is escaped: its first word is
// LBLK_ESC and its second the position of its 9 values K_{8b} .. K_{8b+8}
// (uint32) in the overflow area that follows the array's blocks.
constexpr int LBLK_SHIFT = 3;
constexpr uint32_t LBLK_MAXSPAN = 4095;
constexpr uint32_t LBLK_ESC = 0x80000000u;  // K <= 2^31 - 1, so bit 31 of K_{8b} is free
__host__ __device__ __forceinline__ unsigned long long lblk_count(uint32_t R) { return ((unsigned long long)R + 1ull) / 8ull + 1ull; }

constexpr uint32_t NO_X_IN_IMG = 0xFFFFFFFFu;  // the image does not hold the knots

// 128 bytes per array.
struct __align__(16) ArrDesc {
    long long img;        // byte offset of the staged image in the blob (direct: the rank table;
                          // learned: the cell map, G x {J_g, J_{g+1}})
    long long xg;         // byte offset of the knots (or (X, Y) pairs) in the blob
    long long yoff;       // element offset of the array's knot values Y in the caller's Ycat
    uint32_t img_bytes;   // bytes of the image (multiple of 16), 0 if nothing to stage
    uint32_t x_in_img;    // byte offset of the knots inside the image, or NO_X_IN_IMG
    int32_t n;            // N: the array has N+1 knots
    int32_t mode;         // ArrMode
    uint32_t R;           // direct and learned: largest cell
    int32_t form;         // direct: FForm
    int32_t pbits;        // bisection over all knots: 2^floor(log2 N)
    int32_t aux;          // direct: 1 if the knot fingerprints of the rank table are used
    double H, W, X0;      // direct: parameters in the array's precision (held exactly)
    double XN;            // last knot
    float uscale;         // learned: u = (narrow(z) - x0f) * uscale (float32), 1 / (X_N - X_0)
    float x0f;            // learned: narrow(X0)
    long long n_esc;      // learned: escaped blocks in the overflow area of the cell table
    int32_t seg_off;      // learned: first predictor segment in the model tables
    int32_t seg_n;        // learned: number of predictor segments
    long long ct;          // learned: byte offset of the cell table K (C + 1 values) in the engine's ctab
    uint32_t g_in_img;    // direct: byte offset of the knot fingerprints inside the image
    int32_t xs;           // knot stride: 1 (knots alone) or 2 ((X_i, Y_i) pairs)
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
    const T *Y;                 // caller's knot values (interpolation), or nullptr (stored pairs, or none)
    T *y_out;
    const unsigned char *ctab;  // learned cell tables
    const int *order;           // claim order: position p serves array order[p] (nullptr: p itself)
    long long *chunk_off;       // n_arrays+1 chunk offsets by position (written by the planner)
    unsigned long long *counter;// chunk counter (reset by the planner)
    long long chunk;            // queries per chunk of an array that is not staged (chunk_len)
    uint32_t smem_limit;        // largest image staged in shared memory
    int checked;
    int l2pf;                   // 1: bulk L2 prefetch of the query stream allowed (device memory)
    int *err;
};

// Queries per chunk of an array.  A block stages the image of every chunk it
// claims (its previous chunk is almost always of another array), so a staged
// array gets chunks of about STAGE_Q_PER_BYTE queries per image byte, between
// `base` and STAGE_MAX_CHUNKS * base, a multiple of `base`; the claim order
// serves the largest arrays first, so the long chunks do not end the launch.
constexpr long long STAGE_Q_PER_BYTE = 4;  // 2: 472.5, 4: 481.4 G/s on the 4096-array workload
constexpr long long STAGE_MAX_CHUNKS = 8;

// Images smaller than this are read through L1 rather than staged: their
// chunks are short, and a bulk copy and its barrier would cost more than the
// first-touch misses.
constexpr uint32_t STAGE_MIN_BYTES = 4096;

__host__ __device__ __forceinline__ bool stage_image(const ArrDesc &d, uint32_t smem_limit)
{
    return d.img_bytes >= STAGE_MIN_BYTES && d.img_bytes <= smem_limit;
}

__host__ __device__ __forceinline__ long long chunk_len(const ArrDesc &d, long long base, uint32_t smem_limit)
{
    if (!stage_image(d, smem_limit)) return base;
    const long long want = (long long)d.img_bytes * STAGE_Q_PER_BYTE;
    const long long n = (want + base - 1) / base;
    return (n < 1 ? 1 : (n > STAGE_MAX_CHUNKS ? STAGE_MAX_CHUNKS : n)) * base;
}

// Chunk offsets from the query offsets, in claim order; resets the chunk
// counters: counter[0] = 0, and counter[1] = the first chunk of claim
// position `split` (the second launch's first chunk when the arrays are
// served by two launches, positions [0, split) and [split, n_arrays); the
// second launch's positions have their own chunk base and staging limit,
// chunk1 and smem_limit1).  One block.
__global__ void k_plan_chunks(const long long *z_off, long long m_single, int n_arrays, long long chunk,
                              const ArrDesc *desc, const int *order, uint32_t smem_limit, long long *chunk_off,
                              unsigned long long *counter, int split, long long chunk1, uint32_t smem_limit1);

__device__ __forceinline__ long long q_begin(const long long *z_off, int a) { return z_off ? z_off[a] : 0; }

// ------------------------------------------------------------------ per-query pieces
// Cell j = trunc(v) (negative and NaN -> 0, saturated at 2^32 - 1) and the
// knot fingerprint g = floor(256 (v - j)), the top 8 bits of the fractional
// part of v (FP_ABOVE for v >= 2^32).  Within one cell g is a non-decreasing
// function of v, so g(v) < g(w) implies v < w and g(v) > g(w) implies v > w.
// float: in float arithmetic, where v - j is exact (j <= v < j + 1, Sterbenz)
// and so is the product by 256 (negative and NaN v give g = 0); double: from
// the bit pattern (cell_fp_bits), which keeps the scarce FP64 pipe free.
__device__ __forceinline__ uint32_t cell_fp(float v, uint32_t *g)
{
    const uint32_t j = __float2uint_rz(v);
    *g = __float2uint_rz(__fmul_rn(__fsub_rn(v, __uint2float_rn(j)), (float)FP_ABOVE));
    return j;
}
__device__ __forceinline__ uint32_t cell_fp(double v, uint32_t *g) { return cell_fp_bits(v, g); }

// f of a direct array for its queries and knots.  float: both forms as one
// subtraction and one fused multiply-add, f = m(H m(z - x0) + c), with
// (x0, c) = (X_0, 0) for Eq. f (H y + 0 rounds like the product H y) and
// (0, -W) for the FMA form (z - 0 = z); double keeps one FP64 operation per
// query where the form allows it.
template <typename T> struct CellF;
template <> struct CellF<float> {
    float H, x0, c;
    __device__ __forceinline__ explicit CellF(const ArrDesc &d)
        : H((float)d.H), x0(d.form == F_FMA ? 0.0f : (float)d.X0), c(d.form == F_FMA ? -(float)d.W : 0.0f)
    {
    }
    __device__ __forceinline__ float operator()(float z) const { return __fmaf_rn(H, __fsub_rn(z, x0), c); }
    // 2^FP_BITS f(z), exactly: scaling by a power of two commutes with the
    // rounding of the fused multiply-add, except where f(z) is subnormal, and
    // there both give cell 0 and fingerprint 0
    __device__ __forceinline__ float scaled(float z) const
    {
        return __fmaf_rn(H * (float)FP_ABOVE, __fsub_rn(z, x0), c * (float)FP_ABOVE);
    }
};
template <> struct CellF<double> {
    double H, W, X0;
    int form;
    __device__ __forceinline__ explicit CellF(const ArrDesc &d) : H(d.H), W(d.W), X0(d.X0), form(d.form) {}
    __device__ __forceinline__ double operator()(double z) const
    {
        if (form == F_FMA) return __fma_rn(H, z, -W);
        if (form == F_PLAIN_X0ZERO) return __dmul_rn(H, z);
        return __dmul_rn(H, __dsub_rn(z, X0));
    }
};

// Cell and fingerprint of a query; a query past the last cell R gets cell R
// and fingerprint FP_ABOVE, above every knot's.  FASTF (float, R < 2^24 - 1):
// both from one conversion, q = trunc(2^FP_BITS f(z)) = 2^FP_BITS j + g, which
// stays below 2^32 up to cell 2^24 - 1 and saturates above, past R.
template <typename T, bool FASTF = false>
__device__ __forceinline__ uint32_t cell_q(const CellF<T> &f, uint32_t R, T z, uint32_t *g)
{
    uint32_t j;
    if constexpr (FASTF) {
        const uint32_t q = __float2uint_rz(f.scaled(z));
        j = q >> FP_BITS;
        *g = q & (FP_ABOVE - 1u);
    } else {
        j = cell_fp(f(z), g);
    }
    if (j > R) {
        *g = FP_ABOVE;
        return R;
    }
    return j;
}
constexpr uint32_t FASTF_MAX_R = (1u << 24) - 2;  // largest R of the one-conversion form

// ------------------------------------------------------------------ rank table
// With pairs (i, i+1) ComputeHR makes F strictly increasing, so a cell holds at
// most one knot and K_j = min{i : F_i >= j} = #{i : F_i < j} (Eq. indexdef):
// K is the rank function of the set of cells that hold a knot.  A direct
// array's image stores it as one 8-byte word per group of 32 cells,
//   x  K_{32 g}, the knots in cells before the group
//   y  bit b set when cell 32 g + b holds a knot
// so K_j = K_{32 g} + popc(y below bit b) (a quarter of a byte per cell),
// followed by one byte per knot, the knot's fingerprint (cell_fp).  A query
// reads one word; if its cell holds a knot, that knot's fingerprint; and the
// knot itself only when the two fingerprints are equal (about 1 in 256).
constexpr int RANK_SHIFT = 5;  // 32 cells per word

struct RankHit {
    uint32_t t;     // K_j
    uint32_t knot;  // 1 if cell j holds knot t (F_t == j)
};

__device__ __forceinline__ RankHit rank_decode(uint2 w, uint32_t j)
{
    RankHit h;
    uint32_t below;  // the b = j mod 32 low bits set
    asm("bmsk.clamp.b32 %0, 0, %1;" : "=r"(below) : "r"(j & 31u));
    h.t = w.x + __popc(w.y & below);
    h.knot = (w.y >> (j & 31u)) & 1u;
    return h;
}

// Bytes of a direct array's rank words (16-byte multiple).
__host__ __device__ __forceinline__ size_t rank_bytes(uint32_t R)
{
    return (((size_t)(R >> RANK_SHIFT) + 1) * 8 + 15) / 16 * 16;
}

template <typename T> __device__ __forceinline__ bool lt_exact(T a, T b)
{
    if constexpr (sizeof(T) == 8) return okey((double)a) < okey((double)b);
    else return a < b;
}

// Largest i in [lo, lo + n - 1] with X_i <= z, given X_lo <= z and
// z < X_{lo+n} (fixed depth, Algorithm binaryoptnopad on X[lo .. lo+n]);
// `top` = 2^floor(log2 n) (or any larger power of two); knot i at X[i xs].
template <typename T>
__device__ __forceinline__ int32_t bisect(const T *X, int xs, int32_t lo, int32_t n, int32_t top, T z, long long n_x,
                                          int *err)
{
    int32_t i = 0;
    for (int32_t k = top; k > 0; k >>= 1) {
        const int32_t r = i | k;
        const int32_t w = r < n ? r : n;
        if (!lt_exact<T>(z, X[(size_t)in_bounds(lo + w, n_x, BS_X, err) * xs])) i = r;
    }
    return lo + (i < n ? i : n);
}

// Pair (X_i, Y_i) of knot i in the pair layout (xs = 2), and an interval
// (X_i, Y_i, X_{i+1}, Y_{i+1}) as two pairs.
template <typename T> struct XYPair { T x, y; };
__device__ __forceinline__ XYPair<float> pair_ld(const float *X, int32_t i)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(X) + i);
    return {v.x, v.y};
}
__device__ __forceinline__ XYPair<double> pair_ld(const double *X, int32_t i)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(X) + i);
    return {v.x, v.y};
}
template <typename T> struct Ival { T x0, y0, x1, y1; };
template <typename T> __device__ __forceinline__ Ival<T> ival_of(XYPair<T> a, XYPair<T> b) { return {a.x, a.y, b.x, b.y}; }

// y = Y_i + (Y_{i+1} - Y_i) ((z - X_i) / (X_{i+1} - X_i)), each step rounded
// once; NaN where i lies outside [0, N-1].
template <typename T>
__device__ __forceinline__ T interp_of(const Ival<T> &v, T z, int32_t i, int32_t n)
{
    using A = Arith<T>;
    const T t = A::div(A::sub(z, v.x0), A::sub(v.x1, v.x0));
    return i >= 0 && i < n ? A::fma(A::sub(v.y1, v.y0), t, v.y0) : T(NAN);
}

// The linear interpolant of NQ queries with answers r.  Xg: the array's
// knots in global memory: the pair layout (xs = 2, two adjacent pairs per
// query) or the knots alone (X from them, Y from the caller's values).
// Every load is issued before the first value is formed.
template <typename T, int NQ>
__device__ __forceinline__ void interp_values(const BatchArgs<T> &a, const ArrDesc &d, const T *Xg, const T *z,
                                              const int32_t *r, T *y)
{
    Ival<T> v[NQ];
    if (d.xs == 2) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int32_t i = r[q] >= 0 && r[q] < d.n ? r[q] : 0;
            v[q] = ival_of<T>(pair_ld(Xg, in_bounds(i, (long long)d.n + 1, BS_X, a.err)),
                              pair_ld(Xg, in_bounds(i + 1, (long long)d.n + 1, BS_X, a.err)));
        }
    } else {
        const T *Y = a.Y + d.yoff;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int32_t i = r[q] >= 0 && r[q] < d.n ? r[q] : 0;
            const long long n1 = (long long)d.n + 1;
            v[q].x0 = __ldg(Xg + in_bounds(i, n1, BS_X, a.err));
            v[q].x1 = __ldg(Xg + in_bounds(i + 1, n1, BS_X, a.err));
            v[q].y0 = __ldg(Y + in_bounds(i, n1, BS_Y, a.err));
            v[q].y1 = __ldg(Y + in_bounds(i + 1, n1, BS_Y, a.err));
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) y[q] = interp_of<T>(v[q], z[q], r[q], d.n);
}

}  // namespace ds
