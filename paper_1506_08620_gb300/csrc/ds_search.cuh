// ds_search.cuh -- the direct-search lookup kernels (Algorithm direct,
// Algorithm directcache, Eq. fma).
//
// One thread answers VPT vectors of queries per tile (4 floats or 2 doubles
// per vector); queries are streamed with evict-first vector loads, results
// with evict-first vector stores.  The table (K and X, or the (K_j, X_{K_j})
// pairs) is either read through the read-only path from global memory, where
// it stays L2-resident, or staged once per block into shared memory with a
// bulk asynchronous copy when it fits.  Blocks are persistent: the grid is one
// wave of resident blocks and each block walks tiles with a grid stride.
//
// Table entries carry a flag in bit 31: set when a knot lies in the cell
// (F_t == j for t = K_j).  A query z in a cell without a knot satisfies
// f(z) = j < F_t = f(X_t), so z < X_t by the monotonicity of f (property
// monotonic of Eq. fprop) and the answer is t - 1 without reading X_t; only
// queries in a cell that holds a knot need the correcting comparison.
//
// DirectGap2 and Gap-q tables (Section 4.7: f(X_{i+q}) > f(X_i), Eq.
// f-monotonic-n) hold t = K_j = max{i : F_i <= j} (Eq. kgeneral) in bits
// 0..29, bit 31 set when F_t >= j (knot t lies in the cell, or the cell is
// below F_0 and t = 0) and bit 30 when F_{t-1} == j (knot t-1 lies in the cell
// too).  Without bit 31, F_t < j = f(z) gives z > X_t and the answer is t;
// without bit 30 the same argument gives z > X_{t-1}.  Otherwise the answer is
// the largest i in [t - q, t] with X_i <= z (X_{t-q} < z because F_{t-q} <
// F_t <= j; X_{-1} = -inf), found by a bisection after the comparisons with
// X_t and X_{t-1}: for q = 2 exactly the comparisons of Algorithm direct-2,
// each made only where the flags say it can be true.
#pragma once

#include "ds_common.cuh"

namespace ds {

// the three forms of f
enum FForm : int { F_PLAIN = 0, F_FMA = 1, F_PLAIN_X0ZERO = 2 };

constexpr uint32_t KNOT_FLAG = 0x80000000u;

constexpr uint32_t KNOT_FLAG2 = 0x40000000u;  // Eq. kgeneral: knot t-1 in the cell as well
constexpr uint32_t GEN_T_MASK = 0x3FFFFFFFu;  // Eq. kgeneral: t in bits 0..29

// Packed table: K in 16-byte blocks of 12 cells, {K of the block's first
// cell, 12 bytes (K_j - base) | flags >> 24}.  K grows by at most 1 per cell
// for Direct (F is strictly increasing) and at most q for Eq. kgeneral
// (F_{i+q} > F_i), so the difference fits 6 bits for q <= 5; bits 6 and 7
// carry the flags of bits 30 and 31.  1.33 bytes per cell instead of 4 keeps
// large tables L2-resident, and a lookup still reads one 16-byte sector.
constexpr int PACK_CELLS = 12;
constexpr int MAX_PACKED_Q = 5;

__device__ __forceinline__ uint32_t unpack_cell(uint4 w, uint32_t j)
{
    const uint32_t b = __umulhi(j, 0xAAAAAAABu) >> 3;  // j / 12
    const uint32_t s = j - b * PACK_CELLS;
    const uint32_t word = s < 4 ? w.y : (s < 8 ? w.z : w.w);
    const uint32_t byte = (word >> ((s & 3u) * 8u)) & 0xFFu;
    return (w.x + (byte & 0x3Fu)) | ((byte & 0xC0u) << 24);
}

template <typename T> struct SearchArgs {
    const uint4 *K16;     // packed table (L2 path), or nullptr
    const uint32_t *K;    // R+1 cells (Eq. indexdef), flag in bit 31
    const T *X;           // N+1 knots
    const Pair<T> *P;     // R+1 (K_j | flag, X_{K_j}) pairs (cache layout)
    const void *smem_src; // contiguous image staged to shared memory
    uint32_t smem_bytes;  // bytes of the image (multiple of 16)
    uint32_t x_smem_off;  // byte offset of X inside the image
    T H, W, X0;
    uint32_t R;
    int32_t q;            // pair distance of an Eq. kgeneral table (Gap-q); 1 for Direct
    int checked;          // NaN -> -1
    const T *Z;
    int32_t *I;
    long long m;
    int *err;
    long long n_x;        // N+1 (the extent of X, for the range-checking build)
};

template <typename T> struct VecOf;
template <> struct VecOf<float> { using V = float4; using IV = int4; static constexpr int L = 4; };
template <> struct VecOf<double> { using V = double2; using IV = int2; static constexpr int L = 2; };

// Cell of a query: j = min(f(z), R).  F_PLAIN: trunc(m(H m(z - X0)))
// (Eq. function); F_PLAIN_X0ZERO: the same with X0 == 0, where m(z - 0) == z
// exactly; F_FMA: trunc(m(H z - W)) (Eq. fma).  Exactly one floating-point
// operation of the array's precision per query besides the conversion, and
// for float64 with INTOPS the conversion is done on the bit pattern by
// integer instructions (the FP64 pipe is the scarce one on GB300).
template <typename T, int FM, bool INTOPS>
__device__ __forceinline__ uint32_t cell_of(T z, const SearchArgs<T> &a)
{
    using A = Arith<T>;
    T v;
    if constexpr (FM == F_FMA) v = A::fma(a.H, z, -a.W);
    else if constexpr (FM == F_PLAIN_X0ZERO) v = A::mul(a.H, z);
    else v = A::mul(a.H, A::sub(z, a.X0));
    uint32_t j;
    if constexpr (INTOPS && sizeof(T) == 8) j = trunc_u32_bits((double)v);
    else j = A::trunc_u32(v);
    return min(j, a.R);
}

// Table entry of cell j: flagged t = K_j, and for the cache layout X_{K_j}.
template <typename T, bool CACHE, bool SMEM>
__device__ __forceinline__ uint32_t gather_k(uint32_t j, const uint32_t *K, const Pair<T> *P, T *x_out,
                                             const SearchArgs<T> &a)
{
    j = in_bounds(j, (long long)a.R + 1, BS_K, a.err);
    if constexpr (CACHE) {
        if constexpr (SMEM) {
            const Pair<T> p = P[j];
            *x_out = p.x;
            return (uint32_t)p.k;
        } else if constexpr (sizeof(T) == 4) {
            const int2 p = __ldg(reinterpret_cast<const int2 *>(P) + j);
            *x_out = __int_as_float(p.y);
            return (uint32_t)p.x;
        } else {
            const longlong2 p = __ldg(reinterpret_cast<const longlong2 *>(P) + j);
            *x_out = __longlong_as_double(p.y);
            return (uint32_t)(p.x & 0xFFFFFFFFll);
        }
    } else {
        if constexpr (SMEM) return K[j];
        else return __ldg(K + j);
    }
}

template <typename T, bool SMEM>
__device__ __forceinline__ T gather_x(int32_t t, const T *X, const SearchArgs<T> &a)
{
    t = in_bounds(t, a.n_x, BS_X, a.err);
    if constexpr (SMEM) return X[t];
    else return __ldg(X + t);
}

template <typename T> __device__ __forceinline__ bool is_nan(T z);
template <> __device__ __forceinline__ bool is_nan<float>(float z) { return !(z == z); }
template <> __device__ __forceinline__ bool is_nan<double>(double z)
{
    return ((unsigned long long)__double_as_longlong(z) & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
}

// Correction step: i = t - [z < X_t] (the comparison only where the cell
// holds a knot); NaN -> -1 when checked.
template <typename T, bool INTOPS>
__device__ __forceinline__ int32_t correct(T z, uint32_t e, T x, int checked)
{
    const int32_t t = (int32_t)(e & ~KNOT_FLAG);
    bool lt = true;
    if (e & KNOT_FLAG) {
        if constexpr (INTOPS && sizeof(T) == 8) lt = okey((double)z) < okey((double)x);
        else lt = z < x;
    }
    int32_t i = t - (int32_t)lt;
    if (checked && is_nan<T>(z)) i = -1;
    return i;
}

template <typename T, bool INTOPS>
__device__ __forceinline__ bool z_less(T z, T x)
{
    if constexpr (INTOPS && sizeof(T) == 8) return okey((double)z) < okey((double)x);
    else return z < x;
}

// Eq. kgeneral correction (Algorithm direct-2 and its q-knot form): x = X_t
// and xp = X_{t-1}, read by the caller under bits 31 and 30.  When
// z < X_{t-1} the answer lies in [max(t - q, -1), t - 2] and is found by
// bisection with X_{t-q} < z.
template <typename T, bool INTOPS, bool SMEM>
__device__ __forceinline__ int32_t correct_gen(T z, uint32_t e, T x, T xp, const T *X, const SearchArgs<T> &args)
{
    const int32_t q = args.q;
    const int checked = args.checked;
    const int32_t t = (int32_t)(e & GEN_T_MASK);
    int32_t i = t;
    if ((e & KNOT_FLAG) && z_less<T, INTOPS>(z, x)) {
        i = t - 1;
        if ((e & KNOT_FLAG2) && z_less<T, INTOPS>(z, xp)) {
            int32_t a = t - q < -1 ? -1 : t - q, b = t - 1;  // X_a <= z < X_b
            while (b - a > 1) {
                const int32_t m = (a + b) >> 1;
                if (z_less<T, INTOPS>(z, gather_x<T, SMEM>(m, X, args))) b = m;
                else a = m;
            }
            i = a;
        }
    }
    if (checked && is_nan<T>(z)) i = -1;
    return i;
}

template <typename T, int FM, bool CACHE, bool SMEM, bool INTOPS, bool GEN = false>
__device__ __forceinline__ int32_t lookup(T z, const uint32_t *K, const T *X, const Pair<T> *P,
                                          const SearchArgs<T> &a)
{
    const uint32_t j = cell_of<T, FM, INTOPS>(z, a);
    T x = T(0);
    const uint32_t e = gather_k<T, CACHE, SMEM>(j, K, P, &x, a);
    if constexpr (GEN) {
        const int32_t t = (int32_t)(e & GEN_T_MASK);
        T xp = T(0);
        if (e & KNOT_FLAG) x = gather_x<T, SMEM>(t, X, a);
        if (e & KNOT_FLAG2) xp = gather_x<T, SMEM>(t - 1, X, a);
        return correct_gen<T, INTOPS, SMEM>(z, e, x, xp, X, a);
    } else {
        if constexpr (!CACHE) {
            if (e & KNOT_FLAG) x = gather_x<T, SMEM>((int32_t)(e & ~KNOT_FLAG), X, a);
        }
        return correct<T, INTOPS>(z, e, x, a.checked);
    }
}

template <typename T, int FM, bool CACHE, bool SMEM, bool INTOPS, int VPT, bool GEN = false>
__global__ void __launch_bounds__(256) k_search_vec(SearchArgs<T> a, long long nvec, long long ntiles)
{
    using V = typename VecOf<T>::V;
    using IV = typename VecOf<T>::IV;
    constexpr int L = VecOf<T>::L;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;

    const uint32_t *K;
    const T *X;
    const Pair<T> *P;
    if constexpr (SMEM) {
        if (!stage_to_smem(smem, a.smem_src, a.smem_bytes, &bar, a.err)) return;
        K = reinterpret_cast<const uint32_t *>(smem);
        X = reinterpret_cast<const T *>(smem + a.x_smem_off);
        P = reinterpret_cast<const Pair<T> *>(smem);
    } else {
        K = a.K;
        X = a.X;
        P = a.P;
    }
    const V *__restrict__ Zv = reinterpret_cast<const V *>(a.Z);
    IV *__restrict__ Iv = reinterpret_cast<IV *>(a.I);

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long b = tile * (long long)VPT * blockDim.x + threadIdx.x;
        V zv[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            if (idx < nvec) zv[v] = __ldcs(Zv + idx);
        }
        // phase 1: cells; phase 2: all table gathers; phase 3: the knot gathers
        // of cells that hold a knot; phase 4: corrections.  Every gather of the
        // thread is in flight at once.
        constexpr int NQ = VPT * L;
        const T *zs = reinterpret_cast<const T *>(zv);
        uint32_t e[NQ];
        T x[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            x[q] = T(0);
            e[q] = cell_of<T, FM, INTOPS>(zs[q], a);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) e[q] = gather_k<T, CACHE, SMEM>(e[q], K, P, &x[q], a);
        int32_t r[NQ];
        if constexpr (GEN) {
            T xp[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t t = (int32_t)(e[q] & GEN_T_MASK);
                xp[q] = T(0);
                if (e[q] & KNOT_FLAG) x[q] = gather_x<T, SMEM>(t, X, a);
                if (e[q] & KNOT_FLAG2) xp[q] = gather_x<T, SMEM>(t - 1, X, a);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) r[q] = correct_gen<T, INTOPS, SMEM>(zs[q], e[q], x[q], xp[q], X, a);
        } else {
            if constexpr (!CACHE) {
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (e[q] & KNOT_FLAG) x[q] = gather_x<T, SMEM>((int32_t)(e[q] & ~KNOT_FLAG), X, a);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) r[q] = correct<T, INTOPS>(zs[q], e[q], x[q], a.checked);
        }
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            if (idx < nvec) {
                IV o;
                if constexpr (L == 4) o = make_int4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
                else o = make_int2(r[2 * v], r[2 * v + 1]);
                __stcs(Iv + idx, o);
            }
        }
    }
    // the last m mod L queries
    if (blockIdx.x == 0) {
        const long long q = nvec * L + threadIdx.x;
        if (q < a.m) a.I[q] = lookup<T, FM, CACHE, SMEM, INTOPS, GEN>(a.Z[q], K, X, P, a);
    }
}

// Scalar path for queries or results that are not aligned for vector access.
template <typename T, int FM, bool CACHE, bool INTOPS, bool GEN = false>
__global__ void __launch_bounds__(256) k_search_scalar(SearchArgs<T> a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.m; q += stride)
        a.I[q] = lookup<T, FM, CACHE, false, INTOPS, GEN>(a.Z[q], a.K, a.X, a.P, a);
}

// Float64 lookups with the data kept as IEEE bit patterns (long long)
// throughout: the only double-precision instruction per query is the DMUL
// (or DFMA, or DADD + DMUL for the plain form with X_0 != 0) of f.  The
// truncation works on the product's bits, the comparison z < X_t on
// order-preserving integer keys, and no double value is ever moved or
// selected, so the compiler has no reason to emit further FP64-pipe
// instructions (GB300's FP64 pipe is its scarce resource).
__device__ __forceinline__ long long okey_bits(long long b) { return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFll); }

template <int FM>
__device__ __forceinline__ uint32_t cell_bits(long long zb, double H, double NW, double X0, uint32_t R)
{
    const double z = __longlong_as_double(zb);
    double v;
    if constexpr (FM == F_FMA) v = __fma_rn(H, z, NW);
    else if constexpr (FM == F_PLAIN_X0ZERO) v = __dmul_rn(H, z);
    else v = __dmul_rn(H, __dsub_rn(z, X0));
    const uint32_t j = trunc_u32_bits(v);
    return j < R ? j : R;
}

__device__ __forceinline__ int32_t correct_bits(long long zb, uint32_t e, long long xb, int checked)
{
    const int32_t t = (int32_t)(e & ~KNOT_FLAG);
    const bool lt = (e & KNOT_FLAG) ? okey_bits(zb) < okey_bits(xb) : true;
    int32_t i = t - (int32_t)lt;
    if (checked && ((unsigned long long)zb & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) i = -1;
    return i;
}

// Eq. kgeneral correction on bit patterns; xb, xpb = bits of X_t, X_{t-1}
// (read by the caller under bits 31 and 30).
template <bool SMEM>
__device__ __forceinline__ int32_t correct_bits_gen(long long zb, uint32_t e, long long xb, long long xpb,
                                                    const long long *Xb, uint64_t keep, int32_t q, int checked,
                                                    long long n_x, int *err)
{
    const long long kz = okey_bits(zb);
    const int32_t t = (int32_t)(e & GEN_T_MASK);
    int32_t i = t;
    if ((e & KNOT_FLAG) && kz < okey_bits(xb)) {
        i = t - 1;
        if ((e & KNOT_FLAG2) && kz < okey_bits(xpb)) {
            int32_t a = t - q < -1 ? -1 : t - q, b = t - 1;  // X_a <= z < X_b
            while (b - a > 1) {
                const int32_t m = (a + b) >> 1;
                const long long *px = Xb + in_bounds(m, n_x, BS_X, err);
                if (kz < okey_bits(SMEM ? *px : ld_keep(px, keep))) b = m;
                else a = m;
            }
            i = a;
        }
    }
    if (checked && ((unsigned long long)zb & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) i = -1;
    return i;
}

template <int FM, bool CACHE, bool SMEM, int VPT, bool PACKED = false, bool GEN = false>
__global__ void __launch_bounds__(256) k_search_f64bits(SearchArgs<double> a, long long nvec, long long ntiles)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    const uint32_t *K;
    const long long *Xb;
    const longlong2 *P;
    if constexpr (SMEM) {
        if (!stage_to_smem(smem, a.smem_src, a.smem_bytes, &bar, a.err)) return;
        K = reinterpret_cast<const uint32_t *>(smem);
        Xb = reinterpret_cast<const long long *>(smem + a.x_smem_off);
        P = reinterpret_cast<const longlong2 *>(smem);
    } else {
        K = a.K;
        Xb = reinterpret_cast<const long long *>(a.X);
        P = reinterpret_cast<const longlong2 *>(a.P);
    }
    const double H = a.H, NW = -a.W, X0 = a.X0;
    const uint32_t R = a.R;
    const uint64_t keep = l2_keep_policy();
    const longlong2 *__restrict__ Zv = reinterpret_cast<const longlong2 *>(a.Z);
    int2 *__restrict__ Iv = reinterpret_cast<int2 *>(a.I);
    constexpr int NQ = 2 * VPT;
    // software pipeline: the next tile's queries are loaded while this tile's
    // gathers are in flight
    long long zn[NQ];
    auto load_tile = [&](long long tile, long long *dst) {
        const long long b = tile * (long long)VPT * blockDim.x + threadIdx.x;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            longlong2 q = make_longlong2(0, 0);
            if (tile < ntiles && idx < nvec) q = __ldcs(Zv + idx);
            dst[2 * v] = q.x;
            dst[2 * v + 1] = q.y;
        }
    };
    load_tile(blockIdx.x, zn);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long b = tile * (long long)VPT * blockDim.x + threadIdx.x;
        long long zb[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) zb[q] = zn[q];
        load_tile(tile + gridDim.x, zn);
        uint32_t e[NQ];
        long long xb[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) e[q] = cell_bits<FM>(zb[q], H, NW, X0, R);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if constexpr (CACHE) {
                const longlong2 *pp = P + in_bounds(e[q], (long long)R + 1, BS_K, a.err);
                const longlong2 p = SMEM ? *pp : ld_keep(pp, keep);
                e[q] = (uint32_t)(p.x & 0xFFFFFFFFll);
                xb[q] = p.y;
            } else if constexpr (PACKED) {
                const uint32_t j = e[q];
                const uint32_t blk = in_bounds(__umulhi(j, 0xAAAAAAABu) >> 3, ((long long)R + PACK_CELLS) / PACK_CELLS,
                                               BS_K16, a.err);
                e[q] = unpack_cell(ld_keep(a.K16 + blk, keep), j);
            } else {
                const uint32_t *pk = K + in_bounds(e[q], (long long)R + 1, BS_K, a.err);
                e[q] = SMEM ? *pk : ld_keep(pk, keep);
            }
        }
        if constexpr (GEN) {
            long long xpb[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t t = (int32_t)(e[q] & GEN_T_MASK);
                xb[q] = 0;
                xpb[q] = 0;
                if (e[q] & KNOT_FLAG) {
                    const long long *px = Xb + in_bounds(t, a.n_x, BS_X, a.err);
                    xb[q] = SMEM ? *px : ld_keep(px, keep);
                }
                if (e[q] & KNOT_FLAG2) {
                    const long long *px = Xb + in_bounds(t - 1, a.n_x, BS_X, a.err);
                    xpb[q] = SMEM ? *px : ld_keep(px, keep);
                }
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const long long idx = b + (long long)v * blockDim.x;
                if (idx < nvec)
                    __stcs(Iv + idx, make_int2(correct_bits_gen<SMEM>(zb[2 * v], e[2 * v], xb[2 * v], xpb[2 * v], Xb,
                                                                      keep, a.q, a.checked, a.n_x, a.err),
                                               correct_bits_gen<SMEM>(zb[2 * v + 1], e[2 * v + 1], xb[2 * v + 1],
                                                                      xpb[2 * v + 1], Xb, keep, a.q, a.checked,
                                                                      a.n_x, a.err)));
            }
        } else {
            if constexpr (!CACHE) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    xb[q] = 0;
                    if (e[q] & KNOT_FLAG) {
                        const long long *px = Xb + in_bounds((int32_t)(e[q] & ~KNOT_FLAG), a.n_x, BS_X, a.err);
                        xb[q] = SMEM ? *px : ld_keep(px, keep);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const long long idx = b + (long long)v * blockDim.x;
                if (idx < nvec)
                    __stcs(Iv + idx,
                           make_int2(correct_bits(zb[2 * v], e[2 * v], xb[2 * v], a.checked),
                                     correct_bits(zb[2 * v + 1], e[2 * v + 1], xb[2 * v + 1], a.checked)));
            }
        }
    }
    if (blockIdx.x == 0) {  // the last m mod 2 queries
        const long long q = nvec * 2 + threadIdx.x;
        if (q < a.m) {
            const long long zq = reinterpret_cast<const long long *>(a.Z)[q];
            uint32_t e = cell_bits<FM>(zq, H, NW, X0, R);
            long long xq = 0;
            if constexpr (CACHE) {
                const longlong2 p = P[in_bounds(e, (long long)R + 1, BS_K, a.err)];
                e = (uint32_t)(p.x & 0xFFFFFFFFll);
                xq = p.y;
            } else if constexpr (PACKED) {
                e = unpack_cell(a.K16[in_bounds(__umulhi(e, 0xAAAAAAABu) >> 3, ((long long)R + PACK_CELLS) / PACK_CELLS,
                                                BS_K16, a.err)],
                                e);
            } else {
                e = K[in_bounds(e, (long long)R + 1, BS_K, a.err)];
            }
            if constexpr (GEN) {
                const int32_t t = (int32_t)(e & GEN_T_MASK);
                const long long xq0 = (e & KNOT_FLAG) ? Xb[in_bounds(t, a.n_x, BS_X, a.err)] : 0;
                const long long xq1 = (e & KNOT_FLAG2) ? Xb[in_bounds(t - 1, a.n_x, BS_X, a.err)] : 0;
                a.I[q] = correct_bits_gen<true>(zq, e, xq0, xq1, Xb, keep, a.q, a.checked, a.n_x, a.err);
            } else {
                if constexpr (!CACHE) {
                    if (e & KNOT_FLAG) xq = Xb[in_bounds((int32_t)(e & ~KNOT_FLAG), a.n_x, BS_X, a.err)];
                }
                a.I[q] = correct_bits(zq, e, xq, a.checked);
            }
        }
    }
}

struct SearchPlan {
    int form;      // FForm
    bool cache, smem, intops, packed;
    bool gen;      // Eq. kgeneral table (q >= 2) and Algorithm direct-2 / its q-knot form
    int block;     // threads per block
    int vpt;       // vectors per thread per tile
    int grid_cap;  // resident blocks (one wave)
};

constexpr int SEARCH_BLOCK = 256;
constexpr int SEARCH_VPT = 4;

// Launch one search (defined in ds_search_f32.cu / ds_search_f64.cu).
template <typename T>
ds_status launch_search(const SearchArgs<T> &a, const SearchPlan &plan, cudaStream_t stream);

// Resident blocks per SM of the vector kernel chosen by `plan` with the given
// dynamic shared memory, and the opt-in of large shared memory.
template <typename T>
ds_status prepare_search(SearchPlan *plan, uint32_t smem_bytes, int num_sms);

}  // namespace ds
