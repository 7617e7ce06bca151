// ds_multi_kernels.cuh -- the persistent ragged search kernel and the
// segmented build kernels shared by the batched and learned forms.
#pragma once

#include "ds_index.cuh"
#include "ds_multi.cuh"

namespace ds {

// ------------------------------------------------------------------ learned predictor
// Float32 image of a query for the predictor: z - X0 scaled to [0, 1].  For
// float64 arrays the query is first narrowed to float32 by truncating its
// significand (integer instructions only; any fixed narrowing is valid
// because the error bound is recorded with this same function).
template <typename T> __device__ __forceinline__ float narrow(T z);
template <> __device__ __forceinline__ float narrow<float>(float z) { return z; }
template <> __device__ __forceinline__ float narrow<double>(double z)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(z);
    const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e == 1024) return __uint_as_float(s | 0x7F800000u | (unsigned)((b & 0x000FFFFFFFFFFFFFull) != 0));
    if (e > 127) return __uint_as_float(s | 0x7F800000u);
    if (e < -126) return __uint_as_float(s);
    return __uint_as_float(s | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

template <typename T>
__device__ __forceinline__ float pred_u(T z, const ArrDesc &d)
{
    return __fmul_rn(__fsub_rn(narrow<T>(z), d.x0f), d.uscale);
}

// ------------------------------------------------------------------ learned cell map
// Cell of z on a learned array: t = u(z) G (exact, G a power of two), macro
// cell g = min(trunc t, G - 1) with its first cells {J_g, J_{g+1}}, and
//   j = J_g + min(trunc(m(D m(t - g))), D),  D = J_{g+1} - J_g.
// Every step is a monotone function of z (rounding is monotone, D >= 0), and
// j lies in [J_g, J_{g+1}] while J is non-decreasing, so f is monotone over
// the whole line: Eq. fprop holds for it, which is all the table of Eq.
// indexdef needs.  Negative t and NaN give cell J_0 = 0, t >= G cell J_G.
template <typename T>
__device__ __forceinline__ uint32_t learned_cell(T z, const ArrDesc &d, const uint2 *M, uint32_t G, int *err)
{
    const float t = __fmul_rn(pred_u<T>(z, d), (float)G);
    uint32_t g = __float2uint_rz(t);
    g = g < G - 1u ? g : G - 1u;
    const float fr = __fsub_rn(t, __uint2float_rn(g));
    const uint2 J = M[in_bounds(g, (long long)G, BS_CMAP, err)];
    const uint32_t D = J.y - J.x;
    const uint32_t k = __float2uint_rz(__fmul_rn(__uint2float_rn(D), fr));
    return J.x + (k < D ? k : D);
}

// K_j and K_{j+1} of a learned array's cell table (a 16-byte block per 8
// cells: K_{8b} and 12-bit differences, or an escaped block's 9 values in the
// overflow area after the lblk_count(R) blocks).
__device__ __forceinline__ uint32_t lblk_field(uint4 w, uint32_t r)
{
    // difference r (1..8) of the block: bits 12 (r - 1) .. 12 r - 1 of (y, z, w)
    const uint32_t o = 12u * (r - 1u);
    const uint32_t lo = o < 32u ? w.y : (o < 64u ? w.z : w.w);
    const uint32_t hi = o < 32u ? w.z : (o < 64u ? w.w : 0u);
    return __funnelshift_r(lo, hi, o & 31u) & 0xFFFu;
}
__device__ __forceinline__ void learned_bounds(const unsigned char *ct, uint32_t R, uint32_t j, uint32_t *t0,
                                               uint32_t *t1, long long n_esc, int *err)
{
    const uint4 w = __ldg(reinterpret_cast<const uint4 *>(ct) +
                          in_bounds(j >> LBLK_SHIFT, (long long)lblk_count(R), BS_CBLOCK, err));
    const uint32_t r = j & 7u;
    if (w.x & LBLK_ESC) {
        const uint32_t *O = reinterpret_cast<const uint32_t *>(ct + lblk_count(R) * 16ull) +
                            (size_t)in_bounds(w.y, n_esc, BS_CESC, err) * 9u;
        *t0 = __ldg(O + r);
        *t1 = __ldg(O + r + 1u);
    } else {
        *t0 = w.x + (r ? lblk_field(w, r) : 0u);
        *t1 = w.x + lblk_field(w, r + 1u);
    }
}

// Table read: shared memory (staged image) or global memory through the
// read-only path (L1-cached: a block works on one array at a time, whose
// table is small enough to get L1 reuse).  Rank words and knot fingerprints
// are marked evict-last in L2 with the policy `pol`, so they stay resident
// under the query stream; knots and learned tables keep the default policy.
template <bool SM> __device__ __forceinline__ uint32_t tab_ld(const uint32_t *p, uint64_t)
{
    if constexpr (SM) return *p;
    else return __ldg(p);
}
template <bool SM> __device__ __forceinline__ float tab_ld(const float *p, uint64_t)
{
    if constexpr (SM) return *p;
    else return __ldg(p);
}
template <bool SM> __device__ __forceinline__ double tab_ld(const double *p, uint64_t)
{
    if constexpr (SM) return *p;
    else return __ldg(p);
}
template <bool SM> __device__ __forceinline__ uint2 tab_ld(const uint2 *p, uint64_t pol)
{
    if constexpr (SM) return *p;
    else return ld_keep_l1(p, pol);
}
template <bool SM> __device__ __forceinline__ uint32_t tab_ld(const uint8_t *p, uint64_t pol)
{
    if constexpr (SM) return *p;
    else return ld_keep_l1(p, pol);
}

// ------------------------------------------------------------------ NQ queries of one array
// Kernel kinds: every mode (fingerprints decided per array at run time), or
// direct arrays only, without or with fingerprints (the other paths compiled
// out, which keeps the register count low), or with fingerprints and the
// one-conversion cell form (float arrays, every R < 2^24 - 1), or learned
// arrays only, or direct arrays whose knots are stored as (X, Y) pairs,
// without fingerprints (KIND_DIRECT_XY: the direct arrays of a learned handle
// that holds its values).  A handle with direct and learned arrays serves
// each group with its own launch and kind.
enum BatchKind : int {
    KIND_ALL = 0, KIND_DIRECT = 1, KIND_DIRECT_FP = 2, KIND_DIRECT_FPF = 3, KIND_LEARNED_ONLY = 4, KIND_DIRECT_XY = 5
};
__host__ __device__ constexpr bool direct_kind(int k)
{
    return k == KIND_DIRECT || k == KIND_DIRECT_FP || k == KIND_DIRECT_FPF || k == KIND_DIRECT_XY;
}

// Learned form: j = f(z) on the learned cell map, (t0, t1) = (K_j, K_{j+1}).
// Knots below t0 lie in cells below j and are < z; knots from t1 on lie in
// cells above j and are > z (f is monotone), so the answer is t0 - 1 plus the
// number of knots i in [t0, t1) with X_i <= z: none for an empty cell, else
// decided by X_{t0} and X_{t1-1}, and between them by a bisection of the
// cell's knots.  img: the cell map (shared or global memory).
template <typename T, int NQ, bool SM>
__device__ __forceinline__ void learned_answer(const BatchArgs<T> &a, const ArrDesc &d, const unsigned char *img,
                                               const T *X, const T *z, int32_t *r)
{
    const uint2 *M = reinterpret_cast<const uint2 *>(img);
    const uint32_t G = d.img_bytes >> 3;
    const unsigned char *ct = a.ctab + d.ct;
    const int xs = d.xs;
    uint32_t t0[NQ], t1[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        learned_bounds(ct, d.R, learned_cell<T>(z[q], d, M, G, a.err), &t0[q], &t1[q], d.n_esc, a.err);
    const long long n1 = (long long)d.n + 1;
    T xa[NQ], xb[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const bool any = t1[q] > t0[q];
        xa[q] = any ? __ldg(X + (size_t)in_bounds(t0[q], n1, BS_X, a.err) * xs) : T(0);
        xb[q] = any ? __ldg(X + (size_t)in_bounds(t1[q] - 1u, n1, BS_X, a.err) * xs) : T(0);
    }
    bool inner = false;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (t1[q] == t0[q] || lt_exact<T>(z[q], xa[q])) r[q] = (int32_t)t0[q] - 1;
        else if (!lt_exact<T>(z[q], xb[q])) r[q] = (int32_t)t1[q] - 1;
        else {
            r[q] = -2;  // X_{t0} <= z < X_{t1-1}: inside the cell's knots
            inner = true;
        }
    }
    if (inner) {
        // X_{t0} <= z < X_{t1-1}: the answer is t0 plus the number of the knots
        // strictly between those two that are <= z (none for two knots, so no
        // read; otherwise a bisection over them alone)
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (r[q] == -2) {
                const int32_t n = (int32_t)(t1[q] - t0[q]) - 2;
                r[q] = n == 0 ? (int32_t)t0[q]
                              : bisect<T>(X, xs, (int32_t)t0[q], n, 1 << (31 - __clz(n)), z[q], n1, a.err);
            }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (a.checked && is_nan<T>(z[q])) r[q] = -1;
}

// img: the array's image (shared or global memory: for a direct array its
// rank words and knot fingerprints, for a learned one its cell map); X: its
// knots (global memory for direct and learned arrays, shared or global for
// bisected ones), knot i at X[i xs].
template <typename T, int NQ, int KIND, bool SM, bool FASTF>
__device__ __forceinline__ void answer_block(const BatchArgs<T> &a, const ArrDesc &d, const CellF<T> &f,
                                             const unsigned char *img, const T *X, const T *z, int32_t *r,
                                             uint64_t pol)
{
    if (direct_kind(KIND) || (KIND == KIND_ALL && d.mode == MODE_DIRECT)) {
        // one rank word per query; for a cell holding a knot, the knot's
        // fingerprint; the knot X_t itself only when the two fingerprints are
        // equal (otherwise they order z and X_t: within a cell the fingerprint
        // is a non-decreasing function of f, Eq. fprop)
        const bool fp = KIND == KIND_DIRECT_FP || KIND == KIND_DIRECT_FPF || (KIND == KIND_ALL && d.aux);
        const uint2 *Rt = reinterpret_cast<const uint2 *>(img);
        const uint8_t *Gt = img + d.g_in_img;
        uint32_t g[NQ], j[NQ];
        uint2 w[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            j[q] = cell_q<T, FASTF>(f, d.R, z[q], &g[q]);
            w[q] = tab_ld<SM>(Rt + in_bounds(j[q] >> RANK_SHIFT, ((long long)d.R >> RANK_SHIFT) + 1, BS_RANK, a.err),
                              pol);
        }
        RankHit h[NQ];
        uint32_t kf[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            h[q] = rank_decode(w[q], j[q]);
            kf[q] = fp && h[q].knot ? tab_ld<SM>(Gt + in_bounds(h[q].t, (long long)d.n + 1, BS_FPRINT, a.err), pol)
                                    : 0u;
        }
        T x[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const bool need = h[q].knot && (!fp || g[q] == kf[q]);
            const uint32_t t = in_bounds(h[q].t, (long long)d.n + 1, BS_X, a.err);
            const size_t xi = KIND == KIND_DIRECT_XY ? (size_t)t * 2u
                              : direct_kind(KIND)        ? (size_t)t
                                                         : (size_t)t * d.xs;
            x[q] = need ? tab_ld<false>(X + xi, pol) : T(0);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            bool lt = true;  // no knot in the cell: z < X_t (Eq. indexdef)
            if (h[q].knot) lt = (fp && g[q] != kf[q]) ? g[q] < kf[q] : lt_exact<T>(z[q], x[q]);
            r[q] = (int32_t)h[q].t - (int32_t)lt;
            if (a.checked && is_nan<T>(z[q])) r[q] = -1;
        }
        return;
    }
    if (KIND == KIND_LEARNED_ONLY || d.mode == MODE_LEARNED) {  // learned arrays
        learned_answer<T, NQ, SM>(a, d, img, X, z, r);
        return;
    }
    // bisected arrays: fixed-depth search over all knots (Algorithm binaryoptnopad)
    int32_t lo[NQ], n[NQ];
    bool done[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        lo[q] = 0;
        n[q] = d.n;
        done[q] = false;
        if (lt_exact<T>(z[q], X[0])) { r[q] = -1; done[q] = true; }
        else if (!lt_exact<T>(z[q], X[(size_t)d.n * d.xs])) { r[q] = d.n; done[q] = true; }
    }
    const int32_t top = d.pbits;
    // interleaved fixed-depth bisection (Algorithm binaryoptnopad)
    int32_t i[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) i[q] = 0;
    for (int32_t k = top; k > 0; k >>= 1) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int32_t rr = i[q] | k;
            const int32_t w = rr < n[q] ? rr : n[q];
            const size_t xi = (size_t)in_bounds(lo[q] + w, (long long)d.n + 1, BS_X, a.err) * d.xs;
            if (!lt_exact<T>(z[q], tab_ld<SM>(X + xi, pol))) i[q] = rr;
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (!done[q]) r[q] = lo[q] + (i[q] < n[q] ? i[q] : n[q] - 1);
        if (a.checked && is_nan<T>(z[q])) r[q] = -1;
    }
}

// Tiles by which the bulk L2 prefetch of the query stream runs ahead.
constexpr int QP_DIST = 4;

// Queries [zs, ze) of one array by `nthr` threads (a block, or a warp); `tid`
// is the thread's rank among them.
template <typename T, int VPT, bool INTERP, bool VEC, int KIND, bool SM>
__device__ __forceinline__ void process_chunk(const BatchArgs<T> &a, const ArrDesc &d, const unsigned char *K,
                                              const T *X, long long zs, long long ze, uint64_t pol, int tid, int nthr)
{
    constexpr bool FASTF = KIND == KIND_DIRECT_FPF;
    const CellF<T> f(d);  // once per chunk
    constexpr int L = VecOf<T>::L;
    long long va, vb;
    if constexpr (VEC) {
        va = (zs + L - 1) / L * L;
        if (va > ze) va = ze;
        vb = va + (ze - va) / L * L;
    } else {
        va = ze;
        vb = ze;
    }
    const T *Xg = reinterpret_cast<const T *>(a.blob + d.xg);  // the knots in global memory (interpolation)
    // scalar head and tail
    auto one = [&](long long q) {
        T z = a.Z[q];
        int32_t r;
        answer_block<T, 1, KIND, SM, FASTF>(a, d, f, K, X, &z, &r, pol);
        a.I[q] = r;
        if constexpr (INTERP) {
            T y;
            interp_values<T, 1>(a, d, Xg, &z, &r, &y);
            a.y_out[q] = y;
        }
    };
    for (long long q = zs + tid; q < va; q += nthr) one(q);
    for (long long q = vb + tid; q < ze; q += nthr) one(q);
    if constexpr (VEC) {
        using V = typename VecOf<T>::V;
        using IV = typename VecOf<T>::IV;
        constexpr int NQ = VPT * L;
        const long long v0 = va / L, nv = (vb - va) / L;
        const V *Zv = reinterpret_cast<const V *>(a.Z) + v0;
        IV *Iv = reinterpret_cast<IV *>(a.I) + v0;
        // direct-only kernels: software pipeline, the next tile's queries are
        // loaded while this tile's table gathers are in flight (the general
        // kernel is at its register limit already)
        constexpr bool PREFETCH = direct_kind(KIND);
        V zn[VPT];
        auto load_tile = [&](long long base) {
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const long long idx = base + (long long)v * nthr;
                zn[v] = idx < nv ? __ldcs(Zv + idx) : Zv[0];
            }
        };
        // the query stream is also prefetched into L2, QP_DIST tiles ahead of
        // its loads, by bulk prefetches of whole tiles (no registers held)
        const long long tile = (long long)VPT * nthr;
        auto prefetch_l2 = [&](long long first) {
            if (first < nv) {
                const long long n = nv - first < tile ? nv - first : tile;
                bulk_prefetch_l2(Zv + first, (uint32_t)(n * (long long)sizeof(V)));
            }
        };
        if (PREFETCH && a.l2pf && tid == 0)
            for (int k = 1; k <= QP_DIST; ++k) prefetch_l2((long long)k * tile);
        if (PREFETCH && tid < nv) load_tile(tid);
        for (long long base = tid; base < nv; base += (long long)VPT * nthr) {
            if (PREFETCH && a.l2pf && tid == 0) prefetch_l2(base + (long long)(QP_DIST + 1) * tile);
            V zv[VPT];
            if constexpr (PREFETCH) {
#pragma unroll
                for (int v = 0; v < VPT; ++v) zv[v] = zn[v];
                if (base + (long long)VPT * nthr < nv) load_tile(base + (long long)VPT * nthr);
            } else {
                load_tile(base);
#pragma unroll
                for (int v = 0; v < VPT; ++v) zv[v] = zn[v];
            }
            const T *zs4 = reinterpret_cast<const T *>(zv);
            int32_t r[NQ];
            answer_block<T, NQ, KIND, SM, FASTF>(a, d, f, K, X, zs4, r, pol);
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const long long idx = base + (long long)v * nthr;
                if (idx < nv) {
                    IV o;
                    if constexpr (L == 4) o = make_int4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
                    else o = make_int2(r[2 * v], r[2 * v + 1]);
                    __stcs(Iv + idx, o);
                }
            }
            if constexpr (INTERP) {  // one vector of queries at a time (register pressure)
                V *yv = reinterpret_cast<V *>(a.y_out) + v0;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const long long idx = base + (long long)v * nthr;
                    V o;
                    interp_values<T, L>(a, d, Xg, zs4 + v * L, r + v * L, reinterpret_cast<T *>(&o));
                    if (idx < nv) __stcs(yv + idx, o);
                }
            }
        }
    }
}

// The array owning chunk c: the largest a with chunk_off[a] <= c (arrays
// without queries share their offset with the next one, so the largest is the
// owner).  Called by all 32 lanes of a warp: a 32-way search, each step
// comparing 32 evenly spaced offsets with one ballot (3 dependent loads for
// 4096 arrays instead of 12 for bisection).
__device__ __forceinline__ int owner_of_chunk(const long long *chunk_off, int n_arrays, long long c)
{
    const int lane = threadIdx.x & 31;
    int lo = 0, n = n_arrays;  // the owner lies in [lo, lo + n); chunk_off[lo] <= c
    while (n > 1) {
        const int step = (n + 31) >> 5;
        const int p = lo + lane * step;
        const bool ok = p < lo + n && chunk_off[p] <= c;
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        const int k = 31 - __clz(mask);  // lane 0 always qualifies
        const int nlo = lo + k * step;
        n = (lo + n - nlo) < step ? (lo + n - nlo) : step;
        lo = nlo;
    }
    return lo;
}

// Claim the next chunk for the calling warp: (chunk, claim position of its
// array), position -1 when none is left.  All 32 lanes call; every lane gets
// the result.
__device__ __forceinline__ void claim_chunk(unsigned long long *counter, const long long *chunk_off, int n_arrays,
                                            long long *c_out, int *pos_out)
{
    long long c = 0;
    if ((threadIdx.x & 31) == 0) c = (long long)atomicAdd(counter, 1ull);
    c = __shfl_sync(0xffffffffu, c, 0);
    *c_out = c;
    *pos_out = c < chunk_off[n_arrays] ? owner_of_chunk(chunk_off, n_arrays, c) : -1;
}

// Queries [zs, ze) of chunk c, claimed at position p (array arr).
template <typename T>
__device__ __forceinline__ void chunk_range(const BatchArgs<T> &a, const ArrDesc &d, int arr, int p, long long c,
                                            long long *zs, long long *ze)
{
    const long long zb = q_begin(a.z_off, arr);
    const long long zend = a.z_off ? a.z_off[arr + 1] : a.m_single;
    const long long len = chunk_len(d, a.chunk, a.smem_limit);
    *zs = zb + (c - a.chunk_off[p]) * len;
    *ze = *zs + len < zend ? *zs + len : zend;
}

// KIND: BatchKind (KIND_DIRECT*: every array the launch serves is in direct
// mode; a handle with direct and learned arrays may serve each group with
// its own launch).
// WARPS: no table is staged (a.smem_limit == 0) and every warp claims its own
// chunks, so no block-wide barrier is needed; otherwise the block claims a
// chunk and stages its array's image for all of its warps.
// MAXB: the largest block the kernel is compiled for (1024 only for the
// direct kinds at one vector per thread, which fit 64 registers).  No kind
// gives a minimum of resident blocks: an explicit 1 lets the compiler spend
// up to 128 registers (the direct kind then took 72 instead of 64, one
// 512-thread block per SM instead of two; 4096 float32 arrays, 2^28 queries:
// 492 -> 430 G lookups/s), and a minimum of 2 at 512 threads (64 registers,
// with spills) measured no better for the kinds that serve 256 float32 arrays
// with the interpolation (79.1 without it, 77.8 with it on the learned kind,
// 77.9 on the direct kind over pairs).
template <typename T, int VPT, bool INTERP, bool VEC, int KIND, bool WARPS = false, int MAXB = 512>
__global__ void __launch_bounds__(MAXB) k_batch_search(BatchArgs<T> a)
{
    if constexpr (WARPS) {
        const int lane = threadIdx.x & 31;
        for (;;) {
            long long c;
            int p;
            claim_chunk(a.counter, a.chunk_off, a.n_arrays, &c, &p);
            if (p < 0) break;
            const int arr = a.order ? a.order[p] : p;
            const ArrDesc d = a.desc[arr];
            long long zs, ze;
            chunk_range(a, d, arr, p, c, &zs, &ze);
            process_chunk<T, VPT, INTERP, VEC, KIND, false>(a, d, a.blob + d.img,
                                                            reinterpret_cast<const T *>(a.blob + d.xg), zs, ze,
                                                            l2_keep_policy(), lane, 32);
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    // the block's next chunk, claimed by warp 0 while the current one is worked
    // on; two slots, read at the start of iteration k from slot k & 1
    __shared__ long long s_c[2];
    __shared__ int s_a[2];
    if (threadIdx.x < 32) {
        long long c0;
        int a0;
        claim_chunk(a.counter, a.chunk_off, a.n_arrays, &c0, &a0);
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            s_c[0] = c0;
            s_a[0] = a0;
        }
    }
    __syncthreads();
    uint32_t parity = 0;
    int staged = -1;
    const uint64_t pol = l2_keep_policy();
    for (int it = 0;; ++it) {
        const long long c = s_c[it & 1];
        const int p = s_a[it & 1];
        if (p < 0) break;
        const int arr = a.order ? a.order[p] : p;
        if (threadIdx.x < 32) {
            long long cn;
            int an;
            claim_chunk(a.counter, a.chunk_off, a.n_arrays, &cn, &an);
            if (threadIdx.x == 0) {
                s_c[(it + 1) & 1] = cn;
                s_a[(it + 1) & 1] = an;
            }
        }
        const ArrDesc d = a.desc[arr];
        long long zs, ze;
        chunk_range(a, d, arr, p, c, &zs, &ze);
        const bool use_smem = stage_image(d, a.smem_limit);
        if (use_smem && staged != arr) {
            if (!stage_again(smem, a.blob + d.img, d.img_bytes, &bar, parity, a.err)) return;
            parity ^= 1u;
            staged = arr;
        }
        const unsigned char *K = use_smem ? smem : a.blob + d.img;
        const T *X = reinterpret_cast<const T *>(use_smem && d.x_in_img != NO_X_IN_IMG ? smem + d.x_in_img
                                                                                       : a.blob + d.xg);
        if (use_smem) process_chunk<T, VPT, INTERP, VEC, KIND, true>(a, d, K, X, zs, ze, pol, threadIdx.x, blockDim.x);
        else process_chunk<T, VPT, INTERP, VEC, KIND, false>(a, d, K, X, zs, ze, pol, threadIdx.x, blockDim.x);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ segmented build kernels
// A segment is a range of at most SEG_KNOTS knots of one array; blocks walk
// segments with a grid stride.
struct Segment {
    long long lo, hi;  // global knot range [lo, hi)
    int32_t arr;
    int32_t pad_;
};

template <typename T>
__global__ void k_seg_validate(const T *__restrict__ Xcat, const long long *__restrict__ x_off,
                               const Segment *__restrict__ segs, int n_segs, HRState *st)
{
    using A = Arith<T>;
    for (int s = blockIdx.x; s < n_segs; s += gridDim.x) {
        const Segment sg = segs[s];
        const long long start = x_off[sg.arr];
        const T X0 = Xcat[start];
        HRState *S = st + sg.arr;
        unsigned long long gmin = NONE64;
        for (long long i = sg.lo + threadIdx.x; i < sg.hi; i += blockDim.x) {
            const T xi = Xcat[i];
            const long long li = i - start;
            if (!isfinite(xi)) atomicMin(&S->bad_nonfinite, (unsigned long long)li);
            if (li >= 1) {
                const T xp = Xcat[i - 1];
                if (!(xp < xi)) atomicMin(&S->bad_order, (unsigned long long)li);
                const T dp = A::sub(xp, X0), di = A::sub(xi, X0);
                if (dp == di) atomicMin(&S->bad_indist, (unsigned long long)li);
                const T gap = A::sub(di, dp);
                if (gap > T(0)) {
                    const unsigned long long b = (unsigned long long)A::bits(gap);
                    gmin = b < gmin ? b : gmin;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, gmin, o);
            gmin = other < gmin ? other : gmin;
        }
        if ((threadIdx.x & 31) == 0 && gmin != NONE64) atomicMin(&S->min_gap_bits, gmin);
    }
}

template <typename T, bool FMA>
__global__ void k_seg_hr_init(const T *Xcat, const long long *x_off, int n_arrays, HRState *st)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_arrays) hr_init_one<T, FMA>(Xcat + x_off[a], x_off[a + 1] - x_off[a], st + a);
}

template <typename T, bool FMA>
__global__ void k_seg_hr_check(const T *__restrict__ Xcat, const long long *__restrict__ x_off,
                               const Segment *__restrict__ segs, int n_segs, HRState *st)
{
    using A = Arith<T>;
    for (int s = blockIdx.x; s < n_segs; s += gridDim.x) {
        const Segment sg = segs[s];
        HRState *S = st + sg.arr;
        if (S->done) continue;
        const long long start = x_off[sg.arr];
        const T H = (T)S->H, W = (T)S->W, X0 = Xcat[start];
        long long first = start + S->cursor;
        if (first < sg.lo) first = sg.lo;
        for (long long i = first + threadIdx.x; i < sg.hi; i += blockDim.x) {
            const uint32_t fa = A::trunc_u32(fval<T, FMA>(H, W, X0, Xcat[i - 1]));
            const uint32_t fb = A::trunc_u32(fval<T, FMA>(H, W, X0, Xcat[i]));
            if (fa == fb) atomicMin(&S->first_violation, (unsigned long long)(i - start));
        }
    }
}

template <typename T, bool FMA>
__global__ void k_seg_hr_grow(const T *Xcat, const long long *x_off, int n_arrays, HRState *st)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_arrays) hr_grow_one<T, FMA>(Xcat + x_off[a], x_off[a + 1] - x_off[a], st + a);
}

// Copy every array's knots (with their values Y as (X_i, Y_i) pairs when
// Ycat is given) into its place in the blob; cells F_i of the knots of
// direct arrays into F and their fingerprints into G (packed like Xcat).
template <typename T>
__global__ void k_seg_copy_fill_F(const T *__restrict__ Xcat, const T *__restrict__ Ycat,
                                  const long long *__restrict__ x_off, const Segment *__restrict__ segs, int n_segs,
                                  const ArrDesc *__restrict__ desc, unsigned char *blob, uint32_t *__restrict__ F,
                                  uint8_t *__restrict__ G)
{
    for (int s = blockIdx.x; s < n_segs; s += gridDim.x) {
        const Segment sg = segs[s];
        const ArrDesc d = desc[sg.arr];
        const long long start = x_off[sg.arr];
        T *Xd = reinterpret_cast<T *>(blob + d.xg);
        for (long long i = sg.lo + threadIdx.x; i < sg.hi; i += blockDim.x) {
            const T x = Xcat[i];
            const long long li = i - start;
            if (Ycat) {
                Xd[2 * li] = x;
                Xd[2 * li + 1] = Ycat[i];
            } else {
                Xd[li] = x;
            }
            if (d.mode == MODE_DIRECT) {  // f and fingerprint exactly as a query computes them
                uint32_t g;
                F[i] = cell_fp(CellF<T>(d)(x), &g);
                G[i] = (uint8_t)g;
            }
        }
    }
}

// Rank words and knot fingerprints of every direct array, in two passes (the
// blob is zeroed first).  k_seg_rank_base writes K_{32 g} of every group:
// warps walk 32-knot chunks of all direct arrays (chunk -> array through the
// chunk offsets kc_off) and write the groups whose first cell lies in the
// chunk's cell span.  k_seg_rank_bits sets, for every knot, its cell's bit,
// and stores its fingerprint.
__global__ void k_seg_rank_base(const uint32_t *__restrict__ F, const long long *__restrict__ x_off,
                                const long long *__restrict__ kc_off, int n_arrays, const ArrDesc *__restrict__ desc,
                                unsigned char *blob);
__global__ void k_seg_rank_bits(const uint32_t *__restrict__ F, const uint8_t *__restrict__ G,
                                const Segment *__restrict__ segs, int n_segs, const long long *__restrict__ x_off,
                                const ArrDesc *__restrict__ desc, unsigned char *blob);

}  // namespace ds
