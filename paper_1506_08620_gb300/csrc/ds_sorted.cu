// ds_sorted.cu -- two uses of the search the paper's introduction names
// (Section 1.2): sorted queries, solved in O(M + N) by merging Z into X
// instead of searching each query, and counting the samples that fall in each
// interval [X_i, X_{i+1}) (a histogram), fused with direct search.
//
// Merge path: the merged sequence of X (N+1 knots) and Z (M queries), X_i
// placed before z whenever X_i <= z, is cut into tiles of MP_TILE elements.
// The cut at diagonal d (a + b = d: a knots and b queries precede it) is
// found by a bisection; a block takes a contiguous range of tiles and finds
// their cuts MP_BLOCK at a time.  For each tile it stages the tile's knots
// and queries in shared memory, each thread merges MP_ITEMS consecutive
// elements from its own diagonal, and the answers leave through shared
// memory with coalesced stores.  A query merged after a knots gets the answer
// a - 1 = #{X_i <= z} - 1.  Every element is read once from HBM and every
// answer written once.
#include <algorithm>
#include <cstring>

#include "ds_index.cuh"

namespace ds {

// Comparison key of the merge: floats compare as themselves, doubles as their
// order-preserving integer keys (integer comparisons instead of the FP64 pipe).
template <typename T> struct MergeKey;
template <> struct MergeKey<float> {
    using K = float;
    static __device__ __forceinline__ float of(float v) { return v; }
};
template <> struct MergeKey<double> {
    using K = long long;
    static __device__ __forceinline__ long long of(double v) { return okey(v); }
};

constexpr int MP_BLOCK = 256;
constexpr int MP_ITEMS = 11;  // odd: fewer shared-memory bank conflicts in the per-thread merges
constexpr int MP_TILE = MP_BLOCK * MP_ITEMS;

// Number of knots among the first d elements of the merge (X_i before z when
// X_i <= z): the a in [max(0, d - M), min(d, NX)] at which the order flips.
template <typename T>
__device__ __forceinline__ long long merge_split(const T *X, long long NX, const T *Z, long long M, long long d)
{
    long long lo = d - M > 0 ? d - M : 0, hi = d < NX ? d : NX;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        // X[mid] before Z[d - mid - 1]: the cut takes more knots
        if (!(MergeKey<T>::of(Z[d - mid - 1]) < MergeKey<T>::of(X[mid]))) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(MP_BLOCK) k_merge_search(const T *__restrict__ X, long long NX,
                                                           const T *__restrict__ Z, long long M,
                                                           int32_t *__restrict__ I)
{
    using K = typename MergeKey<T>::K;
    extern __shared__ __align__(16) unsigned char smem[];
    K *sX = reinterpret_cast<K *>(smem);
    K *sZ = sX + MP_TILE;
    int32_t *sI = reinterpret_cast<int32_t *>(sZ + MP_TILE);
    __shared__ long long cuts[MP_BLOCK + 1];
    const long long total = NX + M;
    const long long ntiles = (total + MP_TILE - 1) / MP_TILE;
    // a contiguous range of tiles per block; their cuts are found MP_BLOCK at a
    // time, one bisection per thread, so that the bisections' latencies overlap
    const long long per = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t_begin = blockIdx.x * per;
    const long long t_end = t_begin + per < ntiles ? t_begin + per : ntiles;
    for (long long base = t_begin; base < t_end; base += MP_BLOCK) {
        const int n = (int)(t_end - base < MP_BLOCK ? t_end - base : MP_BLOCK);
        for (int k = threadIdx.x; k <= n; k += blockDim.x) {
            const long long d = (base + k) * MP_TILE;
            cuts[k] = merge_split(X, NX, Z, M, d < total ? d : total);
        }
        __syncthreads();
        // tile j of the round: its cut (a0, b0) and sizes, clamped as described below
        auto tile_of = [&](int j, long long *a0, long long *b0, int *nx, int *nz) {
            const long long d0 = (base + j) * MP_TILE;
            const long long d1 = d0 + MP_TILE < total ? d0 + MP_TILE : total;
            // for sorted inputs a1 - a0 lies in [0, d1 - d0] already; the clamp keeps
            // every index inside the tile and inside X and Z for any input
            long long a1 = cuts[j + 1];
            const long long a1_lo = cuts[j] > d1 - M ? cuts[j] : d1 - M;
            const long long a1_hi = cuts[j] + (d1 - d0) < NX ? cuts[j] + (d1 - d0) : NX;
            a1 = a1 < a1_lo ? a1_lo : (a1 > a1_hi ? a1_hi : a1);
            *a0 = cuts[j];
            *b0 = d0 - cuts[j];
            *nx = (int)(a1 - cuts[j]);
            *nz = (int)((d1 - a1) - *b0);
        };
        // software pipeline: tile j + 1's knots and queries are loaded into
        // registers while tile j is merged
        K vz[MP_ITEMS], vx[MP_ITEMS];
        auto load_regs = [&](int j) {
            long long a0, b0;
            int nx, nz;
            tile_of(j, &a0, &b0, &nx, &nz);
#pragma unroll
            for (int u = 0; u < MP_ITEMS; ++u) {
                const int k = threadIdx.x + u * MP_BLOCK;
                vz[u] = MergeKey<T>::of(k < nz ? __ldcs(Z + b0 + k) : T(0));
                vx[u] = MergeKey<T>::of(k < nx ? X[a0 + k] : T(0));
            }
        };
        if (n > 0) load_regs(0);
        for (int j = 0; j < n; ++j) {
            long long a0, b0;
            int nx, nz;
            tile_of(j, &a0, &b0, &nx, &nz);
#pragma unroll
            for (int u = 0; u < MP_ITEMS; ++u) {
                const int k = threadIdx.x + u * MP_BLOCK;
                if (k < nz) sZ[k] = vz[u];
                if (k < nx) sX[k] = vx[u];
            }
            __syncthreads();
            if (j + 1 < n) load_regs(j + 1);
            // this thread's diagonal inside the tile, then a sequential merge
            const int dt = threadIdx.x * MP_ITEMS;
            if (dt < nx + nz) {
                int lo = dt - nz > 0 ? dt - nz : 0, hi = dt < nx ? dt : nx;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (!(sZ[dt - mid - 1] < sX[mid])) lo = mid + 1;
                    else hi = mid;
                }
                int a = lo, b = dt - lo;
                const int end = dt + MP_ITEMS < nx + nz ? dt + MP_ITEMS : nx + nz;
                for (int k = dt; k < end; ++k) {
                    // take the knot when it precedes the query (or no query is left)
                    const bool take_x = b >= nz || (a < nx && !(sZ[b] < sX[a]));
                    if (take_x) {
                        ++a;
                    } else {
                        sI[b] = (int32_t)(a0 + a - 1);
                        ++b;
                    }
                }
            }
            __syncthreads();
            for (int k = threadIdx.x; k < nz; k += blockDim.x) __stcs(I + b0 + k, sI[k]);
        }
        __syncthreads();
    }
}

// Counts of the answers -1 .. N (bins 0 .. N+1) of direct search; NaN counts
// as -1.  SMH: per-block counters in shared memory, added to the global
// counts at the end.
template <typename T, int FM, bool GEN, bool SMH>
__global__ void __launch_bounds__(256) k_histogram(SearchArgs<T> a, unsigned long long *__restrict__ counts,
                                                   long long nbins)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *h = reinterpret_cast<uint32_t *>(smem);
    if constexpr (SMH) {
        for (long long k = threadIdx.x; k < nbins; k += blockDim.x) h[k] = 0u;
        __syncthreads();
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.m; q += stride) {
        int32_t i;
        if constexpr (sizeof(T) == 8) {
            // doubles as bit patterns: one FP64 instruction per query (as k_search_f64bits)
            const long long zb = __ldcs(reinterpret_cast<const long long *>(a.Z) + q);
            const long long *Xb = reinterpret_cast<const long long *>(a.X);
            const uint32_t j = cell_bits<FM>(zb, (double)a.H, -(double)a.W, (double)a.X0, a.R);
            const uint32_t e = __ldg(a.K + in_bounds(j, (long long)a.R + 1, BS_K, a.err));
            if constexpr (GEN) {
                const int32_t t = (int32_t)(e & GEN_T_MASK);
                const long long xb = (e & KNOT_FLAG) ? __ldg(Xb + in_bounds(t, a.n_x, BS_X, a.err)) : 0;
                const long long xpb = (e & KNOT_FLAG2) ? __ldg(Xb + in_bounds(t - 1, a.n_x, BS_X, a.err)) : 0;
                i = correct_bits_gen<true>(zb, e, xb, xpb, Xb, 0, a.q, 1, a.n_x, a.err);  // plain loads in the bisection
            } else {
                i = correct_bits(zb, e,
                                 (e & KNOT_FLAG) ? __ldg(Xb + in_bounds((int32_t)(e & ~KNOT_FLAG), a.n_x, BS_X, a.err))
                                                 : 0,
                                 1);
            }
        } else {
            i = lookup<T, FM, false, false, false, GEN>(__ldcs(a.Z + q), a.K, a.X, a.P, a);
        }
        const long long bin = i + 1;
        if constexpr (SMH) atomicAdd(&h[bin], 1u);
        else atomicAdd(&counts[bin], 1ull);
    }
    if constexpr (SMH) {
        __syncthreads();
        for (long long k = threadIdx.x; k < nbins; k += blockDim.x)
            if (h[k]) atomicAdd(&counts[k], (unsigned long long)h[k]);
    }
}

template <typename T, int FM, bool GEN>
static const void *hist_pick2(bool smh)
{
    return smh ? (const void *)k_histogram<T, FM, GEN, true> : (const void *)k_histogram<T, FM, GEN, false>;
}
template <typename T, int FM>
static const void *hist_pick1(bool gen, bool smh)
{
    return gen ? hist_pick2<T, FM, true>(smh) : hist_pick2<T, FM, false>(smh);
}
template <typename T>
static const void *hist_pick(int form, bool gen, bool smh)
{
    switch (form) {
    case F_FMA: return hist_pick1<T, F_FMA>(gen, smh);
    case F_PLAIN_X0ZERO: return hist_pick1<T, F_PLAIN_X0ZERO>(gen, smh);
    default: return hist_pick1<T, F_PLAIN>(gen, smh);
    }
}

template <typename T>
static ds_status histogram_typed(const ds_index *idx, const void *Z, long long m, unsigned long long *counts,
                                 cudaStream_t s)
{
    SearchArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.K = reinterpret_cast<const uint32_t *>(idx->tab);
    a.X = reinterpret_cast<const T *>(idx->tab + idx->k_bytes);
    a.H = (T)idx->H;
    a.W = (T)idx->W;
    a.X0 = (T)idx->X0;
    a.R = (uint32_t)idx->R;
    a.q = idx->q;
    a.checked = 1;  // NaN counts as -1
    a.Z = reinterpret_cast<const T *>(Z);
    a.m = m;
    a.err = idx->dev_err;
    a.n_x = idx->n_knots;
    const long long nbins = idx->n_knots + 1;
    const size_t hbytes = (size_t)nbins * sizeof(uint32_t);
    const bool smh = hbytes <= 96 * 1024;
    const void *fn = hist_pick<T>(idx->plan.form, idx->q >= 2, smh);
    if (smh) DS_TRY(allow_dynamic_smem(fn, (int)hbytes));
    int occ = 0;
    DS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smh ? hbytes : 0));
    long long blocks = std::max(1, occ) * (long long)idx->props.num_sms;
    blocks = std::min(blocks, std::max(1ll, (m + 255) / 256));
    long long nb = nbins;
    void *args[] = {&a, &counts, &nb};
    DS_TRY_CUDA(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(256), args, smh ? hbytes : 0, s));
    return DS_OK;
}

template <typename T>
static ds_status merge_typed(const void *X, long long NX, const void *Z, long long M, int32_t *I, cudaStream_t s)
{
    int dev = 0, sms = 0, occ = 0;
    DS_TRY_CUDA(cudaGetDevice(&dev));
    DS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t sbytes = 2 * (size_t)MP_TILE * sizeof(typename MergeKey<T>::K) + (size_t)MP_TILE * sizeof(int32_t);
    DS_TRY(allow_dynamic_smem((const void *)k_merge_search<T>, (int)sbytes));
    DS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_merge_search<T>, MP_BLOCK, sbytes));
    const long long ntiles = (NX + M + MP_TILE - 1) / MP_TILE;
    const long long blocks = std::max(1ll, std::min(ntiles, (long long)std::max(occ, 1) * sms));
    k_merge_search<T><<<(unsigned)blocks, MP_BLOCK, sbytes, s>>>(reinterpret_cast<const T *>(X), NX,
                                                                 reinterpret_cast<const T *>(Z), M, I);
    DS_TRY_CUDA(cudaGetLastError());
    return DS_OK;
}

}  // namespace ds

using namespace ds;

extern "C" ds_status ds_search_sorted(const void *X_dev, int64_t n_knots, ds_dtype dtype, const void *Z_dev, int64_t m,
                                      int32_t *I_dev, void *stream)
{
    if (m == 0) return DS_OK;
    if (!X_dev || !Z_dev || !I_dev || n_knots < 1 || n_knots > (1ll << 31) - 1 || m < 0 ||
        (dtype != DS_F32 && dtype != DS_F64)) {
        set_error("ds_search_sorted: bad argument (X=%p, n_knots=%lld, dtype=%d, Z=%p, m=%lld, I=%p)", X_dev,
                  (long long)n_knots, (int)dtype, Z_dev, (long long)m, (void *)I_dev);
        return DS_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return dtype == DS_F32 ? merge_typed<float>(X_dev, n_knots, Z_dev, m, I_dev, s)
                           : merge_typed<double>(X_dev, n_knots, Z_dev, m, I_dev, s);
}

extern "C" ds_status ds_histogram(const ds_index *idx, const void *Z_dev, int64_t m, uint64_t *counts_dev,
                                  void *stream)
{
    if (!idx || idx->hdr.kind != KIND_INDEX || idx->hdr.magic != HANDLE_MAGIC) {
        set_error("ds_histogram: not an index handle");
        return DS_E_ARG;
    }
    if (m == 0) return DS_OK;
    if (!Z_dev || !counts_dev || m < 0) {
        set_error("ds_histogram: null pointer or negative size");
        return DS_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *c = reinterpret_cast<unsigned long long *>(counts_dev);
    return idx->dtype == DS_F32 ? histogram_typed<float>(idx, Z_dev, m, c, s)
                                : histogram_typed<double>(idx, Z_dev, m, c, s);
}
