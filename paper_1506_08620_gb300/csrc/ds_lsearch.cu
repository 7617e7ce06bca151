// ds_lsearch.cu -- the logarithmic searches of Section 3 as GPU kernels:
// Algorithm naivealg (Classic) and its fixed-iteration form (ClassicMod),
// Algorithm binaryopt (leading-bit search on a right-padded array),
// Algorithm binaryoptnopad (the same with min(r, N) after U iterations),
// Algorithm naiveoffset (Knuth's Algorithm U state: start index and size) and
// Algorithm eytzinger (breadth-first layout padded to 2^L - 1).  They are the
// comparators of direct search (the paper's tables of throughput against the
// size of X) and exact searches in their own right.
//
// Every thread answers VPT vectors of queries, the steps of its queries
// interleaved so that their gathers are in flight together.  The layout is
// staged per block into shared memory by a bulk copy when it fits, otherwise
// read through the read-only path (its top levels stay in L1).  float64 layouts
// are stored as order-preserving integer keys, so every comparison is an
// integer one (GB300's FP64 pipe is its scarce resource).
//
// The paper states these algorithms for X_0 <= z < X_N.  A query outside that
// range (or NaN) is answered from X_0 and X_N directly (-1 below X_0, N at or
// above X_N, -1 for NaN), and the algorithm runs on X_0 instead, which keeps
// every index it forms inside the layout.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "ds_search.cuh"

struct ds_lsearch {
    ds::HandleHeader hdr;
    int32_t dtype;
    int32_t method;
    uint32_t flags;
    long long n_knots;
    long long c[4];       // method constants (ds_lsearch_constants)
    long long len;        // elements of the layout
    unsigned char *lay;   // layout: float values, or int64 keys for float64 arrays
    size_t lay_bytes;     // padded to 16 bytes
    double X0, XN;
    bool smem;
    int grid_cap;
    int *dev_err;
    double build_ms;
    ds::DeviceProps props;
};

namespace ds {

constexpr int LS_BLOCK = 256;
constexpr int LS_VPT = 2;

static long long floor_log2(long long v)
{
    long long r = 0;
    while ((2ll << r) <= v) ++r;
    return r;
}

// Constants of each method (host only).
static ds_status ls_constants(int method, long long n_knots, long long c[4], long long *len)
{
    c[0] = c[1] = c[2] = c[3] = 0;
    const long long N = n_knots - 1;
    if (N < 1) return DS_E_ARG;
    *len = n_knots;
    switch (method) {
    case DS_LS_CLASSIC: return DS_OK;
    case DS_LS_CLASSICMOD: {  // ceil(log2 N) iterations
        long long it = 0;
        while ((1ll << it) < N) ++it;
        c[0] = it;
        return DS_OK;
    }
    case DS_LS_LEADBIT:
    case DS_LS_LEADBIT_NOPAD: {
        const long long P = 1ll << floor_log2(N);  // P = 2^floor(log2 N)
        c[0] = P;
        // partial sums s_u = sum_{k=1..u} P / 2^(k-1)
        long long s = 0, u = 0, U = 0, ubar = -1, s_ubar = 0;
        for (long long k = P; k > 0; k >>= 1) {
            s += k;
            ++u;
            if (s <= N) U = u;                            // U = sup{u : s_u <= N}
            if (ubar < 0 && s >= N) ubar = u, s_ubar = s;  // ubar = inf{u : s_u >= N}
        }
        if (method == DS_LS_LEADBIT) {
            c[1] = 1 + s_ubar;  // Q: the array is padded with X_N up to size Q
            *len = c[1] > n_knots ? c[1] : n_knots;
        } else {
            c[1] = U;
        }
        return DS_OK;
    }
    case DS_LS_OFFSET:
        c[0] = (N + 1) / 2;          // F, mid index
        c[1] = N + 1 - c[0];         // S, mid size
        c[2] = floor_log2(N + 1);    // J, iterations
        return DS_OK;
    case DS_LS_EYTZINGER:
        c[0] = 1 + floor_log2(2 + N);  // L
        *len = (1ll << c[0]) - 1;      // X padded with X_N to 2^L - 1, breadth-first
        return DS_OK;
    default: return DS_E_ARG;
    }
}

// ------------------------------------------------------------------ device
// Comparison key of a query: the float itself, or the order-preserving
// integer key of a double (okey).
template <typename T> struct LsKey;
template <> struct LsKey<float> {
    using K = float;
    static __device__ __forceinline__ float of(float z) { return z; }
    static __device__ __forceinline__ bool nan(float z) { return !(z == z); }
};
template <> struct LsKey<double> {
    using K = long long;
    static __device__ __forceinline__ long long of(double z) { return okey(z); }
    static __device__ __forceinline__ bool nan(double z)
    {
        return ((unsigned long long)__double_as_longlong(z) & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
    }
};

template <typename T> struct LsArgs {
    const typename LsKey<T>::K *Y;  // layout in global memory
    uint32_t lay_bytes;
    int smem;
    long long c0, c1, c2;
    int32_t N;
    typename LsKey<T>::K k0, kN;   // keys of X_0 and X_N
    const T *Z;
    int32_t *I;
    long long m;
    int *err;
    long long len;  // elements of the layout (for the range-checking build)
};

template <typename K, bool SM> __device__ __forceinline__ K ls_ld(const K *Y, long long i, long long len, int *err)
{
    const K *p = Y + in_bounds(i, len, BS_LAYOUT, err);
    if constexpr (SM) return *p;
    else return __ldg(p);
}

// NQ queries (keys kz, already moved into [X_0, X_N)) through one method.
template <typename K, int METHOD, int NQ, bool SM>
__device__ __forceinline__ void ls_run(const K *Y, long long c0, long long c1, long long c2, int32_t N, const K *kz,
                                       int32_t *r, long long len, int *err)
{
    if constexpr (METHOD == DS_LS_CLASSIC) {
        // Algorithm naivealg: low/high bisection with a data-dependent trip count
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            int32_t lo = 0, hi = N;
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (kz[q] < ls_ld<K, SM>(Y, mid, len, err)) hi = mid;
                else lo = mid;
            }
            r[q] = lo;
        }
    } else if constexpr (METHOD == DS_LS_CLASSICMOD) {
        // the same with two conditional assignments and ceil(log2 N) iterations
        int32_t lo[NQ], hi[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) lo[q] = 0, hi[q] = N;
        for (long long it = 0; it < c0; ++it) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t mid = (lo[q] + hi[q]) >> 1;
                const bool lt = kz[q] < ls_ld<K, SM>(Y, mid, len, err);
                hi[q] = lt ? mid : hi[q];
                lo[q] = lt ? lo[q] : mid;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) r[q] = lo[q];
    } else if constexpr (METHOD == DS_LS_LEADBIT) {
        // Algorithm binaryopt: one conditional OR per bit on the padded array
        int32_t i[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) i[q] = 0;
        for (int32_t k = (int32_t)c0; k > 0; k >>= 1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t rr = i[q] | k;
                if (!(kz[q] < ls_ld<K, SM>(Y, rr, len, err))) i[q] = rr;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) r[q] = i[q];
    } else if constexpr (METHOD == DS_LS_LEADBIT_NOPAD) {
        // Algorithm binaryoptnopad: U iterations that cannot pass N, then min(r, N)
        int32_t i[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) i[q] = 0;
        int32_t k = (int32_t)c0;
        for (long long u = 0; u < c1; ++u, k >>= 1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t rr = i[q] | k;
                if (!(kz[q] < ls_ld<K, SM>(Y, rr, len, err))) i[q] = rr;
            }
        }
        for (; k > 0; k >>= 1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t rr = i[q] | k;
                const int32_t w = rr < N ? rr : N;
                if (!(kz[q] < ls_ld<K, SM>(Y, w, len, err))) i[q] = rr;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) r[q] = i[q];
    } else if constexpr (METHOD == DS_LS_OFFSET) {
        // Algorithm naiveoffset: start index i and range size S
        int32_t i[NQ];
        const int32_t F0 = (int32_t)c0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) i[q] = !(kz[q] < ls_ld<K, SM>(Y, F0, len, err)) ? F0 : 0;
        int32_t S = (int32_t)c1;
        for (long long j = 0; j < c2; ++j) {
            const int32_t h = S >> 1;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int32_t F = i[q] + h;
                if (!(kz[q] < ls_ld<K, SM>(Y, F, len, err))) i[q] = F;
            }
            S -= h;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) r[q] = i[q];
    } else {
        // Algorithm eytzinger: breadth-first layout, root at 0, children 2P+1, 2P+2
        int32_t P[NQ];
        const int32_t L = (int32_t)c0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) P[q] = !(kz[q] < ls_ld<K, SM>(Y, 0, len, err)) ? 2 : 1;
        for (int32_t l = 1; l < L; ++l) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) P[q] = 2 * P[q] + (!(kz[q] < ls_ld<K, SM>(Y, P[q], len, err)) ? 2 : 1);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) r[q] = P[q] - (1 << L);
    }
}

template <typename T, int METHOD, bool SM, int NQ>
__device__ __forceinline__ void ls_answer(const typename LsKey<T>::K *Y, const LsArgs<T> &a, const T *z, int32_t *r)
{
    using K = typename LsKey<T>::K;
    K kz[NQ];
    int32_t over[NQ];  // -2: in range; otherwise the answer
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const K k = LsKey<T>::of(z[q]);
        over[q] = LsKey<T>::nan(z[q]) ? -1 : (k < a.k0 ? -1 : (!(k < a.kN) ? a.N : -2));
        kz[q] = over[q] == -2 ? k : a.k0;
    }
    ls_run<K, METHOD, NQ, SM>(Y, a.c0, a.c1, a.c2, a.N, kz, r, a.len, a.err);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (over[q] != -2) r[q] = over[q];
}

template <typename T, int METHOD, bool SM>
__global__ void __launch_bounds__(LS_BLOCK) k_lsearch_vec(LsArgs<T> a, long long nvec, long long ntiles)
{
    using K = typename LsKey<T>::K;
    using V = typename VecOf<T>::V;
    using IV = typename VecOf<T>::IV;
    constexpr int L = VecOf<T>::L;
    constexpr int NQ = LS_VPT * L;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    const K *Y = a.Y;
    if constexpr (SM) {
        if (!stage_to_smem(smem, a.Y, a.lay_bytes, &bar, a.err)) return;
        Y = reinterpret_cast<const K *>(smem);
    }
    const V *__restrict__ Zv = reinterpret_cast<const V *>(a.Z);
    IV *__restrict__ Iv = reinterpret_cast<IV *>(a.I);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long b = tile * (long long)LS_VPT * blockDim.x + threadIdx.x;
        V zv[LS_VPT];
#pragma unroll
        for (int v = 0; v < LS_VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            zv[v] = idx < nvec ? __ldcs(Zv + idx) : Zv[0];
        }
        int32_t r[NQ];
        ls_answer<T, METHOD, SM, NQ>(Y, a, reinterpret_cast<const T *>(zv), r);
#pragma unroll
        for (int v = 0; v < LS_VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            if (idx < nvec) {
                IV o;
                if constexpr (L == 4) o = make_int4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
                else o = make_int2(r[2 * v], r[2 * v + 1]);
                __stcs(Iv + idx, o);
            }
        }
    }
    if (blockIdx.x == 0) {  // the last m mod L queries
        const long long q = nvec * L + threadIdx.x;
        if (q < a.m) {
            const T z = a.Z[q];
            int32_t r;
            ls_answer<T, METHOD, SM, 1>(Y, a, &z, &r);
            a.I[q] = r;
        }
    }
}

// Queries or results not aligned for vector access.
template <typename T, int METHOD>
__global__ void __launch_bounds__(LS_BLOCK) k_lsearch_scalar(LsArgs<T> a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.m; q += stride) {
        const T z = a.Z[q];
        int32_t r;
        ls_answer<T, METHOD, false, 1>(a.Y, a, &z, &r);
        a.I[q] = r;
    }
}

// Layout: float values, or okey of the doubles; padded with X_N (index >= N+1),
// or the breadth-first order of the padded array for Eytzinger.
template <typename T>
__global__ void k_ls_layout(const T *__restrict__ X, long long n_knots, int method, long long len, long long L,
                            typename LsKey<T>::K *__restrict__ Y)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += stride) {
        long long src = k;
        if (method == DS_LS_EYTZINGER) {
            // node k (0-based) at depth d holds rank (2 (k + 1 - 2^d) + 1) 2^(L-1-d) - 1
            const long long k1 = k + 1;
            const int d = 63 - __clzll(k1);
            src = ((2 * (k1 - (1ll << d)) + 1) << (L - 1 - d)) - 1;
        }
        if (src > n_knots - 1) src = n_knots - 1;
        Y[k] = LsKey<T>::of(X[src]);
    }
}

// ------------------------------------------------------------------ host
template <typename T, int METHOD>
static const void *ls_pick(bool vec, bool smem)
{
    if (!vec) return (const void *)k_lsearch_scalar<T, METHOD>;
    return smem ? (const void *)k_lsearch_vec<T, METHOD, true> : (const void *)k_lsearch_vec<T, METHOD, false>;
}

template <typename T>
static const void *ls_kernel(int method, bool vec, bool smem)
{
    switch (method) {
    case DS_LS_CLASSIC: return ls_pick<T, DS_LS_CLASSIC>(vec, smem);
    case DS_LS_CLASSICMOD: return ls_pick<T, DS_LS_CLASSICMOD>(vec, smem);
    case DS_LS_LEADBIT: return ls_pick<T, DS_LS_LEADBIT>(vec, smem);
    case DS_LS_LEADBIT_NOPAD: return ls_pick<T, DS_LS_LEADBIT_NOPAD>(vec, smem);
    case DS_LS_OFFSET: return ls_pick<T, DS_LS_OFFSET>(vec, smem);
    default: return ls_pick<T, DS_LS_EYTZINGER>(vec, smem);
    }
}

static uint32_t ls_smem_limit(const DeviceProps &p)
{
    long long lim = 96 * 1024;
    if (const char *e = getenv("DS_SMEM_LIMIT")) lim = atoll(e);
    const long long cap = (long long)p.max_smem_optin - 1024;
    if (lim > cap) lim = cap;
    return lim < 0 ? 0u : (uint32_t)lim;
}

template <typename T>
static ds_status ls_build_typed(ds_lsearch *h, const T *X, cudaStream_t s)
{
    using K = typename LsKey<T>::K;
    h->lay_bytes = round_up((size_t)h->len * sizeof(K), 16);
    DS_TRY_CUDA(dev_alloc(&h->lay, h->lay_bytes));
    DS_TRY_CUDA(cudaMemsetAsync(h->lay, 0, h->lay_bytes, s));
    const long long blocks = std::min<long long>((h->len + 255) / 256, (long long)h->props.num_sms * 8);
    k_ls_layout<T><<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(X, h->n_knots, h->method, h->len, h->c[0],
                                                                        reinterpret_cast<K *>(h->lay));
    DS_TRY_CUDA(cudaGetLastError());
    DS_TRY_CUDA(cudaStreamSynchronize(s));
    h->smem = !(h->flags & DS_NO_SMEM) && h->lay_bytes <= ls_smem_limit(h->props);
    const void *fn = ls_kernel<T>(h->method, true, h->smem);
    if (h->smem) DS_TRY(allow_dynamic_smem(fn, (int)h->lay_bytes));
    int occ = 0;
    DS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, LS_BLOCK, h->smem ? h->lay_bytes : 0));
    if (occ < 1) {
        set_error("ds_lsearch_build: kernel cannot be resident");
        return DS_E_ARG;
    }
    h->grid_cap = occ * h->props.num_sms;
    return DS_OK;
}

template <typename T>
static ds_status ls_search_typed(const ds_lsearch *h, const void *Z, long long m, int32_t *I, cudaStream_t s)
{
    using K = typename LsKey<T>::K;
    LsArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.Y = reinterpret_cast<const K *>(h->lay);
    a.lay_bytes = (uint32_t)std::min<size_t>(h->lay_bytes, 0xFFFFFFF0u);
    a.c0 = h->c[0];
    a.c1 = h->c[1];
    a.c2 = h->c[2];
    a.N = (int32_t)(h->n_knots - 1);
    if constexpr (sizeof(T) == 8) {
        long long b0, bN;
        memcpy(&b0, &h->X0, 8);
        memcpy(&bN, &h->XN, 8);
        a.k0 = b0 >= 0 ? b0 : -(b0 & 0x7FFFFFFFFFFFFFFFll);
        a.kN = bN >= 0 ? bN : -(bN & 0x7FFFFFFFFFFFFFFFll);
    } else {
        a.k0 = (float)h->X0;
        a.kN = (float)h->XN;
    }
    a.Z = reinterpret_cast<const T *>(Z);
    a.I = I;
    a.m = m;
    a.err = h->dev_err;
    a.len = h->len;
    constexpr int L = VecOf<T>::L;
    const bool vec = ((uintptr_t)Z % 16 == 0) && ((uintptr_t)I % (L * sizeof(int32_t)) == 0);
    const void *fn = ls_kernel<T>(h->method, vec, h->smem);
    if (!vec) {
        long long blocks = std::min<long long>((m + LS_BLOCK - 1) / LS_BLOCK, (long long)h->grid_cap * 4);
        void *args[] = {&a};
        DS_TRY_CUDA(cudaLaunchKernel(fn, dim3((unsigned)std::max<long long>(blocks, 1)), dim3(LS_BLOCK), args, 0, s));
        return DS_OK;
    }
    long long nvec = m / L;
    const long long per_tile = (long long)LS_VPT * LS_BLOCK;
    long long ntiles = (nvec + per_tile - 1) / per_tile;
    long long blocks = std::max<long long>(std::min<long long>(ntiles, h->grid_cap), 1);
    void *args[] = {&a, &nvec, &ntiles};
    DS_TRY_CUDA(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(LS_BLOCK), args, h->smem ? h->lay_bytes : 0, s));
    return DS_OK;
}

void free_lsearch(ds_lsearch *h)
{
    if (!h) return;
    if (h->lay) dev_free(h->lay);
    if (h->dev_err) dev_free(h->dev_err);
    h->hdr.magic = 0;
    delete h;
}

ds_status info_lsearch(const ds_lsearch *h, ds_info_t *o)
{
    o->kind = KIND_LSEARCH;
    o->search_launches = 1;
    o->dtype = h->dtype;
    o->flags = h->flags;
    o->n_arrays = 1;
    o->n_knots = h->n_knots;
    o->X0 = h->X0;
    o->XN = h->XN;
    o->table_bytes = (int64_t)h->lay_bytes;
    o->build_ms = h->build_ms;
    o->smem_resident = h->smem ? 1 : 0;
    o->n_fallback = 1;
    int err = 0;
    if (h->dev_err && cudaMemcpy(&err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
        o->device_error = err;
    return DS_OK;
}

}  // namespace ds

using namespace ds;

extern "C" ds_status ds_lsearch_constants(int32_t method, int64_t n_knots, int64_t consts[4], int64_t *layout_len)
{
    if (!consts || !layout_len) {
        set_error("ds_lsearch_constants: null output");
        return DS_E_ARG;
    }
    long long c[4], len = 0;
    const ds_status rc = ls_constants(method, n_knots, c, &len);
    if (rc != DS_OK) {
        set_error("ds_lsearch_constants: bad method %d or size %lld", method, (long long)n_knots);
        return rc;
    }
    for (int k = 0; k < 4; ++k) consts[k] = c[k];
    *layout_len = len;
    return DS_OK;
}

extern "C" ds_status ds_lsearch_build(const void *X_dev, int64_t n_knots, ds_dtype dtype, int32_t method,
                                      uint32_t flags, void *stream, ds_lsearch **out)
{
    clear_error();
    if (!out) {
        set_error("ds_lsearch_build: out is NULL");
        return DS_E_ARG;
    }
    *out = nullptr;
    if (!X_dev || n_knots < 2 || n_knots > (1ll << 30) || (dtype != DS_F32 && dtype != DS_F64) ||
        method < DS_LS_CLASSIC || method > DS_LS_EYTZINGER || (flags & ~(uint32_t)(DS_CHECKED | DS_NO_SMEM))) {
        set_error("ds_lsearch_build: bad argument (X=%p, n_knots=%lld, dtype=%d, method=%d, flags=%u)", X_dev,
                  (long long)n_knots, (int)dtype, method, flags);
        return DS_E_ARG;
    }
    const double t0 = now_ms();
    cudaStream_t s = (cudaStream_t)stream;
    ds_lsearch *h = new ds_lsearch;
    memset(h, 0, sizeof(*h));
    h->hdr.kind = KIND_LSEARCH;
    h->hdr.magic = HANDLE_MAGIC;
    h->dtype = dtype;
    h->method = method;
    h->flags = flags;
    h->n_knots = n_knots;
    ds_status rc = device_props(&h->props);
    if (rc == DS_OK) rc = ls_constants(method, n_knots, h->c, &h->len);
    if (rc == DS_OK && h->len > (1ll << 30)) {  // node indices and 2^L stay within int32
        set_error("ds_lsearch_build: the layout would hold %lld elements (at most 2^30)", h->len);
        rc = DS_E_ARG;
    }
    if (rc == DS_OK) {
        cudaError_t e = dev_alloc(&h->dev_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, sizeof(int));
        const size_t esz = dtype == DS_F32 ? 4 : 8;
        unsigned char ends[16];
        if (e == cudaSuccess) e = cudaMemcpy(ends, X_dev, esz, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(ends + 8, (const unsigned char *)X_dev + (n_knots - 1) * esz, esz, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("ds_lsearch_build: %s", cudaGetErrorString(e));
            rc = e == cudaErrorMemoryAllocation ? DS_E_NOMEM : DS_E_CUDA;
        } else if (dtype == DS_F32) {
            float a, b;
            memcpy(&a, ends, 4);
            memcpy(&b, ends + 8, 4);
            h->X0 = a;
            h->XN = b;
        } else {
            memcpy(&h->X0, ends, 8);
            memcpy(&h->XN, ends + 8, 8);
        }
    }
    if (rc == DS_OK)
        rc = dtype == DS_F32 ? ls_build_typed<float>(h, (const float *)X_dev, s)
                             : ls_build_typed<double>(h, (const double *)X_dev, s);
    if (rc != DS_OK) {
        free_lsearch(h);
        return rc;
    }
    h->build_ms = now_ms() - t0;
    *out = h;
    return DS_OK;
}

extern "C" ds_status ds_lsearch_search(const ds_lsearch *h, const void *Z_dev, int64_t m, int32_t *I_dev,
                                       void *stream)
{
    if (!h || h->hdr.magic != HANDLE_MAGIC || h->hdr.kind != KIND_LSEARCH) {
        set_error("ds_lsearch_search: not a log-search handle");
        return DS_E_ARG;
    }
    if (m == 0) return DS_OK;
    if (!Z_dev || !I_dev || m < 0) {
        set_error("ds_lsearch_search: null pointer or negative size");
        return DS_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return h->dtype == DS_F32 ? ls_search_typed<float>(h, Z_dev, m, I_dev, s)
                              : ls_search_typed<double>(h, Z_dev, m, I_dev, s);
}
