// ds_cluster.cu -- float64 direct search with the table held in the
// distributed shared memory of a thread-block cluster (DS_CLUSTER_TABLE).
//
// The table of Eq. indexdef is held as a rank table (with pairs (i, i+1) a
// cell holds at most one knot, so K_j = #{i : F_i < j}): one word per 64
// cells, K at the word's first cell (uint32) and a 64-bit mask of the cells
// holding a knot, so K_j = base + popc(mask below j mod 64).  The words are
// sliced over the CTAs of a 16-CTA cluster (16384 words, 192 KB, per CTA),
// so a cluster holds up to 2^20 words = 2^26 cells.  Every CTA loads its
// slice once per launch; a query's word is then read from the shared memory
// of the CTA that owns it (ld.shared::cluster), instead of from L2 through
// the L1TEX request path.  The knot X_t of a cell holding a knot is read from
// global memory as in the other kernels.
#include "ds_index.cuh"
#include "ds_search.cuh"

namespace ds {

constexpr int CL_CTAS = 16;                     // CTAs per cluster
constexpr int CL_WPC_SHIFT = 14;                // 16384 words per CTA
constexpr uint32_t CL_WPC = 1u << CL_WPC_SHIFT;
constexpr size_t CL_SMEM = (size_t)CL_WPC * 12; // masks (8 B) then bases (4 B): 192 KB
constexpr int CL_THREADS = 1024;
constexpr int CL_VPT = 2;                       // double2 vectors of queries per thread per tile

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives, then waits for all (the
// smem writes before it are visible to the cluster after it).
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_rank(uint32_t cta_addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(cta_addr), "r"(rank));
    return r;
}
__device__ __forceinline__ unsigned long long ld_cluster_u64(uint32_t addr)
{
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// Words from the table K (flag bit 31: the cell holds its knot): word w
// covers cells 64 w .. 64 w + 63 (cells past R: no knot).
__global__ void k_cluster_words(const uint32_t *__restrict__ K, unsigned long long cells,
                                unsigned long long *__restrict__ mask, uint32_t *__restrict__ base, uint32_t words)
{
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
        const unsigned long long c0 = (unsigned long long)w * 64ull;
        unsigned long long m = 0;
        for (int b = 0; b < 64; ++b)
            if (c0 + b < cells && (K[c0 + b] & KNOT_FLAG)) m |= 1ull << b;
        mask[w] = m;
        base[w] = K[c0] & ~KNOT_FLAG;
    }
}

struct ClusterArgs {
    const unsigned long long *mask;
    const uint32_t *base;
    uint32_t words;
    const long long *X;  // knots as bit patterns
    double H, NW, X0;
    uint32_t R;
    int checked;
    const double *Z;
    int32_t *I;
    long long m, nvec, ntiles;
};

template <int FM>
__global__ void __launch_bounds__(CL_THREADS) k_search_f64_cluster(ClusterArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sm_mask = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *sm_base = reinterpret_cast<uint32_t *>(smem + (size_t)CL_WPC * 8);
    const uint32_t rank = cluster_rank();
    for (uint32_t i = threadIdx.x; i < CL_WPC; i += blockDim.x) {
        const uint32_t w = (rank << CL_WPC_SHIFT) + i;
        sm_mask[i] = w < a.words ? __ldg(a.mask + w) : 0ull;
        sm_base[i] = w < a.words ? __ldg(a.base + w) : 0u;
    }
    cluster_sync_all();
    const uint32_t mask_addr = smem_u32(sm_mask), base_addr = smem_u32(sm_base);
    const uint64_t keep = l2_keep_policy();
    const longlong2 *__restrict__ Zv = reinterpret_cast<const longlong2 *>(a.Z);
    int2 *__restrict__ Iv = reinterpret_cast<int2 *>(a.I);
    constexpr int NQ = 2 * CL_VPT;
    for (long long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const long long b = tile * (long long)CL_VPT * blockDim.x + threadIdx.x;
        long long zb[NQ];
#pragma unroll
        for (int v = 0; v < CL_VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            const longlong2 q = idx < a.nvec ? __ldcs(Zv + idx) : make_longlong2(0, 0);
            zb[2 * v] = q.x;
            zb[2 * v + 1] = q.y;
        }
        uint32_t e[NQ];
        unsigned long long mk[NQ];
        uint32_t bs[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            e[q] = cell_bits<FM>(zb[q], a.H, a.NW, a.X0, a.R);
            const uint32_t w = e[q] >> 6, owner = w >> CL_WPC_SHIFT, li = w & (CL_WPC - 1u);
            mk[q] = ld_cluster_u64(map_rank(mask_addr + li * 8u, owner));
            bs[q] = ld_cluster_u32(map_rank(base_addr + li * 4u, owner));
        }
        long long xb[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint32_t bit = e[q] & 63u;
            const unsigned long long below = bit ? mk[q] & ((1ull << bit) - 1ull) : 0ull;
            const uint32_t t = bs[q] + (uint32_t)__popcll(below);
            const bool knot = (mk[q] >> bit) & 1ull;
            e[q] = t | (knot ? KNOT_FLAG : 0u);
            xb[q] = knot ? ld_keep(a.X + t, keep) : 0ll;
        }
#pragma unroll
        for (int v = 0; v < CL_VPT; ++v) {
            const long long idx = b + (long long)v * blockDim.x;
            if (idx < a.nvec)
                __stcs(Iv + idx, make_int2(correct_bits(zb[2 * v], e[2 * v], xb[2 * v], a.checked),
                                           correct_bits(zb[2 * v + 1], e[2 * v + 1], xb[2 * v + 1], a.checked)));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (a.m & 1)) {  // the last query of an odd count
        const long long zq = reinterpret_cast<const long long *>(a.Z)[a.m - 1];
        uint32_t e = cell_bits<FM>(zq, a.H, a.NW, a.X0, a.R);
        const uint32_t w = e >> 6, owner = w >> CL_WPC_SHIFT, li = w & (CL_WPC - 1u);
        const unsigned long long mk = ld_cluster_u64(map_rank(mask_addr + li * 8u, owner));
        const uint32_t bs = ld_cluster_u32(map_rank(base_addr + li * 4u, owner));
        const uint32_t bit = e & 63u;
        const uint32_t t = bs + (uint32_t)__popcll(bit ? mk & ((1ull << bit) - 1ull) : 0ull);
        const bool knot = (mk >> bit) & 1ull;
        const long long xq = knot ? a.X[t] : 0ll;
        a.I[a.m - 1] = correct_bits(zq, t | (knot ? KNOT_FLAG : 0u), xq, a.checked);
    }
    cluster_sync_all();  // no CTA leaves while the cluster may still read its slice
}

template <int FM>
static ds_status launch_cluster(const ds_index *idx, const void *Z, long long m, int32_t *I, cudaStream_t s)
{
    const void *fn = (const void *)k_search_f64_cluster<FM>;
    DS_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    DS_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = CL_SMEM;
    cfg.stream = s;
    cfg.gridDim = dim3(CL_CTAS);
    int clusters = 0;
    DS_TRY_CUDA(cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg));
    if (clusters < 1) {
        set_error("cluster search: a cluster of %d CTAs with %zu bytes of shared memory each cannot be resident",
                  CL_CTAS, CL_SMEM);
        return DS_E_UNIMPLEMENTED;
    }
    cfg.gridDim = dim3((unsigned)(clusters * CL_CTAS));
    ClusterArgs a;
    a.mask = idx->cw_mask;
    a.base = idx->cw_base;
    a.words = idx->cw_words;
    a.X = reinterpret_cast<const long long *>(idx->tab + idx->k_bytes);
    a.H = idx->H;
    a.NW = -idx->W;
    a.X0 = idx->X0;
    a.R = (uint32_t)idx->R;
    a.checked = (idx->flags & DS_CHECKED) != 0;
    a.Z = (const double *)Z;
    a.I = I;
    a.m = m;
    a.nvec = m / 2;
    a.ntiles = (a.nvec + (long long)CL_VPT * CL_THREADS - 1) / ((long long)CL_VPT * CL_THREADS);
    DS_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_search_f64_cluster<FM>, a));
    return DS_OK;
}

ds_status build_cluster_words(ds_index *idx, cudaStream_t s)
{
    const unsigned long long cells = idx->R + 1ull;
    const unsigned long long words = (cells + 63ull) / 64ull;
    if (words > (unsigned long long)CL_CTAS * CL_WPC) {
        set_error("DS_CLUSTER_TABLE: %llu cells exceed a cluster's %llu", cells,
                  (unsigned long long)CL_CTAS * CL_WPC * 64ull);
        return DS_E_TABLE_TOO_LARGE;
    }
    idx->cw_words = (uint32_t)words;
    DS_TRY_CUDA(cudaMalloc(&idx->cw_mask, words * sizeof(unsigned long long)));
    DS_TRY_CUDA(cudaMalloc(&idx->cw_base, words * sizeof(uint32_t)));
    const int grid = (int)std::min<unsigned long long>((words + 255) / 256, (unsigned long long)idx->props.num_sms * 8);
    k_cluster_words<<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(idx->tab), cells, idx->cw_mask,
                                         idx->cw_base, (uint32_t)words);
    DS_TRY_CUDA(cudaGetLastError());
    DS_TRY_CUDA(cudaStreamSynchronize(s));
    idx->table_bytes += words * 12;
    return DS_OK;
}

ds_status search_cluster(const ds_index *idx, const void *Z, long long m, int32_t *I, cudaStream_t s)
{
    if (((uintptr_t)Z % 16) || ((uintptr_t)I % 8)) {
        set_error("cluster search: queries and results must be 16- and 8-byte aligned");
        return DS_E_ARG;
    }
    switch (idx->plan.form) {
    case F_FMA: return launch_cluster<F_FMA>(idx, Z, m, I, s);
    case F_PLAIN_X0ZERO: return launch_cluster<F_PLAIN_X0ZERO>(idx, Z, m, I, s);
    default: return launch_cluster<F_PLAIN>(idx, Z, m, I, s);
    }
}

}  // namespace ds
