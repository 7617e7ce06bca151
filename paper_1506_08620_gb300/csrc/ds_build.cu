// ds_build.cu -- single-array build (Section 4: ComputeHR, Eq. indexdef,
// Section 4.8 pairs) and the single-array search entry.
#include <cstdlib>
#include <cstring>

#include "ds_index.cuh"

namespace ds {

__global__ void k_hr_state_init(HRState *st, int count, int gap)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= count) return;
    HRState s;
    memset(&s, 0, sizeof(s));
    s.first_violation = NONE64;
    s.bad_nonfinite = NONE64;
    s.bad_order = NONE64;
    s.bad_indist = NONE64;
    s.min_gap_bits = NONE64;
    s.gap = gap;
    st[a] = s;
}

__global__ void k_pack_cells(const uint32_t *__restrict__ K, unsigned long long R, uint4 *__restrict__ P, bool gen)
{
    const unsigned long long nblk = (R + PACK_CELLS) / PACK_CELLS;
    const uint32_t flags = gen ? KNOT_FLAG | KNOT_FLAG2 : KNOT_FLAG;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < (long long)nblk; b += step) {
        const unsigned long long j0 = (unsigned long long)b * PACK_CELLS;
        const uint32_t base = K[j0] & ~flags;
        uint32_t w[3] = {0u, 0u, 0u};
        for (int s = 0; s < PACK_CELLS; ++s) {
            const unsigned long long j = j0 + s;
            if (j > R) break;
            const uint32_t e = K[j];
            const uint32_t byte = ((e & ~flags) - base) | ((e & flags) >> 24);
            w[s >> 2] |= byte << ((s & 3) * 8);
        }
        P[b] = make_uint4(base, w[0], w[1], w[2]);
    }
}

__global__ void k_clear_flags(uint32_t *p, long long count, int stride, uint32_t flag_mask)
{
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += step)
        p[i * stride] &= ~flag_mask;
}

__global__ void k_fill_K_general(const uint32_t *__restrict__ F, long long n_knots, unsigned long long R,
                                 uint32_t *__restrict__ K)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long N = n_knots - 1;
    const long long nchunks = (n_knots + 31) / 32;
    for (long long c = warp; c < nchunks; c += nwarps) {
        const long long i = c * 32 + lane;
        const long long Fi = i <= N ? (long long)F[i] : (1ll << 32);  // lanes past X_N never qualify
        const long long lo = c == 0 ? 0 : (long long)F[c * 32];
        const long long hi = c + 1 == nchunks ? (long long)R + 1 : (long long)F[c * 32 + 32];
        const long long before = c == 0 ? -1 : (long long)F[c * 32 - 1];  // F_{32c-1}
        for (long long base = lo; base < hi; base += 32) {
            const long long j = base + lane;
            // largest lane k with F_{32c+k} <= j (lane 0 qualifies except in the
            // cells below F_0, where K_j = 0)
            int k = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const long long Fc = __shfl_sync(0xffffffffu, Fi, (k + s) & 31);
                if (k + s <= 31 && Fc <= j) k += s;
            }
            const long long Fk = __shfl_sync(0xffffffffu, Fi, k);
            const long long Fkm = __shfl_sync(0xffffffffu, Fi, (k + 31) & 31);
            const long long Fprev = k == 0 ? before : Fkm;  // F_{t-1}
            if (j < hi)
                K[j] = (uint32_t)(c * 32 + k) | (Fk >= j ? KNOT_FLAG : 0u) | (Fprev == j ? KNOT_FLAG2 : 0u);
        }
    }
}

static int grid_for(const DeviceProps &p, long long work, int block)
{
    long long want = (work + block - 1) / block;
    long long cap = (long long)p.num_sms * 8;
    if (want > cap) want = cap;
    return want < 1 ? 1 : (int)want;
}

static uint32_t smem_limit_bytes(const DeviceProps &p)
{
    long long lim = 96 * 1024;
    if (const char *e = getenv("DS_SMEM_LIMIT")) lim = atoll(e);
    long long cap = (long long)p.max_smem_optin - 1024;  // room for the static barrier
    if (lim > cap) lim = cap;
    return lim < 0 ? 0u : (uint32_t)lim;
}

static bool f64_intops_default()
{
    if (const char *e = getenv("DS_F64_INTOPS")) return atoi(e) != 0;
    return true;
}

// ComputeHR on the device, driven from the host: validation, start, then
// rounds of (pair scan, growth step) until done.  Writes the final state to
// *host_st.  `st` is device scratch for one HRState.
template <typename T, bool FMA>
static ds_status run_compute_hr(const T *X, long long n_knots, HRState *st, HRState *host_st, cudaStream_t s,
                                const DeviceProps &props, int gap)
{
    const int block = 256;
    const int grid = grid_for(props, n_knots, block);
    k_hr_state_init<<<1, 1, 0, s>>>(st, 1, gap);
    k_validate<T><<<grid, block, 0, s>>>(X, n_knots, st);
    k_hr_init<T, FMA><<<1, 1, 0, s>>>(X, n_knots, st);
    DS_TRY_CUDA(cudaGetLastError());
    for (long long round = 0;; ++round) {
        for (int k = 0; k < 3; ++k) {
            k_hr_check<T, FMA><<<grid, block, 0, s>>>(X, n_knots, st);
            k_hr_grow<T, FMA><<<1, 1, 0, s>>>(X, n_knots, st);
        }
        DS_TRY_CUDA(cudaGetLastError());
        DS_TRY_CUDA(cudaMemcpyAsync(host_st, st, sizeof(HRState), cudaMemcpyDeviceToHost, s));
        DS_TRY_CUDA(cudaStreamSynchronize(s));
        if (host_st->done) break;
        if (round > 1000000) {
            set_error("ComputeHR did not finish");
            return DS_E_NO_CONVERGENCE;
        }
    }
    return DS_OK;
}

// Refinement of H (end of Section 4.4): bisect [last infeasible H, final H]
// on the bit patterns (positive floats order like them), each probe checking
// every pair and the overflow test; hs receives the smallest feasible H
// reached, its W and R.
template <typename T, bool FMA>
static ds_status refine_h(const T *X, long long n_knots, HRState *st, HRState *hs, cudaStream_t s,
                          const DeviceProps &props)
{
    using A = Arith<T>;
    using B = typename A::Bits;
    const int block = 256;
    const int grid = grid_for(props, n_knots, block);
    T lo_h = (T)hs->H_inf, hi_h = (T)hs->H;
    B lo, hi;
    memcpy(&lo, &lo_h, sizeof(T));
    memcpy(&hi, &hi_h, sizeof(T));
    HRState probe;
    while (hi - lo > 1) {
        const B mid = lo + (hi - lo) / 2;
        T Hm;
        memcpy(&Hm, &mid, sizeof(T));
        k_hr_probe<T, FMA><<<1, 1, 0, s>>>(X, n_knots, Hm, st);
        k_hr_check<T, FMA><<<grid, block, 0, s>>>(X, n_knots, st);
        DS_TRY_CUDA(cudaGetLastError());
        DS_TRY_CUDA(cudaMemcpyAsync(&probe, st, sizeof(HRState), cudaMemcpyDeviceToHost, s));
        DS_TRY_CUDA(cudaStreamSynchronize(s));
        if (probe.status == DS_OK && probe.first_violation == NONE64) hi = mid;
        else lo = mid;
    }
    T Hf;
    memcpy(&Hf, &hi, sizeof(T));
    k_hr_probe<T, FMA><<<1, 1, 0, s>>>(X, n_knots, Hf, st);
    DS_TRY_CUDA(cudaGetLastError());
    DS_TRY_CUDA(cudaMemcpyAsync(&probe, st, sizeof(HRState), cudaMemcpyDeviceToHost, s));
    DS_TRY_CUDA(cudaStreamSynchronize(s));
    hs->H = probe.H;
    hs->W = probe.W;
    hs->R = probe.R;
    return DS_OK;
}

template <typename T, bool FMA>
static ds_status build_typed(const T *X_user, long long n_knots, uint32_t flags, int q, cudaStream_t s, ds_index *idx,
                             bool x0zero)
{
    const DeviceProps &props = idx->props;
    HRState *st = nullptr;
    DS_TRY_CUDA(dev_alloc(&st, sizeof(HRState)));
    HRState hs;
    // Gap-q separates the pairs (i, i+q); with fewer than q+1 knots the pair distance is N
    const bool gen = q >= 2;
    const int gap = (long long)q < n_knots - 1 ? q : (int)(n_knots - 1);
    idx->q = q;
    ds_status rc = run_compute_hr<T, FMA>(X_user, n_knots, st, &hs, s, props, gap);
    if (rc == DS_OK && hs.status == DS_OK && hs.updates > 0 && (flags & DS_REFINE_H))
        rc = refine_h<T, FMA>(X_user, n_knots, st, &hs, s, props);
    dev_free(st);
    if (rc != DS_OK) return rc;
    idx->updates = hs.updates;
    idx->passes = hs.passes;
    idx->H = hs.H;
    idx->W = hs.W;
    if (hs.status != DS_OK) {
        set_error("ds_build: %s (knot %lld)", hr_message(hs.status), hr_bad_knot(hs));
        return (ds_status)hs.status;
    }
    const unsigned long long R = hs.R;
    idx->R = R;
    idx->k_bytes = round_up((size_t)(R + 1) * sizeof(int32_t), 16);
    idx->x_bytes = round_up((size_t)n_knots * sizeof(T), 16);
    const bool cache = (flags & DS_CACHE_LAYOUT) != 0;
    idx->pair_bytes = cache ? round_up((size_t)(R + 1) * sizeof(Pair<T>), 16) : 0;
    idx->table_bytes = idx->k_bytes + idx->x_bytes + idx->pair_bytes;
    const size_t budget = table_budget_bytes();
    if (idx->table_bytes > budget) {
        set_error("ds_build: table needs %zu bytes, budget is %zu (R = %llu)", idx->table_bytes, budget, R);
        return DS_E_TABLE_TOO_LARGE;
    }
    DS_TRY_CUDA(dev_alloc(&idx->tab, idx->k_bytes + idx->x_bytes));
    DS_TRY_CUDA(cudaMemsetAsync(idx->tab, 0, idx->k_bytes + idx->x_bytes, s));
    T *Xc = reinterpret_cast<T *>(idx->tab + idx->k_bytes);
    uint32_t *K = reinterpret_cast<uint32_t *>(idx->tab);
    DS_TRY_CUDA(cudaMemcpyAsync(Xc, X_user, (size_t)n_knots * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (cache) DS_TRY_CUDA(dev_alloc(&idx->pairs, idx->pair_bytes));
    uint32_t *F = nullptr;
    DS_TRY_CUDA(dev_alloc(&F, (size_t)n_knots * sizeof(uint32_t)));
    const int block = 256;
    k_fill_F<T, FMA><<<grid_for(props, n_knots, block), block, 0, s>>>(Xc, n_knots, (T)hs.H, (T)hs.W, F);
    long long warps_work = (n_knots + 31) / 32 * 32;
    if (gen)
        k_fill_K_general<<<grid_for(props, warps_work, block), block, 0, s>>>(F, n_knots, R, K);
    else
        k_fill_K<T><<<grid_for(props, warps_work, block), block, 0, s>>>(
            F, n_knots, K, cache ? reinterpret_cast<Pair<T> *>(idx->pairs) : nullptr, Xc);
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(s);
    dev_free(F);
    if (le != cudaSuccess || se != cudaSuccess) {
        set_error("ds_build: table fill failed: %s", cudaGetErrorString(le != cudaSuccess ? le : se));
        return DS_E_CUDA;
    }
    // search plan
    SearchPlan &plan = idx->plan;
    plan.form = FMA ? F_FMA : (x0zero ? F_PLAIN_X0ZERO : F_PLAIN);
    plan.cache = cache;
    plan.gen = gen;
    plan.intops = sizeof(T) == 8 && f64_intops_default();
    plan.block = SEARCH_BLOCK;
    plan.vpt = SEARCH_VPT;
    if (sizeof(T) == 8 && plan.intops) {
        plan.vpt = 2;  // measured best for the float64 kernel (more resident warps)
        if (const char *e = getenv("DS_F64_VPT")) plan.vpt = atoi(e) == 4 || atoi(e) == 8 ? atoi(e) : 2;
    }
    const size_t image = cache ? idx->pair_bytes : idx->k_bytes + idx->x_bytes;
    plan.smem = !(flags & DS_NO_SMEM) && image <= smem_limit_bytes(props);
    idx->smem_bytes = plan.smem ? (uint32_t)image : 0;
    plan.packed = false;
    if (sizeof(T) == 8 && plan.intops && !plan.smem && !cache && q <= MAX_PACKED_Q) {
        const char *e = getenv("DS_PACKED");
        if (!e || atoi(e) != 0) {
            const unsigned long long nblk = (R + PACK_CELLS) / PACK_CELLS;
            idx->k16_bytes = (size_t)nblk * sizeof(uint4);
            DS_TRY_CUDA(dev_alloc(&idx->k16, idx->k16_bytes));
            k_pack_cells<<<grid_for(props, (long long)nblk, 256), 256, 0, s>>>(K, R, idx->k16, gen);
            DS_TRY_CUDA(cudaGetLastError());
            DS_TRY_CUDA(cudaStreamSynchronize(s));
            idx->table_bytes += idx->k16_bytes;
            plan.packed = true;
        }
    }
    DS_TRY(prepare_search<T>(&plan, idx->smem_bytes, props.num_sms));
    return DS_OK;
}

// Smallest q in 1..q_max for which ComputeHR over the pairs (i, i+q) succeeds
// and the table image (K and X, each padded to 16 bytes) fits budget_bytes;
// 0 if none does.
template <typename T, bool FMA>
static ds_status select_q(const T *X, long long n_knots, long long budget_bytes, int q_max, cudaStream_t s,
                          const DeviceProps &props, int *q_out)
{
    *q_out = 0;
    HRState *st = nullptr;
    DS_TRY_CUDA(dev_alloc(&st, sizeof(HRState)));
    ds_status rc = DS_OK;
    const size_t x_bytes = round_up((size_t)n_knots * sizeof(T), 16);
    for (int q = 1; q <= q_max; ++q) {
        const int gap = (long long)q < n_knots - 1 ? q : (int)(n_knots - 1);
        HRState hs;
        rc = run_compute_hr<T, FMA>(X, n_knots, st, &hs, s, props, gap);
        if (rc != DS_OK) break;
        if (hs.status == DS_E_NOT_INCREASING) {  // no q helps
            rc = DS_E_NOT_INCREASING;
            set_error("ds_build_q: %s (knot %lld)", hr_message(hs.status),
                      (long long)(hs.bad_nonfinite != NONE64 ? hs.bad_nonfinite : hs.bad_order));
            break;
        }
        if (hs.status != DS_OK) continue;
        const size_t bytes = round_up((size_t)(hs.R + 1) * sizeof(int32_t), 16) + x_bytes;
        if ((long long)bytes <= budget_bytes) {
            *q_out = q;
            break;
        }
    }
    dev_free(st);
    return rc;
}

ds_status build_single(const void *X_dev, long long n_knots, ds_dtype dtype, uint32_t flags, int q, int q_max,
                       long long budget_bytes, cudaStream_t s, ds_index **out)
{
    const double t0 = now_ms();
    ds_index *idx = new ds_index;
    memset(idx, 0, sizeof(*idx));
    idx->hdr.kind = KIND_INDEX;
    idx->hdr.magic = HANDLE_MAGIC;
    idx->dtype = dtype;
    idx->flags = flags;
    idx->n_knots = n_knots;
    ds_status rc = device_props(&idx->props);
    if (rc == DS_OK) {
        cudaError_t e = dev_alloc(&idx->dev_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(idx->dev_err, 0, sizeof(int));
        if (e != cudaSuccess) {
            set_error("ds_build: %s", cudaGetErrorString(e));
            rc = e == cudaErrorMemoryAllocation ? DS_E_NOMEM : DS_E_CUDA;
        }
    }
    // first and last knot on the host (X_0 == 0 selects the subtraction-free form)
    if (rc == DS_OK) {
        const size_t esz = dtype == DS_F32 ? sizeof(float) : sizeof(double);
        unsigned char e2[16];
        cudaError_t e = cudaMemcpy(e2, X_dev, esz, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(e2 + 8, (const unsigned char *)X_dev + (n_knots - 1) * esz, esz, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("ds_build: cannot read X: %s", cudaGetErrorString(e));
            rc = DS_E_CUDA;
        } else if (dtype == DS_F32) {
            float a, b;
            memcpy(&a, e2, 4);
            memcpy(&b, e2 + 8, 4);
            idx->X0 = a;
            idx->XN = b;
        } else {
            memcpy(&idx->X0, e2, 8);
            memcpy(&idx->XN, e2 + 8, 8);
        }
    }
    const bool fma = (flags & DS_FMA) != 0;
    if (rc == DS_OK && q == 0) {  // the memory-budget choice of q (Section 4.7)
        if (budget_bytes <= 0) budget_bytes = (long long)smem_limit_bytes(idx->props);
        if (dtype == DS_F32)
            rc = fma ? select_q<float, true>((const float *)X_dev, n_knots, budget_bytes, q_max, s, idx->props, &q)
                     : select_q<float, false>((const float *)X_dev, n_knots, budget_bytes, q_max, s, idx->props, &q);
        else
            rc = fma ? select_q<double, true>((const double *)X_dev, n_knots, budget_bytes, q_max, s, idx->props,
                                              &q)
                     : select_q<double, false>((const double *)X_dev, n_knots, budget_bytes, q_max, s, idx->props,
                                               &q);
        if (rc == DS_OK && q == 0) {
            set_error("ds_build_q: no q in 1..%d gives a feasible table of at most %lld bytes", q_max, budget_bytes);
            rc = DS_E_TABLE_TOO_LARGE;
        }
    }
    if (rc == DS_OK) {
        const bool x0zero = idx->X0 == 0.0;
        if (dtype == DS_F32) {
            rc = fma ? build_typed<float, true>((const float *)X_dev, n_knots, flags, q, s, idx, x0zero)
                     : build_typed<float, false>((const float *)X_dev, n_knots, flags, q, s, idx, x0zero);
        } else {
            rc = fma ? build_typed<double, true>((const double *)X_dev, n_knots, flags, q, s, idx, x0zero)
                     : build_typed<double, false>((const double *)X_dev, n_knots, flags, q, s, idx, x0zero);
        }
    }
    if (rc != DS_OK) {
        free_index(idx);
        return rc;
    }
    idx->build_ms = now_ms() - t0;
    *out = idx;
    return DS_OK;
}

template <typename T>
static ds_status search_typed(const ds_index *idx, const void *Z, long long m, int32_t *I, cudaStream_t s)
{
    SearchArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.K = reinterpret_cast<const uint32_t *>(idx->tab);
    a.K16 = idx->k16;
    a.X = reinterpret_cast<const T *>(idx->tab + idx->k_bytes);
    a.P = reinterpret_cast<const Pair<T> *>(idx->pairs);
    a.smem_src = idx->plan.cache ? idx->pairs : (const void *)idx->tab;
    a.smem_bytes = idx->smem_bytes;
    a.x_smem_off = (uint32_t)idx->k_bytes;
    a.H = (T)idx->H;
    a.W = (T)idx->W;
    a.X0 = (T)idx->X0;
    a.R = (uint32_t)idx->R;
    a.q = idx->q;
    a.checked = (idx->flags & DS_CHECKED) != 0;
    a.Z = reinterpret_cast<const T *>(Z);
    a.I = I;
    a.m = m;
    a.err = idx->dev_err;
    a.n_x = idx->n_knots;
    return launch_search<T>(a, idx->plan, s);
}

ds_status search_index(const ds_index *idx, const void *Z, long long m, int32_t *I, cudaStream_t s)
{
    if (m == 0) return DS_OK;
    if (!Z || !I || m < 0) {
        set_error("ds_search: null pointer or negative size");
        return DS_E_ARG;
    }
    return idx->dtype == DS_F32 ? search_typed<float>(idx, Z, m, I, s) : search_typed<double>(idx, Z, m, I, s);
}

}  // namespace ds

extern "C" ds_status ds_index_tables(const ds_index *idx, const int32_t **K_dev, const void **X_dev,
                                     const void **pairs_dev)
{
    if (!idx || idx->hdr.kind != ds::KIND_INDEX) {
        ds::set_error("ds_index_tables: not an index handle");
        return DS_E_ARG;
    }
    if (K_dev) *K_dev = reinterpret_cast<const int32_t *>(idx->tab);
    if (X_dev) *X_dev = idx->tab + idx->k_bytes;
    if (pairs_dev) *pairs_dev = idx->pairs;
    return DS_OK;
}

extern "C" ds_status ds_index_export(const ds_index *idx, int32_t *K_out_dev, void *X_out_dev, void *pairs_out_dev,
                                     void *stream)
{
    if (!idx || idx->hdr.kind != ds::KIND_INDEX || idx->hdr.magic != ds::HANDLE_MAGIC) {
        ds::set_error("ds_index_export: not an index handle");
        return DS_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t esz = idx->dtype == DS_F32 ? 4 : 8;
    const long long cells = (long long)idx->R + 1;
    const int grid = (int)((cells + 255) / 256 < idx->props.num_sms * 8 ? (cells + 255) / 256 : idx->props.num_sms * 8);
    if (K_out_dev) {
        DS_TRY_CUDA(cudaMemcpyAsync(K_out_dev, idx->tab, (size_t)cells * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        ds::k_clear_flags<<<grid, 256, 0, s>>>(reinterpret_cast<uint32_t *>(K_out_dev), cells, 1,
                                               idx->q >= 2 ? ds::KNOT_FLAG | ds::KNOT_FLAG2 : ds::KNOT_FLAG);
        DS_TRY_CUDA(cudaGetLastError());
    }
    if (X_out_dev)
        DS_TRY_CUDA(cudaMemcpyAsync(X_out_dev, idx->tab + idx->k_bytes, (size_t)idx->n_knots * esz,
                                    cudaMemcpyDeviceToDevice, s));
    if (pairs_out_dev) {
        if (!idx->pairs) {
            ds::set_error("ds_index_export: the index has no pair table (built without DS_CACHE_LAYOUT)");
            return DS_E_ARG;
        }
        DS_TRY_CUDA(cudaMemcpyAsync(pairs_out_dev, idx->pairs, (size_t)cells * (esz == 4 ? 8 : 16),
                                    cudaMemcpyDeviceToDevice, s));
        ds::k_clear_flags<<<grid, 256, 0, s>>>(reinterpret_cast<uint32_t *>(pairs_out_dev), cells, esz == 4 ? 2 : 4,
                                               ds::KNOT_FLAG);
        DS_TRY_CUDA(cudaGetLastError());
    }
    return DS_OK;
}
