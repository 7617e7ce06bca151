// ds_search_impl.cuh -- kernel selection and launch for one element type.
// Included by exactly one translation unit per type (ds_search_f32.cu,
// ds_search_f64.cu) so the two sets of instantiations compile in parallel.
#pragma once

#include "ds_search.cuh"

namespace ds {

template <int FM, bool CACHE, bool SMEM>
static const void *pick_f64bits(int vpt, bool packed)
{
    if constexpr (!CACHE && !SMEM) {
        if (packed) return vpt == 2 ? (const void *)k_search_f64bits<FM, false, false, 2, true>
                                    : (const void *)k_search_f64bits<FM, false, false, 4, true>;
    }
    (void)packed;
    switch (vpt) {
    case 2: return (const void *)k_search_f64bits<FM, CACHE, SMEM, 2>;
    case 8: return (const void *)k_search_f64bits<FM, CACHE, SMEM, 8>;
    default: return (const void *)k_search_f64bits<FM, CACHE, SMEM, 4>;
    }
}

template <typename T, int FM, bool CACHE, bool SMEM>
static const void *pick_vec4(bool intops, int vpt, bool packed)
{
    if constexpr (sizeof(T) == 8) {
        if (intops) return pick_f64bits<FM, CACHE, SMEM>(vpt, packed);
    }
    (void)vpt;
    (void)packed;
    (void)intops;
    return (const void *)k_search_vec<T, FM, CACHE, SMEM, false, SEARCH_VPT>;
}
template <typename T, int FM, bool CACHE>
static const void *pick_vec3(bool smem, bool intops, int vpt, bool packed)
{
    return smem ? pick_vec4<T, FM, CACHE, true>(intops, vpt, packed)
                : pick_vec4<T, FM, CACHE, false>(intops, vpt, packed);
}
template <typename T, int FM>
static const void *pick_vec2(bool cache, bool smem, bool intops, int vpt, bool packed)
{
    return cache ? pick_vec3<T, FM, true>(smem, intops, vpt, packed)
                 : pick_vec3<T, FM, false>(smem, intops, vpt, packed);
}
// Eq. kgeneral kernels (q >= 2): no cache layout; float64 on bit patterns with VPT 2 or 4.
template <typename T, int FM, bool SMEM>
static const void *pick_gen_3(const SearchPlan &p)
{
    if constexpr (sizeof(T) == 8) {
        if (p.intops) {
            if constexpr (!SMEM) {
                if (p.packed) return p.vpt == 4 ? (const void *)k_search_f64bits<FM, false, false, 4, true, true>
                                                : (const void *)k_search_f64bits<FM, false, false, 2, true, true>;
            }
            return p.vpt == 4 ? (const void *)k_search_f64bits<FM, false, SMEM, 4, false, true>
                              : (const void *)k_search_f64bits<FM, false, SMEM, 2, false, true>;
        }
    }
    return (const void *)k_search_vec<T, FM, false, SMEM, false, SEARCH_VPT, true>;
}
template <typename T, int FM>
static const void *pick_gen_2(const SearchPlan &p)
{
    return p.smem ? pick_gen_3<T, FM, true>(p) : pick_gen_3<T, FM, false>(p);
}

template <typename T>
static const void *pick_vec(const SearchPlan &p)
{
    if (p.gen) {
        switch (p.form) {
        case F_FMA: return pick_gen_2<T, F_FMA>(p);
        case F_PLAIN_X0ZERO: return pick_gen_2<T, F_PLAIN_X0ZERO>(p);
        default: return pick_gen_2<T, F_PLAIN>(p);
        }
    }
    switch (p.form) {
    case F_FMA: return pick_vec2<T, F_FMA>(p.cache, p.smem, p.intops, p.vpt, p.packed);
    case F_PLAIN_X0ZERO: return pick_vec2<T, F_PLAIN_X0ZERO>(p.cache, p.smem, p.intops, p.vpt, p.packed);
    default: return pick_vec2<T, F_PLAIN>(p.cache, p.smem, p.intops, p.vpt, p.packed);
    }
}

template <typename T, int FM, bool CACHE>
static const void *pick_scalar3(bool intops)
{
    if constexpr (sizeof(T) == 8) {
        if (intops) return (const void *)k_search_scalar<T, FM, CACHE, true>;
    }
    (void)intops;
    return (const void *)k_search_scalar<T, FM, CACHE, false>;
}
template <typename T, int FM>
static const void *pick_scalar2(bool cache, bool intops)
{
    return cache ? pick_scalar3<T, FM, true>(intops) : pick_scalar3<T, FM, false>(intops);
}
template <typename T, int FM>
static const void *pick_scalar_gen(bool intops)
{
    if constexpr (sizeof(T) == 8) {
        if (intops) return (const void *)k_search_scalar<T, FM, false, true, true>;
    }
    (void)intops;
    return (const void *)k_search_scalar<T, FM, false, false, true>;
}

template <typename T>
static const void *pick_scalar(const SearchPlan &p)
{
    if (p.gen) {
        switch (p.form) {
        case F_FMA: return pick_scalar_gen<T, F_FMA>(p.intops);
        case F_PLAIN_X0ZERO: return pick_scalar_gen<T, F_PLAIN_X0ZERO>(p.intops);
        default: return pick_scalar_gen<T, F_PLAIN>(p.intops);
        }
    }
    switch (p.form) {
    case F_FMA: return pick_scalar2<T, F_FMA>(p.cache, p.intops);
    case F_PLAIN_X0ZERO: return pick_scalar2<T, F_PLAIN_X0ZERO>(p.cache, p.intops);
    default: return pick_scalar2<T, F_PLAIN>(p.cache, p.intops);
    }
}

template <typename T>
ds_status prepare_search(SearchPlan *plan, uint32_t smem_bytes, int num_sms)
{
    const void *fn = pick_vec<T>(*plan);
    if (plan->smem) DS_TRY(allow_dynamic_smem(fn, (int)smem_bytes));
    int occ = 0;
    DS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, plan->block, plan->smem ? smem_bytes : 0));
    if (occ < 1) {
        set_error("search kernel cannot be resident with %u bytes of shared memory", smem_bytes);
        return DS_E_ARG;
    }
    plan->grid_cap = occ * num_sms;
    return DS_OK;
}

template <typename T>
ds_status launch_search(const SearchArgs<T> &a, const SearchPlan &plan, cudaStream_t stream)
{
    if (a.m <= 0) return DS_OK;
    constexpr int L = VecOf<T>::L;
    const bool aligned = (((uintptr_t)a.Z) % 16 == 0) && (((uintptr_t)a.I) % (L * sizeof(int32_t)) == 0);
    if (!aligned) {
        SearchPlan p = plan;
        p.smem = false;
        const void *fn = pick_scalar<T>(p);
        long long blocks = (a.m + plan.block - 1) / plan.block;
        if (blocks > (long long)plan.grid_cap * 4) blocks = (long long)plan.grid_cap * 4;
        SearchArgs<T> args = a;
        void *kargs[] = {&args};
        DS_TRY_CUDA(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(plan.block), kargs, 0, stream));
        return DS_OK;
    }
    const void *fn = pick_vec<T>(plan);
    long long nvec = a.m / L;
    long long per_tile = (long long)plan.vpt * plan.block;
    long long ntiles = (nvec + per_tile - 1) / per_tile;
    long long blocks = ntiles < plan.grid_cap ? ntiles : plan.grid_cap;
    if (blocks < 1) blocks = 1;  // the tail (m < L) still needs one block
    SearchArgs<T> args = a;
    void *kargs[] = {&args, &nvec, &ntiles};
    DS_TRY_CUDA(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(plan.block), kargs,
                                 plan.smem ? a.smem_bytes : 0, stream));
    return DS_OK;
}

}  // namespace ds
