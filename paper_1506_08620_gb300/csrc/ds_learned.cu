// ds_learned.cu -- learned-index form: MLP training kernels, error bound,
// bounded-window search with certificate and fall-back, fused interpolation.
#include <cstring>

#include "ds_index.cuh"

struct ds_learned {
    ds::HandleHeader hdr;
    int32_t dtype;
};

namespace ds {
void free_learned(ds_learned *L) { delete L; }
ds_status info_learned(const ds_learned *L, ds_info_t *o)
{
    o->kind = KIND_LEARNED;
    o->dtype = L->dtype;
    return DS_OK;
}
}  // namespace ds

extern "C" {
void ds_learned_cfg_default(ds_learned_cfg *cfg)
{
    memset(cfg, 0, sizeof(*cfg));
    cfg->steps = 2000;
    cfg->batch = 8192;
    cfg->n_queries = 1 << 20;
    cfg->lr = 1e-3f;
    cfg->seed = 1506086200ull;
}
ds_status ds_learned_build(const void *, const int64_t *, int32_t, int64_t, ds_dtype, const ds_learned_cfg *,
                           void *, ds_learned **out)
{
    if (out) *out = nullptr;
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_learned_search(const ds_learned *, const void *, const int64_t *, int64_t, const void *, void *,
                            int32_t *, void *)
{
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_learned_array(const ds_learned *, int32_t, float *, int32_t *, int32_t *, int32_t *)
{
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_mlp_forward(const float *, const float *, int64_t, float *, void *) { return DS_E_UNIMPLEMENTED; }
ds_status ds_mlp_loss_grad(const float *, const float *, const float *, int64_t, float *, float *, void *)
{
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_adam_step(float *, float *, float *, const float *, int32_t, float, void *)
{
    return DS_E_UNIMPLEMENTED;
}
}
