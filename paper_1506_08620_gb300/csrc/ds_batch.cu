// ds_batch.cu -- many independent knot arrays (CSR): segmented build and the
// persistent ragged search.
#include <cstring>

#include "ds_index.cuh"

struct ds_batch {
    ds::HandleHeader hdr;
    int32_t dtype;
    uint32_t flags;
};

namespace ds {
void free_batch(ds_batch *b) { delete b; }
ds_status info_batch(const ds_batch *b, ds_info_t *o)
{
    o->kind = KIND_BATCH;
    o->dtype = b->dtype;
    return DS_OK;
}
}  // namespace ds

extern "C" {
ds_status ds_batch_build(const void *, const int64_t *, int32_t, ds_dtype, uint32_t, void *, ds_batch **out)
{
    if (out) *out = nullptr;
    ds::set_error("ds_batch_build: not implemented yet");
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_batch_search(const ds_batch *, const void *, const int64_t *, int32_t *, void *)
{
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_batch_autotune(ds_batch *, const void *, const int64_t *, int32_t *, void *, ds_tune_t *)
{
    return DS_E_UNIMPLEMENTED;
}
ds_status ds_batch_set_tune(ds_batch *, const ds_tune_t *) { return DS_E_UNIMPLEMENTED; }
ds_status ds_batch_get_tune(const ds_batch *, ds_tune_t *) { return DS_E_UNIMPLEMENTED; }
ds_status ds_batch_array(const ds_batch *, int32_t, double *, double *, uint64_t *, int32_t *)
{
    return DS_E_UNIMPLEMENTED;
}
}
