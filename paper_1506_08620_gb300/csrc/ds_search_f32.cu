// Direct-search lookup kernels for float32 knot arrays.
#include "ds_search_impl.cuh"

namespace ds {
template ds_status prepare_search<float>(SearchPlan *, uint32_t, int);
template ds_status launch_search<float>(const SearchArgs<float> &, const SearchPlan &, cudaStream_t);
}  // namespace ds
