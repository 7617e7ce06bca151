// Direct-search lookup kernels for float64 knot arrays.
#include "ds_search_impl.cuh"

namespace ds {
template ds_status prepare_search<double>(SearchPlan *, uint32_t, int);
template ds_status launch_search<double>(const SearchArgs<double> &, const SearchPlan &, cudaStream_t);
}  // namespace ds
