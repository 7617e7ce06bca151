// ds_static.cu -- table build that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a table:
// code running under a host framework that owns every device allocation (a
// fixed memory pool handed out at start-up), real-time loops where an
// allocation's implicit device synchronisation is not allowed, or plug-ins
// whose allocations are forbidden after initialisation.  For them this entry
// point builds H, W, R and the K table of one array into a buffer the caller
// already owns, using as scratch a fixed array that lives in the library's own
// device image instead of a fresh allocation.
//
// The scratch (one ComputeHR state and the cells F_i of up to
// DS_STATIC_MAX_KNOTS knots) is a file-scope __device__ array: every GPU that
// loads libds.so holds it until the process exits.  All calls share it and it
// keeps the previous call's contents, so each call re-initialises what must
// start from a known value; two calls whose GPU work overlaps (two streams,
// two host threads) race on it.
#include <cstring>

#include "ds_index.cuh"

namespace ds {

constexpr long long STATIC_MAX_KNOTS = DS_STATIC_MAX_KNOTS;
constexpr size_t STATIC_HR_BYTES = 256;  // HRState, padded to the 256-byte alignment of F
constexpr size_t STATIC_BYTES = STATIC_HR_BYTES + (size_t)STATIC_MAX_KNOTS * sizeof(uint32_t);
static_assert(sizeof(HRState) <= STATIC_HR_BYTES, "HRState must fit its slot");

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side stand-in, never the device memory itself, so
// the address is looked up with cudaGetSymbolAddress (which allocates
// nothing).  It is looked up on every call rather than cached: a context
// destroyed by cudaDeviceReset and created again may place the array
// elsewhere, and a cached address would then point at memory the library
// does not own.
static void *static_scratch_address(ds_status *rc)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
        set_error("ds_build_table_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        *rc = DS_E_CUDA;
        return nullptr;
    }
    *rc = DS_OK;
    return p;
}

template <typename T, bool FMA>
static ds_status static_build(const T *X, long long n_knots, int32_t *K_out, long long K_capacity, double *H_out,
                              double *W_out, uint64_t *R_out, cudaStream_t s, unsigned char *scratch)
{
    DeviceProps props;
    DS_TRY(device_props(&props));
    HRState *st = reinterpret_cast<HRState *>(scratch);
    uint32_t *F = reinterpret_cast<uint32_t *>(scratch + STATIC_HR_BYTES);
    const int block = 256;
    long long want = (n_knots + block - 1) / block;
    const int grid = (int)(want < props.num_sms * 8 ? (want < 1 ? 1 : want) : props.num_sms * 8);

    // ComputeHR: the state slot is re-initialised on every call
    k_hr_state_init<<<1, 1, 0, s>>>(st, 1, 1);
    k_validate<T><<<grid, block, 0, s>>>(X, n_knots, st);
    k_hr_init<T, FMA><<<1, 1, 0, s>>>(X, n_knots, st);
    HRState hs;
    for (long long round = 0;; ++round) {
        for (int k = 0; k < 3; ++k) {
            k_hr_check<T, FMA><<<grid, block, 0, s>>>(X, n_knots, st);
            k_hr_grow<T, FMA><<<1, 1, 0, s>>>(X, n_knots, st);
        }
        DS_TRY_CUDA(cudaGetLastError());
        DS_TRY_CUDA(cudaMemcpyAsync(&hs, st, sizeof(HRState), cudaMemcpyDeviceToHost, s));
        DS_TRY_CUDA(cudaStreamSynchronize(s));
        if (hs.done) break;
        if (round > 1000000) {
            set_error("ds_build_table_static: ComputeHR did not finish");
            return DS_E_NO_CONVERGENCE;
        }
    }
    *H_out = hs.H;
    *W_out = hs.W;
    *R_out = hs.R;
    if (hs.status != DS_OK) {
        set_error("ds_build_table_static: %s (knot %lld)", hr_message(hs.status), hr_bad_knot(hs));
        return (ds_status)hs.status;
    }
    if ((long long)hs.R + 1 > K_capacity) {
        set_error("ds_build_table_static: K needs %llu entries, the buffer holds %lld", hs.R + 1, K_capacity);
        return DS_E_ARG;
    }
    // cells of the knots into the static scratch, then the caller's table
    k_fill_F<T, FMA><<<grid, block, 0, s>>>(X, n_knots, (T)hs.H, (T)hs.W, F);
    long long wwant = (n_knots + block - 1) / block;
    const int wgrid = (int)(wwant < props.num_sms * 8 ? (wwant < 1 ? 1 : wwant) : props.num_sms * 8);
    k_fill_K<T><<<wgrid, block, 0, s>>>(F, n_knots, reinterpret_cast<uint32_t *>(K_out), nullptr, X);
    // the caller receives the plain K of Eq. indexdef
    k_clear_flags<<<wgrid, block, 0, s>>>(reinterpret_cast<uint32_t *>(K_out), (long long)hs.R + 1, 1, KNOT_FLAG);
    DS_TRY_CUDA(cudaGetLastError());
    DS_TRY_CUDA(cudaStreamSynchronize(s));
    return DS_OK;
}

}  // namespace ds

extern "C" ds_status ds_build_table_static(const void *X_dev, int64_t n_knots, ds_dtype dtype, uint32_t flags,
                                           int32_t *K_out_dev, int64_t K_capacity, double *H_out, double *W_out,
                                           uint64_t *R_out, void *stream)
{
    ds::clear_error();
    if (!X_dev || !K_out_dev || !H_out || !W_out || !R_out || n_knots < 2 || (dtype != DS_F32 && dtype != DS_F64) ||
        (flags & ~(uint32_t)DS_FMA)) {
        ds::set_error("ds_build_table_static: bad argument");
        return DS_E_ARG;
    }
    if (n_knots > ds::STATIC_MAX_KNOTS) {
        ds::set_error("ds_build_table_static: %lld knots exceed the static scratch limit of %lld knots "
                      "(DS_STATIC_MAX_KNOTS); use ds_build", (long long)n_knots, ds::STATIC_MAX_KNOTS);
        return DS_E_ARG;
    }
    ds_status rc;
    unsigned char *scratch = (unsigned char *)ds::static_scratch_address(&rc);
    if (!scratch) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool fma = (flags & DS_FMA) != 0;
    if (dtype == DS_F32)
        return fma ? ds::static_build<float, true>((const float *)X_dev, n_knots, K_out_dev, K_capacity, H_out, W_out,
                                                   R_out, s, scratch)
                   : ds::static_build<float, false>((const float *)X_dev, n_knots, K_out_dev, K_capacity, H_out,
                                                    W_out, R_out, s, scratch);
    return fma ? ds::static_build<double, true>((const double *)X_dev, n_knots, K_out_dev, K_capacity, H_out, W_out,
                                                R_out, s, scratch)
               : ds::static_build<double, false>((const double *)X_dev, n_knots, K_out_dev, K_capacity, H_out, W_out,
                                                 R_out, s, scratch);
}
