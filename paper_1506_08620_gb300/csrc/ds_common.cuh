// ds_common.cuh -- internal definitions shared by the libds translation units.
//
// Floating-point discipline: every step of the map f (Eq. function, Eq. fma)
// is written with explicit round-to-nearest intrinsics (__fmul_rn, __fsub_rn,
// __fmaf_rn, __dmul_rn, ...), which the compiler never contracts or
// reassociates, so the table built on the device and the lookups that read it
// evaluate exactly the same rounded expression (Section 4.4: "all phases of the
// algorithm ... consistently use the function").
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "ds.h"

namespace ds {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();

// ------------------------------------------------------------------ device memory
// Every device allocation of the library goes through these: they keep a
// count of the live allocations and bytes (ds_debug_alloc_stats), and
// ds_debug_fail_alloc can make a chosen allocation fail with
// cudaErrorMemoryAllocation without allocating, so that tests reach every
// error path of a build on the host.
cudaError_t dev_alloc(void **p, size_t bytes);
cudaError_t dev_alloc_async(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p);
void dev_free_async(void *p, cudaStream_t s);
template <typename T> inline cudaError_t dev_alloc(T **p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T> inline cudaError_t dev_alloc_async(T **p, size_t bytes, cudaStream_t s)
{
    return dev_alloc_async(reinterpret_cast<void **>(p), bytes, s);
}

#define DS_TRY_CUDA(call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            ::ds::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                            __LINE__);                                                          \
            return e_ == cudaErrorMemoryAllocation ? DS_E_NOMEM : DS_E_CUDA;                    \
        }                                                                                       \
    } while (0)

#define DS_TRY(expr)                          \
    do {                                      \
        ds_status s_ = (expr);                \
        if (s_ != DS_OK) return s_;           \
    } while (0)

// ------------------------------------------------------------------ handles
enum Kind : int32_t { KIND_INDEX = 1, KIND_BATCH = 2, KIND_LEARNED = 3, KIND_LSEARCH = 4 };
constexpr int32_t HANDLE_MAGIC = 0x0D5E5C;

struct HandleHeader {
    int32_t kind;
    int32_t magic;
};

// Status words written by device code (bounded waits, bounds checks; the
// values of ds.h's DS_DEVERR_*).
enum DeviceErr : int32_t { DEVERR_NONE = 0, DEVERR_TIMEOUT = DS_DEVERR_TIMEOUT, DEVERR_BOUNDS = DS_DEVERR_BOUNDS };

// Range-checking build.  Compiled with -DDS_DEBUG_BOUNDS (the library variant
// libds_bounds.so), every table and knot gather of the search kernels checks
// its index against the extent it reads: an index outside [0, n) is recorded
// in the error word as DEVERR_BOUNDS | site << 8 (the first such index only)
// and replaced by 0, so that the read stays inside its table.  The normal
// build compiles the checks away (in_bounds returns its index).
// The sites are ds.h's DS_BS_*.
enum BoundsSite : int32_t {
    BS_K = DS_BS_K, BS_K16 = DS_BS_K16, BS_X = DS_BS_X, BS_RANK = DS_BS_RANK, BS_FPRINT = DS_BS_FPRINT,
    BS_CMAP = DS_BS_CMAP, BS_CBLOCK = DS_BS_CBLOCK, BS_CESC = DS_BS_CESC, BS_Y = DS_BS_Y, BS_LAYOUT = DS_BS_LAYOUT
};
#ifdef DS_DEBUG_BOUNDS
constexpr bool BOUNDS_CHECKS = true;
#else
constexpr bool BOUNDS_CHECKS = false;
#endif
template <typename I>
__device__ __forceinline__ I in_bounds(I i, long long n, int site, int *err)
{
    if constexpr (BOUNDS_CHECKS) {
        if ((unsigned long long)(long long)i >= (unsigned long long)n) {
            if (err) atomicCAS(err, 0, (int)DEVERR_BOUNDS | (site << 8));
            return I(0);
        }
    }
    return i;
}

// Device-resident state of ComputeHR (one per array).  H, W, P are kept in
// the array's precision; they are stored in double slots, which hold float
// values exactly.
struct HRState {
    double H, W, P;
    double H_inf;                        // the last H found infeasible by the growth loop
    unsigned long long R;
    long long updates, passes, cursor;
    int status, done, grew;
    int gap;                             // pair distance: 1 (Direct) or 2 (DirectGap2)
    unsigned long long first_violation;  // atomicMin target of the pair scan
    unsigned long long bad_nonfinite;    // first knot that is NaN/Inf
    unsigned long long bad_order;        // first i with !(X_{i-1} < X_i)
    unsigned long long bad_indist;       // first i with D_{i-1} == D_i
    unsigned long long min_gap_bits;     // min m(D_i - D_{i-1}) as bits (positive floats order like uints)
};
constexpr unsigned long long NONE64 = ~0ull;
constexpr int MAX_HR_PASSES = 64;

// Message of a ComputeHR failure status, and the knot it names: the first
// non-finite or out-of-order knot, or the first indistinguishable one.
inline const char *hr_message(int status)
{
    switch (status) {
    case DS_E_NOT_INCREASING: return "knots are not strictly increasing finite values";
    case DS_E_INDISTINGUISHABLE:
        return "m(X_i - X_0) == m(X_{i-g} - X_0) (g = 1, or 2 for DirectGap2): direct search infeasible";
    case DS_E_OVERFLOW: return "m(H (X_N - X_0)) >= 2^32: direct search infeasible (Q = 32)";
    case DS_E_NO_CONVERGENCE: return "growth of H did not settle";
    default: return "";
    }
}
inline long long hr_bad_knot(const HRState &hs)
{
    if (hs.status == DS_E_NOT_INCREASING)
        return (long long)(hs.bad_nonfinite != NONE64 ? hs.bad_nonfinite : hs.bad_order);
    return (long long)hs.bad_indist;
}

// ------------------------------------------------------------------ arithmetic
template <typename T> struct Arith;

template <> struct Arith<float> {
    using Bits = uint32_t;
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    // cvt.rzi.u32.f32: toward zero, negatives and NaN -> 0, saturates at 2^32-1
    static __device__ __forceinline__ uint32_t trunc_u32(float v) { return __float2uint_rz(v); }
    static __device__ __forceinline__ Bits bits(float v) { return __float_as_uint(v); }
    static __device__ __forceinline__ float from_bits(Bits b) { return __uint_as_float(b); }
};

template <> struct Arith<double> {
    using Bits = unsigned long long;
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ uint32_t trunc_u32(double v) { return __double2uint_rz(v); }
    static __device__ __forceinline__ Bits bits(double v) { return (Bits)__double_as_longlong(v); }
    static __device__ __forceinline__ double from_bits(Bits b) { return __longlong_as_double((long long)b); }
};

// phi(x) of Section 4.4: the smallest float greater than x, for x >= 0
// (positive finite floats are ordered like their bit patterns; +inf stays).
template <typename T> __device__ __forceinline__ T next_up(T x)
{
    using A = Arith<T>;
    if (!(x < T(INFINITY))) return x;
    return A::from_bits(A::bits(x) + 1);
}

// trunc to 32 bits from the IEEE-754 bit pattern of a double, with the
// semantics of cvt.rzi.u32.f64 (toward zero; negative, zero and NaN -> 0;
// >= 2^32 -> 2^32-1), using integer instructions only.
__device__ __forceinline__ uint32_t trunc_u32_bits(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if ((long long)b < 0 || e < 0) return 0u;
    if (e >= 32) return (b & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull ? 0u : 0xFFFFFFFFu;
    const unsigned long long mant = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    return (uint32_t)(mant >> (52 - e));
}

// Cell j = trunc(v) (as trunc_u32 / cvt.rzi.u32: negatives and NaN -> 0,
// saturated at 2^32 - 1) and fingerprint g = floor(256 (v - trunc(v))), the
// top 8 bits of the fractional part, 0 for negatives and NaN and FP_ABOVE for
// v >= 2^32, computed exactly from the bit pattern of a double.  Within one
// cell g is a non-decreasing function of v, so g(v) < g(w) implies v < w and
// g(v) > g(w) implies v > w: comparing fingerprints decides most comparisons
// of a query with the knot of its cell without reading the knot.
constexpr uint32_t FP_BITS = 8;
constexpr uint32_t FP_ABOVE = 1u << FP_BITS;  // fingerprint of a value past the last cell

__device__ __forceinline__ uint32_t cell_fp_bits(double v, uint32_t *g)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if ((long long)b < 0 || e < -(int)FP_BITS || (b & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) {
        *g = 0u;
        return 0u;
    }
    if (e >= 32) {
        *g = FP_ABOVE;
        return 0xFFFFFFFFu;
    }
    const unsigned long long mant = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    *g = (uint32_t)(mant >> (52 - (int)FP_BITS - e)) & (FP_ABOVE - 1u);
    return e < 0 ? 0u : (uint32_t)(mant >> (52 - e));
}

// Signed integer key ordering doubles like their values (+0 and -0 equal);
// for non-NaN a, b:  a < b  <=>  okey(a) < okey(b).
__device__ __forceinline__ long long okey(double v)
{
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFll);
}

// The map f: plain form trunc(m(H m(z - X0))) (Eq. function) or FMA form
// trunc(m(H z - W)) (Eq. fma).  Returns the value before truncation.
template <typename T, bool FMA>
__device__ __forceinline__ T fval(T H, T W, T X0, T z)
{
    using A = Arith<T>;
    if constexpr (FMA) return A::fma(H, z, -W);
    else return A::mul(H, A::sub(z, X0));
}

template <typename T> struct Pair;
template <> struct __align__(8) Pair<float> { int32_t k; float x; };
template <> struct __align__(16) Pair<double> { int32_t k; int32_t pad; double x; };

// ------------------------------------------------------------------ table loads
// Read-only table gathers marked evict-last in L2 (the query stream is
// evict-first), not allocated in L1 (random cells have no L1 reuse).
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t *ptr, uint64_t pol)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ long long ld_keep(const long long *ptr, uint64_t pol)
{
    long long v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ld_keep(const uint4 *ptr, uint64_t pol)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ longlong2 ld_keep(const longlong2 *ptr, uint64_t pol)
{
    longlong2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b64 {%0, %1}, [%2], %3;"
        : "=l"(v.x), "=l"(v.y)
        : "l"(ptr), "l"(pol));
    return v;
}

// The same mark in L2, with L1 allocation (a block works on one array's table
// at a time, so its cells are reused in L1).
__device__ __forceinline__ uint2 ld_keep_l1(const uint2 *ptr, uint64_t pol)
{
    uint2 v;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t ld_keep_l1(const uint8_t *ptr, uint64_t pol)
{
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

// Read-only gathers that skip L1 allocation but keep the default L2 policy
// (for tables larger than L2, where evict-last would crowd out the stream).
__device__ __forceinline__ uint32_t ld_na(const uint32_t *ptr)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(ptr));
    return v;
}
__device__ __forceinline__ long long ld_na(const long long *ptr)
{
    long long v;
    asm("ld.global.nc.L1::no_allocate.b64 %0, [%1];" : "=l"(v) : "l"(ptr));
    return v;
}

// ------------------------------------------------------------------ async copies
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy completed on an mbarrier (TMA, non-tensor form).
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned address and
// size; no shared memory, registers or barrier involved).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bounded wait: gives up after `limit` polls (each poll may suspend the
// thread for a hardware-defined time), returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr uint32_t MBAR_POLL_LIMIT = 1u << 20;
constexpr uint32_t BULK_CHUNK = 32768;  // bytes per cp.async.bulk

// Stage `bytes` (multiple of 16) from global to shared memory with bulk
// copies issued by one thread; every thread of the block waits.  Returns false
// (and records DEVERR_TIMEOUT in *err) if the copy did not complete in time.
__device__ __forceinline__ bool stage_to_smem(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              int *err)
{
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, bytes);
        for (uint32_t off = 0; off < bytes; off += BULK_CHUNK) {
            const uint32_t n = bytes - off < BULK_CHUNK ? bytes - off : BULK_CHUNK;
            bulk_g2s((char *)dst + off, (const char *)src + off, n, bar);
        }
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(bar, 0, MBAR_POLL_LIMIT);
    if (!ok && err) atomicExch(err, (int)DEVERR_TIMEOUT);
    return __syncthreads_and(ok) != 0;
}

// Repeated staging through one mbarrier initialised once per block (thread 0
// called mbar_init and the block synchronised).  The caller synchronises the
// block before the call so that nobody still reads the previous image;
// `parity` is the phase being completed (it flips after every staging).
__device__ __forceinline__ bool stage_again(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                            uint32_t parity, int *err)
{
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, bytes);
        for (uint32_t off = 0; off < bytes; off += BULK_CHUNK) {
            const uint32_t n = bytes - off < BULK_CHUNK ? bytes - off : BULK_CHUNK;
            bulk_g2s((char *)dst + off, (const char *)src + off, n, bar);
        }
    }
    const bool ok = mbar_wait_bounded(bar, parity, MBAR_POLL_LIMIT);
    if (!ok && err) atomicExch(err, (int)DEVERR_TIMEOUT);
    return __syncthreads_and(ok) != 0;
}

// ------------------------------------------------------------------ host helpers
struct DeviceProps {
    int device = 0;
    int num_sms = 0;
    int max_smem_optin = 0;
    int l2_bytes = 0;
};
ds_status device_props(DeviceProps *p);
// Raise a kernel's dynamic shared-memory limit to the most the device allows
// it (the opt-in limit less its static shared memory).  The attribute belongs
// to the kernel, shared by every handle and captured graph, so it is never
// set to one launch's size: a later, smaller setting would make an earlier
// handle's launch invalid.  Fails if need_bytes exceeds that limit.
ds_status allow_dynamic_smem(const void *fn, int need_bytes);
double now_ms();
size_t table_budget_bytes();
size_t round_up(size_t v, size_t a);

}  // namespace ds
