// ds_index.cuh -- the single-array handle and the build kernels it shares
// with the batched build.
#pragma once

#include "ds_search.cuh"

namespace ds {
struct HostPipe;
}

struct ds_index {
    ds::HandleHeader hdr;
    int32_t dtype;
    uint32_t flags;
    long long n_knots;
    double H, W, X0, XN;
    unsigned long long R;
    long long updates, passes;
    double build_ms;
    unsigned char *tab;   // [K: (R+1) uint32 (bit 31: cell holds a knot), padded to 16 B][X copy: N+1 values, padded]
    size_t k_bytes, x_bytes;
    uint4 *k16;           // packed K (12 cells per 16 bytes) for the L2-resident float64 path
    size_t k16_bytes;
    void *pairs;          // (R+1) Pair<T> when DS_CACHE_LAYOUT
    size_t pair_bytes;
    size_t table_bytes;
    ds::SearchPlan plan;
    int q;                // 1: Eq. indexdef table; >= 2: Eq. kgeneral with pairs (i, i+q)
    uint32_t smem_bytes;
    int *dev_err;
    ds::DeviceProps props;
    ds::HostPipe *pipe;
};

namespace ds {

// ---------------------------------------------------------------- kernels
// gap: pair distance of the separation property (1 Direct, 2 DirectGap2).
__global__ void k_hr_state_init(HRState *st, int count, int gap);

// Validation and the minimum gap of the rounded differences D_i = m(X_i - X_0)
// (Eq. distinguishable-exact, Eq. minhnumeric); with pair distance 2
// (DirectGap2, Section 4.7) the differences D_i - D_{i-2} (Eq. fcond11).
template <typename T>
__global__ void k_validate(const T *__restrict__ X, long long n_knots, HRState *st)
{
    using A = Arith<T>;
    const T X0 = X[0];
    const int pg = st->gap;
    unsigned long long gmin = NONE64;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_knots; i += stride) {
        const T xi = X[i];
        if (!isfinite(xi)) atomicMin(&st->bad_nonfinite, (unsigned long long)i);
        if (i >= 1) {
            const T xp = X[i - 1];
            if (!(xp < xi)) atomicMin(&st->bad_order, (unsigned long long)i);
        }
        if (i >= pg) {
            const T dp = A::sub(X[i - pg], X0), di = A::sub(xi, X0);
            if (dp == di) atomicMin(&st->bad_indist, (unsigned long long)i);
            const T gap = A::sub(di, dp);
            if (gap > T(0)) {
                const unsigned long long b = (unsigned long long)A::bits(gap);
                gmin = b < gmin ? b : gmin;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, gmin, o);
        gmin = other < gmin ? other : gmin;
    }
    if ((threadIdx.x & 31) == 0 && gmin != NONE64) atomicMin(&st->min_gap_bits, gmin);
}

// ComputeHR start (Section 4.4): H = phi(m(1/min gap)), overflow check
// (Eq. overflowexact), growth term P = phi(H) - H.  One thread.
template <typename T, bool FMA>
__device__ void hr_init_one(const T *X, long long n_knots, HRState *st)
{
    using A = Arith<T>;
    st->first_violation = NONE64;
    st->updates = 0;
    st->passes = 1;
    st->cursor = st->gap;
    st->grew = 0;
    if (st->bad_nonfinite != NONE64 || st->bad_order != NONE64) {
        st->status = DS_E_NOT_INCREASING;
        st->done = 1;
        return;
    }
    if (st->bad_indist != NONE64) {
        st->status = DS_E_INDISTINGUISHABLE;
        st->done = 1;
        return;
    }
    const T X0 = X[0], XN = X[n_knots - 1];
    const T dmin = A::from_bits((typename A::Bits)st->min_gap_bits);
    const T H = next_up(A::rcp(dmin));
    const T W = A::mul(H, X0);
    st->H = (double)H;
    st->W = (double)W;
    if (!(fval<T, FMA>(H, W, X0, XN) < T(4294967296.0))) {
        st->status = DS_E_OVERFLOW;
        st->done = 1;
        return;
    }
    st->P = (double)A::sub(next_up(H), H);
    st->status = DS_OK;
    st->done = 0;
}

template <typename T, bool FMA>
__global__ void k_hr_init(const T *X, long long n_knots, HRState *st)
{
    hr_init_one<T, FMA>(X, n_knots, st);
}

// First pair (i-1, i), i >= cursor, violating Eq. cond2 under the current H.
template <typename T, bool FMA>
__global__ void k_hr_check(const T *__restrict__ X, long long n_knots, HRState *st)
{
    using A = Arith<T>;
    if (st->done) return;
    const T H = (T)st->H, W = (T)st->W, X0 = X[0];
    const long long c = st->cursor;
    const int pg = st->gap;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = c + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_knots; i += stride) {
        const uint32_t fa = A::trunc_u32(fval<T, FMA>(H, W, X0, X[i - pg]));
        const uint32_t fb = A::trunc_u32(fval<T, FMA>(H, W, X0, X[i]));
        if (fa == fb) atomicMin(&st->first_violation, (unsigned long long)i);
    }
}

// Growth step of ComputeHR for the violation found by k_hr_check, or the end
// of a pass.  A pass that grew H is followed by another full pass (a later
// growth can merge an earlier pair); P keeps doubling across passes.
template <typename T, bool FMA>
__device__ void hr_grow_one(const T *X, long long n_knots, HRState *st)
{
    using A = Arith<T>;
    if (st->done) return;
    const unsigned long long v = st->first_violation;
    st->first_violation = NONE64;
    const T X0 = X[0], XN = X[n_knots - 1];
    T H = (T)st->H, W = (T)st->W, P = (T)st->P;
    if (v == NONE64) {
        if (st->grew) {
            if (st->passes >= MAX_HR_PASSES) {
                st->status = DS_E_NO_CONVERGENCE;
                st->done = 1;
                return;
            }
            st->passes += 1;
            st->grew = 0;
            st->cursor = st->gap;
            return;
        }
        st->R = A::trunc_u32(fval<T, FMA>(H, W, X0, XN));
        st->done = 1;
        return;
    }
    const T xa = X[v - st->gap], xb = X[v];
    while (A::trunc_u32(fval<T, FMA>(H, W, X0, xa)) == A::trunc_u32(fval<T, FMA>(H, W, X0, xb))) {
        st->H_inf = (double)H;
        H = A::add(H, P);
        W = A::mul(H, X0);
        if (!(fval<T, FMA>(H, W, X0, XN) < T(4294967296.0))) {
            st->H = (double)H;
            st->status = DS_E_OVERFLOW;
            st->done = 1;
            return;
        }
        P = A::add(P, P);
        st->updates += 1;
        st->grew = 1;
    }
    st->H = (double)H;
    st->W = (double)W;
    st->P = (double)P;
    st->cursor = (long long)v + 1;
}

template <typename T, bool FMA>
__global__ void k_hr_grow(const T *X, long long n_knots, HRState *st)
{
    hr_grow_one<T, FMA>(X, n_knots, st);
}

// One probe of the refinement of H (end of Section 4.4): state for a pair
// scan by k_hr_check with this H (W = m(H X_0), cursor at the pair distance);
// the overflow test of Eq. overflowexact marks the probe done and infeasible.
template <typename T, bool FMA>
__global__ void k_hr_probe(const T *X, long long n_knots, T H, HRState *st)
{
    using A = Arith<T>;
    const T X0 = X[0], XN = X[n_knots - 1];
    const T W = A::mul(H, X0);
    st->H = (double)H;
    st->W = (double)W;
    st->first_violation = NONE64;
    st->cursor = st->gap;
    const bool over = !(fval<T, FMA>(H, W, X0, XN) < T(4294967296.0));
    st->status = over ? DS_E_OVERFLOW : DS_OK;
    st->done = over ? 1 : 0;
    st->R = over ? 0 : A::trunc_u32(fval<T, FMA>(H, W, X0, XN));
}

// F_i = f(X_i) truncated (the cells of the knots).
template <typename T, bool FMA>
__global__ void k_fill_F(const T *__restrict__ X, long long n_knots, T H, T W, uint32_t *__restrict__ F)
{
    using A = Arith<T>;
    const T X0 = X[0];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_knots; i += stride)
        F[i] = A::trunc_u32(fval<T, FMA>(H, W, X0, X[i]));
}

// K_j = min{ i : F_i >= j }, j = 0..R (Eq. indexdef: K_j = i for
// F_{i-1} < j <= F_i, K_j = 0 for j <= F_0), stored with bit 31 set when the
// cell holds knot K_j (F_{K_j} == j).  One warp per 32 consecutive knots
// writes the concatenation of their cell runs with coalesced stores; each lane
// finds the knot of its cell by a 5-step search over the 32 F values held in
// the warp's registers.
template <typename T>
__global__ void k_fill_K(const uint32_t *__restrict__ F, long long n_knots, uint32_t *__restrict__ K,
                         Pair<T> *__restrict__ pairs, const T *__restrict__ X)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long N = n_knots - 1;
    const long long nchunks = (n_knots + 31) / 32;
    for (long long c = warp; c < nchunks; c += nwarps) {
        const long long i = c * 32 + lane;
        const uint32_t Fi = F[i <= N ? i : N];
        const long long prev = c == 0 ? -1 : (long long)F[c * 32 - 1];
        const long long last = (long long)__shfl_sync(0xffffffffu, Fi, 31);
        for (long long base = prev + 1; base <= last; base += 32) {
            const long long j = base + lane;
            int k = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const uint32_t Fc = __shfl_sync(0xffffffffu, Fi, k + s - 1);
                if ((long long)Fc < j) k += s;
            }
            const uint32_t Fk = __shfl_sync(0xffffffffu, Fi, k);
            if (j <= last) {
                const int32_t kk = (int32_t)(c * 32 + k);
                const uint32_t entry = (uint32_t)kk | ((long long)Fk == j ? KNOT_FLAG : 0u);
                K[j] = entry;
                if (pairs) {
                    Pair<T> p;
                    p.k = (int32_t)entry;
                    if constexpr (sizeof(T) == 8) p.pad = 0;
                    p.x = X[kk];
                    pairs[j] = p;
                }
            }
        }
    }
}

// K_j = max{ i : F_i <= j }, j = 0..R (Eq. kgeneral; 0 below F_0), for
// DirectGap2 and Gap-q, with bit 31 set when F_{K_j} >= j and bit 30 when
// F_{K_j - 1} == j.  Warp c owns the cells [F_{32c}, F_{32c+32}) (chunk 0 from
// 0, the last chunk up to R) and finds each cell's knot by a 5-step search
// over its 32 F values.
__global__ void k_fill_K_general(const uint32_t *__restrict__ F, long long n_knots, unsigned long long R,
                                 uint32_t *__restrict__ K);

// Packed copy of a flagged K (Direct, or Eq. kgeneral with q <= 5 when gen):
// block b = {K_{12b}, 12 bytes (K_j - K_{12b}) | flags >> 24}.
__global__ void k_pack_cells(const uint32_t *__restrict__ K, unsigned long long R, uint4 *__restrict__ P, bool gen);

// Clear the knot flags (flag_mask) of every stride-th 32-bit word: turns a copy
// of the flagged table into the plain K of Eq. indexdef (or Eq. kgeneral).
__global__ void k_clear_flags(uint32_t *p, long long count, int stride, uint32_t flag_mask);

// host side, defined in ds_build.cu
// q >= 1: the table of pair distance q (1: Direct); q == 0: the smallest q in
// 1..q_max whose table fits budget_bytes (<= 0: the shared-memory staging limit).
ds_status build_single(const void *X_dev, long long n_knots, ds_dtype dtype, uint32_t flags, int q, int q_max,
                       long long budget_bytes, cudaStream_t s, ds_index **out);
void free_index(ds_index *idx);
ds_status search_index(const ds_index *idx, const void *Z, long long m, int32_t *I, cudaStream_t s);
ds_status info_index(const ds_index *idx, ds_info_t *out);

}  // namespace ds
