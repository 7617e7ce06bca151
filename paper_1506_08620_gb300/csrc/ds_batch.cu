// ds_batch.cu -- many independent knot arrays (CSR): segmented build of one
// direct-search table per array and the persistent ragged search, with its
// CUDA-graph launch and autotuner.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ds_engine.cuh"

namespace ds {

// ---------------------------------------------------------------- kernels
// Exclusive prefix sum of v over the block; *total gets the block's sum.
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *total)
{
    __shared__ long long warp_sum[33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) / 32;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const long long w = lane < nw ? warp_sum[lane] : 0;
        long long inc2 = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc2, o);
            if (lane >= o) inc2 += y;
        }
        if (lane < nw) warp_sum[lane] = inc2 - w;
        if (lane == 31) warp_sum[32] = inc2;
    }
    __syncthreads();
    const long long r = warp_sum[wid] + incl - v;
    *total = warp_sum[32];
    __syncthreads();  // warp_sum is reused by the next call
    return r;
}

// Positions are taken in rounds of one per thread (coalesced loads); up to
// PLAN_ROUNDS rounds the per-array loads of all rounds are issued together
// before the first scan.
constexpr int PLAN_ROUNDS = 8;

__global__ void k_plan_chunks(const long long *z_off, long long m_single, int n_arrays, long long chunk,
                              const ArrDesc *desc, const int *order, uint32_t smem_limit, long long *chunk_off,
                              unsigned long long *counter, int split, long long chunk1, uint32_t smem_limit1)
{
    // chunks of the array at claim position p
    auto chunks_at = [&](int p) -> long long {
        const int a = order ? order[p] : p;
        long long q = z_off ? z_off[a + 1] - z_off[a] : m_single;
        q = q < 0 ? 0 : q;
        const bool second = split > 0 && p >= split;
        const long long c = chunk_len(desc[a], second ? chunk1 : chunk, second ? smem_limit1 : smem_limit);
        return (q + c - 1) / c;
    };
    const int B = blockDim.x, rounds = (n_arrays + B - 1) / B;
    long long carry = 0;
    if (rounds <= PLAN_ROUNDS) {
        long long cnt[PLAN_ROUNDS];
#pragma unroll
        for (int k = 0; k < PLAN_ROUNDS; ++k) {
            const int p = k * B + threadIdx.x;
            cnt[k] = k < rounds && p < n_arrays ? chunks_at(p) : 0;
        }
#pragma unroll
        for (int k = 0; k < PLAN_ROUNDS; ++k) {
            if (k < rounds) {
                long long total;
                const long long ex = block_exclusive_scan(cnt[k], &total);
                const int p = k * B + threadIdx.x;
                if (p < n_arrays) chunk_off[p] = carry + ex;
                carry += total;
            }
        }
    } else {
        for (int k = 0; k < rounds; ++k) {
            const int p = k * B + threadIdx.x;
            long long total;
            const long long ex = block_exclusive_scan(p < n_arrays ? chunks_at(p) : 0, &total);
            if (p < n_arrays) chunk_off[p] = carry + ex;
            carry += total;
        }
    }
    __syncthreads();  // every chunk_off[p] written
    if (threadIdx.x == 0) {
        chunk_off[n_arrays > 0 ? n_arrays : 0] = carry;
        counter[0] = 0;
        counter[1] = split > 0 && split < n_arrays ? (unsigned long long)chunk_off[split] : 0ull;
    }
}

__global__ void k_seg_rank_base(const uint32_t *__restrict__ F, const long long *__restrict__ x_off,
                                const long long *__restrict__ kc_off, int n_arrays, const ArrDesc *__restrict__ desc,
                                unsigned char *blob)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = kc_off[n_arrays];
    for (long long c = warp; c < total; c += nwarps) {
        int lo = 0, hi = n_arrays - 1;  // array owning chunk c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (kc_off[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const int arr = lo;
        const ArrDesc d = desc[arr];
        const long long lc = c - kc_off[arr];
        const long long start = x_off[arr];
        const long long N = d.n;
        uint32_t *Wd = reinterpret_cast<uint32_t *>(blob + d.img);  // two words per group
        const long long i = lc * 32 + lane;
        const uint32_t Fi = F[start + (i <= N ? i : N)];
        const long long prev = lc == 0 ? -1 : (long long)F[start + lc * 32 - 1];
        const long long last = (long long)__shfl_sync(0xffffffffu, Fi, 31);
        // groups g with prev < 32 g <= last: K_{32 g} is the first lane with F >= 32 g
        const long long g_first = (prev + 32) >> RANK_SHIFT, g_last = last >> RANK_SHIFT;
        for (long long gb = g_first; gb <= g_last; gb += 32) {
            const long long g = gb + lane;
            const long long j = g << RANK_SHIFT;
            int k = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const uint32_t Fc = __shfl_sync(0xffffffffu, Fi, k + s - 1);
                if ((long long)Fc < j) k += s;
            }
            if (g <= g_last) Wd[2 * g] = (uint32_t)(lc * 32 + k);
        }
    }
}

__global__ void k_seg_rank_bits(const uint32_t *__restrict__ F, const uint8_t *__restrict__ G,
                                const Segment *__restrict__ segs, int n_segs, const long long *__restrict__ x_off,
                                const ArrDesc *__restrict__ desc, unsigned char *blob)
{
    for (int s = blockIdx.x; s < n_segs; s += gridDim.x) {
        const Segment sg = segs[s];
        const ArrDesc d = desc[sg.arr];
        if (d.mode != MODE_DIRECT) continue;
        uint32_t *Wd = reinterpret_cast<uint32_t *>(blob + d.img);
        uint8_t *Gd = blob + d.img + d.g_in_img;
        const long long start = x_off[sg.arr];
        for (long long i = sg.lo + threadIdx.x; i < sg.hi; i += blockDim.x) {
            const uint32_t f = F[i];
            atomicOr(&Wd[2 * (long long)(f >> RANK_SHIFT) + 1], 1u << (f & 31u));
            Gd[i - start] = G[i];
        }
    }
}

// ---------------------------------------------------------------- engine (host)
void engine_free(Engine *e)
{
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->gstream) cudaStreamDestroy(e->gstream);
    if (e->desc_dev) dev_free(e->desc_dev);
    if (e->blob) dev_free(e->blob);
    if (e->chunk_off) dev_free(e->chunk_off);
    if (e->order) dev_free(e->order);
    if (e->counter) dev_free(e->counter);
    if (e->dev_err) dev_free(e->dev_err);
    if (e->ctab) dev_free(e->ctab);
    *e = Engine();
}

static std::vector<Segment> make_segments(const std::vector<long long> &x_off)
{
    std::vector<Segment> segs;
    const int A = (int)x_off.size() - 1;
    for (int a = 0; a < A; ++a)
        for (long long lo = x_off[a]; lo < x_off[a + 1]; lo += SEG_KNOTS) {
            Segment s;
            s.lo = lo;
            s.hi = std::min(lo + SEG_KNOTS, x_off[a + 1]);
            s.arr = a;
            s.pad_ = 0;
            segs.push_back(s);
        }
    return segs;
}

static int top_pow2(long long n)
{
    long long t = 1;
    while (t * 2 <= n) t *= 2;
    return (int)t;
}

int lmap_cells(long long n_knots)
{
    const long long g = top_pow2(std::max<long long>(n_knots / 4, 1));
    return (int)std::min<long long>(LMAP_MAX, std::max<long long>(LMAP_MIN, g));
}

static bool feasible_sparse(const HRState &h, long long nk, double max_cells)
{
    return h.status == DS_OK && max_cells > 0.0 && (double)h.R + 1.0 > max_cells * (double)nk;
}

template <typename T, bool FMA>
static ds_status compute_hr_all(const T *Xcat, const long long *x_off_dev, const Segment *segs_dev, int n_segs,
                                int A, cudaStream_t s, const DeviceProps &props, std::vector<HRState> &hs)
{
    HRState *st = nullptr;
    DS_TRY_CUDA(dev_alloc(&st, sizeof(HRState) * (size_t)A));
    const int sgrid = std::max(1, std::min(n_segs, props.num_sms * 8));
    const int agrid = (A + 127) / 128;
    k_hr_state_init<<<agrid, 128, 0, s>>>(st, A, 1);
    k_seg_validate<T><<<sgrid, 256, 0, s>>>(Xcat, x_off_dev, segs_dev, n_segs, st);
    k_seg_hr_init<T, FMA><<<agrid, 128, 0, s>>>(Xcat, x_off_dev, A, st);
    hs.resize(A);
    ds_status rc = DS_OK;
    for (long long round = 0;; ++round) {
        for (int k = 0; k < 3; ++k) {
            k_seg_hr_check<T, FMA><<<sgrid, 256, 0, s>>>(Xcat, x_off_dev, segs_dev, n_segs, st);
            k_seg_hr_grow<T, FMA><<<agrid, 128, 0, s>>>(Xcat, x_off_dev, A, st);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), st, sizeof(HRState) * (size_t)A, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("batched ComputeHR: %s", cudaGetErrorString(e));
            rc = DS_E_CUDA;
            break;
        }
        bool all = true;
        for (int a = 0; a < A && all; ++a) all = hs[a].done != 0;
        if (all) break;
        if (round > 1000000) {
            set_error("batched ComputeHR did not finish");
            rc = DS_E_NO_CONVERGENCE;
            break;
        }
    }
    dev_free(st);
    return rc;
}

// Validate, run ComputeHR per array, lay out the blob and fill every table.
// `want_direct[a] == false` forces array a into `other_mode` (learned build).
template <typename T, bool FMA>
static ds_status build_engine_typed(Engine *e, const T *Xcat, const T *Ycat, const long long *x_off_dev,
                                    const std::vector<long long> &x_off, uint32_t flags, cudaStream_t s,
                                    const std::vector<char> *force_other, int other_mode, std::vector<HRState> *hs_out,
                                    double max_cells)
{
    const int A = e->n_arrays;
    std::vector<Segment> segs = make_segments(x_off);
    const int n_segs = (int)segs.size();
    Segment *segs_dev = nullptr;
    DS_TRY_CUDA(dev_alloc(&segs_dev, sizeof(Segment) * segs.size()));
    ds_status rc = DS_OK;
    std::vector<HRState> hs;
    uint32_t *F = nullptr;
    uint8_t *G = nullptr;
    long long *kc_dev = nullptr;
    do {
        if (cudaMemcpyAsync(segs_dev, segs.data(), sizeof(Segment) * segs.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            set_error("batched build: segment upload failed");
            rc = DS_E_CUDA;
            break;
        }
        rc = compute_hr_all<T, FMA>(Xcat, x_off_dev, segs_dev, n_segs, A, s, e->props, hs);
        if (rc != DS_OK) break;
        // modes and layout
        e->desc_host.assign(A, ArrDesc());
        size_t off = 0;
        std::vector<long long> kc(A + 1, 0);
        for (int a = 0; a < A; ++a) {
            ArrDesc &d = e->desc_host[a];
            memset(&d, 0, sizeof(d));
            const long long nk = x_off[a + 1] - x_off[a];
            d.n = (int32_t)(nk - 1);
            d.yoff = x_off[a];
            d.xs = Ycat ? 2 : 1;
            d.pbits = top_pow2(d.n);
            e->h_updates += hs[a].updates;
            const bool feasible = hs[a].status == DS_OK;
            const bool sparse = feasible_sparse(hs[a], nk, max_cells);
            const bool forced = (force_other && (*force_other)[a]) || sparse;
            if (!feasible && (flags & DS_STRICT)) {
                set_error("array %d: %s", a, ds_status_str((ds_status)hs[a].status));
                rc = (ds_status)hs[a].status;
                break;
            }
            if (hs[a].status == DS_E_NOT_INCREASING) {
                set_error("array %d: knots are not strictly increasing finite values (knot %lld)", a,
                          (long long)(hs[a].bad_nonfinite != NONE64 ? hs[a].bad_nonfinite : hs[a].bad_order));
                rc = DS_E_NOT_INCREASING;
                break;
            }
            d.img = (long long)off;
            if (feasible && !forced) {
                d.mode = MODE_DIRECT;
                d.R = (uint32_t)hs[a].R;
                d.H = hs[a].H;
                d.W = hs[a].W;
                // the image is the rank words and the knot fingerprints; the
                // knots follow it and stay in global memory
                const size_t kb = rank_bytes((uint32_t)hs[a].R), gb = round_up((size_t)nk, 16);
                d.x_in_img = NO_X_IN_IMG;
                d.g_in_img = (uint32_t)std::min<size_t>(kb, 0xFFFFFFFFu);
                d.xg = (long long)(off + kb + gb);
                const size_t xb = round_up((size_t)nk * d.xs * sizeof(T), 16);
                // with the knot values stored, the fingerprints are not used (the
                // interpolation reads the knot's pair anyway), so only the rank
                // words are staged
                const size_t ib = Ycat ? kb : kb + gb;
                d.img_bytes = ib <= 0xFFFFFFF0u ? (uint32_t)ib : 0u;
                off += kb + gb + xb;
                kc[a + 1] = (nk + 31) / 32;
                e->n_direct += 1;
                e->R_total += (unsigned long long)hs[a].R + 1;
            } else {
                d.mode = forced ? other_mode : (other_mode == MODE_LEARNED ? MODE_LEARNED : MODE_BISECT);
                d.R = 0;
                d.xg = (long long)off;
                d.x_in_img = 0;
                const size_t xb = round_up((size_t)nk * d.xs * sizeof(T), 16);
                d.img_bytes = d.mode == MODE_BISECT && xb <= 0xFFFFFFF0u ? (uint32_t)xb : 0u;
                off += xb;
                if (d.mode == MODE_LEARNED) {  // the image is the cell map; the knots stay in global memory
                    d.img = (long long)off;
                    d.img_bytes = (uint32_t)lmap_cells(nk) * 8u;
                    d.x_in_img = NO_X_IN_IMG;
                    off += d.img_bytes;
                }
                if (d.mode == MODE_BISECT) e->n_fallback += 1;
                else e->n_learned += 1;
            }
            d.form = FMA ? F_FMA : F_PLAIN;
            // X0 and XN are read back below
        }
        if (rc != DS_OK) break;
        // knot fingerprints of the rank tables: used unless turned off
        e->fingerprints = !(flags & DS_NO_FINGERPRINT) && e->n_direct > 0 && !Ycat;
        for (int a = 0; a < A; ++a)
            if (e->desc_host[a].mode == MODE_DIRECT) e->desc_host[a].aux = e->fingerprints ? 1 : 0;
        // the one-conversion cell form: float, every direct array with R < 2^24 - 1
        e->fast_cells = sizeof(T) == 4 && e->n_direct > 0;
        for (int a = 0; a < A; ++a)
            if (e->desc_host[a].mode == MODE_DIRECT && e->desc_host[a].R > FASTF_MAX_R) e->fast_cells = false;
        // direct and learned arrays (and no bisected ones): each group gets its
        // own launch of a kernel kind that holds only its path (fewer registers
        // than one kind holding both), the direct arrays first in the claim order
        if (e->n_direct > 0 && e->n_learned > 0 && e->n_fallback == 0) {
            e->order_host.resize((size_t)A);
            for (int a = 0; a < A; ++a) e->order_host[(size_t)a] = a;
            std::stable_sort(e->order_host.begin(), e->order_host.end(), [&](int p, int q) {
                const bool dp = e->desc_host[(size_t)p].mode == MODE_DIRECT;
                const bool dq = e->desc_host[(size_t)q].mode == MODE_DIRECT;
                if (dp != dq) return dp;
                return x_off[p + 1] - x_off[p] > x_off[q + 1] - x_off[q];
            });
            e->split = e->n_direct;
            cudaMemcpyAsync(e->order, e->order_host.data(), sizeof(int) * (size_t)A, cudaMemcpyHostToDevice, s);
        }
        // knots X_0, X_N per array (for the descriptors)
        {
            std::vector<T> ends(2 * (size_t)A);
            for (int a = 0; a < A; ++a) {
                cudaMemcpyAsync(&ends[2 * a], Xcat + x_off[a], sizeof(T), cudaMemcpyDeviceToHost, s);
                cudaMemcpyAsync(&ends[2 * a + 1], Xcat + x_off[a + 1] - 1, sizeof(T), cudaMemcpyDeviceToHost, s);
            }
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                set_error("batched build: cannot read knots");
                rc = DS_E_CUDA;
                break;
            }
            for (int a = 0; a < A; ++a) {
                ArrDesc &d = e->desc_host[a];
                d.X0 = (double)ends[2 * a];
                d.XN = (double)ends[2 * a + 1];
                if (!FMA && d.X0 == 0.0) d.form = F_PLAIN_X0ZERO;
            }
        }
        for (int a = 0; a < A; ++a) kc[a + 1] += kc[a];
        e->blob_bytes = off;
        e->table_bytes = off;
        const size_t budget = table_budget_bytes();
        if (off > budget) {
            set_error("batched build: tables need %zu bytes, budget is %zu", off, budget);
            rc = DS_E_TABLE_TOO_LARGE;
            break;
        }
        if (dev_alloc(&e->blob, std::max<size_t>(off, 16)) != cudaSuccess ||
            dev_alloc(&e->desc_dev, sizeof(ArrDesc) * (size_t)A) != cudaSuccess ||
            dev_alloc(&F, sizeof(uint32_t) * std::max<long long>(x_off[A], 1)) != cudaSuccess ||
            dev_alloc(&G, std::max<long long>(x_off[A], 1)) != cudaSuccess ||
            dev_alloc(&kc_dev, sizeof(long long) * (size_t)(A + 1)) != cudaSuccess) {
            set_error("batched build: device allocation failed");
            rc = DS_E_NOMEM;
            break;
        }
        cudaMemsetAsync(e->blob, 0, std::max<size_t>(off, 16), s);
        cudaMemcpyAsync(e->desc_dev, e->desc_host.data(), sizeof(ArrDesc) * (size_t)A, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(kc_dev, kc.data(), sizeof(long long) * (size_t)(A + 1), cudaMemcpyHostToDevice, s);
        const int sgrid = std::max(1, std::min(n_segs, e->props.num_sms * 8));
        k_seg_copy_fill_F<T><<<sgrid, 256, 0, s>>>(Xcat, Ycat, x_off_dev, segs_dev, n_segs, e->desc_dev, e->blob, F,
                                                   G);
        const long long kchunks = kc[A];
        if (kchunks > 0) {
            const long long kgrid = std::min<long long>((kchunks * 32 + 255) / 256, (long long)e->props.num_sms * 16);
            k_seg_rank_base<<<(int)kgrid, 256, 0, s>>>(F, x_off_dev, kc_dev, A, e->desc_dev, e->blob);
            k_seg_rank_bits<<<sgrid, 256, 0, s>>>(F, G, segs_dev, n_segs, x_off_dev, e->desc_dev, e->blob);
        }
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            set_error("batched build: table fill failed: %s", cudaGetErrorString(ce));
            rc = DS_E_CUDA;
            break;
        }
    } while (0);
    dev_free(segs_dev);
    if (F) dev_free(F);
    if (G) dev_free(G);
    if (kc_dev) dev_free(kc_dev);
    if (hs_out) *hs_out = hs;
    return rc;
}

ds_status engine_build(Engine *e, const void *Xcat, const void *Ycat, const long long *x_off_dev, int n_arrays,
                       ds_dtype dtype, uint32_t flags, cudaStream_t s, const std::vector<char> *force_other,
                       int other_mode, std::vector<long long> *x_off_host, std::vector<HRState> *hs_out,
                       double max_cells)
{
    e->dtype = dtype;
    e->xy = Ycat != nullptr;
    e->flags = flags;
    e->n_arrays = n_arrays;
    DS_TRY(device_props(&e->props));
    std::vector<long long> x_off(n_arrays + 1);
    DS_TRY_CUDA(cudaMemcpy(x_off.data(), x_off_dev, sizeof(long long) * (size_t)(n_arrays + 1),
                           cudaMemcpyDeviceToHost));
    if (x_off[0] != 0) {
        set_error("x_off[0] must be 0");
        return DS_E_ARG;
    }
    for (int a = 0; a < n_arrays; ++a) {
        if (x_off[a + 1] - x_off[a] < 2) {
            set_error("array %d has %lld knots (at least 2 needed)", a, x_off[a + 1] - x_off[a]);
            return DS_E_ARG;
        }
        if (x_off[a + 1] - x_off[a] > (1ll << 31) - 1) {
            set_error("array %d: at most 2^31-1 knots (int32 results)", a);
            return DS_E_ARG;
        }
    }
    e->n_knots = x_off[n_arrays];
    if (x_off_host) *x_off_host = x_off;
    DS_TRY_CUDA(dev_alloc(&e->chunk_off, sizeof(long long) * (size_t)(n_arrays + 1)));
    {  // claim order: the arrays with the most knots first (longest-processing-time first)
        std::vector<int> order(n_arrays);
        for (int a = 0; a < n_arrays; ++a) order[a] = a;
        std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
            return x_off[p + 1] - x_off[p] > x_off[q + 1] - x_off[q];
        });
        DS_TRY_CUDA(dev_alloc(&e->order, sizeof(int) * (size_t)std::max(n_arrays, 1)));
        DS_TRY_CUDA(cudaMemcpy(e->order, order.data(), sizeof(int) * (size_t)n_arrays, cudaMemcpyHostToDevice));
    }
    DS_TRY_CUDA(dev_alloc(&e->counter, 2 * sizeof(unsigned long long)));
    DS_TRY_CUDA(cudaMemset(e->counter, 0, 2 * sizeof(unsigned long long)));
    DS_TRY_CUDA(dev_alloc(&e->dev_err, sizeof(int)));
    DS_TRY_CUDA(cudaMemset(e->dev_err, 0, sizeof(int)));
    const bool fma = (flags & DS_FMA) != 0;
    if (dtype == DS_F32) {
        const float *X = (const float *)Xcat, *Y = (const float *)Ycat;
        return fma ? build_engine_typed<float, true>(e, X, Y, x_off_dev, x_off, flags, s, force_other, other_mode,
                                                     hs_out, max_cells)
                   : build_engine_typed<float, false>(e, X, Y, x_off_dev, x_off, flags, s, force_other, other_mode,
                                                      hs_out, max_cells);
    }
    const double *X = (const double *)Xcat, *Y = (const double *)Ycat;
    return fma ? build_engine_typed<double, true>(e, X, Y, x_off_dev, x_off, flags, s, force_other, other_mode,
                                                  hs_out, max_cells)
               : build_engine_typed<double, false>(e, X, Y, x_off_dev, x_off, flags, s, force_other, other_mode,
                                                   hs_out, max_cells);
}

// ---------------------------------------------------------------- launch
// Warp-claimed kernels exist for the vector path (the scalar path, for
// misaligned buffers, always claims per block); 1024-thread blocks for the
// direct kinds at one vector per thread, block-claimed.
template <typename T, int VPT, bool INTERP, int KIND>
static const void *pick4(bool vec, bool warps, bool big)
{
    if constexpr (VPT == 1 && direct_kind(KIND) && KIND != KIND_DIRECT_XY)
        if (vec && !warps && big) return (const void *)k_batch_search<T, 1, INTERP, true, KIND, false, 1024>;
    if (vec && warps) return (const void *)k_batch_search<T, VPT, INTERP, true, KIND, true>;
    return vec ? (const void *)k_batch_search<T, VPT, INTERP, true, KIND>
               : (const void *)k_batch_search<T, VPT, INTERP, false, KIND>;
}
template <typename T, int VPT, bool INTERP>
static const void *pick3(bool vec, bool warps, bool big, int kind)
{
    switch (kind) {
    case KIND_DIRECT: return pick4<T, VPT, INTERP, KIND_DIRECT>(vec, warps, big);
    case KIND_DIRECT_FP: return pick4<T, VPT, INTERP, KIND_DIRECT_FP>(vec, warps, big);
    case KIND_DIRECT_FPF:
        if constexpr (sizeof(T) == 4) return pick4<T, VPT, INTERP, KIND_DIRECT_FPF>(vec, warps, big);
        else return pick4<T, VPT, INTERP, KIND_DIRECT_FP>(vec, warps, big);
    case KIND_LEARNED_ONLY: return pick4<T, VPT, INTERP, KIND_LEARNED_ONLY>(vec, warps, big);
    case KIND_DIRECT_XY: return pick4<T, VPT, INTERP, KIND_DIRECT_XY>(vec, warps, big);
    default: return pick4<T, VPT, INTERP, KIND_ALL>(vec, warps, big);
    }
}
template <typename T, int VPT>
static const void *pick2(bool interp, bool vec, bool warps, bool big, int kind)
{
    return interp ? pick3<T, VPT, true>(vec, warps, big, kind) : pick3<T, VPT, false>(vec, warps, big, kind);
}
template <typename T>
static const void *pick1(int vpt, bool interp, bool vec, bool warps, bool big, int kind)
{
    switch (vpt) {
    case 1: return pick2<T, 1>(interp, vec, warps, big, kind);
    case 2: return pick2<T, 2>(interp, vec, warps, big, kind);
    default: return pick2<T, 4>(interp, vec, warps, big, kind);
    }
}
// every array in direct mode, searched on its rank table with the knots alone
// (the direct kinds but KIND_DIRECT_XY read knot t at X[t])
static bool direct_only(const Engine *e) { return e->n_learned == 0 && e->n_fallback == 0 && !e->xy; }
// the direct kind for a handle's direct arrays
static int direct_kind_of(const Engine *e)
{
    return e->xy ? KIND_DIRECT_XY : !e->fingerprints ? KIND_DIRECT : e->fast_cells ? KIND_DIRECT_FPF : KIND_DIRECT_FP;
}
// group: 0 for the launch over every array (or, on a split handle, over its
// direct arrays), 1 for a split handle's learned arrays
static const void *pick_kernel(const Engine *e, int vpt, bool interp, bool vec, bool warps, bool big, int group = 0)
{
    // (without a split, a handle with learned arrays and no bisected ones has
    // no direct arrays either)
    const int kind = e->split > 0 ? (group == 0 ? direct_kind_of(e) : KIND_LEARNED_ONLY)
                     : e->n_fallback > 0 ? KIND_ALL
                     : e->n_learned == 0 ? direct_kind_of(e)
                                         : KIND_LEARNED_ONLY;
    return e->dtype == DS_F32 ? pick1<float>(vpt, interp, vec, warps, big, kind)
                              : pick1<double>(vpt, interp, vec, warps, big, kind);
}

static int clamp_vpt(int v) { return v == 1 || v == 2 ? v : 4; }
// The block size a configuration runs with: 128, 256 or 512, or 1024 where a
// 1024-thread kernel exists (direct arrays only, one vector per thread, block
// claims, aligned buffers); a 1024 request falls back to 512 elsewhere.
static int eff_block(const Engine *e, const ds_tune_t &t, bool vec)
{
    if (t.block == 1024)
        return direct_only(e) && clamp_vpt(t.items) == 1 && vec && t.smem_limit >= 0 ? 1024 : 512;
    return t.block == 128 || t.block == 512 ? t.block : 256;
}

// Resident blocks for a configuration (and the shared-memory opt-in), for
// the launch of one group (pick_kernel).
static ds_status occupancy(const Engine *e, const ds_tune_t &t, bool interp, bool vec, int *grid, int group = 0)
{
    const int block = eff_block(e, t, vec);
    const void *fn = pick_kernel(e, clamp_vpt(t.items), interp, vec, t.smem_limit < 0, block == 1024, group);
    const int smem = std::max(0, t.smem_limit);
    if (smem > 0) DS_TRY(allow_dynamic_smem(fn, smem));
    int occ = 0;
    DS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem));
    if (occ < 1) {
        set_error("batched search: configuration cannot be resident (block %d, smem %d)", t.block, smem);
        return DS_E_ARG;
    }
    if (t.blocks_per_sm > 0) occ = std::min(occ, t.blocks_per_sm);
    *grid = occ * e->props.num_sms;
    return DS_OK;
}

// One search kernel over the claim positions [0, n_pos) whose chunks are
// counted from *counter (the planner has set it).
template <typename T>
static ds_status launch_search(const Engine *e, const void *fn, int grid, int block, uint32_t smem_limit,
                               long long chunk, int n_pos, unsigned long long *counter, const void *Z,
                               const long long *z_off, long long m_single, const void *Y, void *y_out, int32_t *I,
                               cudaStream_t s, bool host_io)
{
    BatchArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.desc = e->desc_dev; a.blob = e->blob; a.z_off = z_off; a.m_single = m_single; a.n_arrays = n_pos;
    a.Z = (const T *)Z; a.I = I; a.Y = (const T *)Y; a.y_out = (T *)y_out;
    a.order = e->order; a.chunk_off = e->chunk_off; a.counter = counter;
    a.chunk = chunk; a.smem_limit = smem_limit; a.checked = (e->flags & DS_CHECKED) != 0;
    a.err = e->dev_err; a.ctab = e->ctab; a.l2pf = host_io ? 0 : 1;
    void *args[] = {&a};
    DS_TRY_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, (size_t)smem_limit, s));
    return DS_OK;
}

ds_status engine_launch_direct(const Engine *e, const ds_tune_t &t, const void *Z, const long long *z_off,
                               long long m_single, const void *Y, void *y_out, int32_t *I, cudaStream_t s,
                               bool host_io, const ds_tune_t *t2)
{
    const bool interp = y_out != nullptr;
    const int L = e->dtype == DS_F32 ? 4 : 2;
    const bool vec = ((uintptr_t)Z % 16 == 0) && ((uintptr_t)I % (L * 4) == 0) &&
                     (!interp || (uintptr_t)y_out % 16 == 0);
    const int n_launch = e->split > 0 ? 2 : 1;
    // each launch's configuration: block, vectors per thread, claims, chunk base, staging limit
    struct Cfg {
        int grid, block, vpt;
        bool warps;
        long long chunk;
        uint32_t smem_limit;
    } c[2];
    for (int g = 0; g < n_launch; ++g) {
        const ds_tune_t &tg = g == 1 && t2 ? *t2 : t;
        DS_TRY(occupancy(e, tg, interp, vec, &c[g].grid, g));
        c[g].block = eff_block(e, tg, vec);
        c[g].vpt = clamp_vpt(tg.items);
        c[g].warps = vec && tg.smem_limit < 0;  // nothing staged, and warps claim their own chunks
        const int tiles = c[g].warps ? CHUNK_TILES_WARP : direct_only(e) ? CHUNK_TILES_DIRECT : CHUNK_TILES;
        c[g].chunk = (long long)(c[g].warps ? 32 : c[g].block) * c[g].vpt * L * tiles;
        c[g].smem_limit = (uint32_t)std::max(0, tg.smem_limit);
    }
    const Cfg &c1 = c[n_launch - 1];
    k_plan_chunks<<<1, 1024, 0, s>>>(z_off, m_single, e->n_arrays, c[0].chunk, e->desc_dev, e->order, c[0].smem_limit,
                                     e->chunk_off, e->counter, e->split, c1.chunk, c1.smem_limit);
    DS_TRY_CUDA(cudaGetLastError());
    for (int g = 0; g < n_launch; ++g) {
        // split handle: the direct arrays' positions [0, split), then the learned ones
        const int n_pos = n_launch == 2 && g == 0 ? e->split : e->n_arrays;
        const void *fn = pick_kernel(e, c[g].vpt, interp, vec, c[g].warps, c[g].block == 1024, g);
        unsigned long long *counter = e->counter + g;
        DS_TRY(e->dtype == DS_F32
                   ? launch_search<float>(e, fn, c[g].grid, c[g].block, c[g].smem_limit, c[g].chunk, n_pos, counter, Z,
                                          z_off, m_single, Y, y_out, I, s, host_io)
                   : launch_search<double>(e, fn, c[g].grid, c[g].block, c[g].smem_limit, c[g].chunk, n_pos, counter,
                                           Z, z_off, m_single, Y, y_out, I, s, host_io));
    }
    return DS_OK;
}

// Launch through a CUDA graph holding (planner, search) for these pointers;
// the graph is re-captured when the pointers or the tuning change.  When the
// caller's stream is itself being captured the kernels are launched directly
// (and become part of the caller's graph).
ds_status engine_launch(Engine *e, const void *Z, const long long *z_off, long long m_single, const void *Y,
                        void *y_out, int32_t *I, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DS_TRY_CUDA(cudaStreamIsCapturing(s, &cs));
    static const bool no_graph = getenv("DS_NO_GRAPH") != nullptr;
    if (cs != cudaStreamCaptureStatusNone || no_graph)
        return engine_launch_direct(e, e->tune, Z, z_off, m_single, Y, y_out, I, s, false, &e->tune2);
    const void *key[6] = {Z, z_off, (const void *)(uintptr_t)m_single, Y, y_out, I};
    const bool same = e->gexec && !memcmp(key, e->gkey, sizeof(key)) && !memcmp(&e->tune, &e->gtune, sizeof(ds_tune_t)) &&
                      !memcmp(&e->tune2, &e->gtune2, sizeof(ds_tune_t));
    if (!same) {
        if (e->gexec) {
            cudaGraphExecDestroy(e->gexec);
            e->gexec = nullptr;
        }
        if (!e->gstream) DS_TRY_CUDA(cudaStreamCreateWithFlags(&e->gstream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        DS_TRY_CUDA(cudaStreamBeginCapture(e->gstream, cudaStreamCaptureModeThreadLocal));
        ds_status rc = engine_launch_direct(e, e->tune, Z, z_off, m_single, Y, y_out, I, e->gstream, false, &e->tune2);
        cudaError_t ce = cudaStreamEndCapture(e->gstream, &g);
        if (rc != DS_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) {
            set_error("graph capture failed: %s", cudaGetErrorString(ce));
            return DS_E_CUDA;
        }
        ce = cudaGraphInstantiate(&e->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            set_error("graph instantiation failed: %s", cudaGetErrorString(ce));
            e->gexec = nullptr;
            return DS_E_CUDA;
        }
        memcpy(e->gkey, key, sizeof(key));
        e->gtune = e->tune;
        e->gtune2 = e->tune2;
    }
    DS_TRY_CUDA(cudaGraphLaunch(e->gexec, s));
    return DS_OK;
}

// A launch configuration given by the caller: values normalised as the
// launch normalises them, and checked for residency.
ds_status engine_set_tune(Engine *e, const ds_tune_t &cfg)
{
    if (cfg.smem_limit < -1 || cfg.smem_limit > e->props.max_smem_optin - 2048) {
        set_error("set_tune: smem_limit %d outside [-1, %d]", cfg.smem_limit, e->props.max_smem_optin - 2048);
        return DS_E_ARG;
    }
    ds_tune_t t = cfg;
    t.block = t.block == 128 || t.block == 512 || t.block == 1024 ? t.block : 256;
    t.items = t.items == 1 || t.items == 2 ? t.items : 4;
    int grid = 0;
    for (int g = 0; g < (e->split > 0 ? 2 : 1); ++g) DS_TRY(occupancy(e, t, false, true, &grid, g));
    e->tune = t;
    e->tune2 = t;
    return DS_OK;
}

// Times every configuration (4 block sizes x 3 vectors per thread x 7
// staging settings) and keeps the fastest.  On a split handle it then tunes
// each launch with the other fixed at the best so far: the direct launch,
// then the learned one.
ds_status engine_autotune(Engine *e, const void *Z, const long long *z_off, long long m_single, const void *Y,
                          void *y_out, int32_t *I, cudaStream_t s, ds_tune_t *best_out)
{
    const int blocks[] = {128, 256, 512, 1024};
    const int items[] = {1, 2, 4};
    const int smems[] = {-1, 0, 24 * 1024, 48 * 1024, 96 * 1024, 136 * 1024, 200 * 1024};
    cudaEvent_t e0, e1;
    DS_TRY_CUDA(cudaEventCreate(&e0));
    DS_TRY_CUDA(cudaEventCreate(&e1));
    const bool interp = y_out != nullptr;
    // the best of three timings of two launches each (a single timing lets
    // clock and power swings pick the configuration); ms < 0 on an error
    auto time_of = [&](const ds_tune_t &t0, const ds_tune_t &t1, ds_status *rc) -> float {
        *rc = engine_launch_direct(e, t0, Z, z_off, m_single, Y, y_out, I, s, false, &t1);
        if (*rc != DS_OK) return -1.f;
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2; ++r) engine_launch_direct(e, t0, Z, z_off, m_single, Y, y_out, I, s, false, &t1);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                *rc = DS_E_CUDA;
                set_error("autotune: %s", cudaGetErrorString(cudaGetLastError()));
                return -1.f;
            }
            float one = 0;
            cudaEventElapsedTime(&one, e0, e1);
            ms = std::min(ms, one / 2);
        }
        return ms;
    };
    // phase 0: one configuration for every launch; 1: the direct launch; 2: the learned one
    ds_tune_t best[2];
    memset(best, 0, sizeof(best));
    float best_ms = 1e30f;
    ds_status rc = DS_OK;
    const int phases = e->split > 0 ? 3 : 1;
    for (int phase = 0; phase < phases && rc == DS_OK; ++phase) {
        for (int b : blocks)
            for (int it : items)
                for (int sm : smems) {
                    if (rc != DS_OK) break;
                    if (sm > e->props.max_smem_optin - 2048) continue;
                    if (b == 1024 && (it != 1 || sm < 0 || !direct_only(e))) continue;  // runs as 512
                    ds_tune_t t;
                    memset(&t, 0, sizeof(t));
                    t.block = b;
                    t.items = it;
                    t.smem_limit = sm;
                    const ds_tune_t t0 = phase == 2 ? best[0] : t, t1 = phase == 1 ? best[1] : t;
                    int grid = 0;
                    if (occupancy(e, t0, interp, true, &grid) != DS_OK) continue;
                    if (e->split > 0 && occupancy(e, t1, interp, true, &grid, 1) != DS_OK) continue;
                    const float ms = time_of(t0, t1, &rc);
                    if (rc == DS_OK && ms < best_ms) {
                        best_ms = ms;
                        best[0] = t0;
                        best[1] = t1;
                    }
                }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DS_OK) return rc;
    best[0].ms = best[1].ms = best_ms;
    e->tune = best[0];
    e->tune2 = best[1];
    if (best_out) *best_out = best[0];
    return DS_OK;
}

ds_tune_t default_tune()
{
    ds_tune_t t;
    memset(&t, 0, sizeof(t));
    t.block = 256;
    t.items = 4;
    t.smem_limit = 48 * 1024;
    t.blocks_per_sm = 0;
    return t;
}

}  // namespace ds

// ---------------------------------------------------------------- handle and API
struct ds_batch {
    ds::HandleHeader hdr;
    ds::Engine eng;
};

namespace ds {
void free_batch(ds_batch *b)
{
    engine_free(&b->eng);
    b->hdr.magic = 0;
    delete b;
}
ds_status info_batch(const ds_batch *b, ds_info_t *o)
{
    const Engine &e = b->eng;
    o->kind = KIND_BATCH;
    o->dtype = e.dtype;
    o->flags = e.flags;
    o->n_arrays = e.n_arrays;
    o->n_knots = e.n_knots;
    o->R = e.R_total;
    o->table_bytes = (int64_t)e.table_bytes;
    o->h_updates = e.h_updates;
    o->build_ms = e.build_ms;
    o->n_direct = e.n_direct;
    o->n_fallback = e.n_fallback;
    o->n_learned = e.n_learned;
    o->search_launches = e.split > 0 ? 3 : 2;
    int err = 0;
    if (e.dev_err && cudaMemcpy(&err, e.dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
        o->device_error = err;
    return DS_OK;
}
}  // namespace ds

static bool batch_ok(const ds_batch *b)
{
    return b && b->hdr.magic == ds::HANDLE_MAGIC && b->hdr.kind == ds::KIND_BATCH;
}

extern "C" {

ds_status ds_batch_build(const void *Xcat_dev, const int64_t *x_off_dev, int32_t n_arrays, ds_dtype dtype,
                         uint32_t flags, void *stream, ds_batch **out)
{
    ds::clear_error();
    if (!out) {
        ds::set_error("ds_batch_build: out is NULL");
        return DS_E_ARG;
    }
    *out = nullptr;
    if (!Xcat_dev || !x_off_dev || n_arrays < 1 || (dtype != DS_F32 && dtype != DS_F64) ||
        (flags & ~(uint32_t)(DS_FMA | DS_CHECKED | DS_STRICT | DS_NO_SMEM | DS_NO_FINGERPRINT))) {
        ds::set_error("ds_batch_build: bad argument");
        return DS_E_ARG;
    }
    const double t0 = ds::now_ms();
    ds_batch *b = new ds_batch;
    b->hdr.kind = ds::KIND_BATCH;
    b->hdr.magic = ds::HANDLE_MAGIC;
    ds_status rc = ds::engine_build(&b->eng, Xcat_dev, nullptr, (const long long *)x_off_dev, n_arrays, dtype, flags,
                                    (cudaStream_t)stream, nullptr, ds::MODE_BISECT, nullptr, nullptr);
    if (rc != DS_OK) {
        ds::free_batch(b);
        return rc;
    }
    b->eng.tune = ds::default_tune();
    if (flags & DS_NO_SMEM) b->eng.tune.smem_limit = 0;
    b->eng.tune2 = b->eng.tune;
    b->eng.build_ms = ds::now_ms() - t0;
    *out = b;
    return DS_OK;
}

ds_status ds_batch_search(const ds_batch *b, const void *Zcat_dev, const int64_t *z_off_dev, int32_t *Icat_dev,
                          void *stream)
{
    if (!batch_ok(b) || !Zcat_dev || !z_off_dev || !Icat_dev) {
        ds::set_error("ds_batch_search: bad argument");
        return DS_E_ARG;
    }
    return ds::engine_launch(const_cast<ds::Engine *>(&b->eng), Zcat_dev, (const long long *)z_off_dev, 0, nullptr,
                             nullptr, Icat_dev, (cudaStream_t)stream);
}

ds_status ds_batch_autotune(ds_batch *b, const void *Zcat_dev, const int64_t *z_off_dev, int32_t *Icat_dev,
                            void *stream, ds_tune_t *best)
{
    if (!batch_ok(b) || !Zcat_dev || !z_off_dev || !Icat_dev) {
        ds::set_error("ds_batch_autotune: bad argument");
        return DS_E_ARG;
    }
    return ds::engine_autotune(&b->eng, Zcat_dev, (const long long *)z_off_dev, 0, nullptr, nullptr, Icat_dev,
                               (cudaStream_t)stream,
                               best);
}

ds_status ds_batch_set_tune(ds_batch *b, const ds_tune_t *cfg)
{
    if (!batch_ok(b) || !cfg) {
        ds::set_error("ds_batch_set_tune: bad argument");
        return DS_E_ARG;
    }
    return ds::engine_set_tune(&b->eng, *cfg);
}
ds_status ds_batch_get_tune(const ds_batch *b, ds_tune_t *cfg)
{
    if (!batch_ok(b) || !cfg) return DS_E_ARG;
    *cfg = b->eng.tune;
    return DS_OK;
}

ds_status ds_batch_array(const ds_batch *b, int32_t a, double *H, double *W, uint64_t *R, int32_t *mode)
{
    if (!batch_ok(b) || a < 0 || a >= b->eng.n_arrays) {
        ds::set_error("ds_batch_array: bad argument");
        return DS_E_ARG;
    }
    const ds::ArrDesc &d = b->eng.desc_host[a];
    if (H) *H = d.H;
    if (W) *W = d.W;
    if (R) *R = d.R;
    if (mode) *mode = d.mode;
    return DS_OK;
}

}  // extern "C"
