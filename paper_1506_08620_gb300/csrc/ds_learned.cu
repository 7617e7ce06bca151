// ds_learned.cu -- learned-index form (not in the paper): a 1 -> 32 -> 32 -> 1
// ReLU network g predicting i / N = u + g(u) from u = (z - X_0) / (X_N - X_0)
// (the network learns the deviation from the uniform-grid model N u, and its
// output layer starts at zero, so the untrained model is that linear model),
// trained on the GPU by the forward/backward/Adam kernels below.  Its exact
// piecewise-linear form gives the recorded error bound and, sampled at G
// uniform points and made monotone, the learned cell map: cells of equal
// predicted rank instead of equal width in z.  Direct search runs on that map
// (MODE_LEARNED in ds_multi_kernels.cuh) with the table K of Eq. indexdef over
// its cells, so every answer is exact by construction; a cell may hold several
// knots, and the largest cell population is the bounded window recorded at
// build time.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ds_engine.cuh"

namespace ds {

constexpr int HID = 32;
constexpr int NP = HID + HID + HID * HID + HID + HID + 1;  // 1153
constexpr int OW1 = 0, OB1 = 32, OW2 = 64, OB2 = 64 + 1024, OW3 = OB2 + 32, OB3 = OW3 + 32;
constexpr int TB = 128;  // samples (threads) per training block
static_assert(TB == 128, "the tensor-core gradient tiles W2 over four warps");
constexpr size_t TH_BYTES = ((NP * sizeof(float) + 15) / 16) * 16;  // parameters at the head of shared memory
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

// ------------------------------------------------------------------ Philox-4x32-10
// Counter-based generator of Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
// multiplications with the published multipliers and Weyl key increments.
struct P4 {
    uint32_t v[4];
};
__device__ __forceinline__ P4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
        const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    P4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ uint32_t below(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * n) >> 32); }

// ------------------------------------------------------------------ network
__device__ __forceinline__ float relu(float a) { return a > 0.f ? a : 0.f; }

// Shared-memory image of the parameters: theta, then W2 transposed (W2T[m][n]
// = W2[n][m]), so that both the forward layer (column m of W2 times h1_m) and
// the backward product (row m of W2T times da2) read 32 consecutive floats.
constexpr size_t W2T_OFF = TH_BYTES;
constexpr size_t PARAM_SMEM = TH_BYTES + HID * HID * sizeof(float);

__device__ __forceinline__ void load_params(const float *theta, float *sm)
{
    float *w2t = sm + W2T_OFF / sizeof(float);
    for (int p = threadIdx.x; p < NP; p += blockDim.x) sm[p] = theta[p];
    for (int p = threadIdx.x; p < HID * HID; p += blockDim.x) {
        const int n = p / HID, m = p % HID;
        w2t[m * HID + n] = theta[OW2 + p];
    }
}

// Shared-memory tile of one block's samples and the block's gradient sum.
struct GradTile {
    float U[TB], DOUT[TB], LOSS[TB];
    float H1[TB][HID + 1], DA1[TB][HID + 1], DA2[TB][HID + 1], H2[TB][HID + 1];
};

// ------------------------------------------------------------------ tensor cores for the 32x32 layer
// The three products of the 32x32 layer in a training step (forward
// A2 = H1 W2^T, backward DA1 = DA2 W2, gradient dW2 = DA2^T H1 over the
// block's samples) run on the tensor cores as warp-level mma.sync m16n8k8 with
// TF32 operands and FP32 accumulation, each operand split into a TF32 part
// and a TF32 remainder (x = big + small, both exact in FP32) so that
// big*big + big*small + small*big carries FP32 accuracy (the small*small term
// lies below it).  The tiles are 32 samples x 32 units per warp (forward,
// backward) and 16 x 16 units over the block's 128 samples (gradient).
__device__ __forceinline__ uint32_t tf32_of(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &big, uint32_t &small)
{
    big = tf32_of(x);
    small = tf32_of(x - __uint_as_float(big));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// acc[rt][ct] += A B over k in [0, K) for the output tiles (rows 16 rt .. +16,
// columns 8 ct .. +8); A(row, k) and B(k, col) read the operands.  Fragment
// layout of m16n8k8: lane = 4 g + c; A holds (g, c), (g+8, c), (g, c+4),
// (g+8, c+4); B holds (c, g), (c+4, g); the accumulator (g, 2c), (g, 2c+1),
// (g+8, 2c), (g+8, 2c+1).
template <int RT, int CT, typename FA, typename FB>
__device__ __forceinline__ void warp_mma_3xtf32(float (&acc)[RT][CT][4], int K, FA A, FB B)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += 8) {
        uint32_t ab[RT][4], as[RT][4], bb[CT][2], bs[CT][2];
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) {
            split_tf32(A(16 * rt + g, k0 + c), ab[rt][0], as[rt][0]);
            split_tf32(A(16 * rt + g + 8, k0 + c), ab[rt][1], as[rt][1]);
            split_tf32(A(16 * rt + g, k0 + c + 4), ab[rt][2], as[rt][2]);
            split_tf32(A(16 * rt + g + 8, k0 + c + 4), ab[rt][3], as[rt][3]);
        }
#pragma unroll
        for (int ct = 0; ct < CT; ++ct) {
            split_tf32(B(k0 + c, 8 * ct + g), bb[ct][0], bs[ct][0]);
            split_tf32(B(k0 + c + 4, 8 * ct + g), bb[ct][1], bs[ct][1]);
        }
#pragma unroll
        for (int rt = 0; rt < RT; ++rt)
#pragma unroll
            for (int ct = 0; ct < CT; ++ct) {
                mma_tf32(acc[rt][ct], as[rt], bb[ct]);
                mma_tf32(acc[rt][ct], ab[rt], bs[ct]);
                mma_tf32(acc[rt][ct], ab[rt], bb[ct]);
            }
    }
}
// Visit the accumulator's elements: f(row, col, value).
template <int RT, int CT, typename F>
__device__ __forceinline__ void warp_acc_each(const float (&acc)[RT][CT][4], F f)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int rt = 0; rt < RT; ++rt)
#pragma unroll
        for (int ct = 0; ct < CT; ++ct) {
            f(16 * rt + g, 8 * ct + 2 * c, acc[rt][ct][0]);
            f(16 * rt + g, 8 * ct + 2 * c + 1, acc[rt][ct][1]);
            f(16 * rt + g + 8, 8 * ct + 2 * c, acc[rt][ct][2]);
            f(16 * rt + g + 8, 8 * ct + 2 * c + 1, acc[rt][ct][3]);
        }
}

// Forward and backward of the block's samples, one per thread (all threads
// of each warp take part; a thread without a sample passes valid = false and
// contributes nothing), written into the tile; returns the thread's out.
// dscale = 2 / (batch size).
__device__ __forceinline__ float mlp_sample(const float *sm, float u, float y, float dscale, bool valid, GradTile &t)
{
    const float *th = sm;
    const float *w2t = sm + W2T_OFF / sizeof(float);
    const int s = threadIdx.x, w0 = s & ~31;
    // layer 1 (CUDA cores): h1 = relu(W1 u + b1)
#pragma unroll 4
    for (int m = 0; m < HID; ++m) t.H1[s][m] = relu(__fmaf_rn(th[OW1 + m], u, th[OB1 + m]));
    __syncwarp();
    // layer 2 (tensor cores): A2 = H1 W2^T + b2 for the warp's 32 samples, into H2
    {
        float acc[2][4][4];
#pragma unroll
        for (int ct = 0; ct < 4; ++ct) {
            const int col = 8 * ct + 2 * (s & 3);
#pragma unroll
            for (int rt = 0; rt < 2; ++rt) {
                acc[rt][ct][0] = acc[rt][ct][2] = th[OB2 + col];
                acc[rt][ct][1] = acc[rt][ct][3] = th[OB2 + col + 1];
            }
        }
        warp_mma_3xtf32<2, 4>(acc, HID, [&](int r, int k) { return t.H1[w0 + r][k]; },
                              [&](int k, int n) { return w2t[k * HID + n]; });
        warp_acc_each<2, 4>(acc, [&](int r, int n, float v) { t.H2[w0 + r][n] = v; });
    }
    __syncwarp();
    // output, loss and the output gradient (CUDA cores); da2 into DA2
    float out = th[OB3];
#pragma unroll 4
    for (int n = 0; n < HID; ++n) out = __fmaf_rn(th[OW3 + n], relu(t.H2[s][n]), out);
    const float d = valid ? dscale * (out - y) : 0.f;
#pragma unroll 4
    for (int n = 0; n < HID; ++n) {
        const float a2 = t.H2[s][n];
        t.DA2[s][n] = a2 > 0.f ? d * th[OW3 + n] : 0.f;
        t.H2[s][n] = relu(a2);
    }
    __syncwarp();
    // back through layer 2 (tensor cores): DA1 = (DA2 W2) where a1 > 0
    {
        float acc[2][4][4] = {};
        warp_mma_3xtf32<2, 4>(acc, HID, [&](int r, int k) { return t.DA2[w0 + r][k]; },
                              [&](int k, int m) { return th[OW2 + k * HID + m]; });
        warp_acc_each<2, 4>(acc, [&](int r, int m, float v) {
            t.DA1[w0 + r][m] = t.H1[w0 + r][m] > 0.f ? v : 0.f;  // a1 > 0 exactly where h1 > 0
        });
    }
    t.U[s] = u;
    t.DOUT[s] = d;
    const float r = out - y;
    t.LOSS[s] = valid ? r * r : 0.f;
    return out;
}

__device__ __forceinline__ float mlp_forward1(const float *sm, float u)
{
    const float *th = sm;
    const float4 *w2t = reinterpret_cast<const float4 *>(sm + W2T_OFF / sizeof(float));
    float a2[HID];
#pragma unroll
    for (int n = 0; n < HID; ++n) a2[n] = th[OB2 + n];
#pragma unroll 1
    for (int m = 0; m < HID; ++m) {
        const float h = relu(__fmaf_rn(th[OW1 + m], u, th[OB1 + m]));
#pragma unroll
        for (int q = 0; q < HID / 4; ++q) {
            const float4 w = w2t[m * (HID / 4) + q];
            a2[4 * q + 0] = __fmaf_rn(w.x, h, a2[4 * q + 0]);
            a2[4 * q + 1] = __fmaf_rn(w.y, h, a2[4 * q + 1]);
            a2[4 * q + 2] = __fmaf_rn(w.z, h, a2[4 * q + 2]);
            a2[4 * q + 3] = __fmaf_rn(w.w, h, a2[4 * q + 3]);
        }
    }
    float out = th[OB3];
#pragma unroll
    for (int n = 0; n < HID; ++n) out = __fmaf_rn(th[OW3 + n], relu(a2[n]), out);
    return out;
}

// Sum of the per-sample gradients of the tile's `count` samples, in parameter
// order (rows past `count` hold zero gradients).  The 32x32 block of W2 is the
// product DA2^T H1 over the block's samples, on the tensor cores: warp w of
// the four computes rows 16 (w / 2) .. +16 and columns 16 (w % 2) .. +16; the
// other 129 parameters take one thread each.
__device__ __forceinline__ void tile_gradient(const GradTile &t, int count, float *gout)
{
    const int tid = threadIdx.x;
    {
        const int w = tid >> 5, n0 = 16 * (w >> 1), m0 = 16 * (w & 1);
        float acc[1][2][4] = {};
        warp_mma_3xtf32<1, 2>(acc, TB, [&](int r, int s) { return t.DA2[s][n0 + r]; },
                              [&](int s, int m) { return t.H1[s][m0 + m]; });
        warp_acc_each<1, 2>(acc, [&](int r, int m, float v) { gout[OW2 + (n0 + r) * HID + m0 + m] = v; });
    }
    // W1, b1, b2, W3, b3: 129 sums over the samples
    for (int q = tid; q < 4 * HID + 1; q += blockDim.x) {
        float acc = 0.f;
        int p;
        if (q < HID) {  // W1[m] = sum DA1[s][m] u_s
            for (int s = 0; s < count; ++s) acc = __fmaf_rn(t.DA1[s][q], t.U[s], acc);
            p = OW1 + q;
        } else if (q < 2 * HID) {  // b1
            for (int s = 0; s < count; ++s) acc += t.DA1[s][q - HID];
            p = OB1 + q - HID;
        } else if (q < 3 * HID) {  // b2
            for (int s = 0; s < count; ++s) acc += t.DA2[s][q - 2 * HID];
            p = OB2 + q - 2 * HID;
        } else if (q < 4 * HID) {  // W3[n] = sum DOUT[s] H2[s][n]
            for (int s = 0; s < count; ++s) acc = __fmaf_rn(t.DOUT[s], t.H2[s][q - 3 * HID], acc);
            p = OW3 + q - 3 * HID;
        } else {  // b3
            for (int s = 0; s < count; ++s) acc += t.DOUT[s];
            p = OB3;
        }
        gout[p] = acc;
    }
}

__device__ __forceinline__ float tile_loss(const GradTile &t, int count)
{
    float l = 0.f;
    for (int s = 0; s < count; ++s) l += t.LOSS[s];
    return l;
}

// Gradient of the mean squared error over explicit samples: block b writes
// the sum over its samples into partial[b][*] and partial_loss[b].
__global__ void __launch_bounds__(TB) k_grad_explicit(const float *theta, const float *u, const float *y, long long n,
                                                      float *partial, float *partial_loss)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float *sm = reinterpret_cast<float *>(sm_raw);
    GradTile &t = *reinterpret_cast<GradTile *>(sm_raw + PARAM_SMEM);
    load_params(theta, sm);
    __syncthreads();
    const long long i = (long long)blockIdx.x * TB + threadIdx.x;
    const int count = (int)min((long long)TB, n - (long long)blockIdx.x * TB);
    const bool valid = i < n;  // every thread takes part in the warps' tensor-core products
    mlp_sample(sm, valid ? u[i] : 0.f, valid ? y[i] : 0.f, 2.0f / (float)n, valid, t);
    __syncthreads();
    tile_gradient(t, count, partial + (size_t)blockIdx.x * NP);
    if (threadIdx.x == 0) partial_loss[blockIdx.x] = tile_loss(t, count);
}

__global__ void k_reduce_grad(const float *partial, const float *partial_loss, int nblocks, long long n, float *grad,
                              float *loss)
{
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < nblocks; ++b) acc += partial[(size_t)b * NP + p];
        grad[p] = acc;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += partial_loss[b];
        *loss = l / (float)n;
    }
}

__device__ __forceinline__ void adam_update(float *theta, float *m, float *v, int p, float g, int t, float lr)
{
    const float mm = ADAM_B1 * m[p] + (1.f - ADAM_B1) * g;
    const float vv = ADAM_B2 * v[p] + (1.f - ADAM_B2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mhat = mm / (1.f - powf(ADAM_B1, (float)t));
    const float vhat = vv / (1.f - powf(ADAM_B2, (float)t));
    theta[p] -= lr * mhat / (sqrtf(vhat) + ADAM_EPS);
}

__global__ void k_adam_explicit(float *theta, float *m, float *v, const float *grad, int t, float lr)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x)
        adam_update(theta, m, v, p, grad[p], t, lr);
}

__global__ void k_forward(const float *theta, const float *u, long long n, float *out)
{
    __shared__ __align__(16) float sm[PARAM_SMEM / sizeof(float)];
    load_params(theta, sm);
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = mlp_forward1(sm, u[i]);
}

// ------------------------------------------------------------------ training on an array
struct TrainArgs {
    const ArrDesc *desc;
    const unsigned char *blob;
    const int *model_arr;      // model -> array
    const float2 *pool;        // (u, i/N) of exact-answer query samples
    const long long *pool_off; // n_models+1
    float *theta;              // n_models x NP
    float *m, *v;              // Adam moments
    float *partial;            // n_models x gb x NP
    float *partial_loss;       // n_models x gb
    float *loss;               // n_models
    int *step;                 // n_models (1-based step of the next update = step + 1)
    int gb;                    // blocks per model (batch = gb * TB)
    int steps;                 // schedule length
    float lr;
    uint32_t seed_lo, seed_hi;
};

template <typename T>
__global__ void __launch_bounds__(TB) k_train_grad(TrainArgs a)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float *sm = reinterpret_cast<float *>(sm_raw);
    GradTile &t = *reinterpret_cast<GradTile *>(sm_raw + PARAM_SMEM);
    const int model = blockIdx.y;
    load_params(a.theta + (size_t)model * NP, sm);
    const ArrDesc d = a.desc[a.model_arr[model]];
    const T *X = reinterpret_cast<const T *>(a.blob + d.xg);
    const int step = a.step[model];
    __syncthreads();
    const P4 r = philox((uint32_t)step, (uint32_t)model, blockIdx.x, threadIdx.x, a.seed_lo, a.seed_hi);
    const long long p0 = a.pool_off[model], np = a.pool_off[model + 1] - p0;
    float u, y;
    if ((r.v[0] & 1u) && np > 0) {
        const float2 s = a.pool[p0 + below(r.v[1], (uint32_t)np)];
        u = s.x;
        y = s.y;
    } else {
        const int32_t i = (int32_t)below(r.v[1], (uint32_t)d.n + 1u);
        u = pred_u<T>(X[(size_t)i * d.xs], d);
        y = (float)i / (float)d.n;
    }
    const float res = y - u;  // the network's target: deviation from the linear model
    mlp_sample(sm, u, res, 2.0f / (float)(a.gb * TB), true, t);
    __syncthreads();
    tile_gradient(t, TB, a.partial + ((size_t)model * a.gb + blockIdx.x) * NP);
    if (threadIdx.x == 0) a.partial_loss[(size_t)model * a.gb + blockIdx.x] = tile_loss(t, TB);
}

// Adam on each model with a cosine-decayed step size; advances the model's
// step counter (so a captured graph can be replayed).
__global__ void k_train_adam(TrainArgs a)
{
    const int model = blockIdx.x;
    const int t = a.step[model] + 1;
    const float frac = fminf((float)t / (float)a.steps, 1.f);
    const float lr = a.lr * (0.05f + 0.95f * 0.5f * (1.f + cospif(frac)));
    float *theta = a.theta + (size_t)model * NP;
    float *m = a.m + (size_t)model * NP;
    float *v = a.v + (size_t)model * NP;
    const float *part = a.partial + (size_t)model * a.gb * NP;
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        float g = 0.f;
        for (int b = 0; b < a.gb; ++b) g += part[(size_t)b * NP + p];
        adam_update(theta, m, v, p, g, t, lr);
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int b = 0; b < a.gb; ++b) l += a.partial_loss[(size_t)model * a.gb + b];
        a.loss[model] = l / (float)(a.gb * TB);
    }
    __syncthreads();
    if (threadIdx.x == 0) a.step[model] = t;
}

// Initial network: hinge units W1 = +-1 with their kinks spread over [0, 1],
// He-normal W2 (Box-Muller on Philox uniforms), output layer zero (the
// starting model is the linear one).
__global__ void k_init_params(float *theta, int n_models, uint32_t seed_lo, uint32_t seed_hi)
{
    const int model = blockIdx.x;
    float *th = theta + (size_t)model * NP;
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        const P4 r = philox(0xA5A5A5A5u, (uint32_t)model, (uint32_t)p, 0x5EEDu, seed_lo, seed_hi);
        const float g = sqrtf(-2.f * logf(fmaxf(u01(r.v[0]), 1e-7f))) * cospif(2.f * u01(r.v[1]));
        float val = 0.f;
        if (p < OB1) val = (r.v[2] & 1u) ? 1.f : -1.f;          // W1: +-1
        else if (p >= OW2 && p < OB2) val = g * sqrtf(2.f / HID);  // W2: He normal
        th[p] = val;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < HID; m += blockDim.x) {
        const P4 r = philox(0x0C0FFEEu, (uint32_t)model, (uint32_t)m, 7u, seed_lo, seed_hi);
        const float kink = u01(r.v[0]);
        th[OB1 + m] = -th[OW1 + m] * kink;  // unit m bends at u = kink
    }
}

// Exact-answer query samples: z uniform over [X_0, X_N), answered by the
// fixed-depth bisection over all knots, stored as (u(z), i / N).
template <typename T>
__global__ void k_pool_queries(const ArrDesc *desc, const unsigned char *blob, const int *model_arr,
                               const long long *pool_off, float2 *pool, int n_models, uint32_t seed_lo,
                               uint32_t seed_hi)
{
    const int model = blockIdx.y;
    const ArrDesc d = desc[model_arr[model]];
    const T *X = reinterpret_cast<const T *>(blob + d.xg);
    const long long p0 = pool_off[model], np = pool_off[model + 1] - p0;
    const T X0 = (T)d.X0, XN = (T)d.XN;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (long long)gridDim.x * blockDim.x) {
        const P4 r = philox((uint32_t)k, (uint32_t)(k >> 32), (uint32_t)model, 0xB0B0u, seed_lo, seed_hi);
        const double f = ((double)r.v[0] * 4294967296.0 + (double)r.v[1]) * (1.0 / 18446744073709551616.0);
        T z = (T)((double)X0 + f * ((double)XN - (double)X0));
        if (!(z < XN)) z = X[(size_t)(d.n - 1) * d.xs];
        if (z < X0) z = X0;
        const int32_t i = bisect<T>(X, d.xs, 0, d.n, d.pbits, z, (long long)d.n + 1, nullptr);
        pool[p0 + k] = make_float2(pred_u<T>(z, d), (float)i / (float)d.n);
    }
}

// Piecewise-linear served form of the network: segment k covers
// [seg_x[k], seg_x[k+1]) (seg_x[0] = -inf), value seg_a[k] * u + seg_b[k].
__device__ __forceinline__ float pred_eval(float u, const float *sx, const float *sa, const float *sb, int n,
                                           int top)
{
    int k = 0;
    for (int s = top; s > 0; s >>= 1) {
        const int r = k + s;
        if (r < n && sx[r] <= u) k = r;
    }
    return __fmaf_rn(sa[k], u, sb[k]);
}

__device__ __forceinline__ int32_t floor_clamped(float p, int32_t n)
{
    // floor, with NaN and out-of-range predictions pinned inside [-2^30, 2^30]
    if (!(p > -1073741824.0f)) p = -1073741824.0f;
    if (p > 1073741824.0f) p = 1073741824.0f;
    return __float2int_rd(p);
}

// Error bound of the served predictor: at every knot i (answer i) and at the
// largest value of every interval, nextafter(X_{i+1}, -inf) (answer i).
template <typename T> __device__ __forceinline__ T next_down(T x)
{
    using A = Arith<T>;
    if constexpr (sizeof(T) == 8) {
        const long long k = okey((double)x) - 1;
        const long long b = k >= 0 ? k : ((-k) | (long long)0x8000000000000000ull);
        return __longlong_as_double(b);
    } else {
        const int ib = __float_as_int(x);
        const int k = (ib >= 0 ? ib : -(ib & 0x7FFFFFFF)) - 1;
        const int b = k >= 0 ? k : ((-k) | (int)0x80000000u);
        return __int_as_float(b);
    }
}

template <typename T>
__global__ void k_error_bound(const ArrDesc *desc, const unsigned char *blob, const int *model_arr,
                              const float *seg_x, const float *seg_a, const float *seg_b, int *e_lo, int *e_hi)
{
    const int model = blockIdx.y;
    const ArrDesc d = desc[model_arr[model]];
    const T *X = reinterpret_cast<const T *>(blob + d.xg);
    const float *sx = seg_x + d.seg_off, *sa = seg_a + d.seg_off, *sb = seg_b + d.seg_off;
    int top = 1;
    while (top * 2 <= d.seg_n) top *= 2;
    int lo = 0, hi = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= d.n; i += (long long)gridDim.x * blockDim.x) {
        const int32_t pf = floor_clamped(pred_eval(pred_u<T>(X[(size_t)i * d.xs], d), sx, sa, sb, d.seg_n, top), d.n);
        lo = max(lo, (int)min((long long)pf - i, (long long)1 << 30));
        hi = max(hi, (int)min(i - (long long)pf, (long long)1 << 30));
        if (i < d.n) {
            const T z = next_down<T>(X[(size_t)(i + 1) * d.xs]);
            const int32_t pz = floor_clamped(pred_eval(pred_u<T>(z, d), sx, sa, sb, d.seg_n, top), d.n);
            lo = max(lo, (int)min((long long)pz - i, (long long)1 << 30));
            hi = max(hi, (int)min(i - (long long)pz, (long long)1 << 30));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = max(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(e_lo + model, lo);
        atomicMax(e_hi + model, hi);
    }
}

// ------------------------------------------------------------------ learned cell tables
// F_i = f(X_i) on the learned cell map, exactly as a query computes it, for
// the knots of every model's array (model k's knots start at F + kbase[k]).
template <typename T>
__global__ void k_learned_F(const ArrDesc *desc, const unsigned char *blob, const int *model_arr,
                            const long long *kbase, uint32_t *F)
{
    const int model = blockIdx.y;
    const ArrDesc d = desc[model_arr[model]];
    const T *X = reinterpret_cast<const T *>(blob + d.xg);
    const uint2 *M = reinterpret_cast<const uint2 *>(blob + d.img);
    const uint32_t G = d.img_bytes >> 3;
    uint32_t *Fm = F + kbase[model];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= d.n;
         i += (long long)gridDim.x * blockDim.x)
        Fm[i] = learned_cell<T>(X[(size_t)i * d.xs], d, M, G, nullptr);
}

// #{i in [lo, n1) : F_i < v} + lo for non-decreasing F, given F_i < v below lo.
__device__ __forceinline__ uint32_t count_below(const uint32_t *F, uint32_t lo, uint32_t n1, uint32_t v)
{
    uint32_t hi = n1;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (F[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct LStats {
    unsigned int max_pop;           // largest K_{j+1} - K_j
    unsigned int escaped;           // blocks of 8 cells holding more than LBLK_MAXSPAN knots
    unsigned long long nonempty;    // cells holding a knot
    unsigned long long sum_pop2;    // sum over cells of (K_{j+1} - K_j)^2
};

// Blocks of 8 cells of every model's cell table: K_j = #{i : F_i < j} (Eq.
// indexdef; cells at or past C count every knot).  fill = 0: statistics per
// model; fill = 1: write the table (K_{8b} and the differences K_{8b+r} -
// K_{8b}, r = 1..8, 12 bits each; an escaped block takes the next slot of its
// model's overflow area, counted in st[model].escaped, which starts at 0).
__global__ void k_learned_cells(const ArrDesc *desc, const int *model_arr, const long long *kbase, const uint32_t *F,
                                LStats *st, unsigned char *ctab, int fill)
{
    const int model = blockIdx.y;
    const ArrDesc d = desc[model_arr[model]];
    const uint32_t *Fm = F + kbase[model];
    const uint32_t n1 = (uint32_t)d.n + 1u;
    const unsigned long long C = (unsigned long long)d.R + 1ull;
    const unsigned long long nb = lblk_count(d.R);
    unsigned int max_pop = 0, esc = 0;
    unsigned long long ne = 0, p2 = 0;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t K[9];
        uint32_t lo = 0;
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const unsigned long long j = (b << LBLK_SHIFT) + r;
            K[r] = j >= C ? n1 : count_below(Fm, lo, n1, (uint32_t)j);
            lo = K[r];
        }
        const bool escaped = K[8] - K[0] > LBLK_MAXSPAN;
        if (!fill) {
            esc += escaped;
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if ((b << LBLK_SHIFT) + r < C) {
                    const unsigned int pop = K[r + 1] - K[r];
                    max_pop = max(max_pop, pop);
                    ne += pop > 0;
                    p2 += (unsigned long long)pop * pop;
                }
            continue;
        }
        uint4 *blk = reinterpret_cast<uint4 *>(ctab + d.ct);
        if (escaped) {
            const unsigned int slot = atomicAdd(&st[model].escaped, 1u);
            uint32_t *O = reinterpret_cast<uint32_t *>(ctab + d.ct + nb * 16ull) + (size_t)slot * 9u;
#pragma unroll
            for (int r = 0; r < 9; ++r) O[r] = K[r];
            blk[b] = make_uint4(LBLK_ESC, slot, 0u, 0u);
        } else {
            uint32_t w[3] = {0u, 0u, 0u};
#pragma unroll
            for (int r = 1; r <= 8; ++r) {
                const uint32_t v = K[r] - K[0], o = 12u * (r - 1);
                w[o >> 5] |= v << (o & 31u);
                if ((o & 31u) > 20u) w[(o >> 5) + 1] |= v >> (32u - (o & 31u));
            }
            blk[b] = make_uint4(K[0], w[0], w[1], w[2]);
        }
    }
    if (fill) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        max_pop = max(max_pop, __shfl_xor_sync(0xffffffffu, max_pop, o));
        esc += __shfl_xor_sync(0xffffffffu, esc, o);
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st[model].max_pop, max_pop);
        atomicAdd(&st[model].escaped, esc);
        atomicAdd(&st[model].nonempty, ne);
        atomicAdd(&st[model].sum_pop2, p2);
    }
}

// K_0 .. K_C of one learned array's cell table, decoded (for inspection).
__global__ void k_export_cells(const unsigned char *ct, uint32_t R, long long n_esc, uint32_t *K)
{
    const unsigned long long n = (unsigned long long)R + 2ull;
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t t0, t1;
        learned_bounds(ct, R, (uint32_t)(j <= R ? j : R), &t0, &t1, n_esc, nullptr);
        K[j] = j <= R ? t0 : t1;
    }
}

// ------------------------------------------------------------------ piecewise-linear form
// The network restricted to a scalar input is piecewise linear: its kinks are
// the zeros of the first layer's units and, between those, the zeros of the
// second layer's (affine) pre-activations.  Computed in double from the
// float32 parameters; the served form is whatever these rounded tables give,
// and the error bound is measured on it.
struct Segments {
    std::vector<float> x, a, b;
};

static void pwl_of(const float *thf, double scale, Segments &out)
{
    double W1[HID], b1[HID], W2[HID][HID], b2[HID], w3[HID], b3;
    for (int m = 0; m < HID; ++m) {
        W1[m] = thf[OW1 + m];
        b1[m] = thf[OB1 + m];
        b2[m] = thf[OB2 + m];
        w3[m] = thf[OW3 + m];
        for (int k = 0; k < HID; ++k) W2[m][k] = thf[OW2 + m * HID + k];
    }
    b3 = thf[OB3];
    std::vector<double> bp;
    for (int m = 0; m < HID; ++m)
        if (W1[m] != 0.0) {
            const double t = -b1[m] / W1[m];
            if (std::isfinite(t) && t > -4.0 && t < 5.0) bp.push_back(t);
        }
    std::sort(bp.begin(), bp.end());
    bp.erase(std::unique(bp.begin(), bp.end()), bp.end());
    std::vector<double> edges;
    edges.push_back(-INFINITY);
    for (double t : bp) edges.push_back(t);
    edges.push_back(INFINITY);
    std::vector<double> sx, sa, sb;
    for (size_t k = 0; k + 1 < edges.size(); ++k) {
        const double lo = edges[k], hi = edges[k + 1];
        const double mid = std::isinf(lo) ? (std::isinf(hi) ? 0.5 : hi - 1.0) : (std::isinf(hi) ? lo + 1.0 : 0.5 * (lo + hi));
        double al[HID], be[HID];
        for (int m = 0; m < HID; ++m) {
            const bool on = W1[m] * mid + b1[m] > 0.0;
            al[m] = on ? W1[m] : 0.0;
            be[m] = on ? b1[m] : 0.0;
        }
        double s[HID], c[HID];
        for (int n = 0; n < HID; ++n) {
            double ss = 0, cc = b2[n];
            for (int m = 0; m < HID; ++m) {
                ss += W2[n][m] * al[m];
                cc += W2[n][m] * be[m];
            }
            s[n] = ss;
            c[n] = cc;
        }
        std::vector<double> sub;
        sub.push_back(lo);
        for (int n = 0; n < HID; ++n)
            if (s[n] != 0.0) {
                const double t = -c[n] / s[n];
                if (t > lo && t < hi && t > -4.0 && t < 5.0) sub.push_back(t);
            }
        std::sort(sub.begin() + 1, sub.end());
        sub.push_back(hi);
        for (size_t q = 0; q + 1 < sub.size(); ++q) {
            const double l2 = sub[q], h2 = sub[q + 1];
            if (!(h2 > l2)) continue;
            const double m2 = std::isinf(l2) ? (std::isinf(h2) ? 0.5 : h2 - 1.0) : (std::isinf(h2) ? l2 + 1.0 : 0.5 * (l2 + h2));
            double slope = 0, icpt = b3;
            for (int n = 0; n < HID; ++n)
                if (s[n] * m2 + c[n] > 0.0) {
                    slope += w3[n] * s[n];
                    icpt += w3[n] * c[n];
                }
            sx.push_back(l2);
            sa.push_back((slope + 1.0) * scale);  // prediction N (u + g(u))
            sb.push_back(icpt * scale);
        }
    }
    out.x.clear();
    out.a.clear();
    out.b.clear();
    for (size_t k = 0; k < sx.size(); ++k) {
        const float fx = k == 0 ? -INFINITY : (float)sx[k];
        if (k > 0 && !(fx > out.x.back())) {  // kinks closer than a float apart: keep the later piece
            out.a.back() = (float)sa[k];
            out.b.back() = (float)sb[k];
            continue;
        }
        out.x.push_back(fx);
        out.a.push_back((float)sa[k]);
        out.b.push_back((float)sb[k]);
    }
}

// The learned cell map of one array: the served prediction p sampled at
// u = g / G, g = 0..G, made non-decreasing by rearrangement (the sampled
// values sorted: Chernozhukov, Fernandez-Val and Galichon, "Improving point
// and interval estimators of monotone functions by rearrangement",
// Biometrika 2009; for a prediction that dips it keeps the rise spread over
// the dip, where a running maximum would pile its knots into one cell), then
// J_g = floor(p C / (N + 1)) clamped into [0, C - 1], with J_0 = 0 and
// J_G = C - 1 (so the map covers every cell); entry g holds {J_g, J_{g+1}}.
// Any non-decreasing J gives exact answers (the search kernel's f is
// monotone); a good p gives cells of equal population.
static void cell_map(const Segments &sg, long long n_knots, unsigned long long C, int G, std::vector<uint2> &out)
{
    std::vector<double> p(G + 1);
    size_t k = 0;
    for (int g = 0; g <= G; ++g) {
        const double u = (double)g / (double)G;
        while (k + 1 < sg.x.size() && (double)sg.x[k + 1] <= u) ++k;
        p[g] = (double)sg.a[k] * u + (double)sg.b[k];
        if (!(p[g] == p[g])) p[g] = 0.0;  // NaN: never from finite parameters; kept in range regardless
    }
    std::sort(p.begin(), p.end());
    std::vector<unsigned long long> J(G + 1);
    for (int g = 0; g <= G; ++g) {
        double c = std::floor(p[g] * (double)C / (double)n_knots);
        if (!(c >= 0.0)) c = 0.0;
        if (c > (double)(C - 1)) c = (double)(C - 1);
        J[g] = (unsigned long long)c;
    }
    J[0] = 0;
    J[G] = C - 1;
    for (int g = 1; g <= G; ++g) J[g] = std::max(J[g], J[g - 1]);
    out.resize(G);
    for (int g = 0; g < G; ++g) out[g] = make_uint2((uint32_t)J[g], (uint32_t)J[g + 1]);
}

}  // namespace ds

// ------------------------------------------------------------------ handle
struct ds_learned {
    ds::HandleHeader hdr;
    ds::Engine eng;
    std::vector<int> model_arr;        // model -> array
    std::vector<int> arr_model;        // array -> model or -1
    std::vector<float> theta_host;     // n_models x NP
    int steps = 0;
    double train_ms = 0, final_loss = 0;
    long long max_window = 0;
    // per model: cells C, largest cell population, cells holding a knot, uint32 table
    std::vector<int> e_lo, e_hi;       // per model: recorded error bounds of the network's prediction
    std::vector<unsigned long long> cells;
    std::vector<unsigned int> max_pop;
    std::vector<unsigned long long> nonempty;
    std::vector<unsigned int> escaped;
    std::vector<double> mean_pop;      // sum of squared cell populations / (N + 1)
    std::vector<int> from_network;     // 1: the map comes from the network, 0: from the linear model
    long long *zoff_dev = nullptr;     // device copy of the query offsets of ds_learned_search_host
};

namespace ds {
void free_learned(ds_learned *L)
{
    if (L->zoff_dev) dev_free(L->zoff_dev);
    engine_free(&L->eng);
    L->hdr.magic = 0;
    delete L;
}
ds_status info_learned(const ds_learned *L, ds_info_t *o)
{
    const Engine &e = L->eng;
    o->kind = KIND_LEARNED;
    o->dtype = e.dtype;
    o->flags = e.flags;
    o->n_arrays = e.n_arrays;
    o->n_knots = e.n_knots;
    o->R = e.R_total;
    o->table_bytes = (int64_t)e.table_bytes;
    o->h_updates = e.h_updates;
    o->build_ms = e.build_ms;
    o->n_direct = e.n_direct;
    o->n_learned = e.n_learned;
    o->n_fallback = e.n_fallback;
    o->max_window = L->max_window;
    o->train_steps = L->steps;
    o->train_ms = L->train_ms;
    o->final_loss = L->final_loss;
    if (e.n_arrays == 1) {
        const ArrDesc &d = e.desc_host[0];
        o->X0 = d.X0;
        o->XN = d.XN;
        o->H = d.H;
        o->W = d.W;
    }
    o->fallback_queries = 0;  // exact by construction: no query needs a fall-back
    o->search_launches = e.split > 0 ? 3 : 2;
    int err = 0;
    if (e.dev_err && cudaMemcpy(&err, e.dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
        o->device_error = err;
    return DS_OK;
}

template <typename T>
static ds_status train_and_bound(ds_learned *L, const ds_learned_cfg &cfg, cudaStream_t s)
{
    Engine &e = L->eng;
    const int nm = (int)L->model_arr.size();
    if (nm == 0) return DS_OK;
    const double t0 = now_ms();
    const uint32_t slo = (uint32_t)cfg.seed, shi = (uint32_t)(cfg.seed >> 32);
    const bool linear = (cfg.flags & DS_LEARNED_LINEAR) != 0;
    std::vector<long long> pool_off(nm + 1, 0);
    for (int k = 0; k < nm; ++k) {
        const ArrDesc &d = e.desc_host[L->model_arr[k]];
        long long nq = cfg.n_queries > 0 ? cfg.n_queries : 0;
        if (linear || cfg.steps <= 0) nq = 0;
        pool_off[k + 1] = pool_off[k] + std::min<long long>(nq, 4ll * (d.n + 1) + 4096);
    }
    const int gb = std::max(1, cfg.batch / TB);
    int *model_arr = nullptr, *step = nullptr, *elo = nullptr, *ehi = nullptr;
    long long *pool_off_d = nullptr;
    float2 *pool = nullptr;
    float *theta = nullptr, *mom = nullptr, *vel = nullptr, *part = nullptr, *plos = nullptr, *loss = nullptr;
    float *seg_x = nullptr, *seg_a = nullptr, *seg_b = nullptr;
    uint32_t *Fk = nullptr;
    long long *kbase_d = nullptr;
    LStats *lst = nullptr;
    ds_status rc = DS_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cs = nullptr;
    do {
        cudaError_t ce = cudaSuccess;
        auto A = [&](void **p, size_t bytes) {
            if (ce == cudaSuccess) ce = dev_alloc(p, std::max<size_t>(bytes, 16));
        };
        A((void **)&model_arr, sizeof(int) * nm);
        A((void **)&step, sizeof(int) * nm);
        A((void **)&elo, sizeof(int) * nm);
        A((void **)&ehi, sizeof(int) * nm);
        A((void **)&pool_off_d, sizeof(long long) * (nm + 1));
        A((void **)&pool, sizeof(float2) * (size_t)pool_off[nm]);
        A((void **)&theta, sizeof(float) * (size_t)nm * NP);
        A((void **)&mom, sizeof(float) * (size_t)nm * NP);
        A((void **)&vel, sizeof(float) * (size_t)nm * NP);
        A((void **)&part, sizeof(float) * (size_t)nm * gb * NP);
        A((void **)&plos, sizeof(float) * (size_t)nm * gb);
        A((void **)&loss, sizeof(float) * nm);
        if (ce != cudaSuccess) {
            set_error("learned build: allocation failed: %s", cudaGetErrorString(ce));
            rc = DS_E_NOMEM;
            break;
        }
        cudaMemcpyAsync(model_arr, L->model_arr.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(pool_off_d, pool_off.data(), sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(step, 0, sizeof(int) * nm, s);
        cudaMemsetAsync(mom, 0, sizeof(float) * (size_t)nm * NP, s);
        cudaMemsetAsync(vel, 0, sizeof(float) * (size_t)nm * NP, s);
        cudaMemsetAsync(loss, 0, sizeof(float) * nm, s);
        k_init_params<<<nm, 256, 0, s>>>(theta, nm, slo, shi);
        if (pool_off[nm] > 0)
            k_pool_queries<T><<<dim3(std::max(1, std::min(e.props.num_sms * 4 / std::max(1, nm), 1024)), nm), 256, 0, s>>>(
                e.desc_dev, e.blob, model_arr, pool_off_d, pool, nm, slo, shi);
        if (!linear && cfg.steps > 0) {
            TrainArgs ta;
            ta.desc = e.desc_dev; ta.blob = e.blob; ta.model_arr = model_arr; ta.pool = pool; ta.pool_off = pool_off_d;
            ta.theta = theta; ta.m = mom; ta.v = vel; ta.partial = part; ta.partial_loss = plos; ta.loss = loss;
            ta.step = step; ta.gb = gb; ta.steps = cfg.steps; ta.lr = cfg.lr; ta.seed_lo = slo; ta.seed_hi = shi;
            const size_t smem = PARAM_SMEM + sizeof(GradTile);
            ce = cudaFuncSetAttribute(k_train_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            // one graph of `per` steps, replayed
            const int per = std::min(cfg.steps, 50);
            if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                for (int k = 0; k < per; ++k) {
                    k_train_grad<T><<<dim3(gb, nm), TB, smem, cs>>>(ta);
                    k_train_adam<<<nm, 256, 0, cs>>>(ta);
                }
                ce = cudaStreamEndCapture(cs, &graph);
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&gexec, graph, 0);
            int done = 0;
            while (ce == cudaSuccess && done + per <= cfg.steps) {
                ce = cudaGraphLaunch(gexec, cs);
                done += per;
            }
            for (; ce == cudaSuccess && done < cfg.steps; ++done) {
                k_train_grad<T><<<dim3(gb, nm), TB, smem, cs>>>(ta);
                k_train_adam<<<nm, 256, 0, cs>>>(ta);
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
            if (ce != cudaSuccess) {
                set_error("learned build: training failed: %s", cudaGetErrorString(ce));
                rc = DS_E_CUDA;
                break;
            }
            L->steps = cfg.steps;
        }
        // parameters to the host, piecewise-linear form, back to the device
        L->theta_host.resize((size_t)nm * NP);
        std::vector<float> lh(nm);
        ce = cudaMemcpyAsync(L->theta_host.data(), theta, sizeof(float) * (size_t)nm * NP, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(lh.data(), loss, sizeof(float) * nm, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            set_error("learned build: %s", cudaGetErrorString(ce));
            rc = DS_E_CUDA;
            break;
        }
        double ls = 0;
        for (float v : lh) ls += v;
        L->final_loss = ls / nm;
        std::vector<Segments> segs(nm);
        Segments all;
        for (int k = 0; k < nm; ++k) {
            ArrDesc &d = e.desc_host[L->model_arr[k]];
            Segments &one = segs[k];
            if (linear) {
                one.x.assign(1, -INFINITY);
                one.a.assign(1, (float)d.n);
                one.b.assign(1, 0.f);
            } else {
                pwl_of(&L->theta_host[(size_t)k * NP], (double)d.n, one);
            }
            d.seg_off = (int32_t)all.x.size();
            d.seg_n = (int32_t)one.x.size();
            all.x.insert(all.x.end(), one.x.begin(), one.x.end());
            all.a.insert(all.a.end(), one.a.begin(), one.a.end());
            all.b.insert(all.b.end(), one.b.begin(), one.b.end());
        }
        const size_t nseg = all.x.size();
        A((void **)&seg_x, sizeof(float) * nseg);
        A((void **)&seg_a, sizeof(float) * nseg);
        A((void **)&seg_b, sizeof(float) * nseg);
        if (ce != cudaSuccess) {
            set_error("learned build: allocation failed");
            rc = DS_E_NOMEM;
            break;
        }
        cudaMemcpyAsync(seg_x, all.x.data(), sizeof(float) * nseg, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(seg_a, all.a.data(), sizeof(float) * nseg, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(seg_b, all.b.data(), sizeof(float) * nseg, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(e.desc_dev, e.desc_host.data(), sizeof(ArrDesc) * e.desc_host.size(), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(elo, 0, sizeof(int) * nm, s);
        cudaMemsetAsync(ehi, 0, sizeof(int) * nm, s);
        k_error_bound<T><<<dim3(std::max(1, std::min(e.props.num_sms * 8 / std::max(1, nm), 2048)), nm), 256, 0, s>>>(
            e.desc_dev, e.blob, model_arr, seg_x, seg_a, seg_b, elo, ehi);
        std::vector<int> hlo(nm), hhi(nm);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(hlo.data(), elo, sizeof(int) * nm, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(hhi.data(), ehi, sizeof(int) * nm, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            set_error("learned build: error bound failed: %s", cudaGetErrorString(ce));
            rc = DS_E_CUDA;
            break;
        }
        // the cell maps: C cells per array, the served prediction sampled at G
        // points (the network's, and the linear model's), each made monotone
        // default: one cell per knot, two where the handle holds the knot values
        // (every lookup then goes on to its answer's pairs, and an empty cell
        // answers without reading a knot: with two cells per knot about 61% of
        // uniform queries land in empty cells, against 37%)
        const double cpk = cfg.cells_per_knot > 0.f ? (double)cfg.cells_per_knot : e.xy ? 2.0 : 1.0;
        std::vector<std::vector<uint2>> net_maps(nm), lin_maps(nm);
        std::vector<long long> kbase(nm + 1, 0);
        L->cells.assign(nm, 0);
        L->e_lo.assign(nm, 0);
        L->e_hi.assign(nm, 0);
        Segments linseg;
        for (int k = 0; k < nm; ++k) {
            ArrDesc &d = e.desc_host[L->model_arr[k]];
            L->e_lo[k] = hlo[k];
            L->e_hi[k] = hhi[k];
            const double want = std::ceil(cpk * (double)(d.n + 1));
            const unsigned long long C =
                (unsigned long long)std::min(std::max(want, 1.0), (double)(0xFFFFFFFFull - 1));
            L->cells[k] = C;
            d.R = (uint32_t)(C - 1);
            const int G = (int)(d.img_bytes >> 3);
            linseg.x.assign(1, -INFINITY);
            linseg.a.assign(1, (float)d.n);
            linseg.b.assign(1, 0.f);
            cell_map(segs[k], (long long)d.n + 1, C, G, net_maps[k]);
            cell_map(linseg, (long long)d.n + 1, C, G, lin_maps[k]);
            kbase[k + 1] = kbase[k] + d.n + 1;
        }
        A((void **)&Fk, sizeof(uint32_t) * (size_t)kbase[nm]);
        A((void **)&kbase_d, sizeof(long long) * (size_t)(nm + 1));
        A((void **)&lst, sizeof(LStats) * nm);
        if (ce != cudaSuccess) {
            set_error("learned build: allocation failed");
            rc = DS_E_NOMEM;
            break;
        }
        cudaMemcpyAsync(kbase_d, kbase.data(), sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(e.desc_dev, e.desc_host.data(), sizeof(ArrDesc) * e.desc_host.size(), cudaMemcpyHostToDevice, s);
        const dim3 lgrid(std::max(1, std::min(e.props.num_sms * 8 / std::max(1, nm), 2048)), nm);
        // statistics of the maps in the blob: cell of every knot, then the cells' populations
        auto map_stats = [&](const std::vector<std::vector<uint2>> &maps, std::vector<LStats> &hst) {
            for (int k = 0; k < nm; ++k) {
                const ArrDesc &d = e.desc_host[L->model_arr[k]];
                cudaMemcpyAsync(e.blob + d.img, maps[k].data(), d.img_bytes, cudaMemcpyHostToDevice, s);
            }
            cudaMemsetAsync(lst, 0, sizeof(LStats) * nm, s);
            k_learned_F<T><<<lgrid, 256, 0, s>>>(e.desc_dev, e.blob, model_arr, kbase_d, Fk);
            k_learned_cells<<<lgrid, 256, 0, s>>>(e.desc_dev, model_arr, kbase_d, Fk, lst, nullptr, 0);
            hst.resize(nm);
            cudaError_t c2 = cudaGetLastError();
            if (c2 == cudaSuccess) c2 = cudaMemcpyAsync(hst.data(), lst, sizeof(LStats) * nm, cudaMemcpyDeviceToHost, s);
            if (c2 == cudaSuccess) c2 = cudaStreamSynchronize(s);
            return c2;
        };
        // each array keeps the map whose cells a query shares with fewer knots
        // (sum of squared populations: the mean population seen by queries
        // distributed like the knots); the network's map only where it wins
        std::vector<LStats> st_lin, st_net;
        ce = map_stats(lin_maps, st_lin);
        if (ce == cudaSuccess && !linear) ce = map_stats(net_maps, st_net);
        if (ce != cudaSuccess) {
            set_error("learned build: cell statistics failed: %s", cudaGetErrorString(ce));
            rc = DS_E_CUDA;
            break;
        }
        L->from_network.assign(nm, 0);
        std::vector<std::vector<uint2>> chosen(nm);
        for (int k = 0; k < nm; ++k) {
            const bool net = !linear && st_net[k].sum_pop2 < st_lin[k].sum_pop2;
            L->from_network[k] = net ? 1 : 0;
            chosen[k] = net ? net_maps[k] : lin_maps[k];
        }
        std::vector<LStats> hst;
        ce = map_stats(chosen, hst);
        if (ce != cudaSuccess) {
            set_error("learned build: cell statistics failed: %s", cudaGetErrorString(ce));
            rc = DS_E_CUDA;
            break;
        }
        size_t cbytes = 0;
        L->max_pop.assign(nm, 0);
        L->nonempty.assign(nm, 0);
        L->escaped.assign(nm, 0);
        L->mean_pop.assign(nm, 0.0);
        for (int k = 0; k < nm; ++k) {
            ArrDesc &d = e.desc_host[L->model_arr[k]];
            d.aux = 0;
            d.ct = (long long)cbytes;
            d.n_esc = (long long)hst[k].escaped;
            cbytes += round_up((size_t)lblk_count(d.R) * 16 + (size_t)hst[k].escaped * 36, 16);
            L->max_pop[k] = hst[k].max_pop;
            L->nonempty[k] = hst[k].nonempty;
            L->escaped[k] = hst[k].escaped;
            L->mean_pop[k] = (double)hst[k].sum_pop2 / (double)(d.n + 1);
            L->max_window = std::max(L->max_window, (long long)hst[k].max_pop + 1);
        }
        ce = dev_alloc(&e.ctab, std::max<size_t>(cbytes, 16));
        if (ce != cudaSuccess) {
            e.ctab = nullptr;
            set_error("learned build: cell tables (%zu bytes): allocation failed", cbytes);
            rc = DS_E_NOMEM;
            break;
        }
        e.ctab_bytes = cbytes;
        e.table_bytes += cbytes;
        cudaMemcpyAsync(e.desc_dev, e.desc_host.data(), sizeof(ArrDesc) * e.desc_host.size(), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(lst, 0, sizeof(LStats) * nm, s);  // escaped slots are handed out from 0
        k_learned_cells<<<lgrid, 256, 0, s>>>(e.desc_dev, model_arr, kbase_d, Fk, lst, e.ctab, 1);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            set_error("learned build: cell table fill failed: %s", cudaGetErrorString(ce));
            rc = DS_E_CUDA;
        }
    } while (0);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    for (void *p : {(void *)model_arr, (void *)step, (void *)elo, (void *)ehi, (void *)pool_off_d, (void *)pool,
                    (void *)theta, (void *)mom, (void *)vel, (void *)part, (void *)plos, (void *)loss, (void *)seg_x,
                    (void *)seg_a, (void *)seg_b, (void *)Fk, (void *)kbase_d, (void *)lst})
        if (p) dev_free(p);
    L->train_ms = now_ms() - t0;
    return rc;
}

}  // namespace ds

static bool learned_ok(const ds_learned *L)
{
    return L && L->hdr.magic == ds::HANDLE_MAGIC && L->hdr.kind == ds::KIND_LEARNED;
}

extern "C" {

void ds_learned_cfg_default(ds_learned_cfg *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->steps = 6000;
    cfg->batch = 8192;
    cfg->n_queries = 1 << 18;
    cfg->lr = 3e-3f;
    cfg->seed = 1506086200ull;
    cfg->flags = 0;
    cfg->max_cells_per_knot = 16;
    cfg->cells_per_knot = 0.0f;
}

ds_status ds_learned_build(const void *Xcat_dev, const int64_t *x_off_dev, int32_t n_arrays, int64_t n_knots_if_single,
                           ds_dtype dtype, const ds_learned_cfg *cfg_in, void *stream, ds_learned **out)
{
    return ds_learned_build_xy(Xcat_dev, nullptr, x_off_dev, n_arrays, n_knots_if_single, dtype, cfg_in, stream, out);
}

ds_status ds_learned_build_xy(const void *Xcat_dev, const void *Ycat_dev, const int64_t *x_off_dev, int32_t n_arrays,
                              int64_t n_knots_if_single, ds_dtype dtype, const ds_learned_cfg *cfg_in, void *stream,
                              ds_learned **out)
{
    ds::clear_error();
    if (!out) {
        ds::set_error("ds_learned_build: out is NULL");
        return DS_E_ARG;
    }
    *out = nullptr;
    ds_learned_cfg cfg;
    if (cfg_in) cfg = *cfg_in;
    else ds_learned_cfg_default(&cfg);
    if (!Xcat_dev || n_arrays < 1 || (dtype != DS_F32 && dtype != DS_F64) || (!x_off_dev && n_arrays != 1) ||
        (!x_off_dev && n_knots_if_single < 2) || cfg.batch < 1 || cfg.steps < 0 || !(cfg.lr > 0.f) ||
        !(cfg.cells_per_knot >= 0.f && cfg.cells_per_knot <= 64.f) ||
        (cfg.flags & ~(uint32_t)(DS_LEARNED_FORCE | DS_LEARNED_LINEAR))) {
        ds::set_error("ds_learned_build: bad argument");
        return DS_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double t0 = ds::now_ms();
    ds_learned *L = new ds_learned;
    L->hdr.kind = ds::KIND_LEARNED;
    L->hdr.magic = ds::HANDLE_MAGIC;
    long long *single_off = nullptr;
    const long long *xo = (const long long *)x_off_dev;
    if (!x_off_dev) {
        long long h[2] = {0, (long long)n_knots_if_single};
        if (ds::dev_alloc(&single_off, sizeof(h)) != cudaSuccess ||
            cudaMemcpy(single_off, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) {
            ds::set_error("ds_learned_build: allocation failed");
            delete L;
            return DS_E_NOMEM;
        }
        xo = single_off;
    }
    std::vector<char> force;
    std::vector<char> *fp = nullptr;
    if (cfg.flags & DS_LEARNED_FORCE) {
        force.assign(n_arrays, 1);
        fp = &force;
    }
    ds_status rc = ds::engine_build(&L->eng, Xcat_dev, Ycat_dev, xo, n_arrays, dtype, 0, s, fp, ds::MODE_LEARNED,
                                    nullptr, nullptr, (double)cfg.max_cells_per_knot);
    if (single_off) ds::dev_free(single_off);
    if (rc == DS_OK) {
        ds::Engine &e = L->eng;
        L->arr_model.assign(n_arrays, -1);
        for (int a = 0; a < n_arrays; ++a) {
            ds::ArrDesc &d = e.desc_host[a];
            if (d.mode != ds::MODE_LEARNED) continue;
            L->arr_model[a] = (int)L->model_arr.size();
            L->model_arr.push_back(a);
            // predictor input u = (narrow(z) - narrow(X_0)) * uscale, in float32
            const double span = d.XN - d.X0;
            float x0f = (float)d.X0;
            if (dtype == DS_F64) {  // truncating narrowing, as on the device
                double x0 = d.X0;
                unsigned long long b;
                memcpy(&b, &x0, 8);
                const int ex = (int)((b >> 52) & 0x7FF) - 1023;
                if (ex < -126) x0f = 0.f * (float)((b >> 63) ? -1 : 1);
                else {
                    uint32_t fb = (uint32_t)((b >> 32) & 0x80000000u) | ((uint32_t)(ex + 127) << 23) |
                                  (uint32_t)((b >> 29) & 0x7FFFFFu);
                    memcpy(&x0f, &fb, 4);
                }
            }
            d.x0f = x0f;
            d.uscale = (float)(1.0 / span);
        }
        if (cudaMemcpyAsync(e.desc_dev, e.desc_host.data(), sizeof(ds::ArrDesc) * e.desc_host.size(),
                            cudaMemcpyHostToDevice, s) != cudaSuccess) {
            ds::set_error("ds_learned_build: descriptor upload failed");
            rc = DS_E_CUDA;
        }
    }
    if (rc == DS_OK) {
        rc = dtype == DS_F32 ? ds::train_and_bound<float>(L, cfg, s) : ds::train_and_bound<double>(L, cfg, s);
    }
    if (rc != DS_OK) {
        ds::free_learned(L);
        return rc;
    }
    L->eng.tune = ds::default_tune();
    L->eng.tune2 = L->eng.tune;
    L->eng.build_ms = ds::now_ms() - t0;
    *out = L;
    return DS_OK;
}

ds_status ds_learned_search(const ds_learned *L, const void *Zcat_dev, const int64_t *z_off_dev, int64_t m,
                            const void *Ycat_dev, void *y_out_dev, int32_t *Icat_dev, void *stream)
{
    if (!learned_ok(L) || !Zcat_dev || !Icat_dev || (!z_off_dev && (m < 0 || L->eng.n_arrays != 1)) ||
        (L->eng.xy ? Ycat_dev != nullptr : (Ycat_dev == nullptr) != (y_out_dev == nullptr))) {
        ds::set_error("ds_learned_search: bad argument%s",
                      L && L->eng.xy && Ycat_dev ? " (this handle holds its knot values: pass Ycat = NULL)" : "");
        return DS_E_ARG;
    }
    if (!z_off_dev && m == 0) return DS_OK;
    return ds::engine_launch(const_cast<ds::Engine *>(&L->eng), Zcat_dev, (const long long *)z_off_dev,
                             z_off_dev ? 0 : m, Ycat_dev, y_out_dev, Icat_dev, (cudaStream_t)stream);
}

ds_status ds_learned_autotune(ds_learned *L, const void *Zcat_dev, const int64_t *z_off_dev, int64_t m,
                              const void *Ycat_dev, void *y_out_dev, int32_t *Icat_dev, void *stream, ds_tune_t *best)
{
    if (!learned_ok(L) || !Zcat_dev || !Icat_dev || (!z_off_dev && (m < 1 || L->eng.n_arrays != 1)) ||
        (L->eng.xy ? Ycat_dev != nullptr : (Ycat_dev == nullptr) != (y_out_dev == nullptr))) {
        ds::set_error("ds_learned_autotune: bad argument");
        return DS_E_ARG;
    }
    return ds::engine_autotune(&L->eng, Zcat_dev, (const long long *)z_off_dev, z_off_dev ? 0 : m, Ycat_dev,
                               y_out_dev, Icat_dev, (cudaStream_t)stream, best);
}

ds_status ds_learned_set_tune(ds_learned *L, const ds_tune_t *cfg)
{
    if (!learned_ok(L) || !cfg) {
        ds::set_error("ds_learned_set_tune: bad argument");
        return DS_E_ARG;
    }
    return ds::engine_set_tune(&L->eng, *cfg);
}

ds_status ds_learned_get_tune(const ds_learned *L, ds_tune_t *cfg)
{
    if (!learned_ok(L) || !cfg) return DS_E_ARG;
    *cfg = L->eng.tune;
    return DS_OK;
}

ds_status ds_learned_array(const ds_learned *L, int32_t a, float *theta_host, int32_t *e_lo, int32_t *e_hi,
                           int32_t *mode)
{
    if (!learned_ok(L) || a < 0 || a >= L->eng.n_arrays) {
        ds::set_error("ds_learned_array: bad argument");
        return DS_E_ARG;
    }
    const ds::ArrDesc &d = L->eng.desc_host[a];
    if (mode) *mode = d.mode;
    const int km = L->arr_model[a];
    if (e_lo) *e_lo = km >= 0 && !L->e_lo.empty() ? L->e_lo[km] : 0;
    if (e_hi) *e_hi = km >= 0 && !L->e_hi.empty() ? L->e_hi[km] : 0;
    if (theta_host) {
        const int k = L->arr_model[a];
        if (k >= 0 && !L->theta_host.empty()) memcpy(theta_host, &L->theta_host[(size_t)k * ds::NP], sizeof(float) * ds::NP);
        else memset(theta_host, 0, sizeof(float) * ds::NP);
    }
    return DS_OK;
}

ds_status ds_mlp_forward(const float *theta_dev, const float *u_dev, int64_t n, float *out_dev, void *stream)
{
    if (!theta_dev || (n > 0 && (!u_dev || !out_dev)) || n < 0) {
        ds::set_error("ds_mlp_forward: bad argument");
        return DS_E_ARG;
    }
    if (n == 0) return DS_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    ds::k_forward<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(theta_dev, u_dev, n, out_dev);
    DS_TRY_CUDA(cudaGetLastError());
    return DS_OK;
}

ds_status ds_mlp_loss_grad(const float *theta_dev, const float *u_dev, const float *y_dev, int64_t n, float *grad_dev,
                           float *loss_dev, void *stream)
{
    if (!theta_dev || !u_dev || !y_dev || !grad_dev || !loss_dev || n < 1 || n > (1ll << 30)) {
        ds::set_error("ds_mlp_loss_grad: bad argument");
        return DS_E_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + ds::TB - 1) / ds::TB);
    float *part = nullptr, *plos = nullptr;
    DS_TRY_CUDA(ds::dev_alloc_async(&part, sizeof(float) * (size_t)nb * ds::NP, s));
    cudaError_t ce = ds::dev_alloc_async(&plos, sizeof(float) * (size_t)nb, s);
    const size_t smem = ds::PARAM_SMEM + sizeof(ds::GradTile);
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(ds::k_grad_explicit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce == cudaSuccess) {
        ds::k_grad_explicit<<<nb, ds::TB, smem, s>>>(theta_dev, u_dev, y_dev, n, part, plos);
        ds::k_reduce_grad<<<1, 256, 0, s>>>(part, plos, nb, n, grad_dev, loss_dev);
        ce = cudaGetLastError();
    }
    ds::dev_free_async(part, s);
    if (plos) ds::dev_free_async(plos, s);
    if (ce != cudaSuccess) {
        ds::set_error("ds_mlp_loss_grad: %s", cudaGetErrorString(ce));
        return ce == cudaErrorMemoryAllocation ? DS_E_NOMEM : DS_E_CUDA;
    }
    return DS_OK;
}

ds_status ds_adam_step(float *theta_dev, float *m_dev, float *v_dev, const float *grad_dev, int32_t t, float lr,
                       void *stream)
{
    if (!theta_dev || !m_dev || !v_dev || !grad_dev || t < 1 || !(lr > 0.f)) {
        ds::set_error("ds_adam_step: bad argument");
        return DS_E_ARG;
    }
    ds::k_adam_explicit<<<5, 256, 0, (cudaStream_t)stream>>>(theta_dev, m_dev, v_dev, grad_dev, t, lr);
    DS_TRY_CUDA(cudaGetLastError());
    return DS_OK;
}

// Device address of host memory: mapped page-locked memory as it is, other
// host memory registered (mapped) for this call; *reg is set when the caller
// must unregister it.
static ds_status host_mapped(void *h, size_t bytes, void **d, bool *reg)
{
    *reg = false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer &&
        at.hostPointer) {
        *d = (char *)at.devicePointer + ((char *)h - (char *)at.hostPointer);
        return DS_OK;
    }
    cudaGetLastError();
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        ds::set_error("ds_learned_search_host: a buffer is device memory (use ds_learned_search)");
        return DS_E_ARG;
    }
    DS_TRY_CUDA(cudaHostRegister(h, bytes, cudaHostRegisterMapped));
    *reg = true;
    const cudaError_t e = cudaHostGetDevicePointer(d, h, 0);
    if (e != cudaSuccess) {
        cudaHostUnregister(h);
        *reg = false;
        ds::set_error("ds_learned_search_host: %s", cudaGetErrorString(e));
        return DS_E_CUDA;
    }
    return DS_OK;
}

ds_status ds_learned_search_host(ds_learned *L, const void *Zcat_host, const int64_t *z_off_host, int64_t m,
                                 void *y_out_host, int32_t *Icat_host, void *stream)
{
    ds::clear_error();
    if (!learned_ok(L) || !Zcat_host || !Icat_host || (!z_off_host && (m < 0 || L->eng.n_arrays != 1)) ||
        (y_out_host && !L->eng.xy)) {
        ds::set_error("ds_learned_search_host: bad argument%s",
                      L && y_out_host && !L->eng.xy ? " (interpolation needs a handle from ds_learned_build_xy)" : "");
        return DS_E_ARG;
    }
    ds::Engine &e = L->eng;
    cudaStream_t s = (cudaStream_t)stream;
    if (z_off_host) {
        if (z_off_host[0] != 0) {
            ds::set_error("ds_learned_search_host: z_off[0] must be 0");
            return DS_E_ARG;
        }
        m = z_off_host[e.n_arrays];
        if (!L->zoff_dev) DS_TRY_CUDA(ds::dev_alloc(&L->zoff_dev, sizeof(long long) * (size_t)(e.n_arrays + 1)));
        DS_TRY_CUDA(cudaMemcpyAsync(L->zoff_dev, z_off_host, sizeof(long long) * (size_t)(e.n_arrays + 1),
                                    cudaMemcpyHostToDevice, s));
    }
    if (m == 0) return DS_OK;
    const size_t esz = e.dtype == DS_F32 ? 4 : 8;
    void *zd = nullptr, *id = nullptr, *yd = nullptr;
    bool rz = false, ri = false, ry = false;
    ds_status rc = host_mapped(const_cast<void *>(Zcat_host), (size_t)m * esz, &zd, &rz);
    if (rc == DS_OK) rc = host_mapped(Icat_host, (size_t)m * 4, &id, &ri);
    if (rc == DS_OK && y_out_host) rc = host_mapped(y_out_host, (size_t)m * esz, &yd, &ry);
    if (rc == DS_OK)
        rc = ds::engine_launch_direct(&e, e.tune, zd, z_off_host ? L->zoff_dev : nullptr, z_off_host ? 0 : m, nullptr,
                                      yd, (int32_t *)id, s, true, &e.tune2);
    const cudaError_t ce = cudaStreamSynchronize(s);
    if (rc == DS_OK && ce != cudaSuccess) {
        ds::set_error("ds_learned_search_host: %s", cudaGetErrorString(ce));
        rc = DS_E_CUDA;
    }
    if (rz) cudaHostUnregister(const_cast<void *>(Zcat_host));
    if (ri) cudaHostUnregister(Icat_host);
    if (ry) cudaHostUnregister(y_out_host);
    return rc;
}

ds_status ds_learned_cells(const ds_learned *L, int32_t a, uint64_t *cells, int32_t *max_pop, int64_t *nonempty,
                           int64_t *escaped, double *mean_pop, int32_t *from_network)
{
    if (!learned_ok(L) || a < 0 || a >= L->eng.n_arrays) {
        ds::set_error("ds_learned_cells: bad argument");
        return DS_E_ARG;
    }
    const int k = L->arr_model[a];
    if (cells) *cells = k < 0 ? 0 : L->cells[k];
    if (max_pop) *max_pop = k < 0 ? 0 : (int32_t)L->max_pop[k];
    if (nonempty) *nonempty = k < 0 ? 0 : (int64_t)L->nonempty[k];
    if (escaped) *escaped = k < 0 ? 0 : (int64_t)L->escaped[k];
    if (mean_pop) *mean_pop = k < 0 ? 0.0 : L->mean_pop[k];
    if (from_network) *from_network = k < 0 ? 0 : L->from_network[k];
    return DS_OK;
}

ds_status ds_learned_export_cells(const ds_learned *L, int32_t a, uint32_t *K_out_dev, void *stream)
{
    if (!learned_ok(L) || a < 0 || a >= L->eng.n_arrays || !K_out_dev || L->arr_model[a] < 0) {
        ds::set_error("ds_learned_export_cells: bad argument (array %d is not served by the learned map)", a);
        return DS_E_ARG;
    }
    const ds::ArrDesc &d = L->eng.desc_host[a];
    const unsigned long long n = (unsigned long long)d.R + 2ull;
    const int grid = (int)std::min<unsigned long long>((n + 255) / 256, 4096ull);
    ds::k_export_cells<<<grid, 256, 0, (cudaStream_t)stream>>>(L->eng.ctab + d.ct, d.R, d.n_esc, K_out_dev);
    DS_TRY_CUDA(cudaGetLastError());
    return DS_OK;
}

}  // extern "C"
