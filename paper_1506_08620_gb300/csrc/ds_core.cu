// ds_core.cu -- C ABI entry points shared by all handle kinds: argument
// checks, errors, handle dispatch, the host-buffer pipeline.
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "ds_index.cuh"

namespace ds {

static thread_local char g_err[1024];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// ------------------------------------------------------------------ device memory
namespace {
std::mutex g_alloc_mu;
std::unordered_map<void *, size_t> g_live;  // live allocations and their sizes
long long g_live_bytes = 0;
long long g_fail_at = -1;  // allocations to let through before one fails (-1: none fails)

// true if this allocation is to fail (the hook counts down under the lock)
bool take_failure()
{
    if (g_fail_at < 0) return false;
    if (g_fail_at == 0) {
        g_fail_at = -1;
        return true;
    }
    --g_fail_at;
    return false;
}
void note_alloc(void *p, size_t bytes)
{
    g_live[p] = bytes;
    g_live_bytes += (long long)bytes;
}
void note_free(void *p)
{
    auto it = g_live.find(p);
    if (it == g_live.end()) return;
    g_live_bytes -= (long long)it->second;
    g_live.erase(it);
}
}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes)
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    *p = nullptr;
    if (take_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) note_alloc(*p, bytes);
    return e;
}
cudaError_t dev_alloc_async(void **p, size_t bytes, cudaStream_t s)
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    *p = nullptr;
    if (take_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) note_alloc(*p, bytes);
    return e;
}
void dev_free(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    note_free(p);
    cudaFree(p);
}
void dev_free_async(void *p, cudaStream_t s)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    note_free(p);
    cudaFreeAsync(p, s);
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t table_budget_bytes()
{
    if (const char *e = getenv("DS_TABLE_BUDGET_BYTES")) return (size_t)strtoull(e, nullptr, 10);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    return free_b / 2;
}

ds_status device_props(DeviceProps *p)
{
    DS_TRY_CUDA(cudaGetDevice(&p->device));
    DS_TRY_CUDA(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    DS_TRY_CUDA(cudaDeviceGetAttribute(&p->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    DS_TRY_CUDA(cudaDeviceGetAttribute(&p->l2_bytes, cudaDevAttrL2CacheSize, p->device));
    return DS_OK;
}

ds_status allow_dynamic_smem(const void *fn, int need_bytes)
{
    int dev = 0, optin = 0;
    DS_TRY_CUDA(cudaGetDevice(&dev));
    DS_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    DS_TRY_CUDA(cudaFuncGetAttributes(&fa, fn));
    const int lim = optin - (int)fa.sharedSizeBytes;
    if (need_bytes > lim) {
        set_error("kernel needs %d bytes of dynamic shared memory, the device allows %d", need_bytes, lim);
        return DS_E_ARG;
    }
    DS_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return DS_OK;
}

// ----------------------------------------------------------------- host pipeline
constexpr int PIPE_BUFS = 3;

struct HostPipe {
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in[PIPE_BUFS] = {}, ev_run[PIPE_BUFS] = {}, ev_out[PIPE_BUFS] = {};
    void *zbuf[PIPE_BUFS] = {};
    int32_t *ibuf[PIPE_BUFS] = {};
    long long chunk = 0;
};

static void destroy_pipe(HostPipe *p)
{
    if (!p) return;
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_run) cudaStreamSynchronize(p->s_run);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    for (int b = 0; b < PIPE_BUFS; ++b) {
        if (p->zbuf[b]) dev_free(p->zbuf[b]);
        if (p->ibuf[b]) dev_free(p->ibuf[b]);
        if (p->ev_in[b]) cudaEventDestroy(p->ev_in[b]);
        if (p->ev_run[b]) cudaEventDestroy(p->ev_run[b]);
        if (p->ev_out[b]) cudaEventDestroy(p->ev_out[b]);
    }
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_run) cudaStreamDestroy(p->s_run);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    delete p;
}

static ds_status make_pipe(HostPipe **out, size_t elem_bytes)
{
    HostPipe *p = new HostPipe;
    p->chunk = 1ll << 23;  // queries per chunk
    if (const char *e = getenv("DS_PIPE_CHUNK")) p->chunk = atoll(e) > 0 ? atoll(e) : p->chunk;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_run, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
    for (int b = 0; b < PIPE_BUFS && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&p->ev_in[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_run[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_out[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = dev_alloc(&p->zbuf[b], (size_t)p->chunk * elem_bytes);
        if (e == cudaSuccess) e = dev_alloc(&p->ibuf[b], (size_t)p->chunk * sizeof(int32_t));
    }
    if (e != cudaSuccess) {
        set_error("ds_search_host: pipeline setup failed: %s", cudaGetErrorString(e));
        destroy_pipe(p);
        return e == cudaErrorMemoryAllocation ? DS_E_NOMEM : DS_E_CUDA;
    }
    *out = p;
    return DS_OK;
}

void free_index(ds_index *idx)
{
    if (!idx) return;
    destroy_pipe(idx->pipe);
    if (idx->tab) dev_free(idx->tab);
    if (idx->pairs) dev_free(idx->pairs);
    if (idx->k16) dev_free(idx->k16);
    if (idx->dev_err) dev_free(idx->dev_err);
    idx->hdr.magic = 0;
    delete idx;
}

ds_status info_index(const ds_index *idx, ds_info_t *o)
{
    o->kind = KIND_INDEX;
    o->dtype = idx->dtype;
    o->flags = idx->flags;
    o->n_arrays = 1;
    o->n_knots = idx->n_knots;
    o->H = idx->H;
    o->W = idx->W;
    o->X0 = idx->X0;
    o->XN = idx->XN;
    o->R = idx->R;
    o->table_bytes = (int64_t)idx->table_bytes;
    o->h_updates = idx->updates;
    o->hr_passes = idx->passes;
    o->build_ms = idx->build_ms;
    o->smem_resident = idx->plan.smem ? 1 : 0;
    o->n_direct = 1;
    o->gap_q = idx->q;
    o->search_launches = 1;
    int err = 0;
    if (idx->dev_err && cudaMemcpy(&err, idx->dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
        o->device_error = err;
    return DS_OK;
}

// defined in ds_batch.cu / ds_learned.cu
void free_batch(ds_batch *b);
ds_status info_batch(const ds_batch *b, ds_info_t *out);
void free_learned(ds_learned *L);
ds_status info_learned(const ds_learned *L, ds_info_t *out);
void free_lsearch(ds_lsearch *h);
ds_status info_lsearch(const ds_lsearch *h, ds_info_t *out);

}  // namespace ds

using namespace ds;

static bool valid_handle(const void *h, int32_t kind)
{
    if (!h) return false;
    const HandleHeader *hh = reinterpret_cast<const HandleHeader *>(h);
    return hh->magic == HANDLE_MAGIC && (kind == 0 || hh->kind == kind);
}

extern "C" {

int32_t ds_abi_version(void) { return 1; }

const char *ds_last_error(void) { return g_err; }

ds_status ds_debug_fail_alloc(int64_t nth)
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_fail_at = nth < 0 ? -1 : (long long)nth;
    return DS_OK;
}

ds_status ds_debug_alloc_stats(int64_t *live_count, int64_t *live_bytes)
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (live_count) *live_count = (int64_t)g_live.size();
    if (live_bytes) *live_bytes = (int64_t)g_live_bytes;
    return DS_OK;
}

const char *ds_status_str(ds_status s)
{
    switch (s) {
    case DS_OK: return "DS_OK";
    case DS_E_ARG: return "DS_E_ARG";
    case DS_E_NOT_INCREASING: return "DS_E_NOT_INCREASING";
    case DS_E_INDISTINGUISHABLE: return "DS_E_INDISTINGUISHABLE";
    case DS_E_OVERFLOW: return "DS_E_OVERFLOW";
    case DS_E_TABLE_TOO_LARGE: return "DS_E_TABLE_TOO_LARGE";
    case DS_E_NOMEM: return "DS_E_NOMEM";
    case DS_E_CUDA: return "DS_E_CUDA";
    case DS_E_TIMEOUT: return "DS_E_TIMEOUT";
    case DS_E_UNIMPLEMENTED: return "DS_E_UNIMPLEMENTED";
    case DS_E_NO_CONVERGENCE: return "DS_E_NO_CONVERGENCE";
    case DS_E_DEVICE: return "DS_E_DEVICE";
    }
    return "DS_E_UNKNOWN";
}

ds_status ds_build(const void *X_dev, int64_t n_knots, ds_dtype dtype, uint32_t flags, void *stream, ds_index **out)
{
    clear_error();
    if (!out) {
        set_error("ds_build: out is NULL");
        return DS_E_ARG;
    }
    *out = nullptr;
    if (!X_dev || n_knots < 2 || (dtype != DS_F32 && dtype != DS_F64) ||
        (flags & ~(uint32_t)(DS_FMA | DS_CACHE_LAYOUT | DS_CHECKED | DS_NO_SMEM | DS_GAP2 | DS_REFINE_H))) {
        set_error("ds_build: bad argument (X=%p, n_knots=%lld, dtype=%d, flags=%u)", X_dev, (long long)n_knots,
                  (int)dtype, flags);
        return DS_E_ARG;
    }
    if (n_knots > (1ll << 31) - 1) {
        set_error("ds_build: at most 2^31-1 knots (int32 results)");
        return DS_E_ARG;
    }
    if ((flags & DS_GAP2) && (flags & DS_CACHE_LAYOUT)) {
        set_error("ds_build: DS_GAP2 has no cache layout (its correction reads two knots)");
        return DS_E_ARG;
    }
    if ((flags & DS_GAP2) && n_knots > (1ll << 30)) {
        set_error("ds_build: DS_GAP2 takes at most 2^30 knots");
        return DS_E_ARG;
    }
    return build_single(X_dev, n_knots, dtype, flags, (flags & DS_GAP2) ? 2 : 1, 0, 0, (cudaStream_t)stream, out);
}

ds_status ds_build_q(const void *X_dev, int64_t n_knots, ds_dtype dtype, uint32_t flags, int32_t q, int32_t q_max,
                     int64_t budget_bytes, void *stream, ds_index **out)
{
    clear_error();
    if (!out) {
        set_error("ds_build_q: out is NULL");
        return DS_E_ARG;
    }
    *out = nullptr;
    if (!X_dev || n_knots < 2 || (dtype != DS_F32 && dtype != DS_F64) || q < 0 || (q == 0 && q_max < 1) ||
        (flags & ~(uint32_t)(DS_FMA | DS_CACHE_LAYOUT | DS_CHECKED | DS_NO_SMEM | DS_REFINE_H))) {
        set_error("ds_build_q: bad argument (X=%p, n_knots=%lld, dtype=%d, flags=%u, q=%d, q_max=%d)", X_dev,
                  (long long)n_knots, (int)dtype, flags, q, q_max);
        return DS_E_ARG;
    }
    if ((flags & DS_CACHE_LAYOUT) && q != 1) {
        set_error("ds_build_q: the cache layout exists for q = 1 only");
        return DS_E_ARG;
    }
    if (n_knots > (q == 1 ? (1ll << 31) - 1 : (1ll << 30))) {
        set_error("ds_build_q: too many knots for q = %d (at most 2^30 for an Eq. kgeneral table)", q);
        return DS_E_ARG;
    }
    return build_single(X_dev, n_knots, dtype, flags, q, q_max, budget_bytes, (cudaStream_t)stream, out);
}

ds_status ds_search(const ds_index *idx, const void *Z_dev, int64_t m, int32_t *I_dev, void *stream)
{
    if (!valid_handle(idx, KIND_INDEX)) {
        set_error("ds_search: not an index handle");
        return DS_E_ARG;
    }
    return search_index(idx, Z_dev, m, I_dev, (cudaStream_t)stream);
}

ds_status ds_search_host(ds_index *idx, const void *Z_host, int64_t m, int32_t *I_host, void *stream)
{
    if (!valid_handle(idx, KIND_INDEX)) {
        set_error("ds_search_host: not an index handle");
        return DS_E_ARG;
    }
    if (m == 0) return DS_OK;
    if (!Z_host || !I_host || m < 0) {
        set_error("ds_search_host: null pointer or negative size");
        return DS_E_ARG;
    }
    cudaStream_t us = (cudaStream_t)stream;
    // Pinned, mapped host buffers (cudaHostAlloc, cudaHostRegister): the search
    // kernel streams the queries from host memory and writes the results there
    // itself, over the CPU-GPU link (NVLink-C2C on Grace-Blackwell), with no
    // staging copies; the table gathers stay in device memory.
    const char *pipe_env = getenv("DS_HOST_PIPE");
    const bool force_pipe = pipe_env && atoi(pipe_env) != 0;
    if (!force_pipe) {
        cudaPointerAttributes az, ai;
        if (cudaPointerGetAttributes(&az, Z_host) == cudaSuccess && az.type == cudaMemoryTypeHost &&
            az.devicePointer && az.hostPointer && cudaPointerGetAttributes(&ai, I_host) == cudaSuccess &&
            ai.type == cudaMemoryTypeHost && ai.devicePointer && ai.hostPointer) {
            // the attributes may describe the enclosing allocation: keep the pointers' offsets into it
            const char *zd = (const char *)az.devicePointer + ((const char *)Z_host - (const char *)az.hostPointer);
            char *id = (char *)ai.devicePointer + ((const char *)I_host - (const char *)ai.hostPointer);
            DS_TRY(search_index(idx, zd, m, reinterpret_cast<int32_t *>(id), us));
            DS_TRY_CUDA(cudaStreamSynchronize(us));
            return DS_OK;
        }
        cudaGetLastError();  // pageable memory: not an error, take the copy pipeline
    }
    const size_t esz = idx->dtype == DS_F32 ? 4 : 8;
    if (!idx->pipe) DS_TRY(make_pipe(&idx->pipe, esz));
    HostPipe *p = idx->pipe;
    DS_TRY_CUDA(cudaEventRecord(p->ev_start, us));
    DS_TRY_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_start, 0));
    const char *zh = reinterpret_cast<const char *>(Z_host);
    long long c = 0;
    for (long long off = 0; off < m; off += p->chunk, ++c) {
        const int b = (int)(c % PIPE_BUFS);
        const long long n = m - off < p->chunk ? m - off : p->chunk;
        if (c >= PIPE_BUFS) DS_TRY_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_out[b], 0));
        DS_TRY_CUDA(cudaMemcpyAsync(p->zbuf[b], zh + off * esz, (size_t)n * esz, cudaMemcpyHostToDevice, p->s_in));
        DS_TRY_CUDA(cudaEventRecord(p->ev_in[b], p->s_in));
        DS_TRY_CUDA(cudaStreamWaitEvent(p->s_run, p->ev_in[b], 0));
        DS_TRY(search_index(idx, p->zbuf[b], n, p->ibuf[b], p->s_run));
        DS_TRY_CUDA(cudaEventRecord(p->ev_run[b], p->s_run));
        DS_TRY_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_run[b], 0));
        DS_TRY_CUDA(cudaMemcpyAsync(I_host + off, p->ibuf[b], (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    p->s_out));
        DS_TRY_CUDA(cudaEventRecord(p->ev_out[b], p->s_out));
    }
    DS_TRY_CUDA(cudaStreamSynchronize(p->s_out));
    return DS_OK;
}

ds_status ds_info(const void *handle, ds_info_t *out)
{
    if (!out || !valid_handle(handle, 0)) {
        set_error("ds_info: bad handle");
        return DS_E_ARG;
    }
    memset(out, 0, sizeof(*out));
    switch (reinterpret_cast<const HandleHeader *>(handle)->kind) {
    case KIND_INDEX: return info_index(reinterpret_cast<const ds_index *>(handle), out);
    case KIND_BATCH: return info_batch(reinterpret_cast<const ds_batch *>(handle), out);
    case KIND_LEARNED: return info_learned(reinterpret_cast<const ds_learned *>(handle), out);
    case KIND_LSEARCH: return info_lsearch(reinterpret_cast<const ds_lsearch *>(handle), out);
    }
    return DS_E_ARG;
}

void ds_free(void *handle)
{
    if (!valid_handle(handle, 0)) return;
    switch (reinterpret_cast<HandleHeader *>(handle)->kind) {
    case KIND_INDEX: free_index(reinterpret_cast<ds_index *>(handle)); break;
    case KIND_BATCH: free_batch(reinterpret_cast<ds_batch *>(handle)); break;
    case KIND_LEARNED: free_learned(reinterpret_cast<ds_learned *>(handle)); break;
    case KIND_LSEARCH: free_lsearch(reinterpret_cast<ds_lsearch *>(handle)); break;
    }
}

}  // extern "C"
