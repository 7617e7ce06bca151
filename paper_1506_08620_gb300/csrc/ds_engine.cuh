// ds_engine.cuh -- host side of the multi-array engine shared by ds_batch and
// ds_learned: per-array descriptors, one device blob holding every array's
// image, the chunk planner's scratch, the tuned launch configuration and the
// cached CUDA graph of a search.
#pragma once

#include <vector>

#include "ds_multi_kernels.cuh"

namespace ds {

constexpr long long SEG_KNOTS = 1 << 16;  // knots per build segment
// tiles per search chunk claimed by a block: direct-only handles 32 (16: 472.5,
// 32: 478.5 G/s on the 4096-array workload), others 16 (the learned workloads)
constexpr int CHUNK_TILES_DIRECT = 32;
constexpr int CHUNK_TILES = 16;
constexpr int CHUNK_TILES_WARP = 32;      // tiles per search chunk claimed by a warp

struct Engine {
    int dtype = 0;
    uint32_t flags = 0;
    int n_arrays = 0;
    long long n_knots = 0;
    DeviceProps props;
    ArrDesc *desc_dev = nullptr;
    std::vector<ArrDesc> desc_host;
    unsigned char *blob = nullptr;
    size_t blob_bytes = 0;
    size_t table_bytes = 0;
    long long *chunk_off = nullptr;
    int *order = nullptr;  // claim order of the arrays: most knots first (within each launch's group)
    std::vector<int> order_host;  // its host copy (read by an asynchronous upload)
    int split = 0;  // > 0: direct arrays at claim positions [0, split), learned ones after, one launch each
    unsigned long long *counter = nullptr;  // [0] chunk counter
    int *dev_err = nullptr;
    unsigned char *ctab = nullptr;  // learned arrays' cell tables
    size_t ctab_bytes = 0;
    bool xy = false;                // knots stored as (X_i, Y_i) pairs
    ds_tune_t tune = {};
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    const void *gkey[6] = {};
    ds_tune_t gtune = {};
    ds_tune_t tune2 = {};   // a split handle's learned launch (tune: its direct launch, or the only one)
    ds_tune_t gtune2 = {};
    long long h_updates = 0;
    unsigned long long R_total = 0;
    int n_direct = 0, n_learned = 0, n_fallback = 0;
    bool fingerprints = false;  // the knot fingerprints of the rank tables are used
    bool fast_cells = false;    // float, every direct R < 2^24 - 1: one conversion per query
    double build_ms = 0;
};

// Validate, ComputeHR per array, lay out and fill all tables.  Arrays with
// force_other[a] set (or infeasible for direct search) get mode other_mode
// (MODE_LEARNED) or MODE_BISECT.
// max_cells_per_knot > 0: a feasible array with (R+1) > max_cells_per_knot (N+1)
// also gets other_mode.  Ycat (same CSR as Xcat, or nullptr): the knot values,
// stored with the knots as intervals (X_i, Y_i, X_{i+1}, Y_{i+1}).  A learned array gets room for
// its cell map in the blob (filled later by the learned build).
ds_status engine_build(Engine *e, const void *Xcat, const void *Ycat, const long long *x_off_dev, int n_arrays,
                       ds_dtype dtype, uint32_t flags, cudaStream_t s, const std::vector<char> *force_other,
                       int other_mode, std::vector<long long> *x_off_host, std::vector<HRState> *hs_out,
                       double max_cells_per_knot = 0.0);
// Interpolation: y_out non-null; the knot values come from the stored
// intervals (Y nullptr) or from the caller's Y.
// host_io: Z, I and y_out are host memory mapped into the device (no bulk L2
// prefetch of the query stream).  t configures the launch (a split handle's
// direct launch), t2 a split handle's learned launch (nullptr: t as well).
ds_status engine_launch_direct(const Engine *e, const ds_tune_t &t, const void *Z, const long long *z_off,
                               long long m_single, const void *Y, void *y_out, int32_t *I, cudaStream_t s,
                               bool host_io = false, const ds_tune_t *t2 = nullptr);
ds_status engine_launch(Engine *e, const void *Z, const long long *z_off, long long m_single, const void *Y,
                        void *y_out, int32_t *I, cudaStream_t s);
ds_status engine_autotune(Engine *e, const void *Z, const long long *z_off, long long m_single, const void *Y,
                          void *y_out, int32_t *I, cudaStream_t s, ds_tune_t *best_out);
// Macro cells G of a learned array's cell map for N + 1 knots: a power of two
// in [LMAP_MIN, LMAP_MAX], about (N + 1) / 4.
int lmap_cells(long long n_knots);
ds_status engine_set_tune(Engine *e, const ds_tune_t &cfg);
void engine_free(Engine *e);
ds_tune_t default_tune();

}  // namespace ds
