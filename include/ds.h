/*
 * ds.h -- C ABI of the GB300 direct-search library (libds.so).
 *
 * Interval lookup by "direct search" (F. Cannizzo, "A Fast and Vectorizable
 * Alternative to Binary Search in O(1) with Wide Applicability to Arrays of
 * Floating Point Numbers", arXiv 1506.08620).
 *
 * Problem (Section 2, "Formal Problem Statement"): given strictly increasing
 * knots X_0 < X_1 < ... < X_N and queries z, return for each z the index i
 * with X_i <= z < X_{i+1}, i.e. the index of the largest knot <= z.
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev are CUDA device pointers (or managed memory); the
 *    caller owns them and keeps them alive until the stream work that uses
 *    them has finished.  Pointers named *_host are host pointers (pinned for
 *    asynchronous copies).  `stream` is a cudaStream_t (NULL = legacy default
 *    stream).
 *  - Knots and queries are float32 (DS_F32) or float64 (DS_F64); results are
 *    int32.  Vector loads are used when Z and I are 16-byte aligned; other
 *    alignments take a scalar path with the same results.
 *  - Result domain: for every non-NaN query the result equals the definition
 *    above extended to the whole line: -1 for z < X_0, N for z >= X_N
 *    (Section 2 restricts z to [X_0, X_N); the table answers the same way
 *    outside it).  A NaN query gives -1 with DS_CHECKED and an unspecified
 *    value in [-1, N] without it.  Every memory access stays in bounds for
 *    every input.
 *  - Builds are synchronous (the table size R must be known on the host) and
 *    return only after the handle is usable; searches are asynchronous,
 *    stream-ordered and allocate nothing.
 *  - Errors are returned as ds_status; nothing is thrown across the ABI.
 *    ds_last_error() gives a message for the calling thread's last failure.
 *  - A handle may be searched from one stream at a time: entry points that
 *    use the handle's scratch words (batched and learned searches) race if
 *    two calls with the same handle overlap on the GPU.
 */
#ifndef DS_H
#define DS_H

#include <stdint.h>

#if defined(__GNUC__)
#define DS_API __attribute__((visibility("default")))
#else
#define DS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ds_status {
    DS_OK = 0,
    DS_E_ARG = 1,               /* bad argument: null pointer, size < 2, bad dtype/flag */
    DS_E_NOT_INCREASING = 2,    /* X not strictly increasing or not finite (Section 2) */
    DS_E_INDISTINGUISHABLE = 3, /* m(X_i - X_0) == m(X_{i-1} - X_0): Eq. distinguishable-exact */
    DS_E_OVERFLOW = 4,          /* m(H D_N) >= 2^32: Eq. overflowexact with Q = 32 */
    DS_E_TABLE_TOO_LARGE = 5,   /* (R+1) table entries exceed the byte budget */
    DS_E_NOMEM = 6,             /* device allocation failed */
    DS_E_CUDA = 7,              /* a CUDA runtime call failed (see ds_last_error) */
    DS_E_TIMEOUT = 8,           /* a bounded device wait gave up */
    DS_E_UNIMPLEMENTED = 9,
    DS_E_NO_CONVERGENCE = 10,   /* ComputeHR growth did not settle in 64 passes */
    DS_E_DEVICE = 11            /* a device-side check recorded an error */
} ds_status;

typedef enum ds_dtype { DS_F32 = 0, DS_F64 = 1 } ds_dtype;

/* build flags */
enum {
    DS_FMA = 1u,          /* f(z) = trunc(H z - W), W = H X_0: Section 4.9 "Fused Multiply Add", Eq. fma */
    DS_CACHE_LAYOUT = 2u, /* table of (K_j, X_{K_j}) pairs: Section 4.8, Algorithm directcache */
    DS_CHECKED = 4u,      /* NaN queries return -1 */
    DS_NO_SMEM = 8u,      /* never stage the table in shared memory (keep it L2/HBM resident) */
    DS_STRICT = 16u,      /* batched builds: an infeasible array is an error instead of a fallback */
    DS_GAP2 = 32u,        /* DirectGap2 (Section 4.7): f need only separate knots two apart
                             (Eq. f-monotonic-2), K_j = max{i : f(X_i) <= j} (Eq. kgeneral), answers by
                             Algorithm direct-2, i = t - [z < X_t] - [z < X_{t-1}]; a smaller table and
                             feasible on more arrays; not combined with DS_CACHE_LAYOUT; the same as
                             ds_build_q with q = 2 */
    DS_NO_FINGERPRINT = 64u, /* batched builds: the 8-bit knot fingerprints are not used, so every
                             query in a cell holding a knot reads the knot (the paper's correcting
                             comparison, always made) */
    DS_REFINE_H = 128u    /* single-array builds: when ComputeHR had to grow H, bisect the interval
                             between the last infeasible H and the final one for a smaller feasible
                             H (end of Section 4.4; every probe checks the whole array) */
};

typedef struct ds_index ds_index;     /* one knot array with its direct-search table */
typedef struct ds_batch ds_batch;     /* many independent knot arrays (CSR) */
typedef struct ds_learned ds_learned; /* learned-index form (one or many arrays) */
typedef struct ds_lsearch ds_lsearch; /* one knot array laid out for a logarithmic search (Section 3) */

/* Summary of a handle.  Fields that do not apply are 0. */
typedef struct ds_info_t {
    int32_t kind;           /* 1 = ds_index, 2 = ds_batch, 3 = ds_learned, 4 = ds_lsearch */
    int32_t dtype;          /* ds_dtype */
    uint32_t flags;
    int32_t n_arrays;
    int64_t n_knots;        /* total knots over all arrays */
    double H;               /* single array: grid density H (Section 4.2) */
    double W;               /* single array, DS_FMA: W = m(H X_0) (Eq. fma) */
    double X0, XN;          /* single array: first and last knot */
    uint64_t R;             /* single array: largest cell index; sum of R+1 over arrays otherwise */
    int64_t table_bytes;    /* device bytes of tables, knots copies and models */
    int64_t h_updates;      /* ComputeHR growth steps (all arrays) */
    int64_t hr_passes;      /* ComputeHR passes (single array) */
    double build_ms;        /* wall time of the build call */
    int32_t smem_resident;  /* single array: 1 if searches stage the table in shared memory */
    int32_t n_direct;       /* arrays served by direct search */
    int32_t n_learned;      /* arrays served by the learned predictor */
    int32_t n_fallback;     /* arrays served by the fixed-depth bisection (Algorithm binaryopt) */
    int64_t max_window;     /* learned: largest bounded window (largest cell population + 1) over arrays */
    int64_t train_steps;    /* learned: Adam steps run per model */
    double train_ms;        /* learned: time spent training */
    double final_loss;      /* learned: mean final training loss */
    uint64_t fallback_queries; /* learned: always 0 (the cell map is exact; no query falls back) */
    int32_t device_error;   /* nonzero if a device-side bounded wait or check recorded an error:
                               DS_DEVERR_TIMEOUT, or (range-checking build) DS_DEVERR_BOUNDS | site << 8 */
    int32_t gap_q;          /* single array: q of the table (1 Direct, 2 DirectGap2, ...); batched: largest q */
    int32_t search_launches; /* kernel launches per search call: 1 for one array; batched and learned
                                handles: the chunk planner and one search kernel, or two where a
                                handle's direct and learned arrays are searched by separate kernels */
    int32_t reserved_;
} ds_info_t;

/* ------------------------------------------------------------------------
 * Single array.
 * ------------------------------------------------------------------------ */

/* Build the direct-search table of one knot array (Section 4): validate X,
 * compute H and R with ComputeHR (Section 4.4, algorithm "Computation of H and
 * R"), fill K by Eq. indexdef, optionally pack (K_j, X_{K_j}) pairs
 * (Section 4.8).
 *   X_dev    n_knots = N+1 strictly increasing finite values of `dtype`; read
 *            once and copied (the handle does not keep the pointer).
 *   flags    DS_FMA | DS_CACHE_LAYOUT | DS_CHECKED | DS_NO_SMEM | DS_GAP2 | DS_REFINE_H.
 *            With DS_GAP2 (Section 4.7) ComputeHR separates the knot pairs
 *            (i, i+2) instead of (i, i+1), K follows Eq. kgeneral and searches
 *            use Algorithm direct-2; at most 2^30 knots, no DS_CACHE_LAYOUT.
 *   out      receives the handle (NULL on failure); release with ds_free.
 * Errors: DS_E_ARG, DS_E_NOT_INCREASING, DS_E_INDISTINGUISHABLE (Section 4.4
 * first counter-example; with DS_GAP2, m(X_{i+2} - X_0) == m(X_i - X_0)),
 * DS_E_OVERFLOW (second counter-example, Eq.
 * overflowexact), DS_E_NO_CONVERGENCE, DS_E_TABLE_TOO_LARGE (budget: half of
 * the free device memory, or the DS_TABLE_BUDGET_BYTES environment variable),
 * DS_E_NOMEM, DS_E_CUDA.  Synchronous: returns after the table is built. */
DS_API ds_status ds_build(const void *X_dev, int64_t n_knots, ds_dtype dtype, uint32_t flags, void *stream,
                   ds_index **out);

/* Gap-q (Section 4.7, Eq. f-monotonic-n): f need only separate knots q apart,
 * f(X_{i+q}) > f(X_i).  ComputeHR runs over the pairs (i, i+q) (pair distance
 * N when N < q) and K follows Eq. kgeneral.  A search answers from the table
 * alone when its cell holds no knot; otherwise it compares z with X_t and, if
 * z < X_t, bisects the knots X_{t-q} < z .. X_{t-1} (at most ceil(log2 q) more
 * comparisons; for q = 2 these are the comparisons of Algorithm direct-2).
 * A larger q gives a smaller table (about (X_N - X_0) / min(X_{i+q} - X_i)
 * cells), and arrays on which Direct is infeasible can become feasible.
 *   q             1 (Direct: the table of Eq. indexdef, as ds_build), >= 2, or
 *                 0 to choose, as the paper suggests for a memory budget, the
 *                 smallest q in 1..q_max for which ComputeHR succeeds and the
 *                 table image (K and X, each padded to 16 bytes) fits budget_bytes.
 *   q_max         the largest q tried when q == 0 (ignored otherwise).
 *   budget_bytes  used when q == 0; <= 0 means the shared-memory staging limit
 *                 of the search (so the table is staged per block).
 *   flags         DS_FMA | DS_CHECKED | DS_NO_SMEM | DS_REFINE_H, and DS_CACHE_LAYOUT for q = 1.
 * At most 2^30 knots for q >= 2.  ds_info reports the q built in gap_q.
 * Errors: as ds_build; DS_E_TABLE_TOO_LARGE when q == 0 and no q qualifies.
 * Synchronous. */
DS_API ds_status ds_build_q(const void *X_dev, int64_t n_knots, ds_dtype dtype, uint32_t flags, int32_t q,
                            int32_t q_max, int64_t budget_bytes, void *stream, ds_index **out);

/* Search m queries (Algorithm direct, Section 4.2): j = min(f(z), R),
 * t = K_j, I = t - [z < X_t]; for a DS_GAP2 index (Algorithm direct-2,
 * Section 4.7) I = t - [z < X_t] - [z < X_{t-1}], and for a Gap-q index
 * I = t - [z < X_t] - ... - [z < X_{t-q+1}] (X_{-1} = ... = X_0), at least -1.
 *   Z_dev  m queries of the index's dtype; I_dev  m int32 results.
 * m == 0 is a no-op.  Asynchronous on `stream`; allocates nothing; safe to
 * capture in a CUDA graph. */
DS_API ds_status ds_search(const ds_index *idx, const void *Z_dev, int64_t m, int32_t *I_dev, void *stream);

/* The same search with HOST buffers.  When both are pinned and mapped
 * (cudaHostAlloc, cudaHostRegister) the search kernel reads the queries from
 * and writes the results to host memory directly over the CPU-GPU link, with no
 * staging; otherwise (or with the environment variable DS_HOST_PIPE=1) queries
 * are copied in and results out in pipelined chunks (host->device, search,
 * device->host on separate streams), with device staging buffers allocated on
 * the first call and kept in the handle.  Returns when the last result has
 * been written to I_host. */
DS_API ds_status ds_search_host(ds_index *idx, const void *Z_host, int64_t m, int32_t *I_host, void *stream);

/* Sorted queries (the O(M + N) case of Section 1.2): merge Z into X instead
 * of searching each query.  The merged order places X_i before z when
 * X_i <= z; a query merged after a knots gets I = a - 1, the same answer as
 * ds_search (the largest i with X_i <= z; -1 below X_0, N at or above X_N).
 *   X_dev  n_knots (1 .. 2^31-1) strictly increasing values of `dtype`.
 *   Z_dev  m queries in non-decreasing order, no NaN; for other inputs the
 *          results are unspecified but every access stays in bounds.
 * Needs no index handle and no table; allocates nothing; asynchronous. */
DS_API ds_status ds_search_sorted(const void *X_dev, int64_t n_knots, ds_dtype dtype, const void *Z_dev, int64_t m,
                                  int32_t *I_dev, void *stream);

/* Counts of the samples in each interval (the distribution use case of
 * Section 1.2), by the index's direct search fused with counting:
 * counts_dev[i + 1] += #{z : answer(z) = i} for i = -1 .. N, so bin 0 counts
 * z < X_0 (and NaN), bin N+1 counts z >= X_N.  counts_dev: N+2 uint64, added
 * to (not cleared).  Shared-memory counters when N+2 of them fit in 96 KB,
 * otherwise global atomics.  Asynchronous; allocates nothing. */
DS_API ds_status ds_histogram(const ds_index *idx, const void *Z_dev, int64_t m, uint64_t *counts_dev, void *stream);

/* Read-only device views of the index's tables (for inspection and tests):
 * K (R+1 int32, Eq. indexdef or Eq. kgeneral, with the search's flags: bit 31
 * set when knot K_j lies in cell j, or for Eq. kgeneral when j < f(X_0); for
 * Eq. kgeneral bit 30 when knot K_j - 1 lies in cell j too), the library's copy
 * of X (N+1 values), and,
 * with DS_CACHE_LAYOUT, the (R+1) pairs (8 bytes for float32: int32 K_j then
 * float X_{K_j}; 16 bytes for float64: int32 K_j, 4 bytes of padding, double
 * X_{K_j}).  Any output pointer may be NULL. */
DS_API ds_status ds_index_tables(const ds_index *idx, const int32_t **K_dev, const void **X_dev,
                          const void **pairs_dev);

/* Copy the same tables into caller-owned device buffers (each may be NULL):
 * K_out (R+1 int32, flags cleared), X_out (N+1 values), pairs_out ((R+1) pairs, only with
 * DS_CACHE_LAYOUT).  Asynchronous on `stream`. */
DS_API ds_status ds_index_export(const ds_index *idx, int32_t *K_out_dev, void *X_out_dev, void *pairs_out_dev,
                                 void *stream);

/* ------------------------------------------------------------------------
 * Logarithmic searches (Section 3): the comparators of direct search.
 * ------------------------------------------------------------------------ */

typedef enum ds_lsearch_method {
    DS_LS_CLASSIC = 0,        /* Algorithm naivealg: low/high bisection, data-dependent trip count */
    DS_LS_CLASSICMOD = 1,     /* the same with conditional assignments, ceil(log2 N) iterations */
    DS_LS_LEADBIT = 2,        /* Algorithm binaryopt: leading-bit search, X padded with X_N to size Q */
    DS_LS_LEADBIT_NOPAD = 3,  /* Algorithm binaryoptnopad: min(r, N) after the first U iterations */
    DS_LS_OFFSET = 4,         /* Algorithm naiveoffset: start index and size (Knuth's Algorithm U) */
    DS_LS_EYTZINGER = 5       /* Algorithm eytzinger: breadth-first layout padded to 2^L - 1 */
} ds_lsearch_method;

/* Constants of a method for N+1 = n_knots knots, as the paper defines them
 * (host only, no device call):
 *   CLASSICMOD  consts[0] = ceil(log2 N) iterations
 *   LEADBIT     consts[0] = P = 2^floor(log2 N), consts[1] = Q = 1 + s_ubar,
 *               s_u = sum_{k=1..u} P / 2^(k-1), ubar = inf{u : s_u >= N}
 *   LEADBIT_NOPAD consts[0] = P, consts[1] = U = sup{u : s_u <= N}
 *   OFFSET      consts[0..2] = F = floor((N+1)/2), S = N+1-F, J = floor(log2(N+1))
 *   EYTZINGER   consts[0] = L = 1 + floor(log2(N+2))
 * *layout_len = elements of the method's layout (N+1, Q, or 2^L - 1). */
DS_API ds_status ds_lsearch_constants(int32_t method, int64_t n_knots, int64_t consts[4], int64_t *layout_len);

/* Lay out one knot array for `method` (a copy of X, right-padded with X_N for
 * LEADBIT, breadth-first for EYTZINGER; float64 knots are stored as
 * order-preserving integer keys).  X_dev: n_knots (2..2^30) strictly
 * increasing values (not validated: the methods are exact only on sorted X);
 * the layout may hold at most 2^30 elements (DS_E_ARG otherwise).
 * flags: DS_CHECKED | DS_NO_SMEM.  Synchronous. */
DS_API ds_status ds_lsearch_build(const void *X_dev, int64_t n_knots, ds_dtype dtype, int32_t method,
                                  uint32_t flags, void *stream, ds_lsearch **out);

/* The same answers as ds_search (the largest i with X_i <= z; -1 below X_0
 * and for NaN, N at or above X_N) by the handle's logarithmic method.
 * Asynchronous; allocates nothing. */
DS_API ds_status ds_lsearch_search(const ds_lsearch *h, const void *Z_dev, int64_t m, int32_t *I_dev, void *stream);

/* ------------------------------------------------------------------------
 * Many independent arrays ("vectorial problem" of Section 2, batched).
 * ------------------------------------------------------------------------ */

/* Build one direct-search table per array.  Array a owns the knots
 * Xcat_dev[x_off[a] .. x_off[a+1]-1] (device CSR offsets, n_arrays+1 int64,
 * x_off[0] = 0, at least 2 knots per array).  Each array is validated and
 * gets its own H, R and K exactly as ds_build would compute them.  An array
 * on which direct search is infeasible is served by the fixed-depth bisection
 * of Algorithm binaryopt (the log-time fall-back the Conclusion names) unless
 * DS_STRICT is set, in which case the build fails with that array's status.
 * Flags: DS_FMA | DS_CHECKED | DS_STRICT | DS_NO_SMEM | DS_NO_FINGERPRINT.
 * K is held as a rank table (not in the paper's layout): with pairs (i, i+1)
 * a cell holds at most one knot, so K_j = #{i : F_i < j}; one 8-byte word per
 * 32 cells holds K at the group's first cell and which cells hold a knot, and
 * one byte per knot an 8-bit fingerprint of its position within its cell, so
 * that a query reads the knot only when the fingerprints are equal;
 * DS_NO_FINGERPRINT turns the fingerprints off.  Synchronous. */
DS_API ds_status ds_batch_build(const void *Xcat_dev, const int64_t *x_off_dev, int32_t n_arrays, ds_dtype dtype,
                         uint32_t flags, void *stream, ds_batch **out);

/* Search every array's queries in one persistent launch: queries of array a
 * are Zcat_dev[z_off[a] .. z_off[a+1]-1] (device CSR, n_arrays+1 int64), their
 * results (local indices into array a) go to the same positions of Icat_dev.
 * Asynchronous, allocation-free and capturable; uses the handle's scratch. */
DS_API ds_status ds_batch_search(const ds_batch *b, const void *Zcat_dev, const int64_t *z_off_dev, int32_t *Icat_dev,
                          void *stream);

/* Launch parameters of the batched search. */
typedef struct ds_tune_t {
    int32_t block;       /* threads per block: 128, 256, 512, or 1024 (direct arrays only, items 1,
                            smem_limit >= 0; otherwise it runs as 512); other values run as 256 */
    int32_t items;       /* vectors of queries per thread per tile: 1, 2 or 4 (others run as 4) */
    int32_t smem_limit;  /* largest per-array table (bytes) staged in shared memory; 0 = never (blocks
                            claim chunks); -1 = never, and each warp claims its own chunks */
    int32_t blocks_per_sm;
    float ms;            /* measured time of the chosen configuration (autotune output) */
} ds_tune_t;

/* Time a fixed set of launch configurations on the given queries (each run
 * several times with CUDA events on `stream`), keep the fastest in the handle
 * and return it in *best.  The outputs are overwritten with valid results.
 * Synchronous. */
DS_API ds_status ds_batch_autotune(ds_batch *b, const void *Zcat_dev, const int64_t *z_off_dev, int32_t *Icat_dev,
                            void *stream, ds_tune_t *best);
DS_API ds_status ds_batch_set_tune(ds_batch *b, const ds_tune_t *cfg);
DS_API ds_status ds_batch_get_tune(const ds_batch *b, ds_tune_t *cfg);

/* Per-array parameters (host copies) for inspection: H, W (as double), R and
 * the mode (0 = direct, 2 = bisection fall-back) of array a. */
DS_API ds_status ds_batch_array(const ds_batch *b, int32_t a, double *H, double *W, uint64_t *R, int32_t *mode);

/* ------------------------------------------------------------------------
 * Learned index (not in the paper): a 1 -> 32 -> 32 -> 1 ReLU network
 * predicting the index from u = (z - X_0) / (X_N - X_0), trained on the GPU by
 * this library's own forward/backward/Adam kernels on the pairs (X_i, i) and
 * on exact answers of sampled queries.  Its largest prediction error over all
 * knots is recorded at build time (e_lo, e_hi: ds_learned_array).  It is
 * served as a learned cell map for direct search (Section 4.2's method on
 * cells of equal predicted rank instead of equal width): the prediction,
 * sampled at G uniform points of u and made non-decreasing (by
 * rearrangement), gives
 * C = ceil(cells_per_knot (N+1)) cells; f(z) is that map rounded down to a
 * cell, computed in float32 so that f is monotone; K_j = #{i : f(X_i) < j}
 * as in Eq. indexdef; and a query answers K_j - 1 plus the number of knots of
 * its cell j that are <= z (none for an empty cell; otherwise X_{K_j} and
 * X_{K_{j+1}-1} decide, and between them a bisection of the cell).  Every
 * answer is exact by construction: the cells replace the certificate.  The
 * bounded compare window of a query is its cell, at most max_window - 1 knots
 * (ds_info), recorded at build time.  Each array keeps the network's map
 * only where its cells are better balanced than those of the linear model
 * (ds_learned_cells).  Arrays on which direct search is
 * feasible with at most max_cells_per_knot cells per knot use plain direct
 * search instead (unless DS_LEARNED_FORCE).
 * ------------------------------------------------------------------------ */
enum {
    DS_LEARNED_FORCE = 1u,    /* use the learned map even where direct search is feasible */
    DS_LEARNED_LINEAR = 2u    /* no network: the map of the linear model N u, i.e. cells of equal width in z
                                 (the method "without it", for comparison) */
};

typedef struct ds_learned_cfg {
    int32_t steps;       /* Adam steps per model (0 = untrained initial network); default 6000 */
    int32_t batch;       /* samples per step */
    int32_t n_queries;   /* exact-answer query samples per model, in addition to the knots */
    float lr;            /* Adam step size */
    uint64_t seed;       /* Philox-4x32-10 key for initialisation and sampling */
    uint32_t flags;      /* DS_LEARNED_* */
    int32_t max_cells_per_knot; /* direct search only where (R+1) <= this x (N+1) (its table stays small);
                                   other feasible arrays use the learned map; <= 0: no limit */
    float cells_per_knot;       /* cells C of a learned map per knot; 0 (the default): 1, or 2 for a
                                   handle that holds the knot values (ds_learned_build_xy with Y);
                                   C <= 2^32 - 2 */
    int32_t reserved[3];
} ds_learned_cfg;

DS_API void ds_learned_cfg_default(ds_learned_cfg *cfg);

/* Build the learned form.  Single array: x_off_dev = NULL, n_arrays = 1 and
 * n_knots_if_single = N+1.  Batched: device CSR offsets as in ds_batch_build.
 * The cell tables take 2 bytes per cell (16-byte blocks of 8 cells: K of the
 * first cell and 12-bit differences; a block whose cells hold more than 4095
 * knots keeps its 9 values as uint32 in an overflow area).  Synchronous. */
DS_API ds_status ds_learned_build(const void *Xcat_dev, const int64_t *x_off_dev, int32_t n_arrays,
                           int64_t n_knots_if_single, ds_dtype dtype, const ds_learned_cfg *cfg, void *stream,
                           ds_learned **out);

/* The same build with the knot values Y of the interpolation (Ycat_dev: same
 * dtype and CSR layout as Xcat_dev, copied): the handle stores every knot
 * with its value as an (X_i, Y_i) pair, so that a lookup's four operands
 * X_i, Y_i, X_{i+1}, Y_{i+1} lie in 16 contiguous bytes (float32; 32 for
 * float64): the paper's DirectCache idea (Section 4.8, keeping what one
 * lookup reads together) carried to the interpolation.  Searches interpolate
 * from them (ds_learned_search with Ycat_dev = NULL); the direct arrays of
 * such a handle compare with the knot itself instead of its fingerprint, as
 * the interpolation reads the knot's pair anyway.  Synchronous. */
DS_API ds_status ds_learned_build_xy(const void *Xcat_dev, const void *Ycat_dev, const int64_t *x_off_dev,
                                     int32_t n_arrays, int64_t n_knots_if_single, ds_dtype dtype,
                                     const ds_learned_cfg *cfg, void *stream, ds_learned **out);

/* Search: single array: z_off_dev = NULL and m queries; batched: device CSR
 * z_off_dev (m ignored).  With y_out_dev non-NULL the linear interpolant
 * y = Y_i + (Y_{i+1} - Y_i) ((z - X_i) / (X_{i+1} - X_i)) (each step rounded
 * once) is written for every query whose index lies in [0, N-1] (the use case
 * of the Introduction); other queries get NaN.  The values Y are the handle's
 * own (ds_learned_build_xy; Ycat_dev must then be NULL) or the caller's
 * Ycat_dev (same dtype and CSR layout as X; a handle from ds_learned_build).
 * y_out_dev 16-byte aligned takes the vector path.  Asynchronous,
 * allocation-free. */
DS_API ds_status ds_learned_search(const ds_learned *L, const void *Zcat_dev, const int64_t *z_off_dev, int64_t m,
                            const void *Ycat_dev, void *y_out_dev, int32_t *Icat_dev, void *stream);

/* The same search with HOST buffers (the end-to-end call): Zcat_host (m
 * queries), Icat_host (m results) and y_out_host (m interpolated values, only
 * for a handle from ds_learned_build_xy, or NULL) are read and written by the
 * search kernel in place over the CPU-GPU link, with no staging copies;
 * page-locked mapped memory (cudaHostAlloc, cudaHostRegister) is used as it
 * is, other host memory is registered for the call and unregistered after it.
 * z_off_host: host CSR offsets (n_arrays + 1 int64; m is then z_off[n_arrays]),
 * or NULL for one array of m queries; copied to a device buffer the handle
 * allocates on its first use.  Returns after the results are in host memory
 * (the call synchronizes `stream`). */
DS_API ds_status ds_learned_search_host(ds_learned *L, const void *Zcat_host, const int64_t *z_off_host, int64_t m,
                                        void *y_out_host, int32_t *Icat_host, void *stream);

/* Time the launch configurations of ds_batch_autotune on these queries (the
 * same engine serves the learned form), keep the fastest in the handle and
 * return it in *best.  Single array: z_off_dev = NULL and m queries.  With
 * y_out_dev (and Ycat_dev, as for ds_learned_search) the configurations are
 * timed with the interpolation.  A handle with direct and learned arrays
 * searches each group with its own kernel launch: after the common
 * configuration the autotuner tunes each launch with the other held fixed,
 * keeps both in the handle, and returns the direct launch's in *best (with
 * the time of the whole search).  The outputs are overwritten with valid
 * results.  Synchronous. */
DS_API ds_status ds_learned_autotune(ds_learned *L, const void *Zcat_dev, const int64_t *z_off_dev, int64_t m,
                                     const void *Ycat_dev, void *y_out_dev, int32_t *Icat_dev, void *stream,
                                     ds_tune_t *best);
/* Set or read the launch configuration of the learned search, as
 * ds_batch_set_tune / ds_batch_get_tune (DS_E_ARG for an smem_limit outside
 * [-1, the device's opt-in limit - 2048] or a configuration that cannot be
 * resident).  Set applies the configuration to every launch of the search;
 * get reads the first launch's (the direct arrays' on a handle with direct
 * and learned arrays). */
DS_API ds_status ds_learned_set_tune(ds_learned *L, const ds_tune_t *cfg);
DS_API ds_status ds_learned_get_tune(const ds_learned *L, ds_tune_t *cfg);

/* Host copy of array a's network parameters (1153 floats: W1[32] b1[32]
 * W2[32][32] b2[32] w3[32] b3) and its recorded error bounds: every knot i
 * satisfies floor(p(X_i)) - e_lo <= i <= floor(p(X_i)) + e_hi for the served
 * prediction p.  mode: 0 direct, 1 learned, 2 bisection. */
DS_API ds_status ds_learned_array(const ds_learned *L, int32_t a, float *theta_host, int32_t *e_lo, int32_t *e_hi,
                           int32_t *mode);

/* Cell table of array a (zeros for an array served by plain direct search):
 * cells C, the largest number of knots in one cell, the number of cells
 * holding a knot, the number of escaped blocks (8 cells holding more than 4095
 * knots, whose K values are kept as uint32), the mean cell population seen by
 * queries distributed like the knots (sum of squared populations / (N + 1)),
 * and 1 if the map comes from the network (0: from the linear model, which
 * the build keeps where the network's map gives the larger mean population).
 * Any output may be NULL. */
DS_API ds_status ds_learned_cells(const ds_learned *L, int32_t a, uint64_t *cells, int32_t *max_pop,
                                  int64_t *nonempty, int64_t *escaped, double *mean_pop, int32_t *from_network);

/* Copy K_0 .. K_C (C + 1 uint32, decoded; K_0 = 0, K_C = N + 1) of a learned
 * array's cell table into caller-owned device memory.  Asynchronous. */
DS_API ds_status ds_learned_export_cells(const ds_learned *L, int32_t a, uint32_t *K_out_dev, void *stream);

/* The training kernels on explicit inputs (used to check gradients):
 * forward output of the network for n inputs u; mean squared error over n
 * samples against targets y and its gradient (1153 floats); one Adam step
 * (t is 1-based) on 1153 parameters in place. */
DS_API ds_status ds_mlp_forward(const float *theta_dev, const float *u_dev, int64_t n, float *out_dev, void *stream);
DS_API ds_status ds_mlp_loss_grad(const float *theta_dev, const float *u_dev, const float *y_dev, int64_t n,
                           float *grad_dev, float *loss_dev, void *stream);
DS_API ds_status ds_adam_step(float *theta_dev, float *m_dev, float *v_dev, const float *grad_dev, int32_t t, float lr,
                       void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free table build.  The paper has no counterpart to this entry
 * point; it exists for callers that may not allocate device memory when
 * they build a table: code under a host framework that owns every device
 * allocation (a fixed pool handed out at start-up), real-time loops where the
 * implicit device synchronisation of cudaMalloc/cudaFree is not acceptable,
 * and plug-ins that are forbidden to allocate after initialisation.
 *
 * It computes H, W and R exactly as ds_build does (ComputeHR, Section 4.4)
 * and writes the K table of Eq. indexdef (R+1 int32) into the caller's
 * buffer K_out_dev of K_capacity entries.  Its scratch is a fixed array inside
 * the library's device image: DS_STATIC_MAX_KNOTS cells (4 bytes each) plus
 * one 256-byte ComputeHR state, about 1 MiB, held by every GPU that loads the
 * library until the process exits.  Arrays with more than DS_STATIC_MAX_KNOTS
 * knots are rejected with DS_E_ARG; a K buffer smaller than R+1 entries is
 * rejected with DS_E_ARG after *R_out has been set, so the caller can size a
 * new buffer.  The call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine) and returns after the table is written.
 *
 * Every call looks up the scratch array's device address on the current
 * device (cudaGetSymbolAddress, which allocates nothing), so the call stays
 * valid after cudaDeviceReset.  The call reads H, W and R back to the host
 * and synchronizes `stream`: it must not be made while the stream is being
 * captured.  Every call uses the same scratch and re-initialises the parts
 * that must start from a known value; calls whose GPU work overlaps (from two
 * streams or two host threads) race on the scratch.  An infeasible array
 * returns the status and message of ds_build (with the offending knot).
 * flags: 0 or DS_FMA.
 * ------------------------------------------------------------------------ */
#define DS_STATIC_MAX_KNOTS 262144
DS_API ds_status ds_build_table_static(const void *X_dev, int64_t n_knots, ds_dtype dtype, uint32_t flags,
                                       int32_t *K_out_dev, int64_t K_capacity, double *H_out, double *W_out,
                                       uint64_t *R_out, void *stream);

/* ------------------------------------------------------------------------
 * Handles and diagnostics.
 * ------------------------------------------------------------------------ */
DS_API ds_status ds_info(const void *handle, ds_info_t *out); /* any handle */
DS_API void ds_free(void *handle);                            /* any handle; NULL is a no-op */
DS_API const char *ds_status_str(ds_status s);
DS_API const char *ds_last_error(void);
DS_API int32_t ds_abi_version(void);

/* ------------------------------------------------------------------------
 * Device error words (ds_info_t.device_error).  DS_DEVERR_TIMEOUT: a bounded
 * wait of a kernel gave up (the kernel returned early).  DS_DEVERR_BOUNDS |
 * site << 8: only in the range-checking build of the library
 * (libds_bounds.so, compiled with -DDS_DEBUG_BOUNDS; the Python package loads
 * it when DS_LIBRARY=bounds), the first table or knot gather of a search whose
 * index fell outside its table; the gather read entry 0 instead.  The normal
 * build has no such checks (indices are in range by construction).
 * ------------------------------------------------------------------------ */
enum { DS_DEVERR_TIMEOUT = 1, DS_DEVERR_BOUNDS = 2 };
enum {
    DS_BS_K = 1,       /* single array: K_j (R + 1 cells), or its cache-layout pair */
    DS_BS_K16 = 2,     /* single array: packed block of cells */
    DS_BS_X = 3,       /* knots X_t (N + 1), or their (X, Y) pairs */
    DS_BS_RANK = 4,    /* batched: rank word of a cell */
    DS_BS_FPRINT = 5,  /* batched: knot fingerprint */
    DS_BS_CMAP = 6,    /* learned: macro cell of the cell map */
    DS_BS_CBLOCK = 7,  /* learned: cell-table block */
    DS_BS_CESC = 8,    /* learned: escaped block's values */
    DS_BS_Y = 9,       /* the caller's knot values Y_i (interpolation) */
    DS_BS_LAYOUT = 10  /* logarithmic search: element of the layout */
};

/* ------------------------------------------------------------------------
 * Test aids (the paper has no counterpart: they let tests reach the error
 * paths of every build on the host, with no fault on the device).
 *
 * ds_debug_fail_alloc(nth): the device allocation nth + 1 from now (nth = 0:
 * the next one) made by this library fails as if the device were out of
 * memory (cudaErrorMemoryAllocation, reported as DS_E_NOMEM) without
 * allocating; nth < 0 turns the hook off.  One failure per call; process-wide.
 * ds_debug_alloc_stats: the library's live device allocations (count and
 * bytes; either pointer may be NULL).  A handle's allocations stay live until
 * ds_free; a call that fails leaves none behind.  ds_build_table_static
 * allocates nothing and is not counted.
 * ------------------------------------------------------------------------ */
DS_API ds_status ds_debug_fail_alloc(int64_t nth);
DS_API ds_status ds_debug_alloc_stats(int64_t *live_count, int64_t *live_bytes);

#ifdef __cplusplus
}
#endif

#endif /* DS_H */
