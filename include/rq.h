/*
 * rq.h -- C ABI of librq: IVF-RaBitQ index build and search on one GB300.
 *
 * The method is IVF-RaBitQ as described in "Ascend-RaBitQ" (arXiv 2605.16007):
 * an IVF index (Section 2.1.2) whose lists hold 1-bit RaBitQ codes of the
 * normalised residuals (Section 2.2.1, Eqs. 1-3), searched with the RaBitQ
 * distance estimator (Section 2.2.2, Eqs. 4-5) evaluated with bitwise AND +
 * popcount over a 4-bit scalar-quantised query (Section 3.3.2), a bounded
 * top-k over lists visited in centroid order (Section 3.3.3), and an exact
 * re-rank of the candidates on the raw vectors (Section 3.3.4).
 *
 * Conventions that hold for every call:
 *  - Every call returns rq_status; on failure rq_last_error() returns a
 *    thread-local message describing the first error of the calling thread.
 *  - Pointers named "host or device" may point to host memory (pageable or
 *    pinned) or to device memory of the index's GPU; the library checks with
 *    cudaPointerGetAttributes. Inputs are never modified; host inputs are
 *    copied. Outputs are always caller-allocated.
 *  - A call that writes host outputs returns after they are written. A call
 *    whose outputs are all device memory only enqueues its work on `stream`
 *    (a cudaStream_t, NULL = the legacy default stream) and returns.
 *  - Vectors are row-major float32 (or uint8 for RQ_U8 raw data). D_p is the
 *    dimension rounded up to a multiple of 128; vectors are zero-padded to it.
 *  - Ids are 0-based row numbers of the base matrix given to rq_build.
 *  - Distances are squared L2. Where fewer than k results exist, the output
 *    is padded with id -1 and distance +inf.
 *  - Limits: 1 <= dim <= 2048, n < 2^32, 1 <= nlist <= min(n, 2^20),
 *    1 <= nprobe <= min(nlist, 4096), 1 <= k <= n_rerank <= 4096
 *    (or n_rerank = 0, see rq_search).
 */
#ifndef RQ_H
#define RQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point is exported from librq.so (the library is otherwise
 * built with hidden symbols). */
#if defined(__GNUC__)
#define RQ_API __attribute__((visibility("default")))
#else
#define RQ_API
#endif

typedef enum rq_status {
  RQ_OK = 0,
  RQ_ERR_INVALID_ARG = 1,     /* an argument is out of range or inconsistent */
  RQ_ERR_OOM = 2,             /* a device or host allocation failed */
  RQ_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  RQ_ERR_TIMEOUT = 4,         /* a bounded wait gave up (device or host) */
  RQ_ERR_BUSY = 5,            /* the server is full; retry later */
  RQ_ERR_IO = 6,              /* file read/write failed or bad file */
  RQ_ERR_NOT_IMPLEMENTED = 7, /* the request needs a feature not built */
  RQ_ERR_DEVICE = 8           /* a kernel flagged an internal error */
} rq_status;

typedef enum rq_dtype { RQ_F32 = 0, RQ_U8 = 1 } rq_dtype;

/* How the code scan (Section 3.3.1-3.3.2) is scheduled.
 *  PLAIN:   one thread block per (query, probed list, chunk of 1024 list
 *           vectors), launched per batch (the query-level schedule the paper
 *           starts from, Section 3.3.1); suits few queries per list.
 *  GROUPED: one persistent launch walks a work list of (list, vector block,
 *           group of queries probing that list); the block's codes are loaded
 *           once for the whole group and the popcount estimator runs per pair.
 *  MMA:     as GROUPED, but the integer inner products of a 128-vector tile
 *           with a group of quantised queries come from one tcgen05 tensor-core
 *           MMA (codes and 4-bit query digits both held exactly as FP8).
 *  AUTO:    the fastest of the above for this index, measured by rq_autotune
 *           (GROUPED when no tuning result exists).
 * All modes return bit-identical results. */
typedef enum rq_scan_mode {
  RQ_SCAN_AUTO = 0,
  RQ_SCAN_PLAIN = 1,
  RQ_SCAN_GROUPED = 2,
  RQ_SCAN_MMA = 3
} rq_scan_mode;

/* The estimator of the code scan.
 *  BQ4: the query residual quantised to B_q = 4 bits, the inner product of
 *       Eq. 4 evaluated exactly as an integer by AND + popcount over four
 *       bit-planes (or a tensor-core product), Section 3.3.2.
 *  LUT: the paper's FastScan form: the full-precision residual, float32
 *       tables of 256 entries per 8 dimensions gathered by code byte
 *       (Section 3.3.2); runs on the query-level (PLAIN) schedule; D_p <= 256.
 * The exact re-rank and everything else are the same for both. */
typedef enum rq_estimator { RQ_EST_BQ4 = 0, RQ_EST_LUT = 1 } rq_estimator;

typedef struct rq_build_opts {
  int32_t kmeans_iters; /* Lloyd iterations (default 10; 0 keeps the
                           initial rows as centroids) */
  int32_t keep_float_raw; /* 0 (default): a float32 base whose values are
                           all integers in [0, 255] is kept for the re-rank
                           as uint8 (lossless: every re-rank distance is
                           unchanged, the gather reads 4x fewer bytes);
                           1: always keep float32 */
  int64_t train_size;   /* rows of the k-means training subset; 0 = all rows */
  int32_t raw_on_host;  /* 1: the re-rank reads the raw rows from the
                           caller's base buffer in host memory (page-locked:
                           cudaHostAlloc, cudaMallocHost or
                           cudaHostRegister), through the GPU's mapping of
                           it, instead of a device copy; the base stays in its
                           own dtype. The index keeps a reference: the caller
                           owns the buffer and keeps it alive and unchanged
                           until rq_free. Any other base is INVALID_ARG. 0
                           (default): a device copy (Section 3.3.4 re-ranks
                           on the host to spare the device the raw vectors;
                           here the GPU reads them from host memory) */
} rq_build_opts;

/* Optional device buffers that receive the intermediates of one rq_search
 * call, for stage-by-stage checks. Any field may be NULL. nprobe_max and
 * nsel_max are the largest nprobe and the largest selection size (n_rerank, or
 * k when n_rerank is 0) of the call. */
typedef struct rq_search_dump {
  float* qrot;           /* nq x D_p: P^T q (rotated, zero-padded query) */
  int32_t* probe_ids;    /* nq x nprobe_max: probed lists, ascending (d, id) */
  float* probe_dist;     /* nq x nprobe_max: ||q' - P^T c||^2 of each */
  float* qparams;        /* nq x nprobe_max x 4: vl, delta, nq2, Sq (as float) */
  uint8_t* planes;       /* nq x nprobe_max x 4 x (D_p/8): query bit-planes */
  uint32_t* bound;       /* nq: pruning bound (orderable distance) */
  uint64_t* selected;    /* nq x nsel_max: the selected (estimate, id) keys,
                            padded with all ones; ascending when n_rerank
                            is 0, otherwise in no particular order */
  int32_t* n_candidates; /* nq: candidates that survived pruning */
} rq_search_dump;

/* Stages of one search, for rq_search_opts.stage_ms. */
typedef enum rq_stage {
  RQ_STAGE_ROTATE = 0,   /* q' = P^T q */
  RQ_STAGE_PROBE = 1,    /* centroid distances */
  RQ_STAGE_QUANTIZE = 2, /* per query, one fused step: nprobe selection,
                            residuals to 4-bit planes; the first pruning
                            bound too, except in the tensor-core form */
  RQ_STAGE_BOUND = 3,    /* tensor-core form: the first pruning bound (one
                            grouped pass over the queries' windows, then
                            the n_sel-th smallest per query); other forms
                            read 0 (inside RQ_STAGE_QUANTIZE) */
  RQ_STAGE_WORKLIST = 4, /* (pairs are grouped by list inside
                            RQ_STAGE_QUANTIZE; reads 0) */
  RQ_STAGE_SCAN = 5,     /* the code scan */
  RQ_STAGE_SELECT = 6,   /* candidate collection: survivor keys from the masks */
  RQ_STAGE_RERANK = 7,   /* selection of the n_rerank smallest and exact re-rank */
  RQ_STAGE_COUNT = 8
} rq_stage;

typedef struct rq_search_opts {
  int32_t scan_mode;     /* rq_scan_mode (default AUTO) */
  int32_t no_prune;      /* 1: keep every candidate (no bound); default 0 */
  int32_t use_graph;     /* 1: replay the launch sequence from a CUDA graph
                            cached per (stream, shape); default 0 */
  int32_t test_stall;    /* 0 in normal use. Test hook of the failure path:
                            1 makes the pipelined scan (GROUPED or MMA) hold
                            back its first stage, so that its bounded wait
                            (1 ms under this hook) runs out; the search then
                            returns RQ_ERR_TIMEOUT (synchronous calls) or
                            leaves the code in rq_device_error. */
  rq_search_dump* dump;  /* NULL, or buffers for the intermediates */
  float* stage_ms;       /* NULL, or host array of RQ_STAGE_COUNT floats that
                            receives each stage's device time (CUDA events on
                            the search stream; the call then waits for the
                            device and does not use a graph) */
  int32_t plain_chunk;   /* PLAIN: list vectors per thread block, 1024, 2048
                            or 4096 (0 = 1024, or the tuned size under AUTO;
                            D_p above 256 always uses 1024) */
  int32_t estimator;     /* rq_estimator (default BQ4) */
} rq_search_opts;

typedef struct rq_stats {
  int64_t n;             /* vectors in the index */
  int32_t dim;           /* input dimension D */
  int32_t dim_pad;       /* D_p */
  int32_t nlist;         /* lists */
  int32_t code_bytes;    /* D_p / 8 */
  int64_t min_list;      /* shortest list */
  int64_t max_list;      /* longest list */
  int64_t index_bytes;   /* device bytes of codes, factors, ids, centroids, P */
  int64_t raw_bytes;     /* device bytes of the raw vectors kept for re-rank */
  int32_t auto_scan_mode; /* the scan mode RQ_SCAN_AUTO resolves to */
  int32_t reserved;
} rq_stats;

/* Read-only device pointers into an index (valid until rq_free). Lists are
 * stored back to back in list order; inside a list, in ascending row id. */
typedef struct rq_index_view {
  int64_t n;
  int32_t dim, dim_pad, nlist, code_bytes;
  const double* P;        /* D_p x D_p, float64, row-major; z = P^T u */
  const float* centroids; /* nlist x dim */
  const float* cR;        /* nlist x D_p: P^T c, float32 */
  const int64_t* offsets; /* nlist + 1: list l is slots [offsets[l], offsets[l+1]) */
  const uint8_t* codes;   /* n x code_bytes: bit d of slot s = byte d/8, bit d%8 */
  const float* r;         /* n: ||x - c|| of each slot */
  const float* alpha;     /* n: <P b / sqrt(D_p), u> of each slot (Eq. 3) */
  const float* factors;   /* n x 2: {r^2, r / (sqrt(D_p) alpha)} of each slot */
  const uint32_t* ids;    /* n: row id held by each slot */
  const int32_t* assign;  /* n: list of each row, in row order */
  const void* raw;        /* n x dim raw vectors in row order (float or uint8) */
  int32_t raw_dtype;      /* rq_dtype of raw */
  int32_t reserved;
} rq_index_view;

typedef struct rq_index rq_index;

/* rq_build -- build an IVF-RaBitQ index on the current CUDA device.
 * Steps (Section 3.1.1): k-means over the rows (Phases 1-2, Section 2.1.2),
 * final assignment, random orthogonal P drawn from `seed` (Section 2.2.1),
 * sign codes and factors r, alpha of every row (Eqs. 1-3, Phase 3).
 *   base   host or device, n x dim, float32 (RQ_F32) or uint8 (RQ_U8).
 *   seed   seeds P and the k-means initial rows (Philox4x32-10).
 *   opts   NULL for defaults.
 *   out    receives the index; the caller frees it with rq_free.
 * The index keeps its own device copy of base for the exact re-rank.
 * Errors: INVALID_ARG (sizes out of range, nlist > n, NULL pointers,
 * non-finite values), OOM, CUDA. Synchronous. */
RQ_API rq_status rq_build(const void* base, rq_dtype dtype, int64_t n, int32_t dim,
                   int32_t nlist, uint64_t seed, const rq_build_opts* opts,
                   rq_index** out);

/* rq_build_with -- as rq_build, but with given centroids (nlist x dim,
 * float32) and rotation P (D_p x D_p, float64), both host or device: only the
 * final assignment and the encode (Eqs. 1-3) run. Errors as rq_build. */
RQ_API rq_status rq_build_with(const void* base, rq_dtype dtype, int64_t n,
                        int32_t dim, int32_t nlist, const float* centroids,
                        const double* P, rq_index** out);

/* rq_kmeans -- the k-means stage of rq_build alone (Section 2.1.2; Section
 * 3.1.1 Phases 1-2): `iters` Lloyd iterations from the nlist training rows of
 * smallest Philox rank key. base: host or device, n x dim float32;
 * centroids_out: host or device, nlist x dim float32. Synchronous. */
RQ_API rq_status rq_kmeans(const float* base, int64_t n, int32_t dim, int32_t nlist,
                    uint64_t seed, int32_t iters, int64_t train_size,
                    float* centroids_out);

/* rq_philox_gaussian -- the standard normal draws that rq_build
 * orthogonalises into P: out[i] for i < count, from Philox4x32-10 with key
 * `seed`, counter (i/2, stream) and the Box-Muller transform. out: host or
 * device float64. Synchronous. */
RQ_API rq_status rq_philox_gaussian(uint64_t seed, uint32_t stream, int64_t count,
                             double* out);

/* Device-side failures. Kernels that meet an impossible state or whose
 * bounded wait runs out set the index's error word (rq_device_error). A
 * search whose call waits for the device (host queries or host outputs)
 * reads the word before it returns, clears it, and returns RQ_ERR_TIMEOUT
 * (a bounded wait ran out) or RQ_ERR_DEVICE (any other code); its outputs
 * are then unspecified. A search that only enqueues work (device queries and
 * outputs) cannot see the word: its caller checks rq_device_error after
 * synchronising. */

/* rq_search -- k nearest neighbours of nq queries (Section 2.1.2 query
 * processing; Sections 3.3.1-3.3.4):
 *   1. rotate each query once: q' = P^T q (P^T (q - c) = q' - P^T c),
 *   2. rank the centroids by ||q' - P^T c||^2 (float32, terms added in
 *      increasing dimension) and keep the nprobe nearest by (distance, id);
 *      for nlist <= 4096 and D_p = 128 an approximate ranking with a proven
 *      error bound first narrows the centroids that need the exact value,
 *   3. quantise each residual q' - P^T c to 4 bits (vl, delta, bit-planes),
 *   4. scan the probed lists with the estimator of Eqs. 4-5, keep candidates
 *      at or below a per-query bound set from the nearest lists (Section
 *      3.3.3), select the n_rerank smallest estimates,
 *   5. re-rank them with exact float32 distances to the raw vectors, keep k.
 *   queries   host or device, nq x dim float32 (host queries are checked to be
 *             finite; results for non-finite device queries are unspecified).
 *   out_ids   host or device, nq x k int64; out_dist: nq x k float32
 *             (exact distances; estimated ones when n_rerank == 0, in which
 *             case the top k by the estimate are returned without re-rank).
 *   opts      NULL for defaults. stream: cudaStream_t or NULL.
 * The index is read-only here: concurrent calls on different streams are
 * safe. Errors: INVALID_ARG (ranges above, NULL pointers), OOM, CUDA. */
RQ_API rq_status rq_search(rq_index* ix, const float* queries, int64_t nq,
                    int32_t nprobe, int32_t k, int32_t n_rerank,
                    int64_t* out_ids, float* out_dist,
                    const rq_search_opts* opts, void* stream);

/* rq_search_mixed -- rq_search with per-query nprobe, k and n_rerank
 * (arrays of nq int32, host memory). Results of query i go to row i of
 * out_ids / out_dist (host or device, nq x k_stride, k_stride >= max k); the
 * columns past k[i] are padded with -1 / +inf. Each query's result equals
 * what rq_search returns for it alone. Errors as rq_search. */
RQ_API rq_status rq_search_mixed(rq_index* ix, const float* queries, int64_t nq,
                          const int32_t* nprobe, const int32_t* k,
                          const int32_t* n_rerank, int32_t k_stride,
                          int64_t* out_ids, float* out_dist,
                          const rq_search_opts* opts, void* stream);

/* rq_autotune -- time the scan forms on `nq` sample queries (host or device,
 * nq x dim) at `nprobe`, `n_rerank`: the plain scan with 1024-, 2048- and
 * 4096-vector chunks per thread block, the streaming grouped scan and (D_p =
 * 128) the tensor-core scan. The fastest becomes the choice of RQ_SCAN_AUTO
 * for batches of the sample's class: its size and its pair density (nq x
 * nprobe / nlist), each on a log2 scale; a batch of a class never tuned
 * takes the nearest tuned class. The result is appended to the text file
 * `cache_path` (NULL: no file); a later call for the same index shape and
 * class reuses the stored choice without timing. Every choice returns the
 * same results. Synchronous. */
RQ_API rq_status rq_autotune(rq_index* ix, const float* queries, int64_t nq,
                      int32_t nprobe, int32_t n_rerank, const char* cache_path);

/* rq_get_stats / rq_get_view -- sizes and device pointers of an index. */
RQ_API rq_status rq_get_stats(const rq_index* ix, rq_stats* out);
RQ_API rq_status rq_get_view(const rq_index* ix, rq_index_view* out);

/* rq_export / rq_import -- one flat little-endian file holding the whole
 * index (header "RQIX", version, sizes, then P, centroids, P^T c, offsets,
 * codes, r, alpha, ids, assignments, raw vectors). rq_import rebuilds the
 * index on the current device. Errors: IO, OOM, CUDA, INVALID_ARG. */
RQ_API rq_status rq_export(const rq_index* ix, const char* path);
RQ_API rq_status rq_import(const char* path, rq_index** out);

/* rq_free -- release an index and all its device memory. NULL is a no-op. */
RQ_API void rq_free(rq_index* ix);

/* rq_device_error -- read and clear the index's device error word: 0, or a
 * code set by a kernel that met an impossible state (a bounds check).
 * Synchronises the device. */
RQ_API rq_status rq_device_error(rq_index* ix, int32_t* code);

/* rq_probe_static -- the query rotation and centroid ranking of rq_search
 * (q' = P^T q, then the nprobe lists of smallest ||q' - P^T c||^2, ties by
 * list id), for callers that cannot allocate device memory when they search:
 * processes whose framework hands all device memory to its own allocator (a
 * cudaMalloc of ours would compete with it or fail), and serving threads that
 * cannot take the device-wide synchronisation of cudaMalloc/cudaFree.
 * The paper has no counterpart: it is an interface variant of Phase 1 of the
 * search, which the paper runs as a batch on the NPU.
 * It allocates nothing: its scratch (the rotated queries and the distance
 * keys) is one fixed 16 MiB array in device memory that every GPU loading the
 * library holds until the process exits. A call needs
 * nq * (4 * D_p + 8 * nlist) bytes of it (each part rounded up to 256 bytes);
 * larger calls are rejected with RQ_ERR_INVALID_ARG.
 *   queries   device, nq x dim float32.
 *   out_ids   device, nq x nprobe int32: lists in ascending (distance, id).
 *   out_dist  device, nq x nprobe float32: their squared distances.
 *   stream    cudaStream_t or NULL; the call only enqueues work.
 * The results equal the probe stage of rq_search bit for bit. The first call
 * on a device looks up the array's device address; make that first call
 * before any stream capture. All calls share the one array and it keeps the
 * last call's contents (nothing in it needs to start at zero): calls whose
 * work overlaps on the GPU (on different streams, or from different threads)
 * race on it and must be serialised by the caller.
 * Errors: INVALID_ARG (NULL or host pointers, sizes), CUDA. */
RQ_API rq_status rq_probe_static(const rq_index* ix, const float* queries, int64_t nq,
                                 int32_t nprobe, int32_t* out_ids, float* out_dist,
                                 void* stream);

/* rq_test_fail_allocations -- test hook of the failure paths: the after-th
 * next device allocation this library makes (0 = the very next) fails as if
 * the device were out of memory, and the ones after it succeed again; a
 * negative value disarms the hook. The call that meets the failure returns
 * RQ_ERR_OOM and releases what it had allocated. Process-wide; not for use
 * while other threads call into the library. */
RQ_API void rq_test_fail_allocations(int64_t after);

RQ_API const char* rq_status_str(rq_status s);
RQ_API const char* rq_last_error(void);
RQ_API int32_t rq_version(void);

/* ---------------------------------------------------------------------
 * Serving: continuous batching (the overlapped, multi-request execution the
 * paper names as its next step, Section 3.3.4, here on one GPU).
 * A server thread admits submitted requests as stream slots and device
 * memory become free, merges the requests admitted together into one mixed
 * batch (per-query nprobe, k, n_rerank), and runs up to `slots` batches at a
 * time on separate CUDA streams, so batches admitted later overlap with
 * running ones on the device. Results are those of rq_search_mixed.
 * ------------------------------------------------------------------- */
typedef struct rq_server_opts {
  int32_t slots;            /* batches in flight (streams); default 4 */
  int32_t max_batch;        /* queries merged into one batch; default 1024 */
  int64_t memory_budget;    /* device bytes for in-flight batches;
                               0 = a quarter of free memory */
  int32_t max_queue;        /* queued requests before submit says BUSY;
                               default 65536 */
  int32_t scan_mode;        /* rq_scan_mode for every batch */
} rq_server_opts;

typedef struct rq_server rq_server;

/* Start a server thread on the index (which must outlive the server). */
RQ_API rq_status rq_server_create(rq_index* ix, const rq_server_opts* opts,
                           rq_server** out);
/* Queue a request of nq queries (host memory, copied before return).
 * nprobe, k, n_rerank as rq_search. Errors: INVALID_ARG, BUSY. */
RQ_API rq_status rq_submit(rq_server* s, const float* queries, int64_t nq,
                    int32_t nprobe, int32_t k, int32_t n_rerank,
                    uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a request; on RQ_OK copy its
 * results into host ids (nq x k) and dist (nq x k) and forget the ticket.
 * latency_us (may be NULL) receives submit-to-completion time.
 * Errors: TIMEOUT (the ticket stays valid), INVALID_ARG (unknown ticket),
 * or the error the request's batch met. */
RQ_API rq_status rq_wait(rq_server* s, uint64_t ticket, int64_t* ids, float* dist,
                  int32_t timeout_ms, double* latency_us);
/* Stop admitting, finish queued and running requests, join the thread. */
RQ_API void rq_server_destroy(rq_server* s);

#ifdef __cplusplus
}
#endif

#endif /* RQ_H */
