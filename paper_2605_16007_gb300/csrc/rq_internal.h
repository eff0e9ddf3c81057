// Internal declarations shared by the librq translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <algorithm>
#include <tuple>
#include <utility>
#include <vector>

#include "rq.h"

namespace rq {

constexpr int kMaxDim = 2048;
constexpr int kMaxSelect = 4096;      // largest n_rerank / k / nprobe
// How many candidates, in probe order, set a query's first pruning bound:
// max(1024, n_sel, min(16 n_sel, 32768)).
__host__ __device__ inline int bound_window(int n_sel) {
  const int w = 16 * n_sel < 32768 ? 16 * n_sel : 32768;
  return n_sel > w ? n_sel : (w > 1024 ? w : 1024);
}
constexpr int kMaxNlist = 1 << 20;

// Error bookkeeping: the first error message of the calling thread.
void set_error(const std::string& msg);
rq_status fail(rq_status s, const std::string& msg);
rq_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define RQ_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return ::rq::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define RQ_TRY(call)                         \
  do {                                       \
    rq_status _s = (call);                   \
    if (_s != RQ_OK) return _s;              \
  } while (0)

inline int dim_pad(int d) { return ((d + 127) / 128) * 128; }

// Search shape: one launch sequence (and one workspace) per distinct shape.
struct SearchShape {
  int64_t nq;
  int npmax;      // largest nprobe of the batch
  int nsel_max;   // largest selection size (n_rerank, or k when it is 0)
  int k_stride;   // output row stride
  int mode;       // resolved scan mode
  int prune;
  int withhold;   // test hook: the pipelined scan withholds its first stage
  int chunk;      // plain scan: list vectors per block (a multiple of 1024)
  int lut;        // 1: FastScan estimator (full-precision query, float32 tables)
  bool operator<(const SearchShape& o) const {
    return std::tie(nq, npmax, nsel_max, k_stride, mode, prune, withhold, chunk, lut) <
           std::tie(o.nq, o.npmax, o.nsel_max, o.k_stride, o.mode, o.prune, o.withhold,
                    o.chunk, o.lut);
  }
};

// What the autotuner chose for one class of batches.
struct TunedChoice {
  int mode = RQ_SCAN_GROUPED;
  int chunk = 1024;
};

// The class of a batch for the autotuner: its size and its pair density
// (pairs per list), each on a log2 scale, so that one choice serves the
// batches that stress the scan alike.
inline std::pair<int, int> tune_class(int64_t nq, int64_t sum_nprobe, int nlist) {
  int a = 0, b = 0;
  for (int64_t v = nq; v > 1; v >>= 1) ++a;
  for (int64_t v = (8 * sum_nprobe) / std::max(1, nlist); v > 1; v >>= 1) ++b;
  return {a, b};
}

// Device workspace of one search shape, carved out of one allocation.
struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
  float* q = nullptr;           // nq x dim (input copy)
  float* qrot = nullptr;        // nq x D_p
  uint64_t* pkeys = nullptr;    // nq x nlist exact probe keys, or (nlist <= 4096)
                                // nq x nlist approximate distances (float)
  float* cn = nullptr;          // nlist: ||P^T c||^2 (certified probe selection)
  int32_t* probe_ids = nullptr; // nq x npmax
  float* probe_d = nullptr;     // nq x npmax
  float4* qparams = nullptr;    // nq x npmax: vl, delta, nq2, Sq(bits of int)
  uint32_t* planes = nullptr;   // nq x npmax x 4 x W words
  uint32_t* bound = nullptr;    // nq
  int32_t* counts = nullptr;    // nq: candidates that passed (written by the finalize)
  // Scan output: for probe p of query q, word w of the probed list's
  // survivor mask sits at mask[q * mwords + wbase[q * npmax + p] + w] (bit i:
  // vector 32 w + i passed the bound).
  uint32_t* mask = nullptr;     // nq x mwords
  int32_t* wbase = nullptr;     // nq x npmax: first mask word of each probe
  int32_t* wtotal = nullptr;    // nq: mask words of the query's probes
  uint64_t* sel = nullptr;      // nq x nsel_max
  uint64_t* keys = nullptr;     // nq x kcap survivor keys (collection -> selection)
  int32_t* kcount = nullptr;    // nq: survivors of each query
  int32_t* nprobe = nullptr;    // nq
  int32_t* kq = nullptr;        // nq
  int32_t* nsel = nullptr;      // nq
  int32_t* rerank_on = nullptr; // nq: 1 if n_rerank > 0
  int64_t* out_ids = nullptr;   // nq x k_stride
  float* out_d = nullptr;       // nq x k_stride
  // grouped scans: (query, probe) pairs bucketed by list
  int32_t* list_count = nullptr;  // nlist: pairs probing each list
  int64_t* qwrow = nullptr;       // nlist x nq (stride rounded up to 4, +2): per bucket slot,
                                  // the pair's first mask index
  float* qtau = nullptr;          // nlist x nq (same stride, +4): per bucket slot, the bound
                                  // as a float32 threshold
  int32_t* nchunks = nullptr;     // plain scan: nq x npmax chunk counts
  uint8_t* qdig = nullptr;        // nlist x nq x D_p: per-list buckets of FP8 query digits
  float4* qpb = nullptr;          // nlist x nq (+2): per-list buckets of {vl, delta, nq2, -Sq},
                                  // interleaved by slot couples
  float* resid = nullptr;         // FastScan: nq x npmax x D_p residuals
  uint8_t* qrec = nullptr;        // nlist x nq pair records of the streaming scan
                                  // (pair_rec_bytes(D_p) each)
  // tensor-core scan: the first bound from a grouped pass over each query's
  // window (the first candidates in probe order). Each window pair gets a
  // second slot in a per-list window bucket with its digits and parameters;
  // the pass writes the window's estimates into the query's key buffer
  // (idle until the collection), as uint32 at [q * 2 kcap + position].
  int32_t* wcount = nullptr;      // nlist: window pairs of each list, then
                                  // nlist: the largest window limit of each list
  uint8_t* wqdig = nullptr;       // nlist x nq x D_p (as qdig)
  float4* wqpb = nullptr;         // nlist x nq (+2) (as qpb)
  int64_t* wdest = nullptr;       // nlist x nq (stride of qwrow, +2): first estimate index
  int32_t* wlim = nullptr;        // nlist x nq (same stride, +4): vectors of the list in the window
  int32_t* wtake = nullptr;       // nq: window candidates of each query
  uint32_t* pslot = nullptr;      // nq x npmax: each probe's slot in its list's bucket
  int64_t mwords = 0;             // mask words per query
  int64_t kcap = 0;               // survivor keys each query's buffer holds
};

struct Plan {
  SearchShape shape;
  cudaStream_t stream = nullptr;
  Workspace ws;
  cudaGraphExec_t graph = nullptr;
  int32_t* h_params = nullptr;          // pinned staging of per-query parameters
  int32_t* h_err = nullptr;             // pinned copy of the device error word
  cudaEvent_t params_ready = nullptr;   // the last copy out of h_params has run
  uint64_t last_use = 0;
};

}  // namespace rq

struct rq_index {
  int device = 0;
  int64_t n = 0;
  int dim = 0, dp = 0, nlist = 0, C = 0;  // C = code bytes = dp / 8
  rq_dtype raw_dtype = RQ_F32;
  // device arrays
  double* P = nullptr;        // dp x dp
  float* P32 = nullptr;       // dp x dp
  float* centroids = nullptr; // nlist x dim
  float* cR = nullptr;        // nlist x dp
  int64_t* offsets = nullptr; // nlist + 1
  uint8_t* codes = nullptr;   // n x C
  float* r = nullptr;         // n
  float* alpha = nullptr;     // n
  float2* fac = nullptr;      // n: {r^2, f}
  uint32_t* ids = nullptr;    // n
  int32_t* assign = nullptr;  // n (row order)
  void* raw = nullptr;        // n x dim (float or uint8)
  bool raw_owned = true;      // false: the caller's page-locked host buffer (raw_on_host)
  int32_t* d_err = nullptr;   // device error word
  int2* items = nullptr;      // static scan items (list, first vector)
  int n_items = 0;
  // host copies
  std::vector<int64_t> h_offsets;
  std::vector<int64_t> top_len_prefix;    // sum of the j largest list lengths
  std::vector<int64_t> top_words_prefix;  // sum of the j largest ceil(length / 32)
  int64_t max_list_len = 0;
  // tuned choices for RQ_SCAN_AUTO: per batch class (tune_class), and the
  // latest one as the default for classes never tuned
  std::atomic<int> auto_mode{RQ_SCAN_GROUPED};
  std::map<std::pair<int, int>, rq::TunedChoice> tuned;  // guarded by mu
  // plans (workspaces, graphs) per (stream, shape)
  std::mutex mu;
  std::map<std::pair<cudaStream_t, rq::SearchShape>, std::unique_ptr<rq::Plan>> plans;
  uint64_t plan_clock = 0;
  cudaStream_t graph_stream = nullptr;  // used when a graph is asked on stream 0
};

namespace rq {

// Build (rq_build.cu)
rq_status build_index(const float* d_base_f32, const void* d_raw, rq_dtype dt,
                      int64_t n, int dim, int nlist, uint64_t seed, int iters,
                      int64_t train_size, const float* given_centroids,
                      const double* given_P, rq_index* ix);
rq_status kmeans_device(const float* d_x, int64_t n, int dim, int nlist,
                        uint64_t seed, int iters, int64_t train_size,
                        float* d_centroids);
rq_status philox_gaussian_device(uint64_t seed, uint32_t stream, int64_t count,
                                 double* d_out);
rq_status finish_index_host_side(rq_index* ix);

// Search (rq_search.cu)
rq_status search_run(rq_index* ix, const float* queries, int64_t nq,
                     const int32_t* nprobe, const int32_t* k,
                     const int32_t* n_rerank, int k_stride, int64_t* out_ids,
                     float* out_dist, const rq_search_opts* opts,
                     cudaStream_t stream);
rq_status autotune(rq_index* ix, const float* queries, int64_t nq, const int32_t* nprobe,
                   int n_rerank, const char* cache_path);
void free_plans(rq_index* ix);
size_t search_workspace_bytes(const rq_index* ix, int64_t nq, int npmax, int nsel_max,
                              int k_stride, int mode);

// Memory residence
bool is_device_ptr(const void* p);

// Every device allocation of the library goes through dev_alloc, so that the
// test hook rq_test_fail_allocations can make a chosen one fail.
bool alloc_should_fail();
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// Lets kernel `func` take up to `bytes` of dynamic shared memory on the
// current device. The opt-in above 48 KB is a per-device attribute, so it is
// set once per (kernel, device); safe to call from several threads.
rq_status allow_dynamic_smem(const void* func, int bytes);

}  // namespace rq
