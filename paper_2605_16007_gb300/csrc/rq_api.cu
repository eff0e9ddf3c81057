// C ABI of librq: argument checks, device copies of inputs, index lifetime,
// export/import, and the continuous-batching server.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <set>
#include <tuple>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rq_common.cuh"
#include "rq_internal.h"
#include "rq_scan.cuh"

namespace rq {

static thread_local std::string t_error;

void set_error(const std::string& msg) { t_error = msg; }

rq_status fail(rq_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

rq_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  cudaGetLastError();
  const char* base = strrchr(file, '/');
  set_error(std::string(what) + ": " + cudaGetErrorString(e) + " (" + (base ? base + 1 : file) +
            ":" + std::to_string(line) + ")");
  return (e == cudaErrorMemoryAllocation) ? RQ_ERR_OOM : RQ_ERR_CUDA;
}

// The allocation-failure hook: the countdown-th next device allocation
// fails (0 = the next one); -1 = none.
static std::atomic<int64_t> g_fail_countdown{-1};

bool alloc_should_fail() {
  int64_t c = g_fail_countdown.load();
  while (c >= 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}

rq_status allow_dynamic_smem(const void* func, int bytes) {
  // the limit only grows: a kernel launched with several sizes keeps the
  // largest asked for (setting a smaller one would fail the larger launches)
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> bytes
  int dev = 0;
  RQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(func, dev);
  const auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return RQ_OK;
  RQ_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done[key] = bytes;
  return RQ_OK;
}

namespace {

__global__ void count_nonfinite_kernel(const float* x, int64_t n, int32_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicAdd(out, 1);
}

// Counts values that are not integers in [0, 255].
__global__ void count_non_byte_kernel(const float* x, int64_t n, int32_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = x[i];
    if (!(v >= 0.0f && v <= 255.0f && v == rintf(v))) atomicAdd(out, 1);
  }
}

__global__ void f32_to_u8_kernel(const float* a, uint8_t* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (uint8_t)a[i];
}

__global__ void u8_to_f32_kernel(const uint8_t* a, float* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

rq_status check_finite_device(const float* d, int64_t n, const char* what) {
  int32_t* cnt = nullptr;
  RQ_CUDA(dev_alloc(&cnt, sizeof(int32_t)));
  cudaMemset(cnt, 0, sizeof(int32_t));
  count_nonfinite_kernel<<<(unsigned)std::max<int64_t>(1, (n + 255) / 256), 256>>>(d, n, cnt);
  int32_t h = 0;
  cudaError_t e = cudaMemcpy(&h, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(cnt);
  if (e != cudaSuccess) return cuda_fail(e, "finite check", __FILE__, __LINE__);
  if (h) return fail(RQ_ERR_INVALID_ARG, std::string("non-finite values in ") + what);
  return RQ_OK;
}

void free_index_arrays(rq_index* ix) {
  void* ptrs[] = {ix->P,     ix->P32,   ix->centroids, ix->cR,     ix->offsets, ix->codes,
                  ix->r,     ix->alpha, ix->fac,       ix->ids,    ix->assign,
                  ix->raw_owned ? ix->raw : nullptr, ix->d_err, ix->items};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ix->P = nullptr;
  ix->raw = nullptr;
  ix->items = nullptr;
}

// Copies the base rows to the device: raw (kept for re-rank, in the given
// dtype) and, for uint8, a temporary float32 copy for the build.
rq_status upload_base(const void* base, rq_dtype dt, int64_t n, int dim, void** d_raw,
                      float** d_f32, bool* f32_is_temp) {
  const size_t elt = (dt == RQ_U8) ? 1 : 4;
  const size_t bytes = elt * (size_t)n * dim;
  RQ_CUDA(dev_alloc(d_raw, bytes));
  cudaError_t e = cudaMemcpy(*d_raw, base, bytes, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    cudaFree(*d_raw);
    *d_raw = nullptr;
    return cuda_fail(e, "copy of base vectors", __FILE__, __LINE__);
  }
  if (dt == RQ_F32) {
    *d_f32 = static_cast<float*>(*d_raw);
    *f32_is_temp = false;
    rq_status s = check_finite_device(*d_f32, (int64_t)n * dim, "base");
    if (s != RQ_OK) {
      cudaFree(*d_raw);
      *d_raw = nullptr;
    }
    return s;
  }
  e = dev_alloc(d_f32, sizeof(float) * (size_t)n * dim);
  if (e != cudaSuccess) {
    cudaFree(*d_raw);
    *d_raw = nullptr;
    return cuda_fail(e, "float copy of uint8 base", __FILE__, __LINE__);
  }
  u8_to_f32_kernel<<<(unsigned)std::max<int64_t>(1, ((int64_t)n * dim + 255) / 256), 256>>>(
      static_cast<const uint8_t*>(*d_raw), *d_f32, (int64_t)n * dim);
  *f32_is_temp = true;
  return RQ_OK;
}

rq_status check_build_args(const void* base, rq_dtype dt, int64_t n, int32_t dim,
                           int32_t nlist, rq_index** out) {
  if (!base || !out) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  if (dt != RQ_F32 && dt != RQ_U8) return fail(RQ_ERR_INVALID_ARG, "unknown dtype");
  if (dim < 1 || dim > kMaxDim) return fail(RQ_ERR_INVALID_ARG, "dim outside [1, 2048]");
  if (n < 1 || n >= ((int64_t)1 << 32)) return fail(RQ_ERR_INVALID_ARG, "n outside [1, 2^32)");
  if (nlist < 1 || nlist > kMaxNlist || nlist > n)
    return fail(RQ_ERR_INVALID_ARG, "nlist outside [1, min(n, 2^20)]");
  const int dp = dim_pad(dim);
  if (!(dp / 128 <= 8 || dp == 1536 || dp == 2048))
    return fail(RQ_ERR_INVALID_ARG, "padded dimension " + std::to_string(dp) + " not supported");
  return RQ_OK;
}

// A float32 raw copy whose values are all integers in [0, 255] is replaced
// by a uint8 copy: the re-rank converts each byte back to the same float.
rq_status compress_raw(rq_index* ix) {
  if (ix->raw_dtype != RQ_F32) return RQ_OK;
  const int64_t count = ix->n * ix->dim;
  int32_t* cnt = nullptr;
  RQ_CUDA(dev_alloc(&cnt, sizeof(int32_t)));
  cudaMemset(cnt, 0, sizeof(int32_t));
  const unsigned blocks = (unsigned)std::max<int64_t>(1, (count + 255) / 256);
  count_non_byte_kernel<<<blocks, 256>>>(static_cast<const float*>(ix->raw), count, cnt);
  int32_t h = 1;
  cudaError_t e = cudaMemcpy(&h, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(cnt);
  if (e != cudaSuccess) return cuda_fail(e, "raw check", __FILE__, __LINE__);
  if (h != 0) return RQ_OK;
  uint8_t* r8 = nullptr;
  if (dev_alloc(&r8, (size_t)count + 16) != cudaSuccess) {
    cudaGetLastError();
    return RQ_OK;  // keep the float copy
  }
  f32_to_u8_kernel<<<blocks, 256>>>(static_cast<const float*>(ix->raw), r8, count);
  RQ_CUDA(cudaDeviceSynchronize());
  cudaFree(ix->raw);
  ix->raw = r8;
  ix->raw_dtype = RQ_U8;
  return RQ_OK;
}

rq_status build_common(const void* base, rq_dtype dt, int64_t n, int32_t dim, int32_t nlist,
                       uint64_t seed, int iters, int64_t train, const float* cent,
                       const double* P, rq_index** out, bool keep_float_raw = false,
                       bool raw_on_host = false) {
  RQ_TRY(check_build_args(base, dt, n, dim, nlist, out));
  *out = nullptr;
  void* host_raw = nullptr;  // the GPU's address of the caller's buffer
  if (raw_on_host) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, base) != cudaSuccess || at.type != cudaMemoryTypeHost ||
        !at.devicePointer) {
      cudaGetLastError();
      return fail(RQ_ERR_INVALID_ARG, "raw_on_host needs a page-locked host base buffer");
    }
    host_raw = at.devicePointer;
  }
  std::unique_ptr<rq_index> ix(new rq_index());
  cudaGetDevice(&ix->device);
  void* d_raw = nullptr;
  float* d_f32 = nullptr;
  bool temp = false;
  RQ_TRY(upload_base(base, dt, n, dim, &d_raw, &d_f32, &temp));
  const float* d_cent = nullptr;
  const double* d_P = nullptr;
  float* cent_tmp = nullptr;
  double* P_tmp = nullptr;
  rq_status s = RQ_OK;
  if (cent) {
    const int dp = dim_pad(dim);
    if (dev_alloc(&cent_tmp, sizeof(float) * nlist * dim) != cudaSuccess ||
        dev_alloc(&P_tmp, sizeof(double) * dp * dp) != cudaSuccess) {
      cudaGetLastError();
      s = fail(RQ_ERR_OOM, "given centroids / rotation");
    } else {
      cudaMemcpy(cent_tmp, cent, sizeof(float) * nlist * dim, cudaMemcpyDefault);
      cudaMemcpy(P_tmp, P, sizeof(double) * dp * dp, cudaMemcpyDefault);
      s = check_finite_device(cent_tmp, (int64_t)nlist * dim, "centroids");
      d_cent = cent_tmp;
      d_P = P_tmp;
    }
  }
  if (s == RQ_OK)
    s = build_index(d_f32, d_raw, dt, n, dim, nlist, seed, iters, train, d_cent, d_P, ix.get());
  if (cent_tmp) cudaFree(cent_tmp);
  if (P_tmp) cudaFree(P_tmp);
  if (temp) cudaFree(d_f32);
  if (s == RQ_OK && raw_on_host) {
    // the device copy served the build; the re-rank reads the caller's rows
    cudaFree(ix->raw);
    ix->raw = host_raw;
    ix->raw_owned = false;
  } else if (s == RQ_OK && !keep_float_raw) {
    s = compress_raw(ix.get());
  }
  if (s != RQ_OK) {
    if (ix->raw == nullptr) cudaFree(d_raw);
    free_index_arrays(ix.get());
    return s;
  }
  *out = ix.release();
  return RQ_OK;
}

// ---------------------------------------------------------------------------
// Export / import: "RQIX", version, sizes, then the arrays in a fixed order.
// ---------------------------------------------------------------------------
constexpr uint32_t kFileVersion = 1;

struct FileHeader {
  char magic[4];
  uint32_t version;
  int64_t n;
  int32_t dim, dp, nlist, raw_dtype;
};

struct ArraySpec {
  void** dev;
  size_t bytes;
};

std::vector<ArraySpec> array_specs(rq_index* ix) {
  const size_t n = (size_t)ix->n;
  const size_t raw_elt = ix->raw_dtype == RQ_U8 ? 1 : 4;
  return {
      {(void**)&ix->P, sizeof(double) * ix->dp * ix->dp},
      {(void**)&ix->centroids, sizeof(float) * ix->nlist * ix->dim},
      {(void**)&ix->cR, sizeof(float) * ix->nlist * ix->dp},
      {(void**)&ix->offsets, sizeof(int64_t) * (ix->nlist + 1)},
      {(void**)&ix->codes, n * ix->C},
      {(void**)&ix->r, sizeof(float) * n},
      {(void**)&ix->alpha, sizeof(float) * n},
      {(void**)&ix->fac, sizeof(float2) * n},
      {(void**)&ix->ids, sizeof(uint32_t) * n},
      {(void**)&ix->assign, sizeof(int32_t) * n},
      {(void**)&ix->raw, raw_elt * n * ix->dim},
  };
}

__global__ void p_to_f32_kernel(const double* a, float* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  std::vector<float> q;
  int64_t nq;
  int nprobe, k, nrr;
  std::vector<int64_t> ids;
  std::vector<float> dist;
  rq_status status = RQ_OK;
  std::string error;
  bool done = false;
  Clock::time_point t_submit, t_done;
};

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  std::vector<std::shared_ptr<Request>> reqs;
  int64_t nq = 0, bucket = 0;
  int k_stride = 0;
  size_t mem = 0;
  float* h_q = nullptr;          // pinned
  int64_t* h_ids = nullptr;      // pinned
  float* h_d = nullptr;          // pinned
  float* d_q = nullptr;
  int64_t* d_ids = nullptr;
  float* d_d = nullptr;
  int64_t cap_q = 0, cap_out = 0;  // capacities (elements)
  rq_status launch_status = RQ_OK;
  std::string launch_error;
};

}  // namespace
}  // namespace rq

struct rq_server {
  rq_index* ix = nullptr;
  rq_server_opts opts{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;       // wakes the server thread
  std::condition_variable cv_done;  // wakes waiters
  std::deque<std::shared_ptr<rq::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<rq::Request>> all;
  std::vector<rq::Slot> slots;
  std::vector<int> completed;  // slot ids whose batch finished (host callback)
  uint64_t next_ticket = 1;
  size_t mem_in_use = 0;
  bool stop = false;
};

namespace rq {
namespace {

struct DoneMsg {
  rq_server* s;
  int slot;
};

void CUDART_CB batch_done_cb(void* p) {
  DoneMsg* m = static_cast<DoneMsg*>(p);
  {
    std::lock_guard<std::mutex> lk(m->s->mu);
    m->s->completed.push_back(m->slot);
  }
  m->s->cv.notify_all();
  delete m;
}

int pow2_at_least(int v) {
  int m = 1;
  while (m < v) m <<= 1;
  return m;
}

// Device bytes a batch shape needs (the search workspace) -- the admission
// cost of a batch.
size_t batch_bytes(const rq_index* ix, int64_t nq, int npmax, int nsel, int kst, int mode) {
  return search_workspace_bytes(ix, nq, npmax, nsel, kst, mode) + (size_t)nq * kst * 12 +
         (size_t)nq * ix->dim * 4 + (1 << 20);
}

rq_status slot_reserve(Slot& sl, int64_t nq_elems, int64_t out_elems) {
  if (nq_elems > sl.cap_q) {
    if (sl.h_q) cudaFreeHost(sl.h_q);
    if (sl.d_q) cudaFree(sl.d_q);
    RQ_CUDA(cudaMallocHost(&sl.h_q, sizeof(float) * nq_elems));
    RQ_CUDA(dev_alloc(&sl.d_q, sizeof(float) * nq_elems));
    sl.cap_q = nq_elems;
  }
  if (out_elems > sl.cap_out) {
    if (sl.h_ids) cudaFreeHost(sl.h_ids);
    if (sl.h_d) cudaFreeHost(sl.h_d);
    if (sl.d_ids) cudaFree(sl.d_ids);
    if (sl.d_d) cudaFree(sl.d_d);
    RQ_CUDA(cudaMallocHost(&sl.h_ids, sizeof(int64_t) * out_elems));
    RQ_CUDA(cudaMallocHost(&sl.h_d, sizeof(float) * out_elems));
    RQ_CUDA(dev_alloc(&sl.d_ids, sizeof(int64_t) * out_elems));
    RQ_CUDA(dev_alloc(&sl.d_d, sizeof(float) * out_elems));
    sl.cap_out = out_elems;
  }
  return RQ_OK;
}

// Merge the slot's requests into one mixed batch, padded with placeholder
// queries to a power of two of at least 64 (at least one placeholder) so that
// few distinct shapes occur; one placeholder carries the rounded-up nprobe / selection / k
// so that the shape does not depend on the exact mix.
rq_status launch_batch(rq_server* s, Slot& sl, int npb, int nsb, int kb) {
  rq_index* ix = s->ix;
  const int dim = ix->dim;
  const int64_t nq = sl.nq, bucket = sl.bucket;
  RQ_TRY(slot_reserve(sl, bucket * dim, bucket * kb));
  std::vector<int32_t> np(bucket, 1), kk(bucket, 1), nr(bucket, 1);
  int64_t row = 0;
  for (auto& r : sl.reqs) {
    std::memcpy(sl.h_q + row * dim, r->q.data(), sizeof(float) * r->nq * dim);
    for (int64_t i = 0; i < r->nq; ++i) {
      np[row + i] = r->nprobe;
      kk[row + i] = r->k;
      nr[row + i] = r->nrr;
    }
    row += r->nq;
  }
  for (int64_t i = nq; i < bucket; ++i)
    std::memcpy(sl.h_q + i * dim, sl.h_q, sizeof(float) * dim);
  np[nq] = npb;
  kk[nq] = kb;
  nr[nq] = nsb;
  RQ_CUDA(cudaMemcpyAsync(sl.d_q, sl.h_q, sizeof(float) * bucket * dim, cudaMemcpyHostToDevice,
                          sl.stream));
  rq_search_opts o{};
  o.scan_mode = s->opts.scan_mode;
  o.use_graph = 1;
  sl.k_stride = kb;
  RQ_TRY(search_run(ix, sl.d_q, bucket, np.data(), kk.data(), nr.data(), kb, sl.d_ids, sl.d_d, &o,
                    sl.stream));
  RQ_CUDA(cudaMemcpyAsync(sl.h_ids, sl.d_ids, sizeof(int64_t) * bucket * kb,
                          cudaMemcpyDeviceToHost, sl.stream));
  RQ_CUDA(cudaMemcpyAsync(sl.h_d, sl.d_d, sizeof(float) * bucket * kb, cudaMemcpyDeviceToHost,
                          sl.stream));
  return RQ_OK;
}

void server_loop(rq_server* s) {
  int dev = s->ix->device;
  cudaSetDevice(dev);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // Finish completed batches.
    while (!s->completed.empty()) {
      const int si = s->completed.back();
      s->completed.pop_back();
      Slot& sl = s->slots[si];
      const auto now = Clock::now();
      int64_t row = 0;
      for (auto& r : sl.reqs) {
        if (sl.launch_status == RQ_OK) {
          r->ids.resize(r->nq * r->k);
          r->dist.resize(r->nq * r->k);
          for (int64_t i = 0; i < r->nq; ++i)
            for (int j = 0; j < r->k; ++j) {
              r->ids[i * r->k + j] = sl.h_ids[(row + i) * sl.k_stride + j];
              r->dist[i * r->k + j] = sl.h_d[(row + i) * sl.k_stride + j];
            }
        } else {
          r->status = sl.launch_status;
          r->error = sl.launch_error;
        }
        row += r->nq;
        r->done = true;
        r->t_done = now;
      }
      sl.reqs.clear();
      sl.busy = false;
      s->mem_in_use -= sl.mem;
      sl.mem = 0;
      s->cv_done.notify_all();
    }
    // Admit queued requests into a free slot.
    int free_slot = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
      if (!s->slots[i].busy) {
        free_slot = (int)i;
        break;
      }
    if (free_slot >= 0 && !s->queue.empty()) {
      Slot& sl = s->slots[free_slot];
      int64_t nq = 0;
      int npm = 1, nsm = 1, km = 1;
      std::vector<std::shared_ptr<Request>> take;
      const size_t budget = (size_t)s->opts.memory_budget;
      while (!s->queue.empty()) {
        auto& r = s->queue.front();
        const int64_t nq2 = nq + r->nq;
        if (!take.empty() && nq2 > s->opts.max_batch) break;
        const int np2 = std::max(npm, r->nprobe), ns2 = std::max(nsm, r->nrr > 0 ? r->nrr : r->k),
                  k2 = std::max(km, r->k);
        const int64_t b2 = std::max(64, pow2_at_least((int)nq2 + 1));
        const int npb = std::min(pow2_at_least(np2), std::min(s->ix->nlist, kMaxSelect));
        const int nsb = std::min(pow2_at_least(ns2), kMaxSelect);
        const size_t need = batch_bytes(s->ix, b2, npb, nsb, pow2_at_least(k2), RQ_SCAN_MMA);
        if (!take.empty() && s->mem_in_use + need > budget) break;
        if (take.empty() && s->mem_in_use > 0 && s->mem_in_use + need > budget) break;
        take.push_back(r);
        s->queue.pop_front();
        nq = nq2;
        npm = np2;
        nsm = ns2;
        km = k2;
      }
      if (!take.empty()) {
        sl.reqs = std::move(take);
        sl.nq = nq;
        sl.bucket = std::max(64, pow2_at_least((int)nq + 1));
        const int npb = std::min(pow2_at_least(npm), std::min(s->ix->nlist, kMaxSelect));
        const int nsb = std::min(pow2_at_least(nsm), kMaxSelect);
        const int kb = std::min(pow2_at_least(km), nsb);
        sl.mem = batch_bytes(s->ix, sl.bucket, npb, nsb, kb, RQ_SCAN_MMA);
        s->mem_in_use += sl.mem;
        sl.busy = true;
        lk.unlock();
        sl.launch_status = launch_batch(s, sl, npb, nsb, kb);
        if (sl.launch_status != RQ_OK) sl.launch_error = rq_last_error();
        DoneMsg* m = new DoneMsg{s, free_slot};
        if (sl.launch_status != RQ_OK ||
            cudaLaunchHostFunc(sl.stream, batch_done_cb, m) != cudaSuccess) {
          cudaGetLastError();
          if (sl.launch_status == RQ_OK) {
            sl.launch_status = RQ_ERR_CUDA;
            sl.launch_error = "cudaLaunchHostFunc failed";
          }
          cudaStreamSynchronize(sl.stream);
          batch_done_cb(m);
        }
        lk.lock();
        continue;
      }
    }
    bool any_busy = false;
    for (auto& sl : s->slots) any_busy |= sl.busy;
    if (s->stop && s->queue.empty() && !any_busy) break;
    s->cv.wait(lk, [&] {
      if (!s->completed.empty()) return true;
      if (s->stop && s->queue.empty()) return true;
      if (s->queue.empty()) return false;
      for (auto& sl : s->slots)
        if (!sl.busy) return true;
      return false;
    });
  }
}

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" {

const char* rq_status_str(rq_status s) {
  switch (s) {
    case RQ_OK: return "ok";
    case RQ_ERR_INVALID_ARG: return "invalid argument";
    case RQ_ERR_OOM: return "out of memory";
    case RQ_ERR_CUDA: return "CUDA error";
    case RQ_ERR_TIMEOUT: return "timeout";
    case RQ_ERR_BUSY: return "busy";
    case RQ_ERR_IO: return "I/O error";
    case RQ_ERR_NOT_IMPLEMENTED: return "not implemented";
    case RQ_ERR_DEVICE: return "device error";
  }
  return "unknown status";
}

const char* rq_last_error(void) { return t_error.c_str(); }

void rq_test_fail_allocations(int64_t after) { g_fail_countdown.store(after < 0 ? -1 : after); }

int32_t rq_version(void) { return 10000; }

rq_status rq_build(const void* base, rq_dtype dtype, int64_t n, int32_t dim, int32_t nlist,
                   uint64_t seed, const rq_build_opts* opts, rq_index** out) {
  const int iters = opts ? opts->kmeans_iters : 10;
  const int64_t train = opts ? opts->train_size : 0;
  if (iters < 0) return fail(RQ_ERR_INVALID_ARG, "kmeans_iters < 0");
  if (train < 0) return fail(RQ_ERR_INVALID_ARG, "train_size < 0");
  if (train > 0 && train < nlist) return fail(RQ_ERR_INVALID_ARG, "train_size below nlist");
  return build_common(base, dtype, n, dim, nlist, seed, iters, train, nullptr, nullptr, out,
                      opts && opts->keep_float_raw, opts && opts->raw_on_host);
}

rq_status rq_build_with(const void* base, rq_dtype dtype, int64_t n, int32_t dim, int32_t nlist,
                        const float* centroids, const double* P, rq_index** out) {
  if (!centroids || !P) return fail(RQ_ERR_INVALID_ARG, "NULL centroids or P");
  return build_common(base, dtype, n, dim, nlist, 0, 0, 0, centroids, P, out);
}

rq_status rq_kmeans(const float* base, int64_t n, int32_t dim, int32_t nlist, uint64_t seed,
                    int32_t iters, int64_t train_size, float* centroids_out) {
  if (!centroids_out) return fail(RQ_ERR_INVALID_ARG, "NULL centroids_out");
  rq_index* unused = nullptr;
  RQ_TRY(check_build_args(base, RQ_F32, n, dim, nlist, &unused));
  if (iters < 0 || train_size < 0 || (train_size > 0 && train_size < nlist))
    return fail(RQ_ERR_INVALID_ARG, "bad iters / train_size");
  void* d_raw = nullptr;
  float* d_f32 = nullptr;
  bool temp = false;
  RQ_TRY(upload_base(base, RQ_F32, n, dim, &d_raw, &d_f32, &temp));
  float* d_c = nullptr;
  cudaError_t e = dev_alloc(&d_c, sizeof(float) * nlist * dim);
  if (e != cudaSuccess) {
    cudaFree(d_raw);
    return cuda_fail(e, "centroid buffer", __FILE__, __LINE__);
  }
  rq_status s = kmeans_device(d_f32, n, dim, nlist, seed, iters, train_size, d_c);
  if (s == RQ_OK) {
    e = cudaMemcpy(centroids_out, d_c, sizeof(float) * nlist * dim, cudaMemcpyDefault);
    if (e != cudaSuccess) s = cuda_fail(e, "copy of centroids", __FILE__, __LINE__);
  }
  cudaFree(d_c);
  cudaFree(d_raw);
  return s;
}

rq_status rq_philox_gaussian(uint64_t seed, uint32_t stream, int64_t count, double* out) {
  if (!out || count < 0) return fail(RQ_ERR_INVALID_ARG, "bad output or count");
  if (count == 0) return RQ_OK;
  double* d = nullptr;
  RQ_CUDA(dev_alloc(&d, sizeof(double) * count));
  rq_status s = philox_gaussian_device(seed, stream, count, d);
  if (s == RQ_OK) {
    cudaError_t e = cudaMemcpy(out, d, sizeof(double) * count, cudaMemcpyDefault);
    if (e != cudaSuccess) s = cuda_fail(e, "copy of draws", __FILE__, __LINE__);
  }
  cudaFree(d);
  return s;
}

rq_status rq_search(rq_index* ix, const float* queries, int64_t nq, int32_t nprobe, int32_t k,
                    int32_t n_rerank, int64_t* out_ids, float* out_dist,
                    const rq_search_opts* opts, void* stream) {
  if (nq < 0) return fail(RQ_ERR_INVALID_ARG, "nq < 0");
  if (nq > ((int64_t)1 << 24)) return fail(RQ_ERR_INVALID_ARG, "nq above 2^24 in one call");
  std::vector<int32_t> a(nq, nprobe), b(nq, k), c(nq, n_rerank);
  return search_run(ix, queries, nq, a.data(), b.data(), c.data(), k, out_ids, out_dist, opts,
                    static_cast<cudaStream_t>(stream));
}

rq_status rq_search_mixed(rq_index* ix, const float* queries, int64_t nq, const int32_t* nprobe,
                          const int32_t* k, const int32_t* n_rerank, int32_t k_stride,
                          int64_t* out_ids, float* out_dist, const rq_search_opts* opts,
                          void* stream) {
  return search_run(ix, queries, nq, nprobe, k, n_rerank, k_stride, out_ids, out_dist, opts,
                    static_cast<cudaStream_t>(stream));
}

rq_status rq_autotune(rq_index* ix, const float* queries, int64_t nq, int32_t nprobe,
                      int32_t n_rerank, const char* cache_path) {
  if (nq < 1) return fail(RQ_ERR_INVALID_ARG, "nq < 1");
  std::vector<int32_t> np(nq, nprobe);
  return autotune(ix, queries, nq, np.data(), n_rerank, cache_path);
}

rq_status rq_get_stats(const rq_index* ix, rq_stats* out) {
  if (!ix || !out) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  out->n = ix->n;
  out->dim = ix->dim;
  out->dim_pad = ix->dp;
  out->nlist = ix->nlist;
  out->code_bytes = ix->C;
  int64_t mn = INT64_MAX, mx = 0;
  for (int l = 0; l < ix->nlist; ++l) {
    const int64_t L = ix->h_offsets[l + 1] - ix->h_offsets[l];
    mn = std::min(mn, L);
    mx = std::max(mx, L);
  }
  out->min_list = mn;
  out->max_list = mx;
  const int64_t n = ix->n;
  out->index_bytes = n * (ix->C + 4 + 4 + 8 + 4 + 4) + (int64_t)ix->nlist * (ix->dim + ix->dp) * 4 +
                     (int64_t)(ix->nlist + 1) * 8 + (int64_t)ix->dp * ix->dp * 12;
  out->raw_bytes = n * ix->dim * (ix->raw_dtype == RQ_U8 ? 1 : 4);
  out->auto_scan_mode = ix->auto_mode.load();
  out->reserved = 0;
  return RQ_OK;
}

rq_status rq_get_view(const rq_index* ix, rq_index_view* v) {
  if (!ix || !v) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  v->n = ix->n;
  v->dim = ix->dim;
  v->dim_pad = ix->dp;
  v->nlist = ix->nlist;
  v->code_bytes = ix->C;
  v->P = ix->P;
  v->centroids = ix->centroids;
  v->cR = ix->cR;
  v->offsets = ix->offsets;
  v->codes = ix->codes;
  v->r = ix->r;
  v->alpha = ix->alpha;
  v->factors = reinterpret_cast<const float*>(ix->fac);
  v->ids = ix->ids;
  v->assign = ix->assign;
  v->raw = ix->raw;
  v->raw_dtype = ix->raw_dtype;
  v->reserved = 0;
  return RQ_OK;
}

rq_status rq_export(const rq_index* cix, const char* path) {
  if (!cix || !path) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  rq_index* ix = const_cast<rq_index*>(cix);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(RQ_ERR_IO, std::string("cannot open ") + path);
  FileHeader h{};
  std::memcpy(h.magic, "RQIX", 4);
  h.version = kFileVersion;
  h.n = ix->n;
  h.dim = ix->dim;
  h.dp = ix->dp;
  h.nlist = ix->nlist;
  h.raw_dtype = ix->raw_dtype;
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
  std::vector<char> buf;
  for (auto& a : array_specs(ix)) {
    if (!ok) break;
    buf.resize(a.bytes);
    if (cudaMemcpy(buf.data(), *a.dev, a.bytes, cudaMemcpyDefault) != cudaSuccess) {
      fclose(f);
      return cuda_fail(cudaGetLastError(), "export copy", __FILE__, __LINE__);
    }
    ok = fwrite(buf.data(), 1, a.bytes, f) == a.bytes;
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? RQ_OK : fail(RQ_ERR_IO, std::string("write failed: ") + path);
}

rq_status rq_import(const char* path, rq_index** out) {
  if (!path || !out) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(RQ_ERR_IO, std::string("cannot open ") + path);
  FileHeader h{};
  if (fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "RQIX", 4) != 0 ||
      h.version != kFileVersion || h.n < 1 || h.dim < 1 || h.dim > kMaxDim ||
      h.dp != dim_pad(h.dim) || h.nlist < 1 || h.nlist > h.n ||
      (h.raw_dtype != RQ_F32 && h.raw_dtype != RQ_U8)) {
    fclose(f);
    return fail(RQ_ERR_IO, std::string("not an index file of this version: ") + path);
  }
  std::unique_ptr<rq_index> ix(new rq_index());
  cudaGetDevice(&ix->device);
  ix->n = h.n;
  ix->dim = h.dim;
  ix->dp = h.dp;
  ix->nlist = h.nlist;
  ix->C = h.dp / 8;
  ix->raw_dtype = (rq_dtype)h.raw_dtype;
  std::vector<char> buf;
  rq_status s = RQ_OK;
  for (auto& a : array_specs(ix.get())) {
    buf.resize(a.bytes);
    if (fread(buf.data(), 1, a.bytes, f) != a.bytes) {
      s = fail(RQ_ERR_IO, "truncated index file");
      break;
    }
    // 16 bytes of tail room: bulk copies read whole 16-byte units.
    if (dev_alloc(a.dev, a.bytes + 16) != cudaSuccess) {
      cudaGetLastError();
      *a.dev = nullptr;
      s = fail(RQ_ERR_OOM, "index arrays");
      break;
    }
    if (cudaMemcpy(*a.dev, buf.data(), a.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      s = cuda_fail(cudaGetLastError(), "import copy", __FILE__, __LINE__);
      break;
    }
  }
  fclose(f);
  if (s == RQ_OK) {
    const int64_t nn = (int64_t)h.dp * h.dp;
    if (dev_alloc(&ix->P32, sizeof(float) * nn) != cudaSuccess ||
        dev_alloc(&ix->d_err, sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      s = fail(RQ_ERR_OOM, "index arrays");
    } else {
      p_to_f32_kernel<<<(unsigned)((nn + 255) / 256), 256>>>(ix->P, ix->P32, nn);
      cudaMemset(ix->d_err, 0, sizeof(int32_t));
      if (cudaDeviceSynchronize() != cudaSuccess)
        s = cuda_fail(cudaGetLastError(), "import", __FILE__, __LINE__);
    }
  }
  if (s != RQ_OK) {
    free_index_arrays(ix.get());
    return s;
  }
  s = finish_index_host_side(ix.get());
  if (s != RQ_OK) {
    free_index_arrays(ix.get());
    return s;
  }
  if (ix->h_offsets[ix->nlist] != ix->n) {
    free_index_arrays(ix.get());
    return fail(RQ_ERR_IO, "list offsets do not cover the index");
  }
  *out = ix.release();
  return RQ_OK;
}

void rq_free(rq_index* ix) {
  if (!ix) return;
  cudaDeviceSynchronize();
  free_plans(ix);
  if (ix->graph_stream) cudaStreamDestroy(ix->graph_stream);
  free_index_arrays(ix);
  cudaDeviceSynchronize();
  delete ix;
}

rq_status rq_device_error(rq_index* ix, int32_t* code) {
  if (!ix || !code) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  RQ_CUDA(cudaDeviceSynchronize());
  RQ_CUDA(cudaMemcpy(code, ix->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  RQ_CUDA(cudaMemset(ix->d_err, 0, sizeof(int32_t)));
  return RQ_OK;
}

rq_status rq_server_create(rq_index* ix, const rq_server_opts* opts, rq_server** out) {
  if (!ix || !out) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  std::unique_ptr<rq_server> s(new rq_server());
  s->ix = ix;
  rq_server_opts o{};
  if (opts) o = *opts;
  if (o.slots <= 0) o.slots = 4;
  if (o.slots > 64) return fail(RQ_ERR_INVALID_ARG, "slots above 64");
  if (o.max_batch <= 0) o.max_batch = 1024;
  if (o.max_queue <= 0) o.max_queue = 65536;
  if (o.memory_budget <= 0) {
    size_t fr = 0, tot = 0;
    RQ_CUDA(cudaMemGetInfo(&fr, &tot));
    o.memory_budget = (int64_t)(fr / 4);
  }
  s->opts = o;
  s->slots.resize(o.slots);
  for (auto& sl : s->slots) RQ_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
  rq_server* raw = s.get();
  raw->th = std::thread(server_loop, raw);
  *out = s.release();
  return RQ_OK;
}

rq_status rq_submit(rq_server* s, const float* q, int64_t nq, int32_t nprobe, int32_t k,
                    int32_t n_rerank, uint64_t* ticket) {
  if (!s || !q || !ticket) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  rq_index* ix = s->ix;
  if (nq < 1 || nq > s->opts.max_batch)
    return fail(RQ_ERR_INVALID_ARG, "nq outside [1, max_batch]");
  if (nprobe < 1 || nprobe > std::min(ix->nlist, kMaxSelect))
    return fail(RQ_ERR_INVALID_ARG, "nprobe out of range");
  if (k < 1 || k > kMaxSelect || (n_rerank != 0 && (n_rerank < k || n_rerank > kMaxSelect)))
    return fail(RQ_ERR_INVALID_ARG, "k / n_rerank out of range");
  for (int64_t i = 0; i < nq * ix->dim; ++i)
    if (!std::isfinite(q[i])) return fail(RQ_ERR_INVALID_ARG, "non-finite query value");
  auto r = std::make_shared<Request>();
  r->q.assign(q, q + nq * ix->dim);
  r->nq = nq;
  r->nprobe = nprobe;
  r->k = k;
  r->nrr = n_rerank;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(RQ_ERR_INVALID_ARG, "server is stopping");
    if ((int64_t)s->queue.size() >= s->opts.max_queue) return fail(RQ_ERR_BUSY, "queue full");
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return RQ_OK;
}

rq_status rq_wait(rq_server* s, uint64_t ticket, int64_t* ids, float* dist, int32_t timeout_ms,
                  double* latency_us) {
  if (!s || !ids || !dist) return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(RQ_ERR_INVALID_ARG, "unknown ticket");
  std::shared_ptr<Request> r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
    return fail(RQ_ERR_TIMEOUT, "request not finished within the timeout");
  }
  s->all.erase(ticket);
  lk.unlock();
  if (r->status != RQ_OK) return fail(r->status, r->error);
  std::memcpy(ids, r->ids.data(), sizeof(int64_t) * r->ids.size());
  std::memcpy(dist, r->dist.data(), sizeof(float) * r->dist.size());
  if (latency_us)
    *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
  return RQ_OK;
}

void rq_server_destroy(rq_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.h_q) cudaFreeHost(sl.h_q);
    if (sl.h_ids) cudaFreeHost(sl.h_ids);
    if (sl.h_d) cudaFreeHost(sl.h_d);
    if (sl.d_q) cudaFree(sl.d_q);
    if (sl.d_ids) cudaFree(sl.d_ids);
    if (sl.d_d) cudaFree(sl.d_d);
  }
  // Plans cached for the slot streams must go before the streams do.
  free_plans(s->ix);
  for (auto& sl : s->slots)
    if (sl.stream) cudaStreamDestroy(sl.stream);
  delete s;
}

}  // extern "C"
