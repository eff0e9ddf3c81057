// Index build on the GPU (Section 3.1.1): k-means (Phases 1-2), the random
// orthogonal rotation P (Section 2.2.1), and the encode of every vector into a
// sign code plus the factors r = ||x - c|| and alpha (Eqs. 1-3, Phase 3).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rq_common.cuh"
#include "rq_internal.h"
#include "rq_pairdist.cuh"
#include "rq_scan.cuh"

namespace rq {
namespace {

// Stream ids of the method's random draws (third Philox counter word).
constexpr uint32_t kStreamRotation = 1;
constexpr uint32_t kStreamKmeansInit = 2;
constexpr uint32_t kStreamTrainSample = 3;

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  rq_status alloc(size_t count) {
    n = count;
    cudaError_t e = dev_alloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(RQ_ERR_OOM, "device allocation of " +
                                  std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return RQ_OK;
  }
  T* release() {
    T* q = p;
    p = nullptr;
    return q;
  }
};

inline unsigned blocks_for(int64_t n, int per) {
  return (unsigned)std::max<int64_t>(1, (n + per - 1) / per);
}

// ---------------------------------------------------------------------------
// Philox Gaussian draws (Box-Muller): pair i from block (i, stream).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double unit_open(uint64_t a) {
  return ((double)(a >> 12) + 0.5) * 0x1p-52;
}

__global__ void gaussian_kernel(uint64_t seed, uint32_t stream, int64_t count,
                                double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (2 * i >= count) return;
  const uint4 w = philox_block(seed, stream, (uint64_t)i);
  const uint64_t a = (uint64_t)w.x | ((uint64_t)w.y << 32);
  const uint64_t b = (uint64_t)w.z | ((uint64_t)w.w << 32);
  const double rho = sqrt(-2.0 * log(unit_open(a)));
  const double theta = 6.283185307179586 * unit_open(b);
  out[2 * i] = rho * cos(theta);
  if (2 * i + 1 < count) out[2 * i + 1] = rho * sin(theta);
}

// Row-major Gaussian matrix element (i, j) = g[i * n + j] stored
// column-major for the QR below.
__global__ void to_col_major_kernel(const double* g, double* a, int n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  a[i + (int64_t)j * n] = g[t];
}

// ---------------------------------------------------------------------------
// Householder QR (float64), column-major n x n.
// ---------------------------------------------------------------------------
__device__ double block_sum_double(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// Reflector of column k: v = a - alpha e_k with alpha = -sign(a_k) ||a||,
// beta = 2 / (v . v); column k of A becomes (alpha, 0, ...).
__global__ void house_vec_kernel(double* A, double* V, double* beta, int n, int k) {
  __shared__ double red[32];
  double ss = 0.0;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double a = A[i + (int64_t)k * n];
    ss += a * a;
  }
  const double sigma2 = block_sum_double(ss, red);
  const double sigma = sqrt(sigma2);
  const double akk = A[k + (int64_t)k * n];
  const double alpha = (akk >= 0.0) ? -sigma : sigma;
  const double v0 = akk - alpha;
  const double vn2 = sigma2 - akk * akk + v0 * v0;
  __syncthreads();
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    V[i + (int64_t)k * n] = (i == k) ? v0 : A[i + (int64_t)k * n];
    if (vn2 > 0.0) A[i + (int64_t)k * n] = (i == k) ? alpha : 0.0;
  }
  if (threadIdx.x == 0) beta[k] = (vn2 > 0.0) ? 2.0 / vn2 : 0.0;
}

// Apply H_k = I - beta v v^T to columns j >= j0 of M (rows k..n-1); one warp
// per column.
__global__ void house_apply_kernel(double* M, const double* V, const double* beta,
                                   int n, int k, int j0) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int j = j0 + warp;
  if (j >= n) return;
  const double b = beta[k];
  if (b == 0.0) return;
  const double* v = V + (int64_t)k * n;
  double* col = M + (int64_t)j * n;
  double w = 0.0;
  for (int i = k + lane; i < n; i += 32) w += v[i] * col[i];
  for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  const double s = b * w;
  for (int i = k + lane; i < n; i += 32) col[i] -= s * v[i];
}

__global__ void identity_kernel(double* Q, int n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  Q[t] = ((t % n) == (t / n)) ? 1.0 : 0.0;
}

// P[i][j] (row-major) = Q[i][j] * sign(R[j][j]), sign(0) = +1.
__global__ void sign_fix_kernel(const double* Q, const double* R, double* P,
                                float* P32, int n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  const double s = (R[j + (int64_t)j * n] < 0.0) ? -1.0 : 1.0;
  const double v = Q[i + (int64_t)j * n] * s;
  P[t] = v;
  P32[t] = (float)v;
}

__global__ void to_f32_kernel(const double* a, float* b, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

rq_status random_orthogonal(uint64_t seed, int n, double* d_P, float* d_P32) {
  const int64_t nn = (int64_t)n * n;
  DevBuf<double> g, A, V, beta, Q;
  RQ_TRY(g.alloc(nn));
  RQ_TRY(A.alloc(nn));
  RQ_TRY(V.alloc(nn));
  RQ_TRY(beta.alloc(n));
  RQ_TRY(Q.alloc(nn));
  gaussian_kernel<<<blocks_for((nn + 1) / 2, 256), 256>>>(seed, kStreamRotation, nn, g.p);
  to_col_major_kernel<<<blocks_for(nn, 256), 256>>>(g.p, A.p, n);
  RQ_CUDA(cudaMemset(beta.p, 0, n * sizeof(double)));
  for (int k = 0; k + 1 < n; ++k) {
    house_vec_kernel<<<1, 256>>>(A.p, V.p, beta.p, n, k);
    const int cols = n - k - 1;
    house_apply_kernel<<<blocks_for((int64_t)cols * 32, 256), 256>>>(A.p, V.p, beta.p, n, k, k + 1);
  }
  identity_kernel<<<blocks_for(nn, 256), 256>>>(Q.p, n);
  for (int k = n - 2; k >= 0; --k) {
    const int cols = n - k;
    house_apply_kernel<<<blocks_for((int64_t)cols * 32, 256), 256>>>(Q.p, V.p, beta.p, n, k, k);
  }
  sign_fix_kernel<<<blocks_for(nn, 256), 256>>>(Q.p, A.p, d_P, d_P32, n);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits.
// ---------------------------------------------------------------------------
constexpr int kSortTile = 4096;

__global__ void radix_hist_kernel(const uint64_t* keys, int64_t n, int shift,
                                  int32_t* hist, int ntiles) {
  __shared__ int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t lo = (int64_t)blockIdx.x * kSortTile;
  const int64_t hi = min(n, lo + kSortTile);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&h[(keys[i] >> shift) & 255], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Exclusive scan of m ints in one block (chunked sequential + block scan).
__global__ void exclusive_scan_kernel(const int32_t* in, int64_t* out, int64_t m) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t chunk = (m + T - 1) / T;
  const int64_t lo = min(m, (int64_t)t * chunk), hi = min(m, lo + chunk);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < T; ++i) {
      const int64_t v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t v = in[i];
    out[i] = run;
    run += v;
  }
}

// out[m] = total, for an output sized m + 1.
__global__ void scan_total_kernel(const int32_t* in, int64_t* out, int64_t m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[m] = (m > 0 ? out[m - 1] + in[m - 1] : 0);
}

// One warp per tile keeps the scatter stable: 32 elements at a time in
// order, ranks among equal digits from a match mask.
__global__ void radix_scatter_kernel(const uint64_t* keys, const uint32_t* vals,
                                     int64_t n, int shift, const int64_t* offs,
                                     int ntiles, uint64_t* keys_out,
                                     uint32_t* vals_out) {
  __shared__ int64_t ctr[256];
  const int lane = threadIdx.x;
  for (int i = lane; i < 256; i += 32) ctr[i] = offs[(int64_t)i * ntiles + blockIdx.x];
  __syncwarp();
  const int64_t lo = (int64_t)blockIdx.x * kSortTile;
  const int64_t hi = min(n, lo + kSortTile);
  for (int64_t base = lo; base < hi; base += 32) {
    const int64_t i = base + lane;
    const bool ok = i < hi;
    const unsigned active = __ballot_sync(0xffffffffu, ok);
    uint64_t k = 0;
    uint32_t v = 0;
    int d = -1;
    if (ok) {
      k = keys[i];
      v = vals[i];
      d = (int)((k >> shift) & 255);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d) & active;
    int64_t pos = 0;
    if (ok) {
      const int rank = __popc(peers & ((1u << lane) - 1u));
      pos = ctr[d] + rank;
    }
    __syncwarp();
    if (ok && (__ffs(peers) - 1) == lane) ctr[d] += __popc(peers);
    __syncwarp();
    if (ok) {
      keys_out[pos] = k;
      vals_out[pos] = v;
    }
  }
}

// Sorts keys/vals in place (ping-pong through tmp buffers) on bits
// [lo_bit, hi_bit).
rq_status radix_sort(uint64_t* keys, uint32_t* vals, int64_t n, int lo_bit,
                     int hi_bit) {
  if (n <= 1) return RQ_OK;
  const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  const int64_t m = (int64_t)ntiles * 256;
  DevBuf<uint64_t> k2;
  DevBuf<uint32_t> v2;
  DevBuf<int32_t> hist;
  DevBuf<int64_t> offs;
  RQ_TRY(k2.alloc(n));
  RQ_TRY(v2.alloc(n));
  RQ_TRY(hist.alloc(m));
  RQ_TRY(offs.alloc(m + 1));
  uint64_t* ka = keys;
  uint32_t* va = vals;
  uint64_t* kb = k2.p;
  uint32_t* vb = v2.p;
  int passes = 0;
  for (int shift = lo_bit; shift < hi_bit; shift += 8, ++passes) {
    radix_hist_kernel<<<ntiles, 256>>>(ka, n, shift, hist.p, ntiles);
    exclusive_scan_kernel<<<1, 1024>>>(hist.p, offs.p, m);
    radix_scatter_kernel<<<ntiles, 32>>>(ka, va, n, shift, offs.p, ntiles, kb, vb);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    RQ_CUDA(cudaMemcpy(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice));
    RQ_CUDA(cudaMemcpy(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice));
  }
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

int bits_for(int64_t v) {  // bits needed for values in [0, v)
  int b = 0;
  while (b < 63 && (int64_t(1) << b) < v) ++b;
  return std::max(b, 1);
}

// ---------------------------------------------------------------------------
// Rank keys (Philox word << 32 | row) and small utilities.
// ---------------------------------------------------------------------------
__global__ void row_keys_kernel(uint64_t seed, uint32_t stream, const uint32_t* rows,
                                int64_t n, uint64_t* keys, uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t row = rows ? rows[i] : (uint32_t)i;
  const uint4 w = philox_block(seed, stream, (uint64_t)row);
  keys[i] = ((uint64_t)w.x << 32) | row;
  vals[i] = row;
}

__global__ void iota_keys_kernel(const uint32_t* in, int64_t n, uint64_t* keys,
                                 uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = in[i];
  vals[i] = in[i];
}

__global__ void gather_rows_kernel(const float* x, int dim, const uint32_t* rows,
                                   int64_t m, float* out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m * dim) return;
  const int64_t i = t / dim;
  const int d = (int)(t % dim);
  out[t] = x[(int64_t)rows[i] * dim + d];
}

// ---------------------------------------------------------------------------
// k-means update: mean of each cluster's members, summed in float64 in
// ascending row order, divided in float64, rounded to float32.
// ---------------------------------------------------------------------------
__global__ void histogram_kernel(const int32_t* a, int64_t n, int32_t* counts) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&counts[a[i]], 1);
}

__global__ void cluster_keys_kernel(const int32_t* a, int64_t n, uint64_t* keys,
                                    uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = (uint64_t)(uint32_t)a[i];
  vals[i] = (uint32_t)i;
}

__global__ void centroid_mean_kernel(const float* x, int dim, const uint32_t* rows,
                                     const int64_t* off, float* c) {
  const int j = blockIdx.x;
  const int64_t lo = off[j], hi = off[j + 1];
  if (hi == lo) return;
  for (int d = threadIdx.x; d < dim; d += blockDim.x) {
    double s = 0.0;
    for (int64_t m = lo; m < hi; ++m) s += (double)x[(int64_t)rows[m] * dim + d];
    c[(int64_t)j * dim + d] = (float)(s / (double)(hi - lo));
  }
}

// Empty clusters, in ascending id: take from the largest cluster (ties: lowest
// id) its member farthest from that cluster's new centroid (ties: lowest row).
__global__ void reseed_empty_kernel(const float* x, int dim, int nlist,
                                    const uint32_t* rows, const int64_t* off,
                                    int32_t* a, int32_t* counts, float* c) {
  __shared__ int s_any;
  __shared__ float s_bd[256];
  __shared__ int64_t s_bm[256];
  __shared__ int s_bc[256];
  __shared__ int s_donor;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < nlist; j += blockDim.x)
    if (counts[j] == 0) s_any = 1;
  __syncthreads();
  if (!s_any) return;
  for (int j = 0; j < nlist; ++j) {
    if (counts[j] != 0) continue;  // uniform: every thread reads the same value
    // donor = argmax counts, lowest id on ties
    int bc = -1, bi = 0x7fffffff;
    for (int t = threadIdx.x; t < nlist; t += blockDim.x)
      if (counts[t] > bc) {
        bc = counts[t];
        bi = t;
      }
    s_bc[threadIdx.x] = bc;
    s_bm[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
      int best = -1;
      int64_t bid = 0x7fffffff;
      for (int t = 0; t < (int)blockDim.x; ++t)
        if (s_bc[t] > best || (s_bc[t] == best && s_bm[t] < bid)) {
          best = s_bc[t];
          bid = s_bm[t];
        }
      s_donor = (int)bid;
    }
    __syncthreads();
    const int donor = s_donor;
    const float* cd = c + (int64_t)donor * dim;
    float bd = -1.0f;
    int64_t bm = -1;
    for (int64_t m = off[donor] + threadIdx.x; m < off[donor + 1]; m += blockDim.x) {
      const uint32_t row = rows[m];
      if (a[row] != donor) continue;
      float acc = 0.0f;
      for (int d = 0; d < dim; ++d) {
        const float df = __fsub_rn(x[(int64_t)row * dim + d], cd[d]);
        acc = __fadd_rn(acc, __fmul_rn(df, df));
      }
      if (acc > bd) {  // members visited in ascending row per thread
        bd = acc;
        bm = row;
      }
    }
    s_bd[threadIdx.x] = bd;
    s_bm[threadIdx.x] = bm;
    __syncthreads();
    if (threadIdx.x == 0) {
      float best = -1.0f;
      int64_t brow = -1;
      for (int t = 0; t < (int)blockDim.x; ++t) {
        if (s_bm[t] < 0) continue;
        if (s_bd[t] > best || (s_bd[t] == best && s_bm[t] < brow)) {
          best = s_bd[t];
          brow = s_bm[t];
        }
      }
      s_bm[0] = brow;
    }
    __syncthreads();
    const int64_t far = s_bm[0];
    for (int d = threadIdx.x; d < dim; d += blockDim.x)
      c[(int64_t)j * dim + d] = x[far * dim + d];
    __syncthreads();
    if (threadIdx.x == 0) {
      a[far] = j;
      counts[donor] -= 1;
      counts[j] += 1;
    }
    __syncthreads();
  }
}

rq_status assign_rows(const float* x, int64_t n, int dim, const float* c, int nlist,
                      int32_t* a, float* dmin) {
  pair_dist_kernel<0><<<blocks_for(n, 64), 256>>>(x, n, c, nlist, dim, a, dmin, nullptr);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

// Counting sort of rows by cluster (stable in row order) -> rows, offsets.
rq_status group_by_cluster(const int32_t* a, int64_t n, int nlist, uint32_t* rows,
                           int64_t* off, int32_t* counts) {
  DevBuf<uint64_t> keys;
  RQ_TRY(keys.alloc(n));
  cluster_keys_kernel<<<blocks_for(n, 256), 256>>>(a, n, keys.p, rows);
  RQ_TRY(radix_sort(keys.p, rows, n, 0, bits_for(nlist)));
  RQ_CUDA(cudaMemset(counts, 0, nlist * sizeof(int32_t)));
  histogram_kernel<<<blocks_for(n, 256), 256>>>(a, n, counts);
  exclusive_scan_kernel<<<1, 1024>>>(counts, off, nlist);
  scan_total_kernel<<<1, 1>>>(counts, off, nlist);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

// ---------------------------------------------------------------------------
// Encode. Z = U P for residual rows U = x - c (float32 GEMM, fused epilogue:
// sign bits and per-tile float64 sums of |z|).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
encode_gemm_kernel(const float* __restrict__ x, int dim, const uint32_t* __restrict__ ids,
                   const int32_t* __restrict__ assign, const float* __restrict__ cent,
                   const float* __restrict__ P32, int dp, int64_t n,
                   uint8_t* __restrict__ codes, double* __restrict__ zabs) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][64];
  __shared__ float Zs[64][65];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t s0 = (int64_t)blockIdx.x * 64;
  const int col0 = blockIdx.y * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < dim; k0 += 16) {
    for (int t = threadIdx.x; t < 64 * 16; t += 256) {
      const int r = t >> 4, kk = t & 15;
      const int k = k0 + kk;
      const int64_t s = s0 + r;
      float v = 0.0f;
      if (s < n && k < dim) {
        const uint32_t row = ids[s];
        const int cl = assign[row];
        v = __fsub_rn(x[(int64_t)row * dim + k], cent[(int64_t)cl * dim + k]);
      }
      As[kk][r] = v;
      const int kr = t >> 6, cc = t & 63;
      const int kb = k0 + kr;
      Bs[kr][cc] = (kb < dim) ? P32[(int64_t)kb * dp + col0 + cc] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][4 * ty + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Zs[4 * ty + i][tx + 16 * j] = acc[i][j];
  __syncthreads();
  const int C = dp / 8;
  for (int t = threadIdx.x; t < 64 * 8; t += 256) {
    const int r = t >> 3, b = t & 7;
    const int64_t s = s0 + r;
    if (s >= n) continue;
    uint32_t byte = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) byte |= (Zs[r][8 * b + i] >= 0.0f ? 1u : 0u) << i;
    codes[s * C + col0 / 8 + b] = (uint8_t)byte;
  }
  if (threadIdx.x < 64) {
    const int r = threadIdx.x;
    const int64_t s = s0 + r;
    if (s < n) {
      double sa = 0.0;
      for (int j = 0; j < 64; ++j) sa += (double)fabsf(Zs[r][j]);
      zabs[s * (dp / 64) + blockIdx.y] = sa;
    }
  }
}

// r = ||x - c|| (float64), alpha = sum|z| / (sqrt(D_p) r) (float64; 1 when
// r = 0), then the float32 scan factors {r^2, r / (sqrt(D_p) alpha)}.
__global__ void factors_kernel(const float* x, int dim, const uint32_t* ids,
                               const int32_t* assign, const float* cent, int dp,
                               int64_t n, const double* zabs, float* r_out,
                               float* alpha_out, float2* fac) {
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= n) return;
  const uint32_t row = ids[s];
  const int cl = assign[row];
  double ss = 0.0;
  for (int d = lane; d < dim; d += 32) {
    const double u = (double)x[(int64_t)row * dim + d] - (double)cent[(int64_t)cl * dim + d];
    ss += u * u;
  }
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane != 0) return;
  const double r = sqrt(ss);
  double za = 0.0;
  const int nt = dp / 64;
  for (int t = 0; t < nt; ++t) za += zabs[s * nt + t];
  const double alpha = (r > 0.0) ? za / (sqrt((double)dp) * r) : 1.0;
  const float r32 = (float)r, a32 = (float)alpha;
  r_out[s] = r32;
  alpha_out[s] = a32;
  const float f = __fdiv_rn(r32, __fmul_rn(__fsqrt_rn((float)dp), a32));
  fac[s] = make_float2(__fmul_rn(r32, r32), f);
}

// cR[c][j] = sum_i c[i] P[i][j] (float64, ascending i), rounded to float32.
__global__ void rotate_centroids_kernel(const float* cent, int dim, int nlist,
                                        const double* P, int dp, float* cR) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nlist * dp) return;
  const int c = (int)(t / dp), j = (int)(t % dp);
  double s = 0.0;
  for (int i = 0; i < dim; ++i) s += (double)cent[(int64_t)c * dim + i] * P[(int64_t)i * dp + j];
  cR[t] = (float)s;
}

}  // namespace

// ===========================================================================
rq_status philox_gaussian_device(uint64_t seed, uint32_t stream, int64_t count,
                                 double* d_out) {
  if (count <= 0) return RQ_OK;
  gaussian_kernel<<<blocks_for((count + 1) / 2, 256), 256>>>(seed, stream, count, d_out);
  RQ_CUDA(cudaGetLastError());
  RQ_CUDA(cudaDeviceSynchronize());
  return RQ_OK;
}

rq_status kmeans_device(const float* d_x, int64_t n, int dim, int nlist,
                        uint64_t seed, int iters, int64_t train_size,
                        float* d_centroids) {
  // Training subset: all rows, or the train_size rows of smallest rank key
  // (stream 3), in ascending row order.
  int64_t nt = n;
  DevBuf<uint32_t> trows;
  DevBuf<float> xt_buf;
  const float* xt = d_x;
  DevBuf<uint64_t> keys;
  DevBuf<uint32_t> vals;
  RQ_TRY(keys.alloc(n));
  RQ_TRY(vals.alloc(n));
  if (train_size > 0 && train_size < n) {
    nt = train_size;
    row_keys_kernel<<<blocks_for(n, 256), 256>>>(seed, kStreamTrainSample, nullptr, n, keys.p, vals.p);
    RQ_TRY(radix_sort(keys.p, vals.p, n, 32, 64));
    RQ_TRY(trows.alloc(nt));
    iota_keys_kernel<<<blocks_for(nt, 256), 256>>>(vals.p, nt, keys.p, trows.p);
    RQ_TRY(radix_sort(keys.p, trows.p, nt, 0, bits_for(n)));
    RQ_TRY(xt_buf.alloc((size_t)nt * dim));
    gather_rows_kernel<<<blocks_for(nt * dim, 256), 256>>>(d_x, dim, trows.p, nt, xt_buf.p);
    xt = xt_buf.p;
  }
  // Initial centroids: the nlist training rows of smallest rank key (stream
  // 2), in ascending key order.
  row_keys_kernel<<<blocks_for(nt, 256), 256>>>(seed, kStreamKmeansInit, trows.p, nt, keys.p, vals.p);
  RQ_TRY(radix_sort(keys.p, vals.p, nt, 32, 64));
  gather_rows_kernel<<<blocks_for((int64_t)nlist * dim, 256), 256>>>(d_x, dim, vals.p, nlist, d_centroids);
  RQ_CUDA(cudaGetLastError());
  if (iters <= 0) return RQ_OK;
  DevBuf<int32_t> a, counts;
  DevBuf<uint32_t> rows;
  DevBuf<int64_t> off;
  RQ_TRY(a.alloc(nt));
  RQ_TRY(counts.alloc(nlist));
  RQ_TRY(rows.alloc(nt));
  RQ_TRY(off.alloc(nlist + 1));
  for (int it = 0; it < iters; ++it) {
    RQ_TRY(assign_rows(xt, nt, dim, d_centroids, nlist, a.p, nullptr));
    RQ_TRY(group_by_cluster(a.p, nt, nlist, rows.p, off.p, counts.p));
    centroid_mean_kernel<<<nlist, std::min(1024, ((dim + 31) / 32) * 32)>>>(xt, dim, rows.p, off.p, d_centroids);
    reseed_empty_kernel<<<1, 256>>>(xt, dim, nlist, rows.p, off.p, a.p, counts.p, d_centroids);
    RQ_CUDA(cudaGetLastError());
  }
  return RQ_OK;
}

rq_status build_index(const float* d_base, const void* d_raw, rq_dtype dt,
                      int64_t n, int dim, int nlist, uint64_t seed, int iters,
                      int64_t train_size, const float* given_centroids,
                      const double* given_P, rq_index* ix) {
  const int dp = dim_pad(dim);
  ix->n = n;
  ix->dim = dim;
  ix->dp = dp;
  ix->nlist = nlist;
  ix->C = dp / 8;
  ix->raw_dtype = dt;
  DevBuf<double> P;
  DevBuf<float> P32, cent, cR, r, alpha;
  DevBuf<float2> fac;
  DevBuf<int64_t> off;
  DevBuf<uint8_t> codes;
  DevBuf<uint32_t> ids;
  DevBuf<int32_t> assign, err;
  RQ_TRY(P.alloc((size_t)dp * dp));
  RQ_TRY(P32.alloc((size_t)dp * dp));
  RQ_TRY(cent.alloc((size_t)nlist * dim));
  RQ_TRY(cR.alloc((size_t)nlist * dp));
  RQ_TRY(off.alloc(nlist + 1));
  RQ_TRY(codes.alloc((size_t)n * ix->C));
  RQ_TRY(r.alloc(n));
  RQ_TRY(alpha.alloc(n));
  RQ_TRY(fac.alloc(n + 2));  // 16 bytes of tail room for 16-byte bulk copies
  RQ_TRY(ids.alloc(n + 4));  // tail room for 16-byte bulk copies
  RQ_TRY(assign.alloc(n));
  RQ_TRY(err.alloc(1));
  RQ_CUDA(cudaMemset(err.p, 0, sizeof(int32_t)));

  // P (Section 2.2.1)
  if (given_P) {
    RQ_CUDA(cudaMemcpy(P.p, given_P, sizeof(double) * dp * dp, cudaMemcpyDefault));
    to_f32_kernel<<<blocks_for((int64_t)dp * dp, 256), 256>>>(P.p, P32.p, (int64_t)dp * dp);
  } else {
    RQ_TRY(random_orthogonal(seed, dp, P.p, P32.p));
  }
  // Centroids (Section 2.1.2)
  if (given_centroids) {
    RQ_CUDA(cudaMemcpy(cent.p, given_centroids, sizeof(float) * nlist * dim, cudaMemcpyDefault));
  } else {
    RQ_TRY(kmeans_device(d_base, n, dim, nlist, seed, iters, train_size, cent.p));
  }
  // Final assignment and list layout (ascending row inside each list).
  RQ_TRY(assign_rows(d_base, n, dim, cent.p, nlist, assign.p, nullptr));
  {
    DevBuf<int32_t> counts;
    RQ_TRY(counts.alloc(nlist));
    RQ_TRY(group_by_cluster(assign.p, n, nlist, ids.p, off.p, counts.p));
  }
  // Encode (Eqs. 1-3)
  {
    DevBuf<double> zabs;
    RQ_TRY(zabs.alloc((size_t)n * (dp / 64)));
    dim3 grid(blocks_for(n, 64), dp / 64);
    encode_gemm_kernel<<<grid, 256>>>(d_base, dim, ids.p, assign.p, cent.p, P32.p, dp, n,
                                      codes.p, zabs.p);
    factors_kernel<<<blocks_for(n * 32, 256), 256>>>(d_base, dim, ids.p, assign.p, cent.p, dp,
                                                     n, zabs.p, r.p, alpha.p, fac.p);
    RQ_CUDA(cudaGetLastError());
    RQ_CUDA(cudaDeviceSynchronize());
  }
  rotate_centroids_kernel<<<blocks_for((int64_t)nlist * dp, 256), 256>>>(cent.p, dim, nlist, P.p,
                                                                          dp, cR.p);
  RQ_CUDA(cudaGetLastError());
  RQ_CUDA(cudaDeviceSynchronize());
  ix->P = P.release();
  ix->P32 = P32.release();
  ix->centroids = cent.release();
  ix->cR = cR.release();
  ix->offsets = off.release();
  ix->codes = codes.release();
  ix->r = r.release();
  ix->alpha = alpha.release();
  ix->fac = fac.release();
  ix->ids = ids.release();
  ix->assign = assign.release();
  ix->d_err = err.release();
  ix->raw = const_cast<void*>(d_raw);
  return finish_index_host_side(ix);
}

// Host copies of the list layout, and the static work items of the grouped
// scans: every (list, first vector) block of kGroupVectors vectors.
rq_status finish_index_host_side(rq_index* ix) {
  ix->h_offsets.resize(ix->nlist + 1);
  RQ_CUDA(cudaMemcpy(ix->h_offsets.data(), ix->offsets, sizeof(int64_t) * (ix->nlist + 1),
                     cudaMemcpyDeviceToHost));
  std::vector<int64_t> len(ix->nlist);
  std::vector<int2> items;
  for (int l = 0; l < ix->nlist; ++l) {
    len[l] = ix->h_offsets[l + 1] - ix->h_offsets[l];
    for (int64_t v = 0; v < len[l]; v += kGroupVectors) items.push_back(make_int2(l, (int)v));
  }
  // Persistent scans take items in this order: blocks of the longest lists
  // first (longer lists are near more queries, so their items tend to carry
  // more pairs), full blocks before a list's tail -- the costly items start
  // early and the cheap ones fill the end.
  std::stable_sort(items.begin(), items.end(), [&](const int2& a, const int2& b) {
    const int64_t na = std::min<int64_t>(kGroupVectors, len[a.x] - a.y);
    const int64_t nb = std::min<int64_t>(kGroupVectors, len[b.x] - b.y);
    if (len[a.x] != len[b.x]) return len[a.x] > len[b.x];
    return na > nb;
  });
  std::sort(len.begin(), len.end(), std::greater<int64_t>());
  ix->max_list_len = ix->nlist > 0 ? len[0] : 0;
  ix->top_len_prefix.assign(ix->nlist + 1, 0);
  ix->top_words_prefix.assign(ix->nlist + 1, 0);
  for (int l = 0; l < ix->nlist; ++l) {
    ix->top_len_prefix[l + 1] = ix->top_len_prefix[l] + len[l];
    ix->top_words_prefix[l + 1] = ix->top_words_prefix[l] + (len[l] + 31) / 32;
  }
  if (ix->items) cudaFree(ix->items);
  ix->items = nullptr;
  ix->n_items = (int)items.size();
  RQ_CUDA(dev_alloc(&ix->items, sizeof(int2) * std::max<size_t>(items.size(), 1)));
  RQ_CUDA(cudaMemcpy(ix->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  return RQ_OK;
}

}  // namespace rq
