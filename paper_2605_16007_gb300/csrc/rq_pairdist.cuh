// Pairwise squared distances in the fixed float32 order, shared by the
// k-means assignment (index build) and the centroid ranking (search).
#pragma once

#include "rq_common.cuh"

namespace rq {
namespace {

// For each pair, the terms d = 0, 1, 2, ... are (a - b) rounded, squared and
// rounded, then added and rounded (no fused multiply-add). Tiles of
// (16 RM) x 64 pairs, RM x 4 per thread.
//   MODE 0: per row of A, the nearest row of B (ties: lower id) -> out_arg.
//   MODE 1: the (distance, column) key of every pair -> out_keys (na x nb).
template <int MODE, int RM = 4>
__global__ void __launch_bounds__(256)
pair_dist_kernel(const float* __restrict__ A, int64_t na, const float* __restrict__ B,
                 int nb, int dim, int32_t* out_arg, float* out_min,
                 uint64_t* out_keys) {
  constexpr int ROWS = 16 * RM;
  __shared__ float As[32][ROWS + 1];
  __shared__ float Bs[32][65];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  float best_d[RM];
  int best_c[RM];
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    best_d[i] = __int_as_float(0x7f800000);
    best_c[i] = 0x7fffffff;
  }
  const int ctiles = (MODE == 0) ? (nb + 63) / 64 : 1;
  for (int ct = 0; ct < ctiles; ++ct) {
    const int col0 = (MODE == 0) ? ct * 64 : blockIdx.y * 64;
    float acc[RM][4];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int d0 = 0; d0 < dim; d0 += 32) {
      for (int t = threadIdx.x; t < ROWS * 32; t += 256) {
        const int r = t >> 5, dk = t & 31;
        const int d = d0 + dk;
        const int64_t ar = row0 + r;
        As[dk][r] = (ar < na && d < dim) ? A[ar * dim + d] : 0.0f;
      }
      for (int t = threadIdx.x; t < 64 * 32; t += 256) {
        const int r = t >> 5, dk = t & 31;
        const int d = d0 + dk;
        const int bc = col0 + r;
        Bs[dk][r] = (bc < nb && d < dim) ? B[(int64_t)bc * dim + d] : 0.0f;
      }
      __syncthreads();
#pragma unroll 4
      for (int dk = 0; dk < 32; ++dk) {
        float a[RM], b[4];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = As[dk][RM * ty + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[dk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float df = __fsub_rn(a[i], b[j]);
            acc[i][j] = __fadd_rn(acc[i][j], __fmul_rn(df, df));
          }
      }
      __syncthreads();
    }
    if (MODE == 0) {
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = col0 + tx + 16 * j;
          if (c < nb && acc[i][j] < best_d[i]) {
            best_d[i] = acc[i][j];
            best_c[i] = c;
          }
        }
    } else {
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        const int64_t r = row0 + RM * ty + i;
        if (r >= na) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = col0 + tx + 16 * j;
          if (c < nb) out_keys[r * nb + c] = make_key(acc[i][j], (uint32_t)c);
        }
      }
    }
  }
  if (MODE == 0) {
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      float d = best_d[i];
      int c = best_c[i];
#pragma unroll
      for (int o = 8; o; o >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, d, o);
        const int oc = __shfl_xor_sync(0xffffffffu, c, o);
        if (od < d || (od == d && oc < c)) {
          d = od;
          c = oc;
        }
      }
      const int64_t r = row0 + RM * ty + i;
      if (tx == 0 && r < na) {
        out_arg[r] = c;
        if (out_min) out_min[r] = d;
      }
    }
  }
}

}  // namespace
}  // namespace rq
