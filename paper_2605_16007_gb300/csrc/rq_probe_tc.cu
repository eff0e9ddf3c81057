// The approximate centroid ranking of the certified probe selection on the
// tensor cores: g = ||c||^2 - 2 <q', c> for a 128-query x 128-centroid tile
// per block, the inner products by tcgen05.mma kind::tf32 (Section 3.2.1
// computes the query-centroid distances as one matrix product on the
// accelerator's matrix unit).
//
// TF32 keeps 10 of float32's 23 mantissa bits of each input (the tensor
// core reads the float32 bits and drops the rest), so each input is off by
// less than 2^-10 relative and each product q_d c_d by less than 2^-9
// relative; the products are exact in float32 and at most D_p - 1 float32
// additions follow, in any order, each off by at most 2^-23 relative. So
// |<q', c>_tc - <q', c>| <= (2^-9 + D_p 2^-23) sum_d |q_d c_d|
//                        <= (2^-10 + D_p 2^-24) (||q'||^2 + ||c||^2),
// and with the float32 roundings of ||c||^2, of g and of ||q'||^2 + g, the
// approximate distance is within 2^-8 (||q'||^2 + ||c||^2) of the
// fixed-order exact distance at D_p = 128: the bound the selection then uses
// (kTcProbeEscale).
#include <cuda_runtime.h>

#include <algorithm>

#include "rq_async.cuh"
#include "rq_common.cuh"
#include "rq_internal.h"
#include "rq_scan.cuh"
#include "rq_tc.cuh"

namespace rq {
namespace {

constexpr int kTcM = 128;        // queries per block (TMEM lanes)
constexpr int kTcN = 128;        // centroids per block (TMEM columns)
constexpr int kTcK = 128;        // D_p
constexpr int kTcKb = kTcK / 32; // 128-byte K-blocks of float32 rows
constexpr int kTcThreads = 128;
constexpr int kTcSmA = 0;                            // kTcKb x 128 rows x 128 B
constexpr int kTcSmB = kTcSmA + kTcKb * kTcM * 128;  // kTcKb x 128 rows x 128 B
constexpr int kTcSmCn = kTcSmB + kTcKb * kTcN * 128; // 128 floats
constexpr int kTcSmBar = kTcSmCn + kTcN * 4;         // one mbarrier
constexpr int kTcSmTmem = kTcSmBar + 8;
constexpr int kTcSmAlloc = kTcSmTmem + 4 + 1024;     // + room to align the base

__global__ void __launch_bounds__(kTcThreads, 1)
approx_dist_tc_kernel(const float* __restrict__ qrot, int64_t nq, const float* __restrict__ cR,
                      int nlist, float* __restrict__ g, float* __restrict__ cn_out,
                      int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ volatile int s_ok;
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sbase = smem_u32(sm);
  float* s_cn = reinterpret_cast<float*>(sm + kTcSmCn);
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(sm + kTcSmTmem);
  const uint32_t bar = sbase + kTcSmBar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kTcM;
  const int col0 = blockIdx.y * kTcN;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(sbase + kTcSmTmem, kTcN);
    tmem_relinquish();
  }
  // Thread t stages query row row0 + t and centroid row col0 + t (zeros past
  // the ends) as K-major 128-byte rows with the 128B swizzle, one K-block of
  // 32 floats after another (the loads of a K-block in flight together).
  {
    const bool qa = row0 + tid < nq, cb = col0 + tid < nlist;
    const float4* qs = reinterpret_cast<const float4*>(qrot + (row0 + tid) * kTcK);
    const float4* cs = reinterpret_cast<const float4*>(cR + (int64_t)(col0 + tid) * kTcK);
    float cn = 0.0f;
#pragma unroll 1
    for (int kb = 0; kb < kTcKb; ++kb) {
      float4 va[8], vb[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        va[c] = qa ? __ldg(qs + 8 * kb + c) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        vb[c] = cb ? __ldg(cs + 8 * kb + c) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // 16-byte chunk c of the row's K-block kb
        *reinterpret_cast<float4*>(sm + kTcSmA + kb * kTcM * 128 + sw128_offset(tid, c)) = va[c];
        *reinterpret_cast<float4*>(sm + kTcSmB + kb * kTcN * 128 + sw128_offset(tid, c)) = vb[c];
        cn = fmaf(vb[c].x, vb[c].x, cn);
        cn = fmaf(vb[c].y, vb[c].y, cn);
        cn = fmaf(vb[c].z, vb[c].z, cn);
        cn = fmaf(vb[c].w, vb[c].w, cn);
      }
    }
    s_cn[tid] = cn;
    if (blockIdx.x == 0 && cb) cn_out[col0 + tid] = cn;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_tmem;
  if (tid == 0) {
    const uint32_t id = idesc_tf32_f32(kTcM, kTcN);
#pragma unroll
    for (int kb = 0; kb < kTcKb; ++kb) {
      const uint64_t ad = sdesc_sw128(sbase + kTcSmA + kb * kTcM * 128);
      const uint64_t bd = sdesc_sw128(sbase + kTcSmB + kb * kTcN * 128);
#pragma unroll
      for (int s = 0; s < 4; ++s)  // K = 8 floats (32 bytes) per instruction
        mma_tf32(taddr, ad + (uint64_t)(2 * s), bd + (uint64_t)(2 * s), id, (kb | s) != 0);
    }
    mma_commit(bar);
    const bool ok = mbar_wait_bounded(bar, 0u, kWaitLimitNs);
    if (!ok) {
      flag_error(err, kErrMmaTimeout);
      mbar_wait_bounded(bar, 0u, kWaitLimitNs);  // let it land before the TMEM goes
    }
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  tc_fence_after();
  if (s_ok) {
    // thread t: query row row0 + t = TMEM lane t (warp w: lanes 32 w ..)
    const int64_t r = row0 + tid;
    const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16);
    for (int c8 = 0; c8 < kTcN; c8 += 8) {
      uint32_t v[8];
      tmem_ld8(tl + (uint32_t)c8, v);
      if (r < nq) {
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = fmaf(-2.0f, __uint_as_float(v[j]), s_cn[c8 + j]);
        float* dst = g + r * nlist + col0 + c8;
        if (col0 + c8 + 8 <= nlist && (nlist & 3) == 0) {
          *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
          *reinterpret_cast<float4*>(dst + 4) = make_float4(o[4], o[5], o[6], o[7]);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (col0 + c8 + j < nlist) dst[j] = o[j];
        }
      }
    }
  }
  (void)lane;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(taddr, kTcN);
}

}  // namespace

rq_status launch_approx_dist_tc(const float* qrot, int64_t nq, const float* cR, int nlist, int dp,
                                float* g, float* cn, int32_t* err, cudaStream_t st) {
  if (dp != kTcK) return fail(RQ_ERR_NOT_IMPLEMENTED, "tensor-core centroid ranking: D_p 128 only");
  RQ_TRY(allow_dynamic_smem((const void*)approx_dist_tc_kernel, kTcSmAlloc));
  const dim3 grid((unsigned)((nq + kTcM - 1) / kTcM), (unsigned)((nlist + kTcN - 1) / kTcN));
  approx_dist_tc_kernel<<<grid, kTcThreads, kTcSmAlloc, st>>>(qrot, nq, cR, nlist, g, cn, err);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

}  // namespace rq
