// The RaBitQ estimator on packed codes and query bit-planes (Eqs. 4-5,
// Section 3.3.2), and the survivor output shared by the scan kernels.
#pragma once

#include "rq_common.cuh"
#include "rq_internal.h"

namespace rq {

constexpr int kGroupVectors = 256;  // vectors per work item of the persistent scans

// An integer x with |x| < 2^22 as a float32, exactly, without the
// conversion unit: the bits 0x4B400000 + x are the float 1.5 * 2^23 + x
// (the same exponent for every such x), and subtracting 1.5 * 2^23 is exact.
__device__ __forceinline__ float small_int_to_float(int x) {
  return __fsub_rn(__int_as_float(0x4B400000 + x), 12582912.0f);
}

// With ip = sum_d bit_d q_u,d (bit-planes: ip = sum_j 2^j popc(code & plane_j))
// and pc = popc(code):
//   t  = delta (2 ip - Sq) + vl (2 pc - D_p)
//   d2 = (nq2 + r^2) - 2 (f t),  f = r / (sqrt(D_p) alpha),
// every operation rounded once in float32, then + 0 (turns -0 into +0).
// qp = {vl, delta, nq2, Sq (int bits)}, fac = {r^2, f}; `pl` holds the four
// planes (W words each) in shared memory, 16-byte aligned.
template <int NW4>
__device__ __forceinline__ float estimate_regs(const uint4 (&code)[NW4], int pc, float2 fac,
                                               const uint32_t* pl, float4 qp, int dp) {
  constexpr int W = 4 * NW4;
  int s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  const uint4* p4 = reinterpret_cast<const uint4*>(pl);
#pragma unroll
  for (int i = 0; i < NW4; ++i) {
    const uint4 c = code[i];
    const uint4 a0 = p4[0 * (W / 4) + i];
    const uint4 a1 = p4[1 * (W / 4) + i];
    const uint4 a2 = p4[2 * (W / 4) + i];
    const uint4 a3 = p4[3 * (W / 4) + i];
    s0 += __popc(c.x & a0.x) + __popc(c.y & a0.y) + __popc(c.z & a0.z) + __popc(c.w & a0.w);
    s1 += __popc(c.x & a1.x) + __popc(c.y & a1.y) + __popc(c.z & a1.z) + __popc(c.w & a1.w);
    s2 += __popc(c.x & a2.x) + __popc(c.y & a2.y) + __popc(c.z & a2.z) + __popc(c.w & a2.w);
    s3 += __popc(c.x & a3.x) + __popc(c.y & a3.y) + __popc(c.z & a3.z) + __popc(c.w & a3.w);
  }
  const int ip = s0 + 2 * s1 + 4 * s2 + 8 * s3;
  const int sq = __float_as_int(qp.w);
  const float a = small_int_to_float(2 * ip - sq);
  const float b = small_int_to_float(2 * pc - dp);
  const float t = __fadd_rn(__fmul_rn(qp.y, a), __fmul_rn(qp.x, b));
  const float d = __fsub_rn(__fadd_rn(qp.z, fac.x), __fmul_rn(2.0f, __fmul_rn(fac.y, t)));
  return __fadd_rn(d, 0.0f);
}


// The bound as a float32 threshold. The estimates compared with it are
// never -0 or NaN, and neither is a bound taken from them, so
// orderable(d) <= tau exactly when d <= tau_threshold(tau) (all ones: no
// bound, +inf).
__device__ __forceinline__ float tau_threshold(uint32_t tau) {
  return tau == kU32Max ? __int_as_float(0x7f800000) : from_orderable(tau);
}

// Scan output without atomics: survivor masks only. The vectors of a probed
// list are cut into 32-vector words; word w of probe p of query q has the
// fixed mask index x = q * mwords + wbase[q, p] + w (bit i set: vector
// 32 w + i of the list passed the query's bound). Every word of every probed
// list is written on every search, so the masks are never cleared. The
// finalize kernel recomputes the estimate of each surviving vector (every
// scan form computes the same float32 value) and pairs it with the row id.
// A warp holds one word (lane i = vector 32 w + i).
__device__ __forceinline__ void emit_word(bool pass, int64_t widx, uint32_t* __restrict__ mask,
                                          int lane) {
  const uint32_t m = __ballot_sync(0xffffffffu, pass);
  if (lane == 0) mask[widx] = m;
}

// The same for a chunk of J pairs over one word: bit j of `passbits` says
// whether this lane's vector passes for pair j, whose first mask index is
// wrow[j] (the word's index is wrow[j] + word); lane j writes pair j's mask
// word. Pairs j >= nvalid and words past the list's end (word_valid false,
// where no lane passes) write no mask. All 32 lanes must call it.
template <int J>
__device__ __forceinline__ void emit_chunk(uint32_t passbits, const int64_t* wrow, int nvalid,
                                           int64_t word, bool word_valid,
                                           uint32_t* __restrict__ mask, int lane) {
  uint32_t mine = 0;
  if (__any_sync(0xffffffffu, passbits != 0)) {  // else (the common case) every word is 0
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const uint32_t m = __ballot_sync(0xffffffffu, (passbits >> j) & 1u);
      if (lane == j) mine = m;
    }
  }
  if (word_valid && lane < J && lane < nvalid) mask[wrow[lane] + word] = mine;
}

// FP8 E4M3 encoding of an integer 0..15 (exact): v = 2^e (1 + m/8) with
// e = floor(log2 v), stored as (e + 7) << 3 | m; 0 encodes as 0.
__device__ __forceinline__ uint8_t e4m3_of_int(int v) {
  if (v <= 0) return 0;
  const int e = 31 - __clz(v);
  const int m = (v << (3 - e)) & 7;
  return (uint8_t)(((e + 7) << 3) | m);
}

// Bytes of one pair record of the streaming scan: the four bit-planes
// (4 x D_p/8 bytes), then {vl, delta, nq2, Sq (int bits)} and {query, first
// mask word, bound, 0}, 16 bytes each.
__host__ __device__ constexpr int pair_rec_bytes(int dp) { return dp / 2 + 32; }

// Streaming popcount scan (rq_scan_stream.cu).
rq_status launch_scan_stream(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                             int sms, uint64_t wait_ns, int withhold);

// Tensor-core centroid ranking (rq_probe_tc.cu): g = ||c||^2 - 2 <q', c>
// (nq x nlist) and cn = ||c||^2, D_p 128; its approximate distances are
// within kTcProbeEscale (||q'||^2 + ||c||^2) of the exact ones.
constexpr float kTcProbeEscale = 0.00390625f;  // 2^-8
rq_status launch_approx_dist_tc(const float* qrot, int64_t nq, const float* cR, int nlist, int dp,
                                float* g, float* cn, int32_t* err, cudaStream_t st);

// Tensor-core scan (rq_scan_mma.cu). With `window` it is the first bound's
// grouped pass instead: over the window bucket, writing each window
// candidate's estimate (orderable uint32) into its query's key buffer.
bool mma_supported(const rq_index* ix);
rq_status launch_scan_mma(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                          int sms, int withhold, bool window);
int next_pow2_host(int64_t v);

}  // namespace rq
