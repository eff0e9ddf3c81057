// The RaBitQ estimator on packed codes and query bit-planes (Eqs. 4-5,
// Section 3.3.2), and the candidate append shared by the scan kernels.
#pragma once

#include "rq_common.cuh"
#include "rq_internal.h"

namespace rq {

constexpr int kGroupVectors = 256;  // vectors per grouped work item (one per thread)

// Pairs per grouped work item: query planes of the group sit in shared memory.
inline int group_pairs_for(int dp) { return dp <= 1024 ? 64 : 32; }
template <int NW4>
struct GroupPairs {
  static constexpr int value = (NW4 <= 8) ? 64 : 32;
};

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
  const float a = (float)(2 * ip - sq);
  const float b = (float)(2 * pc - dp);
  const float t = __fadd_rn(__fmul_rn(qp.y, a), __fmul_rn(qp.x, b));
  const float d = __fsub_rn(__fadd_rn(qp.z, fac.x), __fmul_rn(2.0f, __fmul_rn(fac.y, t)));
  return __fadd_rn(d, 0.0f);
}

template <int NW4>
__device__ __forceinline__ float estimate_code(const uint4* __restrict__ cp, float2 fac,
                                               const uint32_t* pl, float4 qp, int dp) {
  uint4 code[NW4];
  int pc = 0;
#pragma unroll
  for (int i = 0; i < NW4; ++i) {
    code[i] = __ldg(cp + i);
    pc += __popc(code[i].x) + __popc(code[i].y) + __popc(code[i].z) + __popc(code[i].w);
  }
  return estimate_regs<NW4>(code, pc, fac, pl, qp, dp);
}

// Append the lanes' passing candidates (distance, id of slot s) to one
// query's buffer with one atomic per warp. All 32 lanes must call it.
__device__ __forceinline__ void append_candidates(bool pass, float d, int64_t s,
                                                  const uint32_t* __restrict__ ids,
                                                  int32_t* count, uint64_t* cand, int64_t cap,
                                                  int lane, int32_t* err) {
  const unsigned mask = __ballot_sync(0xffffffffu, pass);
  if (mask == 0) return;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pass) {
    const int64_t pos = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
    if (pos < cap)
      cand[pos] = make_key(d, ids[s]);
    else
      flag_error(err, kErrCandidateOverflow);
  }
}

// Append for a chunk of J pairs at once: bit j of `passbits` says whether
// this lane's vector (slot s) passes for pair j, whose query is qid[j] and
// estimate d[j]. Lane 0 issues the chunk's counter atomics back to back (they
// are independent), then every lane writes its survivors. All 32 lanes must
// call it.
template <int J>
__device__ __forceinline__ void append_chunk(uint32_t passbits, const float (&d)[J],
                                             const int32_t* qid, int64_t s,
                                             const uint32_t* __restrict__ ids,
                                             int32_t* counts, uint64_t* cand, int64_t cap,
                                             int lane, int32_t* err) {
  uint32_t mk[J];
  int any = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    mk[j] = __ballot_sync(0xffffffffu, (passbits >> j) & 1u);
    any |= mk[j] != 0;
  }
  if (!any) return;
  int base[J];
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < J; ++j) base[j] = mk[j] ? atomicAdd(counts + qid[j], __popc(mk[j])) : 0;
  }
  const uint32_t id = passbits ? ids[s] : 0u;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int b = __shfl_sync(0xffffffffu, base[j], 0);
    if ((passbits >> j) & 1u) {
      const int64_t pos = (int64_t)b + __popc(mk[j] & lt);
      if (pos < cap)
        cand[(int64_t)qid[j] * cap + pos] = make_key(d[j], id);
      else
        flag_error(err, kErrCandidateOverflow);
    }
  }
}

// FP8 E4M3 encoding of an integer 0..15 (exact): v = 2^e (1 + m/8) with
// e = floor(log2 v), stored as (e + 7) << 3 | m; 0 encodes as 0.
__device__ __forceinline__ uint8_t e4m3_of_int(int v) {
  if (v <= 0) return 0;
  const int e = 31 - __clz(v);
  const int m = (v << (3 - e)) & 7;
  return (uint8_t)(((e + 7) << 3) | m);
}

// Tensor-core scan (rq_scan_mma.cu).
bool mma_supported(const rq_index* ix);
rq_status launch_scan_mma(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                          int sms);
int next_pow2_host(int64_t v);

}  // namespace rq
