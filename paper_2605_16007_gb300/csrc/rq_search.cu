// IVF-RaBitQ search on the GPU (Section 2.1.2 query processing; Sections
// 2.2.2 and 3.3): rotate each query once, rank the centroids, quantise each
// probed residual to 4-bit planes, scan the probed lists with the estimator of
// Eqs. 4-5 under a per-query bound (Section 3.3.3), select the best
// candidates and re-rank them exactly (Section 3.3.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rq_async.cuh"
#include "rq_common.cuh"
#include "rq_internal.h"
#include "rq_pairdist.cuh"
#include "rq_scan.cuh"

namespace rq {
namespace {

inline unsigned blocks_for(int64_t n, int per) {
  return (unsigned)std::max<int64_t>(1, (n + per - 1) / per);
}

// Optional CUDA events at stage boundaries: ev[s] marks the start of stage s,
// ev[RQ_STAGE_COUNT] the end of the search.
struct StageTimer {
  cudaEvent_t ev[RQ_STAGE_COUNT + 1] = {};
  bool on = false;
  void mark(int stage, cudaStream_t st) {
    if (on) cudaEventRecord(ev[stage], st);
  }
};

// ---------------------------------------------------------------------------
// Rotation: q' = q P[:D, :] (float32, one multiply-add per term).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
rotate_kernel(const float* __restrict__ q, int64_t nq, int dim,
              const float* __restrict__ P32, int dp, float* __restrict__ qrot) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int col0 = blockIdx.y * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < dim; k0 += 16) {
    for (int t = threadIdx.x; t < 64 * 16; t += 256) {
      const int r = t >> 4, kk = t & 15;
      const int64_t row = r0 + r;
      const int k = k0 + kk;
      As[kk][r] = (row < nq && k < dim) ? q[row * dim + k] : 0.0f;
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
  for (int i = 0; i < 4; ++i) {
    const int64_t row = r0 + 4 * ty + i;
    if (row >= nq) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) qrot[row * dp + col0 + tx + 16 * j] = acc[i][j];
  }
}

// ---------------------------------------------------------------------------
// Per-row selection of the n smallest uint64 keys, ascending, padded with
// all-ones keys to out_width. OUT 0: write keys; OUT 1: write (id, distance)
// of probe keys as int32 / float.
// ---------------------------------------------------------------------------
template <int OUT>
__global__ void __launch_bounds__(1024)
select_rows_kernel(const uint64_t* __restrict__ keys, int64_t row_stride,
                   const int32_t* __restrict__ counts, int64_t fixed_count, int64_t cap,
                   const int32_t* __restrict__ nsel, int nsel_fixed,
                   uint64_t* __restrict__ out, int out_width,
                   int32_t* __restrict__ out_ids, float* __restrict__ out_d,
                   int32_t* err) {
  extern __shared__ uint64_t s_keys[];
  __shared__ int hist[256];
  __shared__ uint64_t bcast[2];
  __shared__ int s_n;
  const int64_t row = blockIdx.x;
  const uint64_t* kr = keys + row * row_stride;
  int64_t count = counts ? (int64_t)counts[row] : fixed_count;
  if (count > cap) {
    if (threadIdx.x == 0) flag_error(err, kErrCandidateOverflow);
    count = cap;
  }
  const int n_sel = nsel ? nsel[row] : nsel_fixed;
  int filled;
  if (count <= kMaxSelect) {
    const int m = next_pow2((int)std::max<int64_t>(count, 1));
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_keys[i] = (i < count) ? kr[i] : kU64Max;
    __syncthreads();
    block_bitonic_sort(s_keys, m);
    filled = (int)std::min<int64_t>(count, n_sel);
  } else {
    const uint64_t T = block_radix_select_u64(kr, count, n_sel, hist, bcast);
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
      const uint64_t k = kr[i];
      if (k < T) {
        const int pos = atomicAdd(&s_n, 1);
        if (pos < n_sel) s_keys[pos] = k;
      }
    }
    __syncthreads();
    const int lt = std::min(s_n, n_sel);
    const int m = next_pow2(n_sel);
    for (int i = lt + threadIdx.x; i < m; i += blockDim.x) s_keys[i] = (i < n_sel) ? T : kU64Max;
    __syncthreads();
    block_bitonic_sort(s_keys, m);
    filled = n_sel;
  }
  for (int j = threadIdx.x; j < out_width; j += blockDim.x) {
    const uint64_t k = (j < filled) ? s_keys[j] : kU64Max;
    if (OUT == 0) {
      out[row * out_width + j] = k;
    } else {
      out_ids[row * out_width + j] = (k == kU64Max) ? -1 : (int32_t)(uint32_t)k;
      out_d[row * out_width + j] =
          (k == kU64Max) ? __int_as_float(0x7f800000) : from_orderable((uint32_t)(k >> 32));
    }
  }
}

// ---------------------------------------------------------------------------
// Quantisation of each probed residual r = q' - P^T c (one warp per pair):
// vl = min r, vr = max r, delta = (vr - vl)/15, inv = 15/(vr - vl),
// q_u = min(15, floor((r - vl) inv + 1/2)) (0 when vr == vl), Sq = sum q_u,
// nq2 = ||r||^2 in the 32-lane order; bit-plane j packs bit j of every q_u
// (dimension d -> word d/32, bit d%32).
// ---------------------------------------------------------------------------
template <int NW4>
__device__ __forceinline__ void quantize_pair(int64_t pair, int64_t q, int c, int slot, int lane,
                                              const float (&qv)[4 * NW4],
                                              const float (&cv)[4 * NW4], int64_t nq, int dp,
                                              float4* __restrict__ qparams,
                                              uint32_t* __restrict__ planes,
                                              uint8_t* __restrict__ qdb,
                                              float4* __restrict__ qpb,
                                              uint8_t* __restrict__ qrec, uint64_t* slot_out,
                                              int wslot, uint8_t* __restrict__ wqdb,
                                              float4* __restrict__ wqpb) {
  constexpr int PER = 4 * NW4;  // values per lane (dp / 32)
  // Streaming scan: the pair's record in its list's bucket (planes, then
  // {vl, delta, nq2, Sq}; query, mask word and bound are added once the
  // bound is known).
  uint32_t* rec = qrec ? reinterpret_cast<uint32_t*>(qrec + ((int64_t)c * nq + slot) * pair_rec_bytes(dp))
                       : nullptr;
  if (lane == 0 && slot_out) *slot_out = ((uint64_t)(uint32_t)slot << 32) | (uint32_t)c;
  float r[PER];
  float vl = __int_as_float(0x7f800000), vr = -vl, acc = 0.0f;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    r[i] = __fsub_rn(qv[i], cv[i]);
    vl = fminf(vl, r[i]);
    vr = fmaxf(vr, r[i]);
    acc = __fadd_rn(acc, __fmul_rn(r[i], r[i]));
  }
  vl = warp_min(vl);
  vr = warp_max(vr);
  const float nq2 = lane_tree_sum(acc);
  const float width = __fsub_rn(vr, vl);
  const bool same = (width == 0.0f);
  const float delta = same ? 0.0f : __fdiv_rn(width, 15.0f);
  const float inv = same ? 0.0f : __fdiv_rn(15.0f, width);
  int sq = 0;
  constexpr int W = PER;  // words per plane
  constexpr int NWD = (4 * W + 31) / 32;  // plane words held per lane
  uint32_t* pl = planes + pair * 4 * W;
  // plane word j W + i goes to lane (j W + i) % 32, so that the words leave
  // in coalesced stores
  uint32_t mine[NWD];
#pragma unroll
  for (int x = 0; x < NWD; ++x) mine[x] = 0u;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int qu = 0;
    if (!same) {
      qu = __float2int_rd(__fadd_rn(__fmul_rn(__fsub_rn(r[i], vl), inv), 0.5f));
      qu = min(qu, 15);
    }
    sq += qu;
    if (qdb) {
      // The tensor-core scan's B rows: FP8 digits in the 128B-swizzled row
      // layout (16-byte chunk d/16 of bucket row `slot` at chunk position
      // (d/16) ^ (slot % 8)), so that one bulk copy lands them in place.
      const int d = lane + 32 * i;
      const uint8_t e = e4m3_of_int(qu);
      qdb[((int64_t)c * nq + slot) * dp + ((((d >> 4) ^ (slot & 7))) << 4) + (d & 15)] = e;
      // a window pair's copy in the window bucket (same layout)
      if (wslot >= 0)
        wqdb[((int64_t)c * nq + wslot) * dp + ((((d >> 4) ^ (wslot & 7))) << 4) + (d & 15)] = e;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t w = __ballot_sync(0xffffffffu, (qu >> j) & 1);
      if (lane == ((j * W + i) & 31)) mine[(j * W + i) >> 5] = w;
    }
  }
#pragma unroll
  for (int x = 0; x < NWD; ++x) {
    const int wi = 32 * x + lane;
    if (wi < 4 * W) {
      pl[wi] = mine[x];
      if (rec) rec[wi] = mine[x];
    }
  }
  sq = warp_sum_int(sq);
  if (lane == 0) {
    const float4 qp = make_float4(vl, delta, nq2, __int_as_float(sq));
    qparams[pair] = qp;
    if (rec) *reinterpret_cast<float4*>(rec + 4 * W) = qp;
    if (qpb) {
      // The tensor-core scan's copy, interleaved by slot couples for its
      // packed float2 arithmetic: slots 2k, 2k + 1 of a bucket hold
      // {vl, vl', delta, delta'} {nq2, nq2', -Sq, -Sq'} (Sq as a float).
      float* cp = reinterpret_cast<float*>(qpb + (int64_t)c * nq + (slot & ~1)) + (slot & 1);
      cp[0] = vl;
      cp[2] = delta;
      cp[4] = nq2;
      cp[6] = -(float)sq;
      if (wslot >= 0) {
        float* wp = reinterpret_cast<float*>(wqpb + (int64_t)c * nq + (wslot & ~1)) + (wslot & 1);
        wp[0] = vl;
        wp[2] = delta;
        wp[4] = nq2;
        wp[6] = -(float)sq;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Plain scan: one block per (query, probed list, chunk of `chunk`
// vectors) -- the query-level schedule of Section 3.3.1, with long lists cut
// into chunks so that they do not leave one block running alone. A thread
// loads the codes of up to eight 128-vector steps before estimating them,
// then each warp writes the survivor mask word of its 32 vectors
// (emit_word).
// ---------------------------------------------------------------------------
constexpr int kPlainChunk = 1024;  // default vectors of one list per block of the plain scan

template <int NW4, int CHUNK>
__global__ void __launch_bounds__(128, NW4 == 1 ? 8 : 4)  // 8 blocks/SM: 3% faster at D_p 128
scan_plain_kernel(const int32_t* __restrict__ nchunks, const int32_t* __restrict__ probe_ids,
                  int npmax, const float4* __restrict__ qparams,
                  const uint32_t* __restrict__ planes, const int64_t* __restrict__ offsets,
                  const uint8_t* __restrict__ codes, const float2* __restrict__ fac,
                  int dp, const uint32_t* __restrict__ bound,
                  const int32_t* __restrict__ wbase, int64_t mwords, uint32_t* __restrict__ mask,
                  int64_t mask_words, int32_t* err) {
  constexpr int W = 4 * NW4;
  constexpr int RB = NW4 >= 8 ? 1 : 8 / NW4;  // 128-vector steps with their loads in flight
  __shared__ __align__(16) uint32_t s_pl[4 * W];
  const int64_t pair = blockIdx.x;
  // block-uniform: a chunk past the list's end, or a probe past the query's
  // nprobe (no chunks), leaves after one load
  if ((int)blockIdx.y >= nchunks[pair]) return;
  const int64_t q = pair / npmax;
  const int c = probe_ids[pair];
  const int64_t lo = offsets[c], hi = offsets[c + 1];
  const int64_t start = lo + (int64_t)blockIdx.y * CHUNK;
  const int64_t end = min(hi, start + CHUNK);
  for (int i = threadIdx.x; i < 4 * W; i += blockDim.x) s_pl[i] = planes[pair * 4 * W + i];
  __syncthreads();
  const float4 qp = qparams[pair];
  const uint32_t tau = bound[q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wrow = q * mwords + wbase[pair];
  for (int64_t b0 = start; b0 < end; b0 += 128 * RB) {
    uint4 code[RB][NW4];
    float2 fv[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t s = b0 + 128 * r + threadIdx.x;
      if (s < end) {
        const uint4* cp = reinterpret_cast<const uint4*>(codes + s * (dp / 8));
#pragma unroll
        for (int w = 0; w < NW4; ++w) code[r][w] = __ldg(cp + w);
        fv[r] = __ldg(fac + s);
      }
    }
    uint32_t passm = 0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t s = b0 + 128 * r + threadIdx.x;
      if (s < end) {
        int pc = 0;
#pragma unroll
        for (int w = 0; w < NW4; ++w)
          pc += __popc(code[r][w].x) + __popc(code[r][w].y) + __popc(code[r][w].z) +
                __popc(code[r][w].w);
        if (orderable(estimate_regs<NW4>(code[r], pc, fv[r], s_pl, qp, dp)) <= tau)
          passm |= 1u << r;
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t s0 = b0 + 128 * r;
      if (s0 + warp * 32 >= end) break;  // warp-uniform: this word is past the chunk's end
      const int64_t widx = wrow + (s0 - lo) / 32 + warp;
      if (!index_ok(widx, mask_words, err)) continue;
      emit_word((passm >> r) & 1u, widx, mask, lane);
    }
  }
}

// ---------------------------------------------------------------------------
// FastScan estimator (Section 3.3.2, the paper's form: the query is not
// quantised). For a rotated residual r, table entry T[g][v] is the float32
// sum of r[8 g + i] over the set bits i of byte v, added in increasing i from
// 0; a code's s is the sum over groups g, in increasing g, of T[g][code byte
// g]; t = 2 s - S (S = sum_d r_d in the 32-lane order) = sum_d b_d r_d, and
// d2 = (nq2 + r_x^2) - 2 (f t), then + 0 -- every operation rounded once.
// ---------------------------------------------------------------------------

// Builds the D_p/8 x 256 tables from r (shared memory, D_p floats) with the
// whole block: level h fills the entries whose highest set bit is h from the
// entry without that bit, so each entry adds its bits in increasing order.
__device__ inline void build_lut(const float* r, float* T, int groups) {
  for (int g = threadIdx.x; g < groups; g += blockDim.x) T[g * 256] = 0.0f;
  __syncthreads();
  for (int h = 0; h < 8; ++h) {
    const int span = 1 << h;
    for (int i = threadIdx.x; i < groups * span; i += blockDim.x) {
      const int g = i >> h, v = span + (i & (span - 1));
      T[g * 256 + v] = __fadd_rn(T[g * 256 + v - span], r[8 * g + h]);
    }
    __syncthreads();
  }
}

template <int NW4>
__device__ __forceinline__ float estimate_lut_regs(const uint4 (&code)[NW4], const float* T,
                                                   float2 fac, float nq2, float S) {
  float sum = 0.0f;
#pragma unroll
  for (int w = 0; w < NW4; ++w) {
    const uint32_t word[4] = {code[w].x, code[w].y, code[w].z, code[w].w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int g = 16 * w + j;
      const float e = T[g * 256 + ((word[j >> 2] >> (8 * (j & 3))) & 255u)];
      sum = (g == 0) ? e : __fadd_rn(sum, e);
    }
  }
  const float t = __fsub_rn(__fmul_rn(2.0f, sum), S);
  const float d = __fsub_rn(__fadd_rn(nq2, fac.x), __fmul_rn(2.0f, __fmul_rn(fac.y, t)));
  return __fadd_rn(d, 0.0f);
}

// The same value without the tables, from the residual r itself (global or
// shared memory): entry T[g][v] is built from T[g][0] = 0 by adding r[8 g + i]
// for the set bits i of v in increasing order, which is what the inner loop
// adds here, in the same order and from the same +0.
template <int NW4>
__device__ __forceinline__ float estimate_lut_direct(const uint4 (&code)[NW4],
                                                     const float* __restrict__ r, float2 fac,
                                                     float nq2, float S) {
  float sum = 0.0f;
#pragma unroll
  for (int w = 0; w < NW4; ++w) {
    const uint32_t word[4] = {code[w].x, code[w].y, code[w].z, code[w].w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int g = 16 * w + j;
      const uint32_t v = (word[j >> 2] >> (8 * (j & 3))) & 255u;
      float e = 0.0f;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if ((v >> i) & 1u) e = __fadd_rn(e, r[8 * g + i]);
      sum = (g == 0) ? e : __fadd_rn(sum, e);
    }
  }
  const float t = __fsub_rn(__fmul_rn(2.0f, sum), S);
  const float d = __fsub_rn(__fadd_rn(nq2, fac.x), __fmul_rn(2.0f, __fmul_rn(fac.y, t)));
  return __fadd_rn(d, 0.0f);
}

// The residual r = q' - P^T c of one (query, probed list) pair into shared
// memory (D_p floats), by the whole block.
__device__ __forceinline__ void residual_to_smem(const float* __restrict__ qrot, int64_t q,
                                                 const float* __restrict__ cR, int c, int dp,
                                                 float* r) {
  for (int d = threadIdx.x; d < dp; d += blockDim.x)
    r[d] = __fsub_rn(qrot[q * dp + d], cR[(int64_t)c * dp + d]);
}

// Plain (query-level) scan with the FastScan estimator: one block per
// (query, probed list, chunk of 1024 list vectors); the block builds its
// pair's tables in shared memory, then each thread estimates its vectors
// (the codes of its 128-vector steps loaded before they are estimated) and
// each warp writes the survivor mask word of its 32 vectors.
template <int NW4>
__global__ void __launch_bounds__(128)
scan_lut_kernel(const int32_t* __restrict__ nchunks, const int32_t* __restrict__ probe_ids,
                int npmax, const float4* __restrict__ qparams, const float* __restrict__ qrot,
                const float* __restrict__ cR, const int64_t* __restrict__ offsets,
                const uint8_t* __restrict__ codes, const float2* __restrict__ fac, int dp,
                const uint32_t* __restrict__ bound, const int32_t* __restrict__ wbase,
                int64_t mwords, uint32_t* __restrict__ mask, int64_t mask_words, int32_t* err) {
  constexpr int RB = NW4 >= 2 ? 4 : 8;
  extern __shared__ __align__(16) float s_lut[];  // D_p/8 x 256 table, then D_p residual
  float* s_r = s_lut + 32 * dp;
  const int64_t pair = blockIdx.x;
  if ((int)blockIdx.y >= nchunks[pair]) return;
  const int64_t q = pair / npmax;
  const int c = probe_ids[pair];
  const int64_t lo = offsets[c], hi = offsets[c + 1];
  const int64_t start = lo + (int64_t)blockIdx.y * 1024;
  const int64_t end = min(hi, start + 1024);
  residual_to_smem(qrot, q, cR, c, dp, s_r);
  __syncthreads();
  build_lut(s_r, s_lut, dp / 8);
  const float4 qp = qparams[pair];
  const uint32_t tau = bound[q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wrow = q * mwords + wbase[pair];
  for (int64_t b0 = start; b0 < end; b0 += 128 * RB) {
    uint4 code[RB][NW4];
    float2 fv[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t sl = b0 + 128 * r + threadIdx.x;
      if (sl < end) {
        const uint4* cp = reinterpret_cast<const uint4*>(codes + sl * (dp / 8));
#pragma unroll
        for (int w = 0; w < NW4; ++w) code[r][w] = __ldg(cp + w);
        fv[r] = __ldg(fac + sl);
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int64_t s0 = b0 + 128 * r;
      if (s0 + warp * 32 >= end) break;  // warp-uniform: this word is past the chunk's end
      const int64_t sl = s0 + threadIdx.x;
      const bool pass =
          sl < end && orderable(estimate_lut_regs<NW4>(code[r], s_lut, fv[r], qp.z, qp.w)) <= tau;
      const int64_t widx = wrow + (s0 - lo) / 32 + warp;
      if (!index_ok(widx, mask_words, err)) continue;
      emit_word(pass, widx, mask, lane);
    }
  }
}

// ---------------------------------------------------------------------------
// The first bound's n-th smallest estimate, kept in shared memory while the
// estimates stream in (Section 3.3.3). The block offers keys in rounds; a
// key below the threshold `thr` goes to the buffer, a key equal to it is
// only counted (eqc), a larger one is dropped. When the buffer could
// overflow in the next round, thr becomes the buffer's n-th smallest key and
// only the keys below it stay. Every dropped key is larger than a threshold
// with at least n keys at or below it, so the n-th smallest of everything
// offered is the n-th smallest of (buffer, eqc copies of thr). The result
// does not depend on the order of the keys.
// ---------------------------------------------------------------------------
struct KthState {
  int nbuf;      // keys in the buffer (all below thr)
  int eqc;       // keys equal to thr seen since thr was set
  uint32_t thr;  // all ones until the first compaction
  int cnt;       // compaction scratch
  int eq2;
};

__device__ __forceinline__ void kth_init(KthState* ks) {
  if (threadIdx.x == 0) {
    ks->nbuf = 0;
    ks->eqc = 0;
    ks->thr = kU32Max;
  }
}

// One key per thread (valid false: none). Every thread of the block calls
// it with the same thr (read after the round's barrier).
__device__ __forceinline__ void kth_offer(KthState* ks, uint32_t* buf, uint32_t thr, uint32_t key,
                                          bool valid) {
  const int lane = threadIdx.x & 31;
  const bool keep = valid && key < thr;
  const uint32_t mk = __ballot_sync(0xffffffffu, keep);
  const uint32_t me = __ballot_sync(0xffffffffu, valid && key == thr);
  int base = 0;
  if (lane == 0) {
    if (mk) base = atomicAdd(&ks->nbuf, __popc(mk));
    if (me) atomicAdd(&ks->eqc, __popc(me));
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (keep) buf[base + __popc(mk & ((1u << lane) - 1u))] = key;
}

// Called by the whole block after a round's barrier: compacts when fewer
// than `room` slots are left (cap >= n + 2 room).
__device__ inline void kth_maybe_compact(KthState* ks, uint32_t* buf, int cap, int room, int n,
                                         int* hist, uint64_t* small, int* ctl) {
  const int nb = ks->nbuf;
  // every thread reads the count before any thread offers the next round's
  // keys, so that all take the same branch
  __syncthreads();
  if (nb <= cap - room) return;
  const uint32_t t2 = block_kth_u32(buf, nb, n, hist, small, ctl);  // nb > n: a key below thr
  if (threadIdx.x == 0) {
    ks->cnt = 0;
    ks->eq2 = 0;
  }
  __syncthreads();
  // keep the keys below t2, in rounds whose reads all come before their
  // writes (a kept key's new position is below every unread position)
  for (int r0 = 0; r0 < nb; r0 += blockDim.x * 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = r0 + threadIdx.x + blockDim.x * u;
      v[u] = i < nb ? buf[i] : kU32Max;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = r0 + threadIdx.x + blockDim.x * u;
      if (i < nb) {
        if (v[u] < t2) buf[atomicAdd(&ks->cnt, 1)] = v[u];
        else if (v[u] == t2) atomicAdd(&ks->eq2, 1);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ks->nbuf = ks->cnt;
    ks->eqc = ks->eq2;
    ks->thr = t2;
  }
  __syncthreads();
}

// The n-th smallest of all keys offered, `total` of them (all ones when
// total < n).
__device__ inline uint32_t kth_result(KthState* ks, uint32_t* buf, int total, int n, int* hist,
                                      uint64_t* small, int* ctl) {
  __syncthreads();
  if (total < n) return kU32Max;
  const int nb = ks->nbuf;
  const uint32_t thr = ks->thr;
  if (nb >= n) return block_kth_u32(buf, nb, n, hist, small, ctl);
  return thr;  // nb < n <= nb + eqc
}

// The FastScan quantities of one pair (a warp): nq2 = ||r||^2 and S = sum_d
// r_d, both in the 32-lane order, stored as {0, 0, nq2, S}; the residual
// itself goes to `resid` (D_p floats per pair) for the finalize kernel.
template <int NW4>
__device__ __forceinline__ void lut_pair(int64_t pair, int64_t q, int c, int lane,
                                         const float* __restrict__ qrot,
                                         const float* __restrict__ cR, int dp,
                                         float4* __restrict__ qparams, float* __restrict__ resid) {
  float acc2 = 0.0f, acc1 = 0.0f;
#pragma unroll
  for (int i = 0; i < 4 * NW4; ++i) {
    const int d = lane + 32 * i;
    const float r = __fsub_rn(qrot[q * dp + d], cR[(int64_t)c * dp + d]);
    resid[pair * dp + d] = r;
    acc2 = __fadd_rn(acc2, __fmul_rn(r, r));
    acc1 = __fadd_rn(acc1, r);
  }
  const float nq2 = lane_tree_sum(acc2);
  const float S = lane_tree_sum(acc1);
  if (lane == 0) qparams[pair] = make_float4(0.0f, 0.0f, nq2, S);
}

// First bound with the FastScan estimator (the same candidates and rank as
// bound_block): per probe the block builds the pair's tables in `lut`
// (D_p/8 x 256 floats, then D_p residual floats) and estimates the list's
// first vectors. `buf` is shared memory for `cap` keys.
template <int NW4>
__device__ inline uint32_t bound_block_lut(int64_t qi, int npmax, int npq, int n_sel,
                                           const uint64_t* lists,
                                           const float4* __restrict__ qparams,
                                           const float* __restrict__ qrot,
                                           const float* __restrict__ cR,
                                           const int64_t* __restrict__ offsets,
                                           const uint8_t* __restrict__ codes,
                                           const float2* __restrict__ fac, int dp,
                                           uint32_t* buf, int cap, float* lut, int* hist,
                                           uint64_t* small, int* ctl) {
  __shared__ KthState ks;
  const int tid = threadIdx.x;
  const int cap1 = bound_window(n_sel);
  float* r = lut + 32 * dp;
  kth_init(&ks);
  int taken = 0;
  for (int p = 0; p < npq && taken < cap1; ++p) {
    const int64_t pair = qi * npmax + p;
    const uint32_t c = (uint32_t)lists[p];
    const int64_t lo = offsets[c];
    const int m = (int)min(offsets[c + 1] - lo, (int64_t)(cap1 - taken));
    __syncthreads();
    residual_to_smem(qrot, qi, cR, (int)c, dp, r);
    __syncthreads();
    build_lut(r, lut, dp / 8);
    const float4 qp = qparams[pair];
    for (int base = 0; base < m; base += blockDim.x) {
      const int i = base + tid;
      uint32_t key = 0;
      if (i < m) {
        uint4 code[NW4];
        const uint4* cp = reinterpret_cast<const uint4*>(codes + (lo + i) * (dp / 8));
#pragma unroll
        for (int w = 0; w < NW4; ++w) code[w] = __ldg(cp + w);
        key = orderable(estimate_lut_regs<NW4>(code, lut, __ldg(fac + lo + i), qp.z, qp.w));
      }
      kth_offer(&ks, buf, ks.thr, key, i < m);
      __syncthreads();
      kth_maybe_compact(&ks, buf, cap, blockDim.x, n_sel, hist, small, ctl);
    }
    taken += m;
  }
  return kth_result(&ks, buf, taken, n_sel, hist, small, ctl);
}

// ---------------------------------------------------------------------------
// Rotation q' = P^T q (float32 FMA): 8 queries x 64 output columns per
// block, K in chunks of 128 staged in shared memory with every load of a
// chunk in flight at once (16-byte loads when the rows allow). The first
// column of blocks also clears the search's counters (zero0[n0], zero1[n1])
// for the later stages.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
rotate_kernel8(const float* __restrict__ q, int64_t nq, int dim, const float* __restrict__ P32,
               int dp, float* __restrict__ qrot, int32_t* __restrict__ zero0, int n0,
               int32_t* __restrict__ zero1, int n1) {
  __shared__ __align__(16) float As[8][132];
  __shared__ __align__(16) float Bs[128][64];
  const int tid = threadIdx.x;
  if (blockIdx.y == 0) {
    for (int i = blockIdx.x * blockDim.x + tid; i < n0; i += gridDim.x * blockDim.x) zero0[i] = 0;
    for (int i = blockIdx.x * blockDim.x + tid; i < n1; i += gridDim.x * blockDim.x) zero1[i] = 0;
  }
  const int r = tid >> 5, cg = tid & 31;
  const int64_t r0 = (int64_t)blockIdx.x * 8;
  const int col0 = blockIdx.y * 64;
  const bool vec = (dim & 3) == 0;
  float acc[2] = {0.0f, 0.0f};
  for (int k0 = 0; k0 < dim; k0 += 128) {
    // A: 8 rows x 128 (one float4 per thread); B: 128 x 64 (eight float4)
    {
      const int rr = tid >> 5, kk = (tid & 31) * 4;
      const int64_t row = r0 + rr;
      float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (row < nq) {
        if (vec && k0 + kk + 3 < dim) {
          v = __ldg(reinterpret_cast<const float4*>(q + row * dim + k0 + kk));
        } else {
          const float* src = q + row * dim + k0 + kk;
          v.x = (k0 + kk + 0 < dim) ? src[0] : 0.0f;
          v.y = (k0 + kk + 1 < dim) ? src[1] : 0.0f;
          v.z = (k0 + kk + 2 < dim) ? src[2] : 0.0f;
          v.w = (k0 + kk + 3 < dim) ? src[3] : 0.0f;
        }
      }
      *reinterpret_cast<float4*>(&As[rr][kk]) = v;
    }
    float4 bv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + 256 * t, kk = e >> 4, c4 = (e & 15) * 4;
      bv[t] = (k0 + kk < dim)
                  ? __ldg(reinterpret_cast<const float4*>(P32 + (int64_t)(k0 + kk) * dp + col0 + c4))
                  : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + 256 * t, kk = e >> 4, c4 = (e & 15) * 4;
      *reinterpret_cast<float4*>(&Bs[kk][c4]) = bv[t];
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 128; ++kk) {
      const float av = As[r][kk];
      acc[0] = fmaf(av, Bs[kk][cg], acc[0]);
      acc[1] = fmaf(av, Bs[kk][cg + 32], acc[1]);
    }
    __syncthreads();
  }
  const int64_t row = r0 + r;
  if (row < nq) {
    qrot[row * dp + col0 + cg] = acc[0];
    qrot[row * dp + col0 + cg + 32] = acc[1];
  }
}

// ---------------------------------------------------------------------------
// Exact squared distances of selected raw rows to the query in the 32-lane
// order: partial sum l takes d = l, l + 32, ... (d < dim) in order, then
// partials l and l + s are added for s = 16, 8, 4, 2, 1. A warp takes eight
// rows at a time, lane l holding partial l of each: every load is a
// coalesced 32-float (or 32-byte) piece of a row, and up to 32 of them (8
// rows x 4 pieces) are in flight per lane; the partials meet by shuffles in
// the same tree. Row i of `keys` (row id in the low word) gets the key
// (distance, id).
// ---------------------------------------------------------------------------
template <typename RawT>
__device__ inline void rerank_rows(const RawT* __restrict__ raw, uint64_t* keys, int n,
                                   const float* __restrict__ qs, int dim) {
  constexpr int G = 8, JB = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int i0 = warp * G; i0 < n; i0 += nwarps * G) {
    uint32_t id[G];
    float acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      id[g] = i0 + g < n ? (uint32_t)keys[i0 + g] : 0u;
      acc[g] = 0.0f;
    }
    for (int d0 = 0; d0 < dim; d0 += 32 * JB) {
      float v[G][JB];
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int jb = 0; jb < JB; ++jb) {
          const int d = d0 + 32 * jb + lane;
          v[g][jb] = (i0 + g < n && d < dim) ? (float)__ldg(raw + (int64_t)id[g] * dim + d) : 0.0f;
        }
#pragma unroll
      for (int jb = 0; jb < JB; ++jb) {
        const int d = d0 + 32 * jb + lane;
        if (d < dim) {
          const float qd = qs[d];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const float df = __fsub_rn(v[g][jb], qd);
            acc[g] = __fadd_rn(acc[g], __fmul_rn(df, df));
          }
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
#pragma unroll
      for (int s2 = 16; s2; s2 >>= 1) acc[g] = __fadd_rn(acc[g], __shfl_down_sync(0xffffffffu, acc[g], s2));
      if (lane == 0 && i0 + g < n) keys[i0 + g] = make_key(acc[g], id[g]);
    }
  }
}

// ---------------------------------------------------------------------------
// Candidate collection, selection and re-rank (three kernels per search).
//
// The survivors are read from the scan's masks and their estimates
// recomputed (every scan form computes the popcount form's float32 value,
// and the FastScan form's direct sums equal its table sums), paired with
// their row ids as (estimate, row id) keys.
//
// 1. collect_kernel: one block per (query, round of kFinRoundWords mask
//    words), the query in x. Thread t holds kFinWordsPerThread consecutive words of the round
//    (four 16-byte loads in flight together); a block scan of the per-thread
//    counts gives each nonzero word a descriptor (position of its first
//    survivor, word offset) and its mask word in shared memory. The survivors
//    are then taken a thread each, up to four at a time with all their loads
//    in flight: the descriptor by binary search, the bit by its rank in the
//    word, the probe by binary search over the probes' first words. The block
//    reserves room in its query's key buffer with one atomic and writes the
//    keys there (in no fixed order; the selection does not depend on it).
// 2. select_kernel: one block per query selects the n_sel smallest keys from
//    the buffer (block radix selection), gathers and re-ranks them exactly and
//    selects the final k.
// 3. finalize_kernel: only for a query with more survivors than its buffer
//    holds (one block per SM walks the queries). It reads the masks again in rounds and keeps the n_sel smallest
//    keys in shared memory by a streaming threshold: a key below the
//    threshold goes to the staging area; when that could overflow in the next
//    step, the n_sel smallest staged keys are kept and the threshold becomes
//    the largest of them. Keys are distinct (one per vector), so a dropped key
//    is above n_sel kept ones and is not among the n_sel smallest of all.
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 256;
constexpr int kFinWordsPerThread = 16;                            // four 16-byte mask loads
constexpr int kFinRoundWords = kFinThreads * kFinWordsPerThread;  // mask words per round
constexpr int64_t kKeyCap = 65536;                                // key buffer per query

// Shared memory of the streaming finalize, in order: selection (P keys),
// top-k (PK keys), staging (S keys), probe slot bases (NP int64), bucket (32
// keys), histogram (256 ints), descriptors and mask words (kFinRoundWords
// each), probe first words (NP ints), query row (dim floats).
struct FinalizeLayout {
  int P, PK, S, NP, dim;
  __host__ __device__ int bytes() const {
    return (P + PK + S + NP + 32) * 8 + 256 * 4 + 2 * kFinRoundWords * 4 +
           ((NP * 4 + 15) & ~15) + ((dim * 4 + 15) & ~15);
  }
  // the collection kernel: probe slot bases, descriptors and words, probe
  // first words
  __host__ __device__ int collect_bytes() const {
    return NP * 8 + 2 * kFinRoundWords * 4 + ((NP * 4 + 15) & ~15);
  }
  // the selection kernel: selection, top-k, bucket, histogram, query row
  __host__ __device__ int select_bytes() const {
    return (P + PK + 32) * 8 + 256 * 4 + ((dim * 4 + 15) & ~15);
  }
};

struct FinalizeArgs {
  const uint32_t* mask;
  const int32_t* wtotal;
  int64_t mwords;
  const int32_t* wbase;      // nq x npmax
  const int32_t* probe_ids;  // nq x npmax
  const int32_t* nprobe;     // nq
  int npmax;
  const int64_t* offsets;
  const uint8_t* codes;
  const float2* fac;
  const uint32_t* planes;    // popcount form: nq x npmax x 4 x W words
  const float4* qparams;     // nq x npmax
  const float* resid;        // FastScan form: nq x npmax x D_p, else null
  int dp;
  const uint32_t* ids;
  int64_t n_slots;
  int32_t* err;
  int32_t* counts;
  const int32_t* nsel;
  const int32_t* kq;
  const int32_t* rerank_on;
  int nsel_max;
  uint64_t* sel;
  const void* raw;
  const float* q;
  int dim, k_stride;
  FinalizeLayout lay;
  int64_t* out_ids;
  float* out_d;
  int64_t nq;
  uint64_t* keys;            // nq x kcap survivor keys (collect -> select)
  int32_t* kcount;           // nq: survivors of each query (cleared before collect)
  int64_t kcap;
};

// One round of a query's mask words from word c0: the descriptors and words
// of the nonzero words into shared memory; every thread gets the round's
// survivor and descriptor counts. All threads call it.
__device__ inline void fin_round(const uint4* __restrict__ mrow4, int T, int c0,
                                 uint32_t* s_desc, uint32_t* s_dword, int* s_warp,
                                 int& tot_keys, int& tot_desc) {
  constexpr int NWARP = kFinThreads / 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wfirst = c0 + tid * kFinWordsPerThread;
  uint32_t w[kFinWordsPerThread];
#pragma unroll
  for (int j = 0; j < kFinWordsPerThread / 4; ++j) {
    const uint4 v = (wfirst + 4 * j < T) ? mrow4[(wfirst >> 2) + j] : make_uint4(0, 0, 0, 0);
    w[4 * j] = v.x;
    w[4 * j + 1] = v.y;
    w[4 * j + 2] = v.z;
    w[4 * j + 3] = v.w;
  }
  int c = 0, nz = 0;
#pragma unroll
  for (int e = 0; e < kFinWordsPerThread; ++e) {
    if (wfirst + e >= T) w[e] = 0u;  // words past the query's last probed list
    const int n = __popc(w[e]);
    c += n;
    nz += n != 0;
  }
  // one scan of both counts: survivors (< 2^18 per round) in the low 18
  // bits, nonzero words (<= kFinRoundWords) above
  const int v = c | (nz << 18);
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();  // the previous round is done with s_warp and the descriptors
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  int ex = incl - v, tot = 0;
#pragma unroll
  for (int i = 0; i < NWARP; ++i) {
    const int sw = s_warp[i];
    if (i < warp) ex += sw;
    tot += sw;
  }
  tot_keys = tot & 0x3FFFF;
  tot_desc = tot >> 18;
  int p = ex & 0x3FFFF, d = ex >> 18;
#pragma unroll
  for (int e = 0; e < kFinWordsPerThread; ++e) {
    const int n = __popc(w[e]);
    if (n) {
      s_desc[d] = ((uint32_t)p << 12) | (uint32_t)(tid * kFinWordsPerThread + e);
      s_dword[d] = w[e];
      ++d;
    }
    p += n;
  }
  __syncthreads();
}

// Up to PT survivors of the round (positions j0 + tid + u kFinThreads) as
// keys: have[u] false past the round's survivors (or for a slot out of range
// in a checked build).
template <int NW4, int PT>
__device__ inline void fin_keys(const FinalizeArgs& a, int64_t row, int c0, int j0, int tot_keys,
                                int tot_desc, const uint32_t* s_desc, const uint32_t* s_dword,
                                const int* s_wb, const int64_t* s_base, int npq,
                                bool (&have)[PT], uint64_t (&key)[PT]) {
  constexpr int W = 4 * NW4;
  int64_t slot[PT], pair[PT];
#pragma unroll
  for (int u = 0; u < PT; ++u) {
    const int j = j0 + threadIdx.x + u * kFinThreads;
    have[u] = j < tot_keys;
    slot[u] = 0;
    pair[u] = row * a.npmax;
    if (have[u]) {
      int lo = 0, hi = tot_desc - 1;  // the last descriptor whose first survivor is <= j
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int)(s_desc[mid] >> 12) <= j) lo = mid; else hi = mid - 1;
      }
      const uint32_t dsc = s_desc[lo];
      const int word = c0 + (int)(dsc & 4095u);
      uint32_t mw = s_dword[lo];  // the survivor's bit: drop the lower set bits
      for (int r = j - (int)(dsc >> 12); r > 0; --r) mw &= mw - 1u;
      const int bit = __ffs(mw) - 1;
      int plo = 0, phi = npq - 1;  // the probe holding `word`
      while (plo < phi) {
        const int mid = (plo + phi + 1) >> 1;
        if (s_wb[mid] <= word) plo = mid; else phi = mid - 1;
      }
      slot[u] = s_base[plo] + (int64_t)(word - s_wb[plo]) * 32 + bit;
      pair[u] = row * a.npmax + plo;
      if (!index_ok(slot[u], a.n_slots, a.err)) have[u] = false;
    }
  }
  // every load of the step in flight: codes, factors, ids, parameters
  uint4 code[PT][NW4];
  float2 fv[PT];
  uint32_t rid[PT];
  float4 qp[PT];
#pragma unroll
  for (int u = 0; u < PT; ++u) {
    if (have[u]) {
      const uint4* cp = reinterpret_cast<const uint4*>(a.codes + slot[u] * (a.dp / 8));
#pragma unroll
      for (int x = 0; x < NW4; ++x) code[u][x] = __ldg(cp + x);
      fv[u] = __ldg(a.fac + slot[u]);
      rid[u] = __ldg(a.ids + slot[u]);
      qp[u] = __ldg(a.qparams + pair[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < PT; ++u) {
    key[u] = kU64Max;
    if (have[u]) {
      float d;
      if (a.resid) {
        d = estimate_lut_direct<NW4>(code[u], a.resid + pair[u] * a.dp, fv[u], qp[u].z, qp[u].w);
      } else {
        int pc = 0;
#pragma unroll
        for (int x = 0; x < NW4; ++x)
          pc += __popc(code[u][x].x) + __popc(code[u][x].y) + __popc(code[u][x].z) +
                __popc(code[u][x].w);
        d = estimate_regs<NW4>(code[u], pc, fv[u], a.planes + pair[u] * 4 * W, qp[u], a.dp);
      }
      key[u] = make_key(d, rid[u]);
    }
  }
}

// Stages the query's probes (first mask word, first slot) in shared memory.
__device__ inline void fin_probes(const FinalizeArgs& a, int64_t row, int npq, int* s_wb,
                                  int64_t* s_base) {
  for (int p = threadIdx.x; p < npq; p += kFinThreads) {
    s_wb[p] = a.wbase[row * a.npmax + p];
    s_base[p] = a.offsets[a.probe_ids[row * a.npmax + p]];
  }
}

// The common end: selection dump, exact re-rank of the `got` selected keys in
// s_sel, top-k and the outputs.
template <typename RawT>
__device__ inline void fin_rerank(const FinalizeArgs& a, int64_t row, uint64_t* s_sel, int got,
                                  uint64_t* s_top, int* hist, uint64_t* small, int* s_ctl,
                                  const float* s_q) {
  const int k = a.kq[row];
  const bool rerank = a.rerank_on[row] != 0;
  const int tid = threadIdx.x;
  for (int j = tid; j < a.nsel_max; j += kFinThreads)
    a.sel[row * a.nsel_max + j] = (j < got) ? s_sel[j] : kU64Max;
  const float inf = __int_as_float(0x7f800000);
  const uint64_t* res = s_sel;
  int kk = min(k, got);
  if (rerank) {
    rerank_rows<RawT>(static_cast<const RawT*>(a.raw), s_sel, got, s_q, a.dim);
    __syncthreads();
    kk = block_select_smallest(s_sel, got, k, s_top, hist, small, s_ctl, true);
    res = s_top;
  }
  for (int j = tid; j < a.k_stride; j += kFinThreads) {
    const uint64_t key = (j < kk) ? res[j] : kU64Max;
    a.out_ids[row * a.k_stride + j] = (key == kU64Max) ? -1 : (int64_t)(uint32_t)key;
    a.out_d[row * a.k_stride + j] = (key == kU64Max) ? inf : from_orderable((uint32_t)(key >> 32));
  }
}

template <int NW4>
__global__ void __launch_bounds__(kFinThreads) collect_kernel(FinalizeArgs a) {
  constexpr int PT = NW4 <= 2 ? 4 : (NW4 <= 4 ? 2 : 1);  // survivors per thread per step
  constexpr int STEP = kFinThreads * PT;
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_warp[kFinThreads / 32];
  __shared__ int s_pos;
  const int64_t row = blockIdx.x;
  const int c0 = blockIdx.y * kFinRoundWords;
  const int T = a.wtotal[row];
  if (c0 >= T) return;  // block-uniform: past the query's mask words
  const FinalizeLayout& lay = a.lay;
  int64_t* s_base = reinterpret_cast<int64_t*>(smem);
  uint32_t* s_desc = reinterpret_cast<uint32_t*>(s_base + lay.NP);
  uint32_t* s_dword = s_desc + kFinRoundWords;
  int* s_wb = reinterpret_cast<int*>(s_dword + kFinRoundWords);
  const int npq = min(a.nprobe[row], a.npmax);
  fin_probes(a, row, npq, s_wb, s_base);
  // mwords is a multiple of 4 and the mask 16-byte aligned
  const uint4* mrow4 = reinterpret_cast<const uint4*>(a.mask + row * a.mwords);
  int tot_keys, tot_desc;
  fin_round(mrow4, T, c0, s_desc, s_dword, s_warp, tot_keys, tot_desc);
  if (tot_keys == 0) return;  // block-uniform
  if (threadIdx.x == 0) s_pos = atomicAdd(&a.kcount[row], tot_keys);
  __syncthreads();
  const int64_t pos0 = s_pos;
  uint64_t* krow = a.keys + row * a.kcap;
  for (int j0 = 0; j0 < tot_keys; j0 += STEP) {
    bool have[PT];
    uint64_t key[PT];
    fin_keys<NW4, PT>(a, row, c0, j0, tot_keys, tot_desc, s_desc, s_dword, s_wb, s_base, npq,
                      have, key);
#pragma unroll
    for (int u = 0; u < PT; ++u) {
      const int64_t at = pos0 + j0 + threadIdx.x + u * kFinThreads;
      if (have[u] && at < a.kcap) krow[at] = key[u];
    }
  }
}

template <typename RawT>
__global__ void __launch_bounds__(kFinThreads) select_kernel(FinalizeArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_ctl[8];
  const int64_t row = blockIdx.x;
  const int count = a.kcount[row];
  if (count > a.kcap) return;  // block-uniform: the streaming finalize takes it
  const FinalizeLayout& lay = a.lay;
  uint64_t* s_sel = reinterpret_cast<uint64_t*>(smem);
  uint64_t* s_top = s_sel + lay.P;
  uint64_t* small = s_top + lay.PK;
  int* hist = reinterpret_cast<int*>(small + 32);
  float* s_q = reinterpret_cast<float*>(hist + 256);
  for (int d = threadIdx.x; d < a.dim; d += kFinThreads) s_q[d] = a.q[row * a.dim + d];
  if (threadIdx.x == 0) a.counts[row] = count;
  // Without re-rank the selection is the answer and is sorted; with re-rank
  // only the set matters and the exact keys are selected below.
  const bool rerank = a.rerank_on[row] != 0;
  const int got = block_select_smallest(a.keys + row * a.kcap, count, a.nsel[row], s_sel, hist,
                                        small, s_ctl, !rerank);
  fin_rerank<RawT>(a, row, s_sel, got, s_top, hist, small, s_ctl, s_q);
}

template <typename RawT, int NW4>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(FinalizeArgs a) {
  constexpr int NWARP = kFinThreads / 32;
  constexpr int PT = NW4 <= 2 ? 4 : (NW4 <= 4 ? 2 : 1);  // survivors per thread per step
  constexpr int STEP = kFinThreads * PT;
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_ctl[8];
  __shared__ int s_warp[NWARP];
  __shared__ int s_nbuf;
  __shared__ uint64_t s_thr;
  // a grid of a few blocks per SM walks the queries; only those whose keys
  // overflowed their buffers are worked on
  for (int64_t row = blockIdx.x; row < a.nq; row += gridDim.x) {
  if (a.kcount[row] <= a.kcap) continue;  // block-uniform: the selection kernel took it
  __syncthreads();  // the previous query's shared memory is free
  const FinalizeLayout& lay = a.lay;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* s_sel = reinterpret_cast<uint64_t*>(smem);
  uint64_t* s_top = s_sel + lay.P;
  uint64_t* s_stage = s_top + lay.PK;
  int64_t* s_base = reinterpret_cast<int64_t*>(s_stage + lay.S);
  uint64_t* small = reinterpret_cast<uint64_t*>(s_base + lay.NP);
  int* hist = reinterpret_cast<int*>(small + 32);
  uint32_t* s_desc = reinterpret_cast<uint32_t*>(hist + 256);
  uint32_t* s_dword = s_desc + kFinRoundWords;
  int* s_wb = reinterpret_cast<int*>(s_dword + kFinRoundWords);
  float* s_q = reinterpret_cast<float*>(s_wb + ((lay.NP + 3) & ~3));
  // mwords is a multiple of 4 and the mask 16-byte aligned
  const uint4* mrow4 = reinterpret_cast<const uint4*>(a.mask + row * a.mwords);
  const int T = a.wtotal[row];
  const int npq = min(a.nprobe[row], a.npmax);
  const int n_sel = a.nsel[row];
  for (int d = tid; d < a.dim; d += kFinThreads) s_q[d] = a.q[row * a.dim + d];
  fin_probes(a, row, npq, s_wb, s_base);
  if (tid == 0) {
    s_nbuf = 0;
    s_thr = kU64Max;
  }
  int64_t count = 0;  // survivors (the same in every thread)
  for (int c0 = 0; c0 < T; c0 += kFinRoundWords) {
    int tot_keys, tot_desc;
    fin_round(mrow4, T, c0, s_desc, s_dword, s_warp, tot_keys, tot_desc);
    count += tot_keys;
    for (int j0 = 0; j0 < tot_keys; j0 += STEP) {
      const uint64_t thr = s_thr;
      bool have[PT];
      uint64_t key[PT];
      fin_keys<NW4, PT>(a, row, c0, j0, tot_keys, tot_desc, s_desc, s_dword, s_wb, s_base, npq,
                        have, key);
      // offer: keys below the threshold go to the staging area
#pragma unroll
      for (int u = 0; u < PT; ++u) {
        const bool keep = have[u] && key[u] < thr;
        const uint32_t mk = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if (lane == 0 && mk) base = atomicAdd(&s_nbuf, __popc(mk));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) s_stage[base + __popc(mk & ((1u << lane) - 1u))] = key[u];
      }
      __syncthreads();
      const int nb = s_nbuf;
      // every thread reads the count before any thread offers the next
      // step's keys, so that all take the same branch
      __syncthreads();
      if (nb > lay.S - STEP) {
        // keep the n_sel smallest (nb > S - STEP > n_sel)
        block_select_smallest(s_stage, nb, n_sel, s_sel, hist, small, s_ctl, false);
        uint64_t mx = 0;
        for (int i = tid; i < n_sel; i += kFinThreads) {
          const uint64_t k = s_sel[i];
          s_stage[i] = k;
          mx = k > mx ? k : mx;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const uint64_t t = __shfl_xor_sync(0xffffffffu, mx, o);
          mx = t > mx ? t : mx;
        }
        if (lane == 0) small[warp] = mx;
        __syncthreads();
        if (tid == 0) {
          uint64_t m2 = 0;
          for (int i = 0; i < NWARP; ++i) m2 = small[i] > m2 ? small[i] : m2;
          s_thr = m2;
          s_nbuf = n_sel;
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  if (tid == 0) a.counts[row] = (int)min(count, (int64_t)INT32_MAX);
  const int staged = s_nbuf;
  const bool rerank = a.rerank_on[row] != 0;
  const int got = block_select_smallest(s_stage, staged, n_sel, s_sel, hist, small, s_ctl, !rerank);
  fin_rerank<RawT>(a, row, s_sel, got, s_top, hist, small, s_ctl, s_q);
  }
}


// Probe selection. Both forms leave the query's np smallest (distance, list)
// keys in dst, ascending, and return how many were found; the distance is
// always the fixed-order float32 one (the terms (q'_d - c_d)^2 added in
// increasing d, no fused multiply-add).
constexpr int kPrepThreads = 256;  // threads of the per-query preparation block
constexpr int kProbeStageKeys = 4096;
constexpr int kProbeCandCap = 1024;
constexpr int kProbeRowStage = 32;  // candidates whose rows are staged in shared memory

// Exact form: select from the full exact ranking (pkeys, nlist keys per
// query), staged in shared memory when it fits.
__device__ inline int probe_select_exact(const uint64_t* __restrict__ pkeys, int nlist, int np,
                                         int64_t row, uint64_t* dst, uint64_t* stage, int* hist,
                                         uint64_t* small, int* ctl) {
  const uint64_t* src = pkeys + row * nlist;
  if (nlist <= kProbeStageKeys) {
#pragma unroll 8
    for (int i = threadIdx.x; i < nlist; i += blockDim.x) stage[i] = src[i];
    __syncthreads();
    src = stage;
  }
  return block_select_smallest(src, nlist, np, dst, hist, small, ctl, true);
}

// The fixed-order squared distance of the query (shared memory) to one
// centroid row.
__device__ __forceinline__ float seq_sqdist(const float* qs, const float* __restrict__ c, int dp) {
  float acc = 0.0f;
  const float4* c4 = reinterpret_cast<const float4*>(c);
  for (int d0 = 0; d0 < dp; d0 += 32) {  // D_p is a multiple of 32
    float4 v[8];                          // a 128-byte row piece in flight
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __ldg(c4 + (d0 >> 2) + j);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int d = d0 + 4 * j;
      float df = __fsub_rn(qs[d], v[j].x);
      acc = __fadd_rn(acc, __fmul_rn(df, df));
      df = __fsub_rn(qs[d + 1], v[j].y);
      acc = __fadd_rn(acc, __fmul_rn(df, df));
      df = __fsub_rn(qs[d + 2], v[j].z);
      acc = __fadd_rn(acc, __fmul_rn(df, df));
      df = __fsub_rn(qs[d + 3], v[j].w);
      acc = __fadd_rn(acc, __fmul_rn(df, df));
    }
  }
  return acc;
}

// Certified form, for nlist <= kProbeStageKeys and D_p 128. From the
// approximate ranking g = ||c||^2 - 2 <q', c> (approx_dist_tc_kernel, on the
// tensor cores in TF32) and ||q'||^2, each centroid's approximate distance
// a = ||q'||^2 + g has |a - exact| <= e with e = kTcProbeEscale (||q'||^2 +
// ||c||^2), exact being the fixed-order float32 distance (the bound is
// derived where g is computed and pinned on the CPU). U = the np-th smallest
// a + e bounds the np-th smallest exact distance from above, so a centroid
// with a - e > U is not among the np nearest (not even on a tie); the others
// (np and a few more) get the exact distance and the exact selection.
// If more than kProbeCandCap remain, every centroid gets the exact distance.
// Shared memory: `region` holds max(nlist keys, kProbeRowStage rows of D_p
// floats) + kProbeCandCap ints + D_p floats.
__device__ inline int probe_select_certified(const float* __restrict__ g,
                                             const float* __restrict__ cn,
                                             const float* __restrict__ qrot,
                                             const float* __restrict__ cR, int nlist, int np,
                                             int dp, int64_t row, uint64_t* dst, uint64_t* region,
                                             int* hist, uint64_t* small, int* ctl) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* ub = reinterpret_cast<uint32_t*>(region);  // nlist upper-bound keys
  uint64_t* keys = region;                            // later: exact keys (reuses ub)
  // in 8-byte units, even so that `cand` and `qs` stay 16-byte aligned
  const int keys_area = (max(nlist, kProbeRowStage * dp / 2) + 1) & ~1;
  int* cand = reinterpret_cast<int*>(region + keys_area);
  float* qs = reinterpret_cast<float*>(cand + kProbeCandCap);
  __shared__ float s_red[32];
  float part = 0.0f;
  for (int d = tid; d < dp; d += blockDim.x) {
    const float v = qrot[row * dp + d];
    qs[d] = v;
    part = fmaf(v, v, part);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  float qn = 0.0f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) qn += s_red[w];
  const float escale = kTcProbeEscale;
  const float* grow = g + row * nlist;
#pragma unroll 8
  for (int c = tid; c < nlist; c += blockDim.x) {
    const float av = qn + grow[c];
    ub[c] = orderable(av + escale * (qn + cn[c]));
  }
  if (tid == 0) ctl[6] = 0;
  __syncthreads();
  // Any U at or above the np-th smallest upper bound keeps the selection
  // exact; the bucket edge of a partial radix search costs fewer passes and
  // admits a few more candidates.
  const uint32_t U = block_kth_upper_u32(ub, nlist, min(np, nlist), 16, hist, small, ctl);
#pragma unroll 8
  for (int c = tid; c < nlist; c += blockDim.x) {
    const float av = qn + grow[c];
    if (orderable(av - escale * (qn + cn[c])) <= U) {
      const int at = atomicAdd(&ctl[6], 1);
      if (at < kProbeCandCap) cand[at] = c;
    }
  }
  __syncthreads();
  const int nc = ctl[6];
  const bool all = nc > kProbeCandCap;
  const int m = all ? nlist : nc;
  if (!all && nc <= kProbeRowStage) {
    // The candidates' rows are staged in shared memory (over the dead upper
    // bounds), every load in flight together, then one thread per candidate
    // adds its terms in order.
    float* rows = reinterpret_cast<float*>(region);
    const int q4 = dp / 4;
    for (int i = tid; i < nc * q4; i += blockDim.x) {
      const int j = i / q4, k4 = i - j * q4;
      reinterpret_cast<float4*>(rows)[i] =
          __ldg(reinterpret_cast<const float4*>(cR + (int64_t)cand[j] * dp) + k4);
    }
    __syncthreads();
    float dist = 0.0f;
    if (tid < nc) {
      const float4* rw = reinterpret_cast<const float4*>(rows + tid * dp);
      const float4* q4p = reinterpret_cast<const float4*>(qs);
#pragma unroll 8
      for (int d4 = 0; d4 < q4; ++d4) {
        const float4 rv = rw[d4], qv = q4p[d4];
        float df = __fsub_rn(qv.x, rv.x);
        dist = __fadd_rn(dist, __fmul_rn(df, df));
        df = __fsub_rn(qv.y, rv.y);
        dist = __fadd_rn(dist, __fmul_rn(df, df));
        df = __fsub_rn(qv.z, rv.z);
        dist = __fadd_rn(dist, __fmul_rn(df, df));
        df = __fsub_rn(qv.w, rv.w);
        dist = __fadd_rn(dist, __fmul_rn(df, df));
      }
    }
    __syncthreads();
    if (tid < nc) keys[tid] = make_key(dist, (uint32_t)cand[tid]);
  } else {
    for (int i = tid; i < m; i += blockDim.x) {
      const int c = all ? i : cand[i];
      keys[i] = make_key(seq_sqdist(qs, cR + (int64_t)c * dp, dp), (uint32_t)c);
    }
  }
  __syncthreads();
  return block_select_smallest(keys, m, np, dst, hist, small, ctl, true);
}

// Writes the selected probes (ids, distances) and, in warp 0, each probe's
// first survivor-mask word: the running sum, in probe order, of the probed
// lists' 32-vector words over the query's own nprobe.
__device__ inline void probe_outputs(const uint64_t* dst, int got, int np, int64_t row,
                                     int32_t* __restrict__ out_ids, float* __restrict__ out_d,
                                     const int64_t* __restrict__ offsets, int npq,
                                     int32_t* __restrict__ wbase, int32_t* __restrict__ wtotal) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j = tid; j < np; j += blockDim.x) {
    const uint64_t k = (j < got) ? dst[j] : kU64Max;
    out_ids[row * np + j] = (k == kU64Max) ? -1 : (int32_t)(uint32_t)k;
    out_d[row * np + j] =
        (k == kU64Max) ? __int_as_float(0x7f800000) : from_orderable((uint32_t)(k >> 32));
  }
  if (warp == 0) {
    const int nw = min(npq, got);
    int carry = 0;
    for (int j0 = 0; j0 < np; j0 += 32) {
      const int j = j0 + lane;
      int w = 0;
      if (j < nw) {
        const uint32_t l = (uint32_t)dst[j];
        w = (int)((offsets[l + 1] - offsets[l] + 31) >> 5);
      }
      int incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (j < np) wbase[row * np + j] = carry + incl - w;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) wtotal[row] = carry;
  }
}

// First bound (Section 3.3.3): lists in probe order give the first
// bound_window(n_sel) candidates, estimated by all kPrepThreads threads (each
// thread's codes loaded before its estimates) and offered to the streaming
// n-th smallest in `buf` (shared memory for `cap` keys); the bound is the
// n_sel-th smallest orderable estimate (all ones when the query has fewer
// candidates). `lists` holds the query's probed list ids (npq of them).
template <int NW4>
__device__ inline uint32_t bound_block(int64_t qi, int npmax, int npq, int n_sel,
                                       const uint64_t* lists, const float4* __restrict__ qparams,
                                       const uint32_t* __restrict__ planes,
                                       const int64_t* __restrict__ offsets,
                                       const uint8_t* __restrict__ codes,
                                       const float2* __restrict__ fac, int dp, uint32_t* buf,
                                       int cap, int* hist, uint64_t* small, int* ctl) {
  constexpr int W = 4 * NW4;
  constexpr int RB = NW4 >= 4 ? 1 : 4 / NW4;  // codes in flight per thread
  __shared__ __align__(16) uint32_t s_pl[4 * W];
  __shared__ KthState ks;
  const int tid = threadIdx.x;
  const int cap1 = bound_window(n_sel);
  kth_init(&ks);
  int taken = 0;
  for (int p = 0; p < npq && taken < cap1; ++p) {
    const int64_t pair = qi * npmax + p;
    const uint32_t c = (uint32_t)lists[p];
    const int64_t lo = offsets[c];
    const int m = (int)min(offsets[c + 1] - lo, (int64_t)(cap1 - taken));
    __syncthreads();
    for (int i = tid; i < 4 * W; i += blockDim.x) s_pl[i] = planes[pair * 4 * W + i];
    __syncthreads();
    const float4 qp = qparams[pair];
    for (int base = 0; base < m; base += kPrepThreads * RB) {
      uint4 code[RB][NW4];
      float2 fv[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = base + tid + kPrepThreads * r;
        if (i < m) {
          const uint4* cp = reinterpret_cast<const uint4*>(codes + (lo + i) * (dp / 8));
#pragma unroll
          for (int w = 0; w < NW4; ++w) code[r][w] = __ldg(cp + w);
          fv[r] = __ldg(fac + lo + i);
        }
      }
      const uint32_t thr = ks.thr;
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = base + tid + kPrepThreads * r;
        uint32_t key = 0;
        if (i < m) {
          int pc = 0;
#pragma unroll
          for (int w = 0; w < NW4; ++w)
            pc += __popc(code[r][w].x) + __popc(code[r][w].y) + __popc(code[r][w].z) +
                  __popc(code[r][w].w);
          key = orderable(estimate_regs<NW4>(code[r], pc, fv[r], s_pl, qp, dp));
        }
        kth_offer(&ks, buf, thr, key, i < m);
      }
      __syncthreads();
      kth_maybe_compact(&ks, buf, cap, kPrepThreads * RB, n_sel, hist, small, ctl);
    }
    taken += m;
  }
  return kth_result(&ks, buf, taken, n_sel, hist, small, ctl);
}

// Query preparation, one block of kPrepThreads threads per query: probe selection,
// then the quantisation of each probed residual (a warp per probe), then the
// first bound. Shared memory: the probe keys (next_pow2(np)), then a region
// used first by the probe selection (nlist keys, plus the certified form's
// candidates and query row) and then for the bound's estimates.
struct PrepArgs {
  const uint64_t* pkeys;  // exact ranking (nlist > kProbeStageKeys), else null
  const float* g;         // approximate ranking (nlist <= kProbeStageKeys), else null
  const float* cn;        // ||c||^2 per centroid (with g)
  int nlist, npmax;
  int64_t nq;
  const int32_t* nprobe;
  const int32_t* nsel;
  const int32_t* no_prune;
  const int64_t* offsets;
  const float* qrot;
  const float* cR;
  int dp;
  int32_t* probe_ids;
  float* probe_d;
  int32_t* wbase;
  int32_t* wtotal;
  float4* qparams;
  uint32_t* planes;
  int32_t* list_count;
  int64_t* qwrow;     // tensor-core scan: per bucket slot, first mask index
  float* qtau;        // ... and the bound as a float32 threshold
  int64_t qstride;    // bucket stride of qwrow / qtau: nq rounded up to 4 (16-byte copies)
  int64_t mwords;
  uint8_t* qdb;
  float4* qpb;
  uint8_t* qrec;      // streaming scan: per-list pair records (null otherwise)
  const uint8_t* codes;
  const float2* fac;
  uint32_t* bound;
  int32_t* nchunks;   // plain scan: `chunk`-vector chunks of each probe (null otherwise)
  int chunk;
  int lut;            // 1: FastScan estimator (residual sums; tables for the bound)
  float* resid;       // FastScan: the residual of each pair (D_p floats)
  int bound_cap;      // keys the shared region holds for the first bound
  int lut_offset;     // byte offset of the table region in dynamic shared memory
  int32_t* err;
  // grouped first bound (null wcount: the block estimates its own window)
  int32_t* wcount;    // nlist window pairs per list, then nlist largest limits
  uint8_t* wqdb;      // window bucket: digits, parameters, first estimate index,
  float4* wqpb;       // vectors of the list in the window
  int64_t* wdest;
  int32_t* wlim;
  int32_t* wtake;     // nq: window size of each query
  uint32_t* pslot;    // nq x npmax: bucket slot of each probe
  int64_t est_stride; // estimates per query in the key buffer
  int win_offset;     // byte offset of the window table (int2 per probe) in dynamic shared memory
};

template <int NW4>
__global__ void __launch_bounds__(kPrepThreads, NW4 >= 4 ? 2 : 4) prep_kernel(PrepArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int hist[256];
  __shared__ uint64_t small[32];
  __shared__ int ctl[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row = blockIdx.x;
  const int P = max(2, next_pow2(a.npmax));  // keeps `region` 16-byte aligned
  uint64_t* dst = reinterpret_cast<uint64_t*>(smem);
  uint64_t* region = dst + P;
  // FastScan tables of the bound (after the region, whose size the host gives)
  float* lut_region = reinterpret_cast<float*>(smem + a.lut_offset);
  const int npq = min(a.nprobe[row], a.npmax);
  const int n_sel = a.nsel[row];
  const bool bound_on = !*a.no_prune && n_sel > 0;
  if (a.wtake && tid == 0) a.wtake[row] = 0;  // until the window is known
  const int got =
      a.g ? probe_select_certified(a.g, a.cn, a.qrot, a.cR, a.nlist, a.npmax, a.dp, row, dst,
                                   region, hist, small, ctl)
          : probe_select_exact(a.pkeys, a.nlist, a.npmax, row, dst, region, hist, small, ctl);
  probe_outputs(dst, got, a.npmax, row, a.probe_ids, a.probe_d, a.offsets, npq, a.wbase,
                a.wtotal);
  if (a.nchunks) {
    for (int p = tid; p < a.npmax; p += blockDim.x) {
      int nc = 0;
      if (p < npq && p < got) {
        const uint32_t l = (uint32_t)dst[p];
        nc = (int)((a.offsets[l + 1] - a.offsets[l] + a.chunk - 1) / a.chunk);
      }
      a.nchunks[row * a.npmax + p] = nc;
    }
  }
  if (got < npq) {
    if (tid == 0) flag_error(a.err, kErrBadProbe);
    return;
  }
  // Grouped first bound: the window is the first bound_window(n_sel)
  // candidates in probe order, so its probes are a prefix of the probes.
  // One warp finds them: per probe its first position in the window and its
  // vectors in the window (s_win), and how many probes reach into it.
  int2* s_win = reinterpret_cast<int2*>(smem + a.win_offset);
  __shared__ int s_pw;
  if (a.wcount && warp == 0) {
    const int cap1 = bound_on ? bound_window(n_sel) : 0;
    int carry = 0, pw = 0;
    for (int b = 0; b < npq && carry < cap1; b += 32) {
      const int p = b + lane;
      int len = 0;
      if (p < npq) {
        const uint32_t l = (uint32_t)dst[p];
        len = (int)min(a.offsets[l + 1] - a.offsets[l], (int64_t)cap1);
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int first = carry + incl - len;  // < 2^31: carry < cap1, 32 lengths <= cap1
      const bool in = p < npq && first < cap1;
      if (in) s_win[p] = make_int2(first, min(len, cap1 - first));
      pw += __popc(__ballot_sync(0xffffffffu, in));
      carry = min(carry + __shfl_sync(0xffffffffu, incl, 31), cap1);
    }
    if (lane == 0) {
      s_pw = pw;
      a.wtake[row] = carry;
    }
  }
  // (dst[p] keeps the list id in its low word; the quantisation puts the
  // pair's bucket slot in the high word, which held the distance: every
  // reader of the distances above is done after this barrier)
  __syncthreads();
  if (a.lut) {
    for (int p = warp; p < npq; p += kPrepThreads / 32)
      lut_pair<NW4>(row * a.npmax + p, row, (int)(uint32_t)dst[p], lane, a.qrot, a.cR, a.dp,
                    a.qparams, a.resid);
  } else {
    // A warp per probe. The query's values are loaded once; the next
    // probe's centroid row and (grouped scans) bucket slot are requested
    // before the current probe is quantised. Grouped scans: a pair takes
    // the next slot of its list's bucket (room for every query of the batch).
    constexpr int PER = 4 * NW4;
    float qv[PER], cv[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) qv[i] = a.qrot[row * a.dp + lane + 32 * i];
    int c = 0, slot = 0, wslot = -1;
    int2 win = make_int2(0, 0);
    auto request = [&](int pp) {
      c = (int)(uint32_t)dst[pp];
#pragma unroll
      for (int i = 0; i < PER; ++i) cv[i] = a.cR[(int64_t)c * a.dp + lane + 32 * i];
      if (a.list_count && lane == 0) slot = atomicAdd(&a.list_count[c], 1);
      // a window pair (with vectors in the window) also takes a window slot
      wslot = -1;
      if (a.wcount && lane == 0 && pp < s_pw) {
        win = s_win[pp];
        if (win.y > 0) {
          wslot = atomicAdd(&a.wcount[c], 1);
          atomicMax(&a.wcount[a.nlist + c], win.y);
        }
      }
    };
    // (no look-ahead above D_p 1024, where the registers run out)
    constexpr bool kAhead = NW4 <= 8;
    if (kAhead && warp < npq) request(warp);
    for (int p = warp; p < npq; p += kPrepThreads / 32) {
      if (!kAhead) request(p);
      float cur[PER];
#pragma unroll
      for (int i = 0; i < PER; ++i) cur[i] = cv[i];
      const int cc = c;
      const int sl = __shfl_sync(0xffffffffu, slot, 0);
      const int wsl = __shfl_sync(0xffffffffu, wslot, 0);
      if (wsl >= 0 && lane == 0) {
        a.wdest[cc * a.qstride + wsl] = row * a.est_stride + win.x;
        a.wlim[cc * a.qstride + wsl] = win.y;
      }
      if (kAhead && p + kPrepThreads / 32 < npq) request(p + kPrepThreads / 32);
      quantize_pair<NW4>(row * a.npmax + p, row, cc, sl, lane, qv, cur, a.nq, a.dp, a.qparams,
                         a.planes, a.qdb, a.qpb, a.qrec,
                         &dst[p], wsl, a.wqdb, a.wqpb);
    }
  }
  // The block's own writes of planes and parameters are visible to it
  // after the barrier.
  __syncthreads();
  uint32_t tau = kU32Max;
  if (!a.wcount && bound_on) {
    uint32_t* bk = reinterpret_cast<uint32_t*>(region);
    if (a.lut)
      tau = bound_block_lut<NW4>(row, a.npmax, npq, n_sel, dst, a.qparams, a.qrot, a.cR,
                                 a.offsets, a.codes, a.fac, a.dp, bk, a.bound_cap, lut_region,
                                 hist, small, ctl);
    else
      tau = bound_block<NW4>(row, a.npmax, npq, n_sel, dst, a.qparams, a.planes, a.offsets,
                             a.codes, a.fac, a.dp, bk, a.bound_cap, hist, small, ctl);
  }
  if (!a.wcount && tid == 0) a.bound[row] = tau;
  if (a.qwrow) {
    // each pair's first mask index and bound, at its bucket slot (with the
    // grouped bound: the slot, for window_bound_kernel to write the bound)
    const float tf = tau_threshold(tau);
    for (int p = tid; p < npq; p += blockDim.x) {
      const uint64_t e = dst[p];
      const int64_t c = (uint32_t)e, slot = (uint32_t)(e >> 32);
      a.qwrow[c * a.qstride + slot] = row * a.mwords + a.wbase[row * a.npmax + p];
      if (a.wcount) a.pslot[row * a.npmax + p] = (uint32_t)slot;
      else a.qtau[c * a.qstride + slot] = tf;
    }
  }
  if (a.qrec) {
    // the rest of each pair record: query, first mask word, bound
    const int rb = pair_rec_bytes(a.dp);
    for (int p = tid; p < npq; p += blockDim.x) {
      const uint64_t e = dst[p];
      const int64_t c = (uint32_t)e, slot = (uint32_t)(e >> 32);
      int4* m = reinterpret_cast<int4*>(a.qrec + (c * a.nq + slot) * rb + a.dp / 2 + 16);
      *m = make_int4((int)row, a.wbase[row * a.npmax + p], (int)tau, 0);
    }
  }
}

// The grouped first bound's last step (Section 3.3.3), one block per
// query: the n_sel-th smallest of the window's estimates, which the
// tensor-core scan's window pass wrote to the query's key buffer (the value
// the preparation block's streaming selection finds from the same
// estimates; all ones when the window holds fewer than n_sel), by block
// radix selection straight from the buffer; then the bound as a float32
// threshold at each of the query's bucket slots.
__global__ void __launch_bounds__(256)
window_bound_kernel(const uint32_t* __restrict__ est, int64_t est_stride,
                    const int32_t* __restrict__ wtake, const int32_t* __restrict__ nsel,
                    const int32_t* __restrict__ no_prune, const int32_t* __restrict__ nprobe,
                    int npmax, const int32_t* __restrict__ probe_ids,
                    const uint32_t* __restrict__ pslot, int nlist, int64_t nq, int64_t qstride,
                    uint32_t* __restrict__ bound, float* __restrict__ qtau) {
  __shared__ int hist[256];
  __shared__ uint64_t small[32];
  __shared__ int ctl[8];
  const int64_t row = blockIdx.x;
  const int n_sel = nsel[row];
  const int n = (int)min((int64_t)wtake[row], est_stride);
  uint32_t tau = kU32Max;
  if (!*no_prune && n_sel > 0 && n >= n_sel)
    tau = block_kth_u32(est + row * est_stride, n, n_sel, hist, small, ctl);
  if (threadIdx.x == 0) bound[row] = tau;
  const float tf = tau_threshold(tau);
  const int npq = min(nprobe[row], npmax);
  for (int p = threadIdx.x; p < npq; p += blockDim.x) {
    const int c = probe_ids[row * npmax + p];
    const uint32_t slot = pslot[row * npmax + p];
    // (a query whose probe selection failed left no slots: skip them)
    if (c >= 0 && c < nlist && slot < (uint32_t)nq) qtau[(int64_t)c * qstride + slot] = tf;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
  size_t off = 0;
  template <typename T>
  size_t take(T** field, int64_t count) {
    const size_t o = off;
    off += align_up(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
    *field = reinterpret_cast<T*>(o);  // offset for now; rebased after allocation
    return o;
  }
};

template <typename T>
void rebase(T*& p, char* base) {
  p = reinterpret_cast<T*>(base + reinterpret_cast<size_t>(p));
}

// Above this many bytes a batch's workspace is split into sub-batches.
constexpr size_t kWorkspaceBudget = size_t(12) << 30;

// The tensor-core form takes its first bound from a grouped pass over the
// queries' windows (the window bucket, then window_bound_kernel); the other
// forms estimate each query's window in its preparation block.
bool grouped_bound(const rq_index* ix, const SearchShape& sh) {
  return sh.mode == RQ_SCAN_MMA && !sh.lut && ix->dp == 128;
}

// Lays out the workspace of a search shape: every field as an offset from
// the base, the total in ws.bytes.
void layout_workspace(const rq_index* ix, const SearchShape& sh, Workspace& ws) {
  const int64_t nq = sh.nq, np = sh.npmax;
  const int W = ix->dp / 32;
  // a multiple of 4: the finalize kernel reads the mask rows 16 bytes at a time
  ws.mwords = (std::max<int64_t>(1, ix->top_words_prefix[std::min(np, (int64_t)ix->nlist)]) + 3) & ~int64_t(3);
  Layout L;
  L.take(&ws.q, nq * ix->dim);
  L.take(&ws.qrot, nq * ix->dp);
  L.take(&ws.pkeys, nq * ix->nlist);
  L.take(&ws.cn, ix->nlist);
  L.take(&ws.probe_ids, nq * np);
  L.take(&ws.probe_d, nq * np);
  L.take(&ws.qparams, nq * np);
  L.take(&ws.planes, nq * np * 4 * W);
  L.take(&ws.bound, nq);
  L.take(&ws.counts, nq);
  L.take(&ws.mask, nq * ws.mwords);
  L.take(&ws.wbase, nq * np);
  L.take(&ws.wtotal, nq);
  L.take(&ws.sel, nq * sh.nsel_max);
  // survivor keys: up to kKeyCap per query (every survivor when the query
  // has fewer scanned vectors); a query with more takes the streaming form
  ws.kcap = std::min<int64_t>(kKeyCap, 32 * ws.mwords);
  L.take(&ws.keys, nq * ws.kcap);
  L.take(&ws.kcount, nq);
  // the per-query parameters in one region (one copy from the pinned staging
  // buffer, which has the same layout): nprobe, k, selection size, re-rank
  // flag (+1: the no-prune flag)
  L.take(&ws.nprobe, 4 * nq + 1);
  L.take(&ws.out_ids, nq * sh.k_stride);
  L.take(&ws.out_d, nq * sh.k_stride);
  if (sh.lut) L.take(&ws.resid, nq * np * ix->dp);
  if (sh.mode != RQ_SCAN_PLAIN) {
    L.take(&ws.list_count, ix->nlist);
  } else {
    L.take(&ws.nchunks, nq * np);
  }
  if (sh.mode == RQ_SCAN_GROUPED) L.take(&ws.qrec, (int64_t)ix->nlist * nq * pair_rec_bytes(ix->dp));
  if (sh.mode == RQ_SCAN_MMA) {
    // bucket stride rounded up to 4 slots, so that every group's copies
    // start 16-byte aligned; + what a group's copy reads past the end
    L.take(&ws.qwrow, (int64_t)ix->nlist * ((nq + 3) & ~int64_t(3)) + 2);
    L.take(&ws.qtau, (int64_t)ix->nlist * ((nq + 3) & ~int64_t(3)) + 4);
    L.take(&ws.qdig, (int64_t)ix->nlist * nq * ix->dp);
    L.take(&ws.qpb, (int64_t)ix->nlist * nq + 2);  // + a couple read past the last bucket
  }
  if (grouped_bound(ix, sh)) {
    // the window bucket, with the strides and tails of the main one
    L.take(&ws.wcount, 2 * (int64_t)ix->nlist);
    L.take(&ws.wqdig, (int64_t)ix->nlist * nq * ix->dp);
    L.take(&ws.wqpb, (int64_t)ix->nlist * nq + 2);
    L.take(&ws.wdest, (int64_t)ix->nlist * ((nq + 3) & ~int64_t(3)) + 2);
    L.take(&ws.wlim, (int64_t)ix->nlist * ((nq + 3) & ~int64_t(3)) + 4);
    L.take(&ws.wtake, nq);
    L.take(&ws.pslot, nq * np);
  }
  ws.bytes = L.off;
}

size_t workspace_bytes(const rq_index* ix, const SearchShape& sh) {
  Workspace ws;
  layout_workspace(ix, sh, ws);
  return ws.bytes;
}

}  // namespace

// Device bytes one search of this shape holds: its workspace, or that of the
// sub-batches it is split into.
size_t search_workspace_bytes(const rq_index* ix, int64_t nq, int npmax, int nsel_max,
                              int k_stride, int mode) {
  SearchShape sh{nq, npmax, nsel_max, k_stride, mode, 0, 0, kPlainChunk, 0};
  size_t b = workspace_bytes(ix, sh);
  while (sh.nq > 1 && b > kWorkspaceBudget) {
    sh.nq = (sh.nq + 1) / 2;
    b = workspace_bytes(ix, sh);
  }
  return b;
}

namespace {

rq_status alloc_workspace(rq_index* ix, const SearchShape& sh, cudaStream_t st, Workspace& ws) {
  const int64_t nq = sh.nq;
  layout_workspace(ix, sh, ws);
  (void)st;
  cudaError_t e = dev_alloc(&ws.base, ws.bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws.base = nullptr;
    return fail(RQ_ERR_OOM, "search workspace of " + std::to_string(ws.bytes) + " bytes");
  }
  char* b = static_cast<char*>(ws.base);
  rebase(ws.q, b);
  rebase(ws.qrot, b);
  rebase(ws.pkeys, b);
  rebase(ws.cn, b);
  rebase(ws.probe_ids, b);
  rebase(ws.probe_d, b);
  rebase(ws.qparams, b);
  rebase(ws.planes, b);
  rebase(ws.bound, b);
  rebase(ws.counts, b);
  rebase(ws.mask, b);
  rebase(ws.wbase, b);
  rebase(ws.wtotal, b);
  rebase(ws.sel, b);
  rebase(ws.keys, b);
  rebase(ws.kcount, b);
  rebase(ws.nprobe, b);
  ws.kq = ws.nprobe + nq;
  ws.nsel = ws.nprobe + 2 * nq;
  ws.rerank_on = ws.nprobe + 3 * nq;
  rebase(ws.out_ids, b);
  rebase(ws.out_d, b);
  if (sh.lut) rebase(ws.resid, b);
  if (sh.mode != RQ_SCAN_PLAIN) {
    rebase(ws.list_count, b);
  } else {
    rebase(ws.nchunks, b);
  }
  if (sh.mode == RQ_SCAN_GROUPED) rebase(ws.qrec, b);
  if (sh.mode == RQ_SCAN_MMA) {
    rebase(ws.qwrow, b);
    rebase(ws.qtau, b);
    rebase(ws.qdig, b);
    rebase(ws.qpb, b);
  }
  if (grouped_bound(ix, sh)) {
    rebase(ws.wcount, b);
    rebase(ws.wqdig, b);
    rebase(ws.wqpb, b);
    rebase(ws.wdest, b);
    rebase(ws.wlim, b);
    rebase(ws.wtake, b);
    rebase(ws.pslot, b);
  }
  return RQ_OK;
}

// The certified probe selection (approximate ranking + exact refinement)
// serves lists up to kProbeStageKeys and D_p 128; otherwise
// every centroid distance is computed exactly.
bool certified_probe(const rq_index* ix) {
  return ix->nlist <= kProbeStageKeys && ix->dp == 128;
}

template <int NW4>
rq_status enqueue_scan_stages(rq_index* ix, const SearchShape& sh, Workspace& ws,
                              cudaStream_t st, StageTimer& tm) {
  const int64_t nq = sh.nq;
  const int np = sh.npmax;
  const int dp = ix->dp;
  const int64_t pairs = nq * np;
  // probe selection, quantisation and first bound: one fused kernel
  tm.mark(RQ_STAGE_QUANTIZE, st);
  const bool grouped = sh.mode != RQ_SCAN_PLAIN;
  {
    PrepArgs a;
    const bool certified = certified_probe(ix);
    a.pkeys = certified ? nullptr : ws.pkeys;
    a.g = certified ? reinterpret_cast<const float*>(ws.pkeys) : nullptr;
    a.cn = ws.cn;
    a.nlist = ix->nlist;
    a.npmax = np;
    a.nq = nq;
    a.nprobe = ws.nprobe;
    a.nsel = ws.nsel;
    a.no_prune = ws.rerank_on + nq;
    a.offsets = ix->offsets;
    a.qrot = ws.qrot;
    a.cR = ix->cR;
    a.dp = dp;
    a.probe_ids = ws.probe_ids;
    a.probe_d = ws.probe_d;
    a.wbase = ws.wbase;
    a.wtotal = ws.wtotal;
    a.qparams = ws.qparams;
    a.planes = ws.planes;
    a.list_count = grouped ? ws.list_count : nullptr;
    a.qwrow = sh.mode == RQ_SCAN_MMA ? ws.qwrow : nullptr;
    a.qtau = ws.qtau;
    a.qstride = (nq + 3) & ~int64_t(3);
    a.mwords = ws.mwords;
    a.qdb = sh.mode == RQ_SCAN_MMA ? ws.qdig : nullptr;
    a.qpb = sh.mode == RQ_SCAN_MMA ? ws.qpb : nullptr;
    a.qrec = sh.mode == RQ_SCAN_GROUPED ? ws.qrec : nullptr;
    a.codes = ix->codes;
    a.fac = ix->fac;
    a.bound = ws.bound;
    a.nchunks = grouped ? nullptr : ws.nchunks;
    a.chunk = sh.chunk;
    a.lut = sh.lut;
    a.resid = ws.resid;
    a.err = ix->d_err;
    // the probe selection's shared region: the certified form's keys, rows,
    // candidates and query; the exact form stages the nlist keys when they fit
    const size_t stage =
        certified ? ((std::max<size_t>((size_t)ix->nlist * 8, (size_t)kProbeRowStage * dp * 4) +
                      15) & ~(size_t)15) + kProbeCandCap * 4 + (size_t)dp * 4
                  : (ix->nlist <= kProbeStageKeys ? (size_t)ix->nlist * 8 : 0);
    // ... and then the first bound's keys: n_sel plus two rounds of
    // estimates (at most 1024 keys each), or the whole window when it is
    // small (no compaction then), up to 8192 keys
    const size_t bound_keys =
        std::max<size_t>(2 * (size_t)sh.nsel_max + 2048,
                         std::min<size_t>((size_t)bound_window(sh.nsel_max) + 1024, 8192));
    const bool gb = grouped_bound(ix, sh);
    const size_t bound_bytes = gb ? 0 : 4 * bound_keys;
    const size_t region = (std::max<size_t>({stage, bound_bytes, 64}) + 15) & ~(size_t)15;
    a.bound_cap = (int)(region / 4);
    size_t smem = (size_t)std::max(2, next_pow2_host(np)) * 8 + region;
    smem = (smem + 15) & ~(size_t)15;
    // the grouped bound's window table
    a.win_offset = (int)smem;
    if (gb) smem += (size_t)np * 8;
    a.wcount = gb ? ws.wcount : nullptr;
    a.wqdb = ws.wqdig;
    a.wqpb = ws.wqpb;
    a.wdest = ws.wdest;
    a.wlim = ws.wlim;
    a.wtake = gb ? ws.wtake : nullptr;
    a.pslot = ws.pslot;
    a.est_stride = 2 * ws.kcap;
    a.lut_offset = (int)smem;
    if (sh.lut) smem += (size_t)(32 * dp + dp) * sizeof(float);
    RQ_TRY(allow_dynamic_smem((const void*)prep_kernel<NW4>, 200 * 1024));
    prep_kernel<NW4><<<(unsigned)nq, kPrepThreads, smem, st>>>(a);
  }
  tm.mark(RQ_STAGE_BOUND, st);
  if (grouped_bound(ix, sh)) {
    // the first bound from one grouped pass over the windows; the estimates
    // go to the key buffers, idle until the collection
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
    RQ_TRY(launch_scan_mma(ix, sh, ws, st, sms, 0, true));
    window_bound_kernel<<<(unsigned)nq, 256, 0, st>>>(
        reinterpret_cast<const uint32_t*>(ws.keys), 2 * ws.kcap, ws.wtake, ws.nsel,
        ws.rerank_on + nq, ws.nprobe, np, ws.probe_ids, ws.pslot, ix->nlist, nq,
        (nq + 3) & ~int64_t(3), ws.bound, ws.qtau);
  }
  tm.mark(RQ_STAGE_WORKLIST, st);
  if (sh.lut) {
    tm.mark(RQ_STAGE_SCAN, st);
    const unsigned chunks = (unsigned)std::max<int64_t>(1, (ix->max_list_len + 1023) / 1024);
    const size_t lsm = (size_t)(32 * dp + dp) * sizeof(float);
    scan_lut_kernel<NW4 <= 2 ? NW4 : 1><<<dim3((unsigned)pairs, chunks), 128, lsm, st>>>(
        ws.nchunks, ws.probe_ids, np, ws.qparams, ws.qrot, ix->cR, ix->offsets, ix->codes,
        ix->fac, dp, ws.bound, ws.wbase, ws.mwords, ws.mask, nq * ws.mwords, ix->d_err);
  } else if (sh.mode == RQ_SCAN_PLAIN) {
    tm.mark(RQ_STAGE_SCAN, st);
    const unsigned chunks =
        (unsigned)std::max<int64_t>(1, (ix->max_list_len + sh.chunk - 1) / sh.chunk);
    auto kern = scan_plain_kernel<NW4, 1024>;
    if (NW4 <= 2 && sh.chunk == 2048) kern = scan_plain_kernel<NW4, (NW4 <= 2 ? 2048 : 1024)>;
    if (NW4 <= 2 && sh.chunk == 4096) kern = scan_plain_kernel<NW4, (NW4 <= 2 ? 4096 : 1024)>;
    kern<<<dim3((unsigned)pairs, chunks), 128, 0, st>>>(
        ws.nchunks, ws.probe_ids, np, ws.qparams, ws.planes, ix->offsets, ix->codes, ix->fac,
        dp, ws.bound, ws.wbase, ws.mwords, ws.mask, nq * ws.mwords, ix->d_err);
  } else {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
    tm.mark(RQ_STAGE_SCAN, st);
    if (sh.mode == RQ_SCAN_MMA) {
      RQ_TRY(launch_scan_mma(ix, sh, ws, st, sms, sh.withhold, false));
    } else {
      RQ_TRY(launch_scan_stream(ix, sh, ws, st, sms, sh.withhold ? kTestWaitLimitNs : kWaitLimitNs,
                                sh.withhold));
    }
  }
  // 5-6. candidate selection and exact re-rank
  tm.mark(RQ_STAGE_SELECT, st);
  FinalizeArgs f;
  f.mask = ws.mask;
  f.wtotal = ws.wtotal;
  f.mwords = ws.mwords;
  f.wbase = ws.wbase;
  f.probe_ids = ws.probe_ids;
  f.nprobe = ws.nprobe;
  f.npmax = np;
  f.offsets = ix->offsets;
  f.codes = ix->codes;
  f.fac = ix->fac;
  f.planes = ws.planes;
  f.qparams = ws.qparams;
  f.resid = sh.lut ? ws.resid : nullptr;
  f.dp = dp;
  f.ids = ix->ids;
  f.n_slots = ix->n;
  f.err = ix->d_err;
  f.counts = ws.counts;
  f.nsel = ws.nsel;
  f.kq = ws.kq;
  f.rerank_on = ws.rerank_on;
  f.nsel_max = sh.nsel_max;
  f.sel = ws.sel;
  f.raw = ix->raw;
  f.q = ws.q;
  f.dim = ix->dim;
  f.k_stride = sh.k_stride;
  // staging: room for n_sel keys plus a step of survivors, with more for
  // large selections (whose first bound lets more survive). With nprobe,
  // n_sel and k at most 4096 and D at most 2048 this is at most 217 KB.
  f.lay = FinalizeLayout{next_pow2_host(sh.nsel_max),
                         next_pow2_host(std::min<int64_t>(sh.k_stride, kMaxSelect)),
                         sh.nsel_max > 512 ? 8192 : 4096, np, ix->dim};
  f.out_ids = ws.out_ids;
  f.out_d = ws.out_d;
  f.nq = nq;
  f.keys = ws.keys;
  f.kcount = ws.kcount;
  f.kcap = ws.kcap;
  const bool u8 = ix->raw_dtype == RQ_U8;
  // collection: one block per (query, round of mask words)
  RQ_CUDA(cudaMemsetAsync(ws.kcount, 0, sizeof(int32_t) * nq, st));
  const int64_t rounds = std::max<int64_t>(1, (ws.mwords + kFinRoundWords - 1) / kFinRoundWords);
  if (rounds > 65535) return fail(RQ_ERR_NOT_IMPLEMENTED, "probed lists too long for one search");
  collect_kernel<NW4><<<dim3((unsigned)nq, (unsigned)rounds), kFinThreads, f.lay.collect_bytes(),
                        st>>>(f);
  // selection and re-rank from the key buffers; the streaming form for the
  // queries whose survivors overflowed them
  tm.mark(RQ_STAGE_RERANK, st);
  auto sel = u8 ? select_kernel<uint8_t> : select_kernel<float>;
  RQ_TRY(allow_dynamic_smem((const void*)sel, 220 * 1024));
  sel<<<(unsigned)nq, kFinThreads, f.lay.select_bytes(), st>>>(f);
  auto fin = u8 ? finalize_kernel<uint8_t, NW4> : finalize_kernel<float, NW4>;
  RQ_TRY(allow_dynamic_smem((const void*)fin, 220 * 1024));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
  fin<<<(unsigned)std::min<int64_t>(nq, sms), kFinThreads, f.lay.bytes(), st>>>(f);
  return RQ_OK;
}

rq_status enqueue_search(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                         StageTimer& tm) {
  const int64_t nq = sh.nq;
  const int dp = ix->dp;
  // 1. rotation, once per query
  tm.mark(RQ_STAGE_ROTATE, st);
  const bool grouped = sh.mode != RQ_SCAN_PLAIN;
  rotate_kernel8<<<dim3(blocks_for(nq, 8), dp / 64), 256, 0, st>>>(
      ws.q, nq, ix->dim, ix->P32, dp, ws.qrot, grouped ? ws.list_count : nullptr,
      grouped ? ix->nlist : 0, ws.wcount, ws.wcount ? 2 * ix->nlist : 0);
  // 2. centroid ranking: approximate (filter of the certified selection)
  // where certified_probe holds, else exact
  tm.mark(RQ_STAGE_PROBE, st);
  if (certified_probe(ix)) {
    RQ_TRY(launch_approx_dist_tc(ws.qrot, nq, ix->cR, ix->nlist, dp,
                                 reinterpret_cast<float*>(ws.pkeys), ws.cn, ix->d_err, st));
  } else {
    pair_dist_kernel<1, 2><<<dim3(blocks_for(nq, 32), blocks_for(ix->nlist, 64)), 256, 0, st>>>(
        ws.qrot, nq, ix->cR, ix->nlist, dp, nullptr, nullptr, ws.pkeys);
  }
  // 3-4. probe selection, quantisation, bound, scan
  switch (dp / 128) {
    case 1: RQ_TRY(enqueue_scan_stages<1>(ix, sh, ws, st, tm)); break;
    case 2: RQ_TRY(enqueue_scan_stages<2>(ix, sh, ws, st, tm)); break;
    case 3: RQ_TRY(enqueue_scan_stages<3>(ix, sh, ws, st, tm)); break;
    case 4: RQ_TRY(enqueue_scan_stages<4>(ix, sh, ws, st, tm)); break;
    case 5: RQ_TRY(enqueue_scan_stages<5>(ix, sh, ws, st, tm)); break;
    case 6: RQ_TRY(enqueue_scan_stages<6>(ix, sh, ws, st, tm)); break;
    case 7: RQ_TRY(enqueue_scan_stages<7>(ix, sh, ws, st, tm)); break;
    case 8: RQ_TRY(enqueue_scan_stages<8>(ix, sh, ws, st, tm)); break;
    case 12: RQ_TRY(enqueue_scan_stages<12>(ix, sh, ws, st, tm)); break;
    case 16: RQ_TRY(enqueue_scan_stages<16>(ix, sh, ws, st, tm)); break;
    default:
      return fail(RQ_ERR_NOT_IMPLEMENTED, "padded dimension " + std::to_string(dp) +
                                              " has no scan kernel (built: 128..1024, 1536, 2048)");
  }
  tm.mark(RQ_STAGE_COUNT, st);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

void destroy_plan(Plan* p) {
  if (p->params_ready) {
    cudaEventSynchronize(p->params_ready);
    cudaEventDestroy(p->params_ready);
  }
  if (p->h_params) cudaFreeHost(p->h_params);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  // cudaFree waits for the device, so the workspace is idle when released
  // (the stream it was used on may no longer exist).
  if (p->ws.base) cudaFree(p->ws.base);
  p->graph = nullptr;
  p->ws.base = nullptr;
  p->h_params = nullptr;
  p->params_ready = nullptr;
}

constexpr size_t kMaxPlans = 64;

rq_status get_plan(rq_index* ix, cudaStream_t st, const SearchShape& sh, Plan** out) {
  std::lock_guard<std::mutex> lk(ix->mu);
  auto key = std::make_pair(st, sh);
  auto it = ix->plans.find(key);
  if (it != ix->plans.end()) {
    it->second->last_use = ++ix->plan_clock;
    *out = it->second.get();
    return RQ_OK;
  }
  if (ix->plans.size() >= kMaxPlans) {
    auto victim = ix->plans.begin();
    for (auto j = ix->plans.begin(); j != ix->plans.end(); ++j)
      if (j->second->last_use < victim->second->last_use) victim = j;
    destroy_plan(victim->second.get());
    ix->plans.erase(victim);
  }
  auto p = std::make_unique<Plan>();
  p->shape = sh;
  p->stream = st;
  RQ_TRY(alloc_workspace(ix, sh, st, p->ws));
  if (cudaMallocHost(&p->h_params, sizeof(int32_t) * (4 * sh.nq + 2)) != cudaSuccess) {
    cudaGetLastError();
    destroy_plan(p.get());
    return fail(RQ_ERR_OOM, "pinned parameter buffer");
  }
  p->h_err = p->h_params + 4 * sh.nq + 1;
  RQ_CUDA(cudaEventCreateWithFlags(&p->params_ready, cudaEventDisableTiming));
  p->last_use = ++ix->plan_clock;
  *out = p.get();
  ix->plans[key] = std::move(p);
  return RQ_OK;
}

}  // namespace

int next_pow2_host(int64_t v) {
  int m = 1;
  while (m < v) m <<= 1;
  return m;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The tuned choice for a batch of the given class: the exact class when it
// was tuned, else the nearest tuned class (batch size and pair density on
// their log2 scales), else the latest tuned mode with the default chunk.
TunedChoice tuned_for(rq_index* ix, std::pair<int, int> cls) {
  std::lock_guard<std::mutex> lk(ix->mu);
  TunedChoice best;
  best.mode = ix->auto_mode.load();
  int best_d = 1 << 30;
  for (const auto& kv : ix->tuned) {
    const int d = std::abs(kv.first.first - cls.first) + std::abs(kv.first.second - cls.second);
    if (d < best_d) {
      best_d = d;
      best = kv.second;
    }
  }
  return best;
}

// Time the scan forms on the sample batch -- the plain scan at each chunk
// size, the streaming scan and (D_p = 128) the tensor-core scan; a warm-up
// run, then the best of three CUDA-event timings each -- and keep the
// fastest for batches of the sample's class (tune_class). Choices are kept
// per (n, dim, nlist, class) in a text cache file, one line each.
rq_status autotune(rq_index* ix, const float* queries, int64_t nq, const int32_t* nprobe,
                   int n_rerank, const char* cache_path) {
  if (!ix || !queries || !nprobe || nq < 1) return fail(RQ_ERR_INVALID_ARG, "bad autotune arguments");
  int64_t sum_np = 0;
  for (int64_t i = 0; i < nq; ++i) sum_np += nprobe[i];
  const std::pair<int, int> cls = tune_class(nq, sum_np, ix->nlist);
  char key[160];
  snprintf(key, sizeof(key), "n=%lld dim=%d nlist=%d nq_class=%d density_class=%d",
           (long long)ix->n, ix->dim, ix->nlist, cls.first, cls.second);
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512];
      int found = -1, chunk = kPlainChunk;
      while (fgets(line, sizeof(line), f)) {
        const size_t kl = strlen(key);
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ') {
          int m = 0, c = 0;
          if (sscanf(line + kl, " mode=%d chunk=%d", &m, &c) == 2) {
            found = m;
            chunk = c;
          }
        }
      }
      fclose(f);
      if (found >= RQ_SCAN_PLAIN && found <= RQ_SCAN_MMA && chunk >= kPlainChunk &&
          chunk % kPlainChunk == 0) {
        std::lock_guard<std::mutex> lk(ix->mu);
        ix->tuned[cls] = TunedChoice{found, chunk};
        ix->auto_mode.store(found);
        return RQ_OK;
      }
    }
  }
  const int k = n_rerank > 0 ? std::min(10, n_rerank) : 10;
  // Everything this call creates is released on every exit path.
  struct Scratch {
    rq_index* ix = nullptr;
    int64_t* d_ids = nullptr;
    float* d_d = nullptr;
    float* d_q = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
      if (st) {
        cudaStreamSynchronize(st);
        // the plans made for this stream go with it
        std::lock_guard<std::mutex> lk(ix->mu);
        for (auto it = ix->plans.begin(); it != ix->plans.end();) {
          if (it->first.first == st) {
            destroy_plan(it->second.get());
            it = ix->plans.erase(it);
          } else {
            ++it;
          }
        }
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (st) cudaStreamDestroy(st);
      if (d_ids) cudaFree(d_ids);
      if (d_d) cudaFree(d_d);
      if (d_q) cudaFree(d_q);
    }
  } sc;
  sc.ix = ix;
  RQ_CUDA(dev_alloc(&sc.d_ids, sizeof(int64_t) * nq * k));
  RQ_CUDA(dev_alloc(&sc.d_d, sizeof(float) * nq * k));
  RQ_CUDA(dev_alloc(&sc.d_q, sizeof(float) * nq * ix->dim));
  RQ_CUDA(cudaMemcpy(sc.d_q, queries, sizeof(float) * nq * ix->dim, cudaMemcpyDefault));
  RQ_CUDA(cudaStreamCreateWithFlags(&sc.st, cudaStreamNonBlocking));
  RQ_CUDA(cudaEventCreate(&sc.e0));
  RQ_CUDA(cudaEventCreate(&sc.e1));
  std::vector<int32_t> kk(nq, k), nr(nq, n_rerank);
  TunedChoice best;
  float best_ms = 1e30f;
  std::string report;
  const TunedChoice forms[] = {{RQ_SCAN_PLAIN, 1024}, {RQ_SCAN_PLAIN, 2048}, {RQ_SCAN_PLAIN, 4096},
                               {RQ_SCAN_GROUPED, 1024}, {RQ_SCAN_MMA, 1024}};
  for (const TunedChoice& fm : forms) {
    if (fm.mode == RQ_SCAN_MMA && !mma_supported(ix)) continue;
    if (fm.mode == RQ_SCAN_PLAIN && fm.chunk > kPlainChunk && ix->max_list_len <= fm.chunk / 2)
      continue;  // no list is long enough for this chunk to differ
    rq_search_opts o{};
    o.scan_mode = fm.mode;
    o.use_graph = 1;
    o.plain_chunk = fm.chunk;
    float ms_best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      RQ_CUDA(cudaEventRecord(sc.e0, sc.st));
      RQ_TRY(search_run(ix, sc.d_q, nq, nprobe, kk.data(), nr.data(), k, sc.d_ids, sc.d_d, &o,
                        sc.st));
      RQ_CUDA(cudaEventRecord(sc.e1, sc.st));
      RQ_CUDA(cudaEventSynchronize(sc.e1));
      float ms = 0.0f;
      RQ_CUDA(cudaEventElapsedTime(&ms, sc.e0, sc.e1));
      if (rep > 0) ms_best = std::min(ms_best, ms);
    }
    report += " mode" + std::to_string(fm.mode) + "_chunk" + std::to_string(fm.chunk) +
              "_ms=" + std::to_string(ms_best);
    if (ms_best < best_ms) {
      best_ms = ms_best;
      best = fm;
    }
  }
  {
    std::lock_guard<std::mutex> lk(ix->mu);
    ix->tuned[cls] = best;
  }
  ix->auto_mode.store(best.mode);
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "%s mode=%d chunk=%d%s\n", key, best.mode, best.chunk, report.c_str());
      fclose(f);
    }
  }
  return RQ_OK;
}

void free_plans(rq_index* ix) {
  std::lock_guard<std::mutex> lk(ix->mu);
  for (auto& kv : ix->plans) destroy_plan(kv.second.get());
  ix->plans.clear();
}

// One launch sequence for a batch whose per-query parameters are already
// checked: h_np, h_k, h_ns (selection sizes) and h_rr (re-rank flags, then
// the no-prune flag at [nq]), searched as shape `sh` (sh.npmax and
// sh.nsel_max may exceed this batch's own, so that a split batch keeps the
// strides of its parent).
rq_status search_part(rq_index* ix, const float* queries, int64_t nq, const int32_t* h_np,
                      const int32_t* h_k, const int32_t* h_ns, const int32_t* h_rr, int k_stride,
                      int64_t* out_ids, float* out_dist, const rq_search_opts* opts,
                      cudaStream_t st, SearchShape sh) {
  const int npmax = sh.npmax, nsel_max = sh.nsel_max;
  float* stage_ms = opts ? opts->stage_ms : nullptr;
  const bool use_graph = opts && opts->use_graph && !stage_ms;
  const rq_search_dump* dump = opts ? opts->dump : nullptr;
  StageTimer tm;
  struct EventsGuard {
    StageTimer& t;
    ~EventsGuard() {
      for (auto& e : t.ev)
        if (e) cudaEventDestroy(e);
    }
  } guard{tm};
  if (stage_ms) {
    for (auto& e : tm.ev) RQ_CUDA(cudaEventCreate(&e));
    tm.on = true;
  }

  const bool q_dev = is_device_ptr(queries);
  if (!q_dev) {
    // branch-free bit test (all-ones exponent: inf or NaN), so that the loop
    // vectorises
    const uint32_t* u = reinterpret_cast<const uint32_t*>(queries);
    uint32_t bad = 0;
    for (int64_t i = 0; i < nq * ix->dim; ++i) bad |= (uint32_t)((u[i] & 0x7f800000u) == 0x7f800000u);
    if (bad) return fail(RQ_ERR_INVALID_ARG, "non-finite query value");
  }
  const bool ids_dev = is_device_ptr(out_ids), d_dev = is_device_ptr(out_dist);

  cudaStream_t run_st = st;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  if (use_graph && st == nullptr) {
    std::lock_guard<std::mutex> lk(ix->mu);
    if (!ix->graph_stream) RQ_CUDA(cudaStreamCreateWithFlags(&ix->graph_stream, cudaStreamNonBlocking));
    run_st = ix->graph_stream;
  }
  Plan* plan = nullptr;
  RQ_TRY(get_plan(ix, run_st, sh, &plan));
  Workspace& ws = plan->ws;
  if (run_st != st) {
    RQ_CUDA(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    RQ_CUDA(cudaEventRecord(ev_in, st));
    RQ_CUDA(cudaStreamWaitEvent(run_st, ev_in, 0));
  }
  // Per-query parameters go through the plan's pinned buffer; the previous
  // call's copy out of it must have run before it is overwritten.
  RQ_CUDA(cudaEventSynchronize(plan->params_ready));
  int32_t* hp = plan->h_params;
  std::memcpy(hp, h_np, sizeof(int32_t) * nq);
  std::memcpy(hp + nq, h_k, sizeof(int32_t) * nq);
  std::memcpy(hp + 2 * nq, h_ns, sizeof(int32_t) * nq);
  std::memcpy(hp + 3 * nq, h_rr, sizeof(int32_t) * (nq + 1));
  RQ_CUDA(cudaMemcpyAsync(ws.nprobe, hp, sizeof(int32_t) * (4 * nq + 1), cudaMemcpyHostToDevice,
                          run_st));
  RQ_CUDA(cudaEventRecord(plan->params_ready, run_st));
  RQ_CUDA(cudaMemcpyAsync(ws.q, queries, sizeof(float) * nq * ix->dim, cudaMemcpyDefault, run_st));
  if (use_graph) {
    if (!plan->graph) {
      cudaGraph_t g = nullptr;
      RQ_CUDA(cudaStreamBeginCapture(run_st, cudaStreamCaptureModeThreadLocal));
      rq_status s = enqueue_search(ix, sh, ws, run_st, tm);
      cudaError_t e = cudaStreamEndCapture(run_st, &g);
      if (s != RQ_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      e = cudaGraphInstantiate(&plan->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    RQ_CUDA(cudaGraphLaunch(plan->graph, run_st));
  } else {
    RQ_TRY(enqueue_search(ix, sh, ws, run_st, tm));
  }
  RQ_CUDA(cudaMemcpyAsync(out_ids, ws.out_ids, sizeof(int64_t) * nq * k_stride, cudaMemcpyDefault,
                          run_st));
  RQ_CUDA(cudaMemcpyAsync(out_dist, ws.out_d, sizeof(float) * nq * k_stride, cudaMemcpyDefault,
                          run_st));
  if (dump) {
    const int W = ix->dp / 32;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> rq_status {
      if (dst) RQ_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, run_st));
      return RQ_OK;
    };
    RQ_TRY(cp(dump->qrot, ws.qrot, sizeof(float) * nq * ix->dp));
    RQ_TRY(cp(dump->probe_ids, ws.probe_ids, sizeof(int32_t) * nq * npmax));
    RQ_TRY(cp(dump->probe_dist, ws.probe_d, sizeof(float) * nq * npmax));
    RQ_TRY(cp(dump->qparams, ws.qparams, sizeof(float4) * nq * npmax));
    RQ_TRY(cp(dump->planes, ws.planes, sizeof(uint32_t) * nq * npmax * 4 * W));
    RQ_TRY(cp(dump->bound, ws.bound, sizeof(uint32_t) * nq));
    RQ_TRY(cp(dump->selected, ws.sel, sizeof(uint64_t) * nq * nsel_max));
    RQ_TRY(cp(dump->n_candidates, ws.counts, sizeof(int32_t) * nq));
  }
  if (run_st != st) {
    RQ_CUDA(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
    RQ_CUDA(cudaEventRecord(ev_out, run_st));
    RQ_CUDA(cudaStreamWaitEvent(st, ev_out, 0));
    cudaEventDestroy(ev_in);
    cudaEventDestroy(ev_out);
  }
  // Host outputs (or host queries read by a pending copy) need the stream
  // to finish before the call returns; device-only calls stay asynchronous.
  // A call that waits also reads the device error word (one 4-byte copy).
  const bool waits = !ids_dev || !d_dev || !q_dev;
  if (waits) {
    RQ_CUDA(cudaMemcpyAsync(plan->h_err, ix->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RQ_CUDA(cudaStreamSynchronize(st));
    const int32_t code = *plan->h_err;
    if (code != 0) {
      RQ_CUDA(cudaMemsetAsync(ix->d_err, 0, sizeof(int32_t), st));
      RQ_CUDA(cudaStreamSynchronize(st));
      if (code == kErrMmaTimeout || code == kErrScanTimeout)
        return fail(RQ_ERR_TIMEOUT, "a bounded wait of the scan ran out (device code " +
                                        std::to_string(code) + ")");
      return fail(RQ_ERR_DEVICE, "a kernel flagged device error " + std::to_string(code));
    }
  }
  if (stage_ms) {
    RQ_CUDA(cudaEventSynchronize(tm.ev[RQ_STAGE_COUNT]));
    for (int i = 0; i < RQ_STAGE_COUNT; ++i) {
      float ms = 0.0f;
      RQ_CUDA(cudaEventElapsedTime(&ms, tm.ev[i], tm.ev[i + 1]));
      stage_ms[i] = ms;
    }
  }
  return RQ_OK;
}


rq_status search_run(rq_index* ix, const float* queries, int64_t nq, const int32_t* nprobe,
                     const int32_t* k, const int32_t* n_rerank, int k_stride, int64_t* out_ids,
                     float* out_dist, const rq_search_opts* opts, cudaStream_t st) {
  if (!ix) return fail(RQ_ERR_INVALID_ARG, "index is NULL");
  if (nq < 0) return fail(RQ_ERR_INVALID_ARG, "nq < 0");
  if (nq == 0) return RQ_OK;
  if (!queries || !out_ids || !out_dist || !nprobe || !k || !n_rerank)
    return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  if (nq > (int64_t)1 << 24) return fail(RQ_ERR_INVALID_ARG, "nq above 2^24 in one call");
  const int pmax_allowed = std::min(ix->nlist, kMaxSelect);
  std::vector<int32_t> h_np(nq), h_k(nq), h_ns(nq), h_rr(nq + 1);
  int npmax = 0, nsel_max = 0, kmax = 0;
  for (int64_t i = 0; i < nq; ++i) {
    const int a = nprobe[i], b = k[i], c = n_rerank[i];
    if (a < 1 || a > pmax_allowed)
      return fail(RQ_ERR_INVALID_ARG, "nprobe " + std::to_string(a) + " outside [1, " +
                                          std::to_string(pmax_allowed) + "]");
    if (b < 1 || b > kMaxSelect) return fail(RQ_ERR_INVALID_ARG, "k outside [1, 4096]");
    if (c != 0 && (c < b || c > kMaxSelect))
      return fail(RQ_ERR_INVALID_ARG, "n_rerank must be 0 or in [k, 4096]");
    h_np[i] = a;
    h_k[i] = b;
    h_ns[i] = c > 0 ? c : b;
    h_rr[i] = c > 0 ? 1 : 0;
    npmax = std::max(npmax, a);
    nsel_max = std::max(nsel_max, h_ns[i]);
    kmax = std::max(kmax, b);
  }
  if (k_stride < kmax) return fail(RQ_ERR_INVALID_ARG, "k_stride below the largest k");
  int mode = opts ? opts->scan_mode : RQ_SCAN_AUTO;
  int chunk = (opts && opts->plain_chunk > 0) ? opts->plain_chunk : kPlainChunk;
  if (mode == RQ_SCAN_AUTO) {
    int64_t sum_np = 0;
    for (int64_t i = 0; i < nq; ++i) sum_np += h_np[i];
    const TunedChoice t = tuned_for(ix, tune_class(nq, sum_np, ix->nlist));
    mode = t.mode;
    if (!(opts && opts->plain_chunk > 0)) chunk = t.chunk;
  }
  if (mode < RQ_SCAN_PLAIN || mode > RQ_SCAN_MMA)
    return fail(RQ_ERR_INVALID_ARG, "unknown scan mode");
  // only the plain scan has chunks; codes wider than 256 bits use 1024
  if (mode != RQ_SCAN_PLAIN || ix->dp > 256) chunk = kPlainChunk;
  if (chunk != 1024 && chunk != 2048 && chunk != 4096)
    return fail(RQ_ERR_INVALID_ARG, "plain_chunk must be 1024, 2048 or 4096");
  if (mode == RQ_SCAN_MMA && !mma_supported(ix)) mode = RQ_SCAN_GROUPED;
  const int estimator = opts ? opts->estimator : RQ_EST_BQ4;
  if (estimator != RQ_EST_BQ4 && estimator != RQ_EST_LUT)
    return fail(RQ_ERR_INVALID_ARG, "unknown estimator");
  if (estimator == RQ_EST_LUT) {
    if (ix->dp > 256)
      return fail(RQ_ERR_NOT_IMPLEMENTED, "the FastScan estimator is built for D_p <= 256");
    mode = RQ_SCAN_PLAIN;  // its scan runs on the query-level schedule
    chunk = kPlainChunk;
  }
  const bool no_prune = opts && opts->no_prune;
  h_rr[nq] = no_prune ? 1 : 0;
  const int withhold = (opts && opts->test_stall && mode != RQ_SCAN_PLAIN) ? 1 : 0;
  SearchShape sh{nq, npmax, nsel_max, k_stride, mode, no_prune ? 1 : 0, withhold, chunk,
                 estimator == RQ_EST_LUT ? 1 : 0};
  // A batch whose workspace would pass the budget runs as consecutive
  // sub-batches of one workspace (the survivor slots grow with the pairs
  // scanned); results and dump rows land where the whole batch puts them.
  int64_t sub = nq;
  while (sub > 1) {
    SearchShape t = sh;
    t.nq = sub;
    if (workspace_bytes(ix, t) <= kWorkspaceBudget) break;
    sub = (sub + 1) / 2;
  }
  if (sub == nq) return search_part(ix, queries, nq, h_np.data(), h_k.data(), h_ns.data(),
                                    h_rr.data(), k_stride, out_ids, out_dist, opts, st, sh);
  float part_ms[RQ_STAGE_COUNT];
  if (opts && opts->stage_ms)
    for (int i = 0; i < RQ_STAGE_COUNT; ++i) opts->stage_ms[i] = 0.0f;
  for (int64_t i0 = 0; i0 < nq; i0 += sub) {
    const int64_t n1 = std::min(sub, nq - i0);
    rq_search_opts po = opts ? *opts : rq_search_opts{};
    rq_search_dump pd{};
    if (opts && opts->dump) {
      const rq_search_dump& d = *opts->dump;
      const int64_t cb = ix->dp / 8;
      pd.qrot = d.qrot ? d.qrot + i0 * ix->dp : nullptr;
      pd.probe_ids = d.probe_ids ? d.probe_ids + i0 * npmax : nullptr;
      pd.probe_dist = d.probe_dist ? d.probe_dist + i0 * npmax : nullptr;
      pd.qparams = d.qparams ? d.qparams + i0 * npmax * 4 : nullptr;
      pd.planes = d.planes ? d.planes + i0 * npmax * 4 * cb : nullptr;
      pd.bound = d.bound ? d.bound + i0 : nullptr;
      pd.selected = d.selected ? d.selected + i0 * nsel_max : nullptr;
      pd.n_candidates = d.n_candidates ? d.n_candidates + i0 : nullptr;
      po.dump = &pd;
    }
    if (opts && opts->stage_ms) po.stage_ms = part_ms;
    std::vector<int32_t> rr(h_rr.begin() + i0, h_rr.begin() + i0 + n1);
    rr.push_back(h_rr[nq]);
    SearchShape t = sh;
    t.nq = n1;
    RQ_TRY(search_part(ix, queries + i0 * ix->dim, n1, h_np.data() + i0, h_k.data() + i0, h_ns.data() + i0, rr.data(),
                       k_stride, out_ids + i0 * k_stride, out_dist + i0 * k_stride, &po, st, t));
    if (opts && opts->stage_ms)
      for (int i = 0; i < RQ_STAGE_COUNT; ++i) opts->stage_ms[i] += part_ms[i];
  }
  return RQ_OK;
}

}  // namespace rq

// ===========================================================================
// Allocation-free variant of the query rotation and centroid ranking.
//
// Some callers cannot allocate device memory at the moment they search:
// processes whose framework hands all device memory to its own caching
// allocator, and latency-critical serving threads that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree. For them, rq_probe_static keeps its scratch (the
// rotated queries and the distance keys) in one fixed array in device memory
// that exists for as long as the library is loaded.
// ===========================================================================
namespace rq {
namespace {

constexpr size_t kProbeScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_probe_scratch[kProbeScratchBytes];

// Device address of g_probe_scratch, looked up once per device. In host code
// the symbol itself is only a host-side stand-in and must never be passed to
// a kernel.
void* g_probe_scratch_addr[kMaxDevices] = {};
std::mutex g_probe_scratch_mu;

rq_status probe_scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return fail(RQ_ERR_INVALID_ARG, "device ordinal above the supported range");
  std::lock_guard<std::mutex> lk(g_probe_scratch_mu);
  if (!g_probe_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_probe_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_probe_scratch)", __FILE__, __LINE__);
    g_probe_scratch_addr[device] = p;
  }
  *out = g_probe_scratch_addr[device];
  return RQ_OK;
}

}  // namespace
}  // namespace rq

extern "C" rq_status rq_probe_static(const rq_index* ix, const float* queries, int64_t nq,
                                     int32_t nprobe, int32_t* out_ids, float* out_dist,
                                     void* stream) {
  using namespace rq;
  if (!ix || !queries || !out_ids || !out_dist)
    return fail(RQ_ERR_INVALID_ARG, "NULL pointer argument");
  if (nq < 1) return fail(RQ_ERR_INVALID_ARG, "nq < 1");
  if (nprobe < 1 || nprobe > std::min(ix->nlist, kMaxSelect))
    return fail(RQ_ERR_INVALID_ARG, "nprobe outside [1, min(nlist, 4096)]");
  const size_t q_bytes = align_up(sizeof(float) * (size_t)nq * ix->dp);
  const size_t k_bytes = align_up(sizeof(uint64_t) * (size_t)nq * ix->nlist);
  if (q_bytes + k_bytes > kProbeScratchBytes)
    return fail(RQ_ERR_INVALID_ARG,
                "rq_probe_static: nq x (4 D_p + 8 nlist) bytes = " +
                    std::to_string(q_bytes + k_bytes) + " exceeds its fixed scratch of " +
                    std::to_string(kProbeScratchBytes) + " bytes; use fewer queries per call");
  if (!is_device_ptr(queries) || !is_device_ptr(out_ids) || !is_device_ptr(out_dist))
    return fail(RQ_ERR_INVALID_ARG, "rq_probe_static takes device pointers only");
  int dev = -1;
  RQ_CUDA(cudaGetDevice(&dev));
  if (dev != ix->device)
    return fail(RQ_ERR_INVALID_ARG, "the current device is not the index's device");
  void* scratch = nullptr;
  RQ_TRY(probe_scratch_address(dev, &scratch));
  float* qrot = static_cast<float*>(scratch);
  uint64_t* pkeys = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + q_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int dp = ix->dp;
  rotate_kernel<<<dim3(blocks_for(nq, 64), dp / 64), 256, 0, st>>>(queries, nq, ix->dim, ix->P32,
                                                                  dp, qrot);
  pair_dist_kernel<1><<<dim3(blocks_for(nq, 64), blocks_for(ix->nlist, 64)), 256, 0, st>>>(
      qrot, nq, ix->cR, ix->nlist, dp, nullptr, nullptr, pkeys);
  const int m = next_pow2_host(std::min<int64_t>(ix->nlist, kMaxSelect));
  const size_t smem = sizeof(uint64_t) * std::max(m, next_pow2_host(nprobe));
  select_rows_kernel<1><<<(unsigned)nq, 1024, smem, st>>>(pkeys, ix->nlist, nullptr, ix->nlist,
                                                         ix->nlist, nullptr, nprobe, nullptr,
                                                         nprobe, out_ids, out_dist, ix->d_err);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}
