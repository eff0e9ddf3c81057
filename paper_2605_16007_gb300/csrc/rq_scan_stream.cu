// Streaming form of the grouped code scan (Eqs. 4-5 with a 4-bit query,
// Section 3.3.2; block-level scheduling across queries, Section 3.3.1).
//
// The scan is bound by the bytes of the probed lists (D_p/8 code bytes and
// the 8-byte {r^2, f} factor per vector) once the index is larger than L2,
// and by the popcounts of the estimator when many queries probe each list,
// so each block keeps a deep ring of list blocks in flight and many of them
// in work at once:
//
//  * Work items are the index's static (list, first vector) blocks of 256
//    vectors, longest lists first. Block b of G takes items b, b + G,
//    b + 2G, ...: its producer warp resolves 256 of them at once (eight per
//    lane: the item, its list's pair count and offsets, each level's loads
//    in flight together), keeps the ones whose list is probed (a ballot), and
//    skips the rest without a further load.
//  * For each kept item the producer waits until the next ring stage is free
//    and issues three TMA bulk copies into it -- the item's codes, its
//    factors, and the first pair records of its list (everything the
//    estimator needs about each (query, probe) pair that probes the list:
//    bit-planes, {vl, delta, nq2, Sq}, query, first mask word, bound; written
//    contiguously per list by the preparation kernel) -- all completing on
//    the stage's `full` mbarrier.
//  * Sixteen consumer warps each take whole items: a warp claims the next
//    ring position from a shared-memory counter, waits until the producer
//    has issued that position (a second counter, so that the stage's
//    mbarrier is never more than one phase behind the wait), waits for its
//    stage, runs
//    the estimator for its 256 vectors (32 at a time, a lane per vector)
//    against every pair of the list, writes the survivor mask words and keys
//    (no atomics), and releases the stage. Up to sixteen items are in work
//    per SM while the producer refills the free stages.
//
// Survivor keys carry the vector's slot in the list layout, not its row id;
// the finalize kernel maps slots to ids for the candidates it collects.
//
// Every wait is bounded (limit given by the host); a wait that runs out sets
// the error word, and the block lets its copies in flight land before it
// returns.
#include <cuda_runtime.h>

#include <algorithm>

#include "rq_async.cuh"
#include "rq_common.cuh"
#include "rq_scan.cuh"

namespace rq {
namespace {

constexpr int kStreamConsumers = 16;                         // warps, one item each
constexpr int kStreamThreads = 32 * (kStreamConsumers + 1);  // plus the producer warp

template <int NW4>
struct StreamCfg {
  static constexpr int kV = kGroupVectors;                 // vectors per item
  static constexpr int kCodeB = kV * 16 * NW4;             // packed codes
  static constexpr int kFacB = kV * 8 + 16;                // {r^2, f}, copied from an even slot
  static constexpr int kRecB = 64 * NW4 + 32;              // one pair record
  static constexpr int kRecCap = 16;                       // records staged per item
  static constexpr int kStageB = kCodeB + kFacB + kRecCap * kRecB;
  static constexpr int kBudget = 200 * 1024;               // one block per SM
  static constexpr int kStagesFit = (kBudget - 1024) / kStageB;
  // at least one stage per consumer warp plus room to refill ahead
  static constexpr int kStages = kStagesFit > 32 ? 32 : kStagesFit;
  static constexpr int kMetaOff = kStages * kStageB;
  static constexpr int kBarOff = kMetaOff + kStages * 32;
  static constexpr int kSmem = kBarOff + 2 * kStages * 8 + 16 + 128;  // + counter, alignment
  static_assert(kStageB % 16 == 0 && kRecB % 16 == 0, "TMA needs 16-byte units");
};

// What the producer tells the consumers about a stage.
struct StreamMeta {
  long long lo;  // first slot of the item
  int l;         // list (-1: no more items)
  int nvec;      // vectors of the item
  int cnt;       // pairs probing the list
  int v0;        // first vector of the item within its list
  int pad0, pad1;
};

template <int NW4>
__device__ void stream_producer(uint8_t* sm, uint32_t sbase, const int2* __restrict__ items,
                                int n_items, const int32_t* __restrict__ list_count,
                                const uint8_t* __restrict__ recs, int64_t pair_stride,
                                const int64_t* __restrict__ offsets,
                                const uint8_t* __restrict__ codes,
                                const float2* __restrict__ fac, volatile int* s_issued,
                                int32_t* err, uint64_t wait_ns, int withhold) {
  using Cfg = StreamCfg<NW4>;
  constexpr int S = Cfg::kStages;
  const int lane = threadIdx.x & 31;
  StreamMeta* meta = reinterpret_cast<StreamMeta*>(sm + Cfg::kMetaOff);
  const uint32_t bar_full = sbase + Cfg::kBarOff;
  const uint32_t bar_empty = bar_full + 8 * S;
  const int64_t G = gridDim.x;
  int i = 0;  // items issued
  bool ok = true;
  // waits until stage i % S is free (true), or gives up (false)
  auto claim = [&](int it) -> bool {
    if (it < S) return true;
    int r = 1;
    if (lane == 0)
      r = mbar_wait_bounded(bar_empty + 8 * (it % S), (uint32_t)(((it / S) - 1) & 1), wait_ns) ? 1
                                                                                              : 0;
    return __shfl_sync(0xffffffffu, r, 0) != 0;
  };
  // Rounds of 32 x kPerLane items: lane j resolves items base + (k 32 + j) G
  // for k < kPerLane, all of one level's loads in flight together (item,
  // then pair count and offsets), then the warp walks the probed ones.
  constexpr int kPerLane = 8;
  for (int64_t base = blockIdx.x; ok && base < n_items; base += 32 * kPerLane * G) {
    int2 w[kPerLane];
#pragma unroll
    for (int k = 0; k < kPerLane; ++k) {
      const int64_t idx = base + (int64_t)(k * 32 + lane) * G;
      w[k] = idx < n_items ? items[idx] : make_int2(-1, 0);
    }
    int cnt[kPerLane];
    long long lo[kPerLane], hi[kPerLane];
#pragma unroll
    for (int k = 0; k < kPerLane; ++k) {
      cnt[k] = 0;
      lo[k] = hi[k] = 0;
      if (w[k].x >= 0) {
        cnt[k] = list_count[w[k].x];
        lo[k] = offsets[w[k].x];
        hi[k] = offsets[w[k].x + 1];
      }
    }
#pragma unroll
    for (int k = 0; k < kPerLane; ++k) {
      uint32_t work = __ballot_sync(0xffffffffu, cnt[k] > 0);
      while (ok && work) {
        const int j = __ffs(work) - 1;
        work &= work - 1;
        const int jl = __shfl_sync(0xffffffffu, w[k].x, j);
        const int jv0 = __shfl_sync(0xffffffffu, w[k].y, j);
        const int jc = __shfl_sync(0xffffffffu, cnt[k], j);
        const long long jlo = __shfl_sync(0xffffffffu, lo[k], j) + jv0;
        const int jn = (int)min((long long)Cfg::kV, __shfl_sync(0xffffffffu, hi[k], j) - jlo);
        if (!claim(i)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          const int st = i % S;
          StreamMeta& m = meta[st];
          m.lo = jlo;
          m.l = jl;
          m.nvec = jn;
          m.cnt = jc;
          m.v0 = jv0;
          const uint32_t stage = sbase + st * Cfg::kStageB;
          const long long lo_al = jlo & ~1ll;
          const uint32_t code_b = (uint32_t)jn * 16 * NW4;
          const uint32_t fac_b = (uint32_t)((((jlo - lo_al) + jn) * 8 + 15) & ~15ll);
          const uint32_t rec_b = (uint32_t)min(jc, Cfg::kRecCap) * Cfg::kRecB;
          if (!(withhold && i == 0)) {
            mbar_expect_tx_arrive(bar_full + 8 * st, code_b + fac_b + rec_b);
            tma_load_1d(stage, codes + jlo * 16 * NW4, code_b, bar_full + 8 * st);
            tma_load_1d(stage + Cfg::kCodeB, fac + lo_al, fac_b, bar_full + 8 * st);
            tma_load_1d(stage + Cfg::kCodeB + Cfg::kFacB,
                        recs + (int64_t)jl * pair_stride * Cfg::kRecB, rec_b, bar_full + 8 * st);
          }
          // (test hook: with `withhold`, the first stage is never filled nor
          // signalled, so the consumers' bounded wait for it runs out)
          __threadfence_block();
          *s_issued = i + 1;
        }
        __syncwarp();
        ++i;
      }
    }
  }
  // End markers: one stage per consumer warp whose meta says "no more
  // items" (each warp claims exactly one of them and leaves).
  for (int e = 0; ok && e < kStreamConsumers; ++e) {
    if (!claim(i + e)) {
      ok = false;
      break;
    }
    if (lane == 0) {
      meta[(i + e) % S].l = -1;
      mbar_arrive(bar_full + 8 * ((i + e) % S));
      __threadfence_block();
      *s_issued = i + e + 1;
    }
    __syncwarp();
  }
  if (lane == 0 && !ok) {
    flag_error(err, kErrScanTimeout);
    // After a wait ran out the consumers may have left: the copies of the
    // last use of every stage land before the block returns. (In a normal
    // run the consumers wait for every stage themselves.)
    for (int s = 0; s < S && s < i; ++s) {
      const int k = s + ((i - 1 - s) / S) * S;  // last item issued into stage s
      if (withhold && k == 0) continue;
      mbar_wait_bounded(bar_full + 8 * s, (uint32_t)((k / S) & 1), wait_ns);
    }
  }
  __syncwarp();
}

// Vectors of an item a consumer warp holds in registers at once: SB blocks
// of 32 (lane t holds vectors t, t + 32, ...), so that every pair record is
// read once per SB blocks and the SB estimates of a pair are independent.
template <int NW4>
struct StreamRegs {
  static constexpr int SB = NW4 >= 4 ? 1 : 8 / NW4;
};

template <int NW4>
__device__ void stream_consumer(const uint8_t* sm, uint32_t sbase, int* s_next,
                                const volatile int* s_issued,
                                const uint8_t* __restrict__ recs, int64_t pair_stride,
                                int64_t mwords, int64_t mask_words, uint32_t* __restrict__ mask,
                                int32_t* err, uint64_t wait_ns) {
  using Cfg = StreamCfg<NW4>;
  constexpr int S = Cfg::kStages;
  constexpr int DP = 128 * NW4;
  constexpr int SB = StreamRegs<NW4>::SB;
  const int lane = threadIdx.x & 31;
  const StreamMeta* meta = reinterpret_cast<const StreamMeta*>(sm + Cfg::kMetaOff);
  const uint32_t bar_full = sbase + Cfg::kBarOff;
  const uint32_t bar_empty = bar_full + 8 * S;
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(s_next, 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    const int st = i % S;
    // Position i is issued once the producer has filled (or withheld) it;
    // from then on stage st's barrier is in phase i / S or just past it, so
    // the parity below names the right phase.
    bool issued = true;
    if (lane == 0) {
      const uint64_t t0 = globaltimer_ns();
      while (*s_issued <= i) {
        if (globaltimer_ns() - t0 > wait_ns) {
          issued = false;
          break;
        }
        __nanosleep(64);
      }
    }
    // every lane observes the phase itself (its own acquire of the copies)
    const bool got = __shfl_sync(0xffffffffu, (int)issued, 0) &&
                     mbar_wait_bounded(bar_full + 8 * st, (uint32_t)((i / S) & 1), wait_ns);
    if (!__all_sync(0xffffffffu, got)) {
      if (lane == 0) flag_error(err, kErrScanTimeout);
      return;
    }
    const StreamMeta m = meta[st];
    if (m.l < 0) {  // an end marker: hand the stage back and leave
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_empty + 8 * st);
      return;
    }
    const uint8_t* stage = sm + st * Cfg::kStageB;
    const uint8_t* srec = stage + Cfg::kCodeB + Cfg::kFacB;
    const uint8_t* grec = recs + (int64_t)m.l * pair_stride * Cfg::kRecB;
    const float2* fac_s = reinterpret_cast<const float2*>(stage + Cfg::kCodeB) + (m.lo & 1);
    for (int b0 = 0; b0 < m.nvec; b0 += 32 * SB) {
      // the codes, factors and popcounts of SB blocks of 32 vectors
      uint4 code[SB][NW4];
      float2 f[SB];
      int pc[SB];
#pragma unroll
      for (int b = 0; b < SB; ++b) {
        const int v = b0 + 32 * b + lane;
        pc[b] = 0;
        f[b] = make_float2(0.0f, 0.0f);
        if (v < m.nvec) {
          const uint4* cp = reinterpret_cast<const uint4*>(stage + v * 16 * NW4);
#pragma unroll
          for (int w = 0; w < NW4; ++w) {
            code[b][w] = cp[w];
            pc[b] += __popc(code[b][w].x) + __popc(code[b][w].y) + __popc(code[b][w].z) +
                     __popc(code[b][w].w);
          }
          f[b] = fac_s[v];
        } else {
#pragma unroll
          for (int w = 0; w < NW4; ++w) code[b][w] = make_uint4(0, 0, 0, 0);
        }
      }
      const int64_t word0 = (m.v0 + b0) / 32;
      for (int g = 0; g < m.cnt; ++g) {
        const uint8_t* rp = g < Cfg::kRecCap ? srec + g * Cfg::kRecB : grec + (int64_t)g * Cfg::kRecB;
        const float4 qp = *reinterpret_cast<const float4*>(rp + 64 * NW4);
        const int4 rm = *reinterpret_cast<const int4*>(rp + 64 * NW4 + 16);  // q, wbase, tau
        const int64_t wrow = (int64_t)rm.x * mwords + rm.y + word0;
        uint32_t mw[SB];
#pragma unroll
        for (int b = 0; b < SB; ++b) {
          const bool valid = b0 + 32 * b + lane < m.nvec;
          const float d = estimate_regs<NW4>(code[b], pc[b], f[b],
                                             reinterpret_cast<const uint32_t*>(rp), qp, DP);
          mw[b] = __ballot_sync(0xffffffffu, valid && orderable(d) <= (uint32_t)rm.z);
        }
        // lane b writes the mask word of block b
#pragma unroll
        for (int b = 0; b < SB; ++b) {
          if (b0 + 32 * b >= m.nvec) break;  // warp-uniform: past the item's end
          if (!index_ok(wrow + b, mask_words, err)) break;
          if (lane == b) mask[wrow + b] = mw[b];
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_empty + 8 * st);
  }
}

template <int NW4>
__global__ void __launch_bounds__(kStreamThreads, 1)
scan_stream_kernel(const int2* __restrict__ items, int n_items,
                   const int32_t* __restrict__ list_count, const uint8_t* __restrict__ recs,
                   int64_t pair_stride, const int64_t* __restrict__ offsets,
                   const uint8_t* __restrict__ codes, const float2* __restrict__ fac,
                   int64_t mwords, uint32_t* __restrict__ mask,
                   int32_t* err, uint64_t wait_ns, int withhold) {
  using Cfg = StreamCfg<NW4>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw_addr + 127u) & ~127u) - raw_addr);
  const uint32_t sbase = smem_u32(sm);
  int* s_next = reinterpret_cast<int*>(sm + Cfg::kBarOff + 2 * Cfg::kStages * 8);
  volatile int* s_issued = s_next + 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(sbase + Cfg::kBarOff + 8 * s, 1);                       // full: the producer
      mbar_init(sbase + Cfg::kBarOff + 8 * (Cfg::kStages + s), 1);  // empty: the consumer warp
    }
    *s_next = 0;
    *s_issued = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if ((int)(threadIdx.x >> 5) == kStreamConsumers)
    stream_producer<NW4>(sm, sbase, items, n_items, list_count, recs, pair_stride, offsets, codes,
                         fac, s_issued, err, wait_ns, withhold);
  else
    stream_consumer<NW4>(sm, sbase, s_next, s_issued, recs, pair_stride, mwords,
                         pair_stride * mwords, mask, err, wait_ns);
}

template <int NW4>
rq_status launch_stream(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                        int sms, uint64_t wait_ns, int withhold) {
  using Cfg = StreamCfg<NW4>;
  RQ_TRY(allow_dynamic_smem((const void*)scan_stream_kernel<NW4>, Cfg::kSmem));
  const unsigned grid = (unsigned)std::max(1, std::min(sms, ix->n_items));
  scan_stream_kernel<NW4><<<grid, kStreamThreads, Cfg::kSmem, st>>>(
      ix->items, ix->n_items, ws.list_count, ws.qrec, sh.nq, ix->offsets, ix->codes, ix->fac,
      ws.mwords, ws.mask, ix->d_err, wait_ns, withhold);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

}  // namespace

rq_status launch_scan_stream(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                             int sms, uint64_t wait_ns, int withhold) {
  switch (ix->dp / 128) {
    case 1: return launch_stream<1>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 2: return launch_stream<2>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 3: return launch_stream<3>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 4: return launch_stream<4>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 5: return launch_stream<5>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 6: return launch_stream<6>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 7: return launch_stream<7>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 8: return launch_stream<8>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 12: return launch_stream<12>(ix, sh, ws, st, sms, wait_ns, withhold);
    case 16: return launch_stream<16>(ix, sh, ws, st, sms, wait_ns, withhold);
    default:
      return fail(RQ_ERR_NOT_IMPLEMENTED, "padded dimension " + std::to_string(ix->dp) +
                                              " has no streaming scan");
  }
}

}  // namespace rq
