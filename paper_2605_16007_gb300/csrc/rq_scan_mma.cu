// Tensor-core form of the grouped code scan (Eqs. 4-5 with a 4-bit query,
// Section 3.3.2), for D_p = 128.
//
// The integer inner product ip = sum_d bit_d * q_u,d of a 128-vector tile
// with a group of up to 64 quantised (query, list) residuals is one
// [128 x 128] x [128 x N] product. Both operands are held exactly in FP8 E4M3
// (a code bit is 0 or 1.0, a query digit an integer 0..15), and the FP32
// accumulation of at most 128 products of integers <= 15 is exact, so ip is
// the same integer the popcount form computes.
//
// Pipeline of one block (persistent over work units = (256-vector block of a
// list, group of up to 64 of the list's pairs)): TMA bulk copies bring the
// unit's B tile (the group's query digits, pre-swizzled in their per-list
// bucket), parameters, per-pair mask rows and bounds -- and, for the first
// group of a block, its packed codes and {r^2, f} factors -- into one of two
// shared-memory stages, completing on that stage's mbarrier, while the block
// works on the other stage. For a block's first group, thread t expands the
// codes of vector t to an FP8 row of the A tile of its 128-vector half (128B
// swizzle) and keeps its vector's popcount and factors in registers for the
// later groups; one thread issues four tcgen05.mma (K = 32 bytes each) per
// tile into that tile's TMEM accumulator (columns [64 tile, 64 tile + 64));
// thread t then reads its own row back with tcgen05.ld (warp w: TMEM lanes
// 32 (w % 4) .. of tile w / 4) for the float32 estimator epilogue, so all
// eight warps share the epilogue.
#include <cuda_runtime.h>

#include <algorithm>

#include "rq_async.cuh"
#include "rq_common.cuh"
#include "rq_scan.cuh"
#include "rq_tc.cuh"

namespace rq {
namespace {

constexpr int kMmaM = 128;        // vectors per tile (TMEM lanes)
constexpr int kMmaNmax = 64;      // pairs per MMA group (TMEM columns)
constexpr int kMmaK = 128;        // D_p
constexpr int kItemV = kGroupVectors;  // 256 vectors per work item = 2 tiles
constexpr int kConsumers = 256;   // eight warps: expansion, MMA issue, epilogue
constexpr int kMmaThreads = kConsumers + 32;  // plus one producer warp
constexpr int kTmemCols = 2 * kMmaNmax;    // one accumulator per tile of the item

// Shared memory of one block (offsets from a 1024-byte aligned base).
constexpr int kSmA = 0;                                  // 2 tiles x 128 x 128 B (128B swizzle)
constexpr int kSmB = kSmA + 2 * kMmaM * kMmaK;           // 2 stages x 64 x 128 B
constexpr int kSmCode = kSmB + 2 * kMmaNmax * kMmaK;     // 2 stages x 256 x 16 B
constexpr int kFacBytes = (kItemV + 2) * 8;              // +1 for alignment, rounded
constexpr int kSmFac = kSmCode + 2 * kItemV * 16;        // 2 stages x 258 x 8 B
constexpr int kSmQp = kSmFac + 2 * kFacBytes;            // 2 stages x 64 x 16 B
constexpr int kSmWr = kSmQp + 2 * kMmaNmax * 16;         // 2 stages x 64 x int64 mask rows
constexpr int kSmTau = kSmWr + 2 * kMmaNmax * 8;         // 2 stages x 64 x float bounds
constexpr int kSmBar = kSmTau + 2 * kMmaNmax * 4;        // mbarriers: full[2], empty[2], mma, aux
constexpr int kSmMeta = kSmBar + 6 * 8;                  // 2 stages x 32-byte meta
constexpr int kSmTmem = kSmMeta + 2 * 32;                // TMEM base address
constexpr int kSmBytes = kSmTmem + 4;
constexpr int kSmAlloc = kSmBytes + 1024;                // room to align the base

// Four code bits (a nibble) -> four FP8 bytes 0x38 (1.0) or 0x00: the
// multiply places bit i at bit 8i without carries (bit i + 7j lands on a
// multiple of 8 only for j = i).
__device__ __forceinline__ uint32_t nibble_to_e4m3(uint32_t n) {
  return ((n * 0x00204081u) & 0x01010101u) * 0x38u;
}

// Work unit meta of one stage: first slot, list (-1: no more units),
// vectors, pairs of the group, first vector within the list, whether this
// is the block's first group (its codes and factors are in the stage).
struct Meta {
  long long lo;
  int l, nvec, np, v0, first, pad;
};

// The estimates of two pairs (columns) for this thread's vector: qa =
// {vl, vl', delta, delta'}, qb = {nq2, nq2', -Sq, -Sq'}, ra / rb the TMEM
// words (ip as float), b2 = (2 pc - D_p) twice, r2 / f2 the vector's r^2 and
// f twice. The popcount form's operations, each rounded once: a = 2 ip - Sq
// is an exact small integer (one FMA with -Sq gives it exactly); x - 2 y is
// x + (-2) y (the negation and the doubling are exact, so one fused
// multiply-add rounds the same); the final + 0 of the popcount form is left
// out because (nq2 + r^2) - x with nq2, r^2 >= +0 is never -0.
__device__ __forceinline__ float2 estimate2(float4 qa, float4 qb, uint32_t ra, uint32_t rb,
                                           float2 b2, float2 r2, float2 f2) {
  const float2 ip = make_float2(__uint_as_float(ra), __uint_as_float(rb));
  const float2 a = __ffma2_rn(make_float2(2.0f, 2.0f), ip, make_float2(qb.z, qb.w));
  // t in scalar operations: a packed multiply feeding a packed add can come
  // out fused into one rounding.
  const float2 t = make_float2(__fadd_rn(__fmul_rn(qa.z, a.x), __fmul_rn(qa.x, b2.x)),
                               __fadd_rn(__fmul_rn(qa.w, a.y), __fmul_rn(qa.y, b2.y)));
  const float2 base = __fadd2_rn(make_float2(qb.x, qb.y), r2);
  return __ffma2_rn(make_float2(-2.0f, -2.0f), __fmul2_rn(f2, t), base);
}

__device__ __forceinline__ void named_bar_consumers() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
}

// Producer (the whole warp). Block b of G takes the static items b, b + G,
// b + 2G, ... (longest lists first): the warp reads 32 of them at once (one
// per lane: item, pair count, offsets) and keeps those whose list is probed,
// so unprobed lists cost no further load. Each kept item is cut into units
// of up to kMmaNmax of its list's pairs. For each unit, once a stage is free
// (its `empty` barrier), lane 0 writes the meta and issues the TMA copies --
// B tile, parameters, mask rows and bounds, and for the first unit of an
// item its codes and factors -- all completing on the stage's `full`
// barrier. No load of the producer depends on another.
__device__ void producer_loop(uint8_t* sm, uint32_t sbase, const int2* __restrict__ items,
                              int n_items, const int32_t* __restrict__ list_count,
                              const int32_t* __restrict__ maxlim, int64_t pair_stride, const int64_t* __restrict__ offsets,
                              const uint8_t* __restrict__ codes, const float2* __restrict__ fac,
                              const uint8_t* __restrict__ qdb, const float4* __restrict__ qpb,
                              const int64_t* __restrict__ qwrow, const float* __restrict__ qtau,
                              int64_t qstride, int32_t* err, uint64_t wait_ns, int withhold) {
  const int lane = threadIdx.x & 31;
  Meta* meta = reinterpret_cast<Meta*>(sm + kSmMeta);
  const int64_t G = gridDim.x;
  int i = 0;                       // units issued
  int last_copy[2] = {-1, -1};     // last unit whose copies went into each stage
  bool ok = true;
  auto claim = [&](int it) -> bool {
    if (it < 2) return true;
    int r = 1;
    if (lane == 0)
      r = mbar_wait_bounded(sbase + kSmBar + 16 + 8 * (it & 1), (uint32_t)(((it >> 1) - 1) & 1),
                            wait_ns)
              ? 1
              : 0;
    return __shfl_sync(0xffffffffu, r, 0) != 0;
  };
  for (int64_t base = blockIdx.x; ok && base < n_items; base += 32 * G) {
    const int64_t idx = base + lane * G;
    int l = 0, cnt = 0, nvec = 0, v0 = 0;
    long long lo = 0;
    if (idx < n_items) {
      const int2 w = items[idx];
      l = w.x;
      v0 = w.y;
      cnt = list_count[l];
      // window pass: past every pair's window end the item has no work
      if (maxlim && v0 >= maxlim[l]) cnt = 0;
      if (cnt > 0) {
        lo = offsets[l] + v0;
        nvec = (int)min((long long)kItemV, (long long)offsets[l + 1] - lo);
      }
    }
    uint32_t work = __ballot_sync(0xffffffffu, cnt > 0);
    while (ok && work) {
      const int j = __ffs(work) - 1;
      work &= work - 1;
      const int jl = __shfl_sync(0xffffffffu, l, j);
      const int jc = __shfl_sync(0xffffffffu, cnt, j);
      const int jn = __shfl_sync(0xffffffffu, nvec, j);
      const int jv0 = __shfl_sync(0xffffffffu, v0, j);
      const long long jlo = __shfl_sync(0xffffffffu, lo, j);
      for (int g0 = 0; g0 < jc; g0 += kMmaNmax) {
        if (!claim(i)) {
          ok = false;
          break;
        }
        const int st = i & 1;
        const uint32_t full = sbase + kSmBar + 8 * st;
        const int np = min(kMmaNmax, jc - g0);
        if (lane == 0) {
          meta[st].lo = jlo;
          meta[st].l = jl;
          meta[st].nvec = jn;
          meta[st].np = np;
          meta[st].v0 = jv0;
          meta[st].first = g0 == 0;
          if (!(withhold && i == 0)) {
            const int64_t b0 = (int64_t)jl * pair_stride + g0;  // first bucket slot
            const int64_t q0 = (int64_t)jl * qstride + g0;      // ... a multiple of 4 here
            const uint32_t b_bytes = (uint32_t)np * kMmaK;
            const uint32_t qp_bytes = (uint32_t)((np + 1) & ~1) * 16;
            const uint32_t wr_bytes = (uint32_t)((np + 1) & ~1) * 8;
            const uint32_t tau_bytes = (uint32_t)((np + 3) & ~3) * 4;
            const long long lo_al = jlo & ~1ll;
            const uint32_t fac_bytes = (uint32_t)((((jlo - lo_al) + jn) * 8 + 15) & ~15ll);
            const uint32_t code_bytes = (uint32_t)jn * 16;
            uint32_t bytes = b_bytes + qp_bytes + wr_bytes + tau_bytes;
            if (g0 == 0) bytes += code_bytes + fac_bytes;
            mbar_expect_tx_arrive(full, bytes);
            if (g0 == 0) {
              tma_load_1d(sbase + kSmCode + st * kItemV * 16, codes + jlo * 16, code_bytes, full);
              tma_load_1d(sbase + kSmFac + st * kFacBytes, fac + lo_al, fac_bytes, full);
            }
            tma_load_1d(sbase + kSmB + st * kMmaNmax * kMmaK, qdb + b0 * kMmaK, b_bytes, full);
            tma_load_1d(sbase + kSmQp + st * kMmaNmax * 16, qpb + b0, qp_bytes, full);
            tma_load_1d(sbase + kSmWr + st * kMmaNmax * 8, qwrow + q0, wr_bytes, full);
            tma_load_1d(sbase + kSmTau + st * kMmaNmax * 4, qtau + q0, tau_bytes, full);
            last_copy[st] = i;
          }
          // (test hook: with `withhold`, the first stage is never filled nor
          // signalled, so the consumers' bounded wait for it runs out)
        }
        __syncwarp();
        ++i;
      }
    }
  }
  if (ok && claim(i)) {
    if (lane == 0) {
      meta[i & 1].l = -1;
      mbar_expect_tx_arrive(sbase + kSmBar + 8 * (i & 1), 0);
    }
  } else {
    ok = false;
  }
  if (lane == 0 && !ok) {
    flag_error(err, kErrMmaTimeout);
    // After a wait ran out the consumers may have left: the copies still in
    // flight land before the block returns.
    for (int s = 0; s < 2; ++s)
      if (last_copy[s] >= 0)
        mbar_wait_bounded(sbase + kSmBar + 8 * s, (uint32_t)((last_copy[s] >> 1) & 1), wait_ns);
  }
  __syncwarp();
}

// Two forms. The scan (kWindow false): per pair its first mask index
// (qwrow) and bound (qtau); survivor mask words out. The first bound's
// window pass (kWindow true): per pair the index of its list's first
// estimate (qwrow) and the list's vectors in the window (qtau, int bits);
// the estimates of those vectors out, as orderable uint32, to `est`; items
// at or past `maxlim` of their list are skipped.
template <bool kWindow>
__global__ void __launch_bounds__(kMmaThreads, 3)
scan_mma_kernel(const int2* __restrict__ items, int n_items,
                const int32_t* __restrict__ list_count, const int32_t* __restrict__ maxlim,
                int64_t pair_stride,
                const float4* __restrict__ qpb, const uint8_t* __restrict__ qdb,
                const int64_t* __restrict__ qwrow, const float* __restrict__ qtau,
                int64_t qstride, const int64_t* __restrict__ offsets,
                const uint8_t* __restrict__ codes, const float2* __restrict__ fac,
                uint32_t* __restrict__ mask, uint32_t* __restrict__ est, int32_t* err,
                uint64_t wait_ns, int withhold) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ volatile int s_ok[4];  // results of the polled waits
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sbase = smem_u32(sm);
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(sm + kSmTmem);
  const Meta* meta = reinterpret_cast<const Meta*>(sm + kSmMeta);
  const uint32_t bar_mma = sbase + kSmBar + 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int b = 0; b < 6; ++b) mbar_init(sbase + kSmBar + 8 * b, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(sbase + kSmTmem, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_tmem;

  if (warp == kConsumers / 32) {
    producer_loop(sm, sbase, items, n_items, list_count, maxlim, pair_stride, offsets, codes, fac,
                  qdb, qpb, qwrow, qtau, qstride, err, wait_ns, withhold);
  } else {
    uint32_t ph_mma = 0;
    bool abort = false, mma_pending = false;
    // this thread's vector of the current block: popcount and factors,
    // kept from the block's first unit for its later ones
    float2 f = make_float2(0.0f, 0.0f);
    int pc = 0;
    for (int i = 0;; ++i) {
      const int st = i & 1;
      const uint32_t full = sbase + kSmBar + 8 * st;
      const uint32_t empty = sbase + kSmBar + 16 + 8 * st;
      // One thread polls each mbarrier; the others wait at the named
      // barrier, which orders the observed data for them, without issuing.
      if (tid == 0) s_ok[0] = mbar_wait_bounded(full, (uint32_t)((i >> 1) & 1), wait_ns) ? 1 : 0;
      named_bar_consumers();
      if (!s_ok[0]) abort = true;
      const Meta m = meta[st];
      if (abort || m.l < 0) break;
      const float4* qp_s = reinterpret_cast<const float4*>(sm + kSmQp + st * kMmaNmax * 16);
      const int64_t* wr_s = reinterpret_cast<const int64_t*>(sm + kSmWr + st * kMmaNmax * 8);
      const float2* tau2 = reinterpret_cast<const float2*>(sm + kSmTau + st * kMmaNmax * 4);
      const uint64_t bdesc = sdesc_sw128(sbase + kSmB + st * kMmaNmax * kMmaK);
      const int np = m.np;
      const int n = max(16, (np + 15) & ~15);
      if (m.first) {
        // A tiles: thread t expands vector t of the block (tile t / 128, row
        // t % 128); they serve every unit of the block.
        const uint8_t* code_s = sm + kSmCode + st * kItemV * 16;
        const float2* fac_s =
            reinterpret_cast<const float2*>(sm + kSmFac + st * kFacBytes) + (m.lo & 1);
        const int tile = tid >> 7, r = tid & (kMmaM - 1);
        uint4 cw = make_uint4(0, 0, 0, 0);
        f = make_float2(0.0f, 0.0f);
        if (tid < m.nvec) {
          cw = *reinterpret_cast<const uint4*>(code_s + tid * 16);
          f = fac_s[tid];
        }
        pc = __popc(cw.x) + __popc(cw.y) + __popc(cw.z) + __popc(cw.w);
        const uint32_t wd[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t w16 = wd[c >> 1] >> ((c & 1) * 16);
          const uint4 val = make_uint4(nibble_to_e4m3(w16 & 15u), nibble_to_e4m3((w16 >> 4) & 15u),
                                       nibble_to_e4m3((w16 >> 8) & 15u),
                                       nibble_to_e4m3((w16 >> 12) & 15u));
          *reinterpret_cast<uint4*>(sm + kSmA + tile * kMmaM * kMmaK + sw128_offset(r, c)) = val;
        }
      }
      fence_async_smem();
      tc_fence_before();
      named_bar_consumers();
      tc_fence_after();
      const int ntiles = (m.nvec + kMmaM - 1) / kMmaM;
      if (tid == 0) {
        const uint32_t id = idesc_e4m3_f32(kMmaM, (uint32_t)n);
        for (int tile = 0; tile < ntiles; ++tile) {
          const uint64_t ad = sdesc_sw128(sbase + kSmA + tile * kMmaM * kMmaK);
#pragma unroll
          for (int k = 0; k < kMmaK / 32; ++k)
            mma_e4m3(taddr + (uint32_t)(tile * kMmaNmax), ad + (uint64_t)(2 * k),
                     bdesc + (uint64_t)(2 * k), id, k > 0);
        }
        mma_commit(bar_mma);
      }
      if (tid == 0) s_ok[1] = mbar_wait_bounded(bar_mma, ph_mma, wait_ns) ? 1 : 0;
      named_bar_consumers();
      if (!s_ok[1]) {
        abort = true;
        mma_pending = true;
        break;
      }
      ph_mma ^= 1u;
      tc_fence_after();
      // Epilogue: thread t = vector t = TMEM lane 32 (w % 4) + lane of
      // tile w / 4; 8 pairs per TMEM load, two at a time in packed float2
      // operations (estimate2). Pairs past np are computed on stale
      // parameters and masked off.
      {
        const int quarter = warp & 3, tile = warp >> 2;
        if (tile < ntiles) {
          const bool valid = tid < m.nvec;
          const float bterm = (float)(2 * pc - kMmaK);
          const float2 b2 = make_float2(bterm, bterm);
          const float2 r2 = make_float2(f.x, f.x);
          const float2 f2 = make_float2(f.y, f.y);
          const uint32_t tl = taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tile * kMmaNmax);
          if constexpr (kWindow) {
            // each pair's estimates of this block's vectors inside its
            // window, at its first estimate index + the vector's position
            const int64_t* dest_s = wr_s;
            const int* lim_s = reinterpret_cast<const int*>(sm + kSmTau + st * kMmaNmax * 4);
            const int v = m.v0 + tid;  // position in the list
            for (int c1 = 0; c1 < np; c1 += 8) {
              uint32_t r[8];
              tmem_ld8(tl + (uint32_t)c1, r);
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const int g = c1 + 2 * h;
                const float2 dd = estimate2(qp_s[g], qp_s[g + 1], r[2 * h], r[2 * h + 1], b2, r2, f2);
                if (valid && g < np && v < lim_s[g]) est[dest_s[g] + v] = orderable(dd.x);
                if (valid && g + 1 < np && v < lim_s[g + 1])
                  est[dest_s[g + 1] + v] = orderable(dd.y);
              }
            }
          } else {
            const float2 mone = make_float2(-1.0f, -1.0f);
            const int64_t word = m.v0 / 32 + warp;
            for (int c1 = 0; c1 < np; c1 += 8) {
              uint32_t r[8];
              tmem_ld8(tl + (uint32_t)c1, r);
              uint32_t sgn[8];  // sign words of tau - d: clear exactly when d <= tau
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const int g = c1 + 2 * h;
                const float2 dd = estimate2(qp_s[g], qp_s[g + 1], r[2 * h], r[2 * h + 1], b2, r2, f2);
                // tau - d rounded once is >= +0 exactly when d <= tau (neither
                // is -0 or NaN; a nonzero difference of floats never rounds to
                // zero; +inf - d = +inf)
                const float2 df = __ffma2_rn(mone, dd, tau2[g >> 1]);
                sgn[2 * h] = __float_as_uint(df.x);
                sgn[2 * h + 1] = __float_as_uint(df.y);
              }
              // the eight sign bits, packed: top bytes gathered by byte
              // permutes, then bits 7, 15, 23, 31 moved to 28..31 by one
              // multiply (its partial products do not overlap)
              const uint32_t b03 = __byte_perm(__byte_perm(sgn[0], sgn[1], 0x0073),
                                               __byte_perm(sgn[2], sgn[3], 0x0073), 0x5410);
              const uint32_t b47 = __byte_perm(__byte_perm(sgn[4], sgn[5], 0x0073),
                                               __byte_perm(sgn[6], sgn[7], 0x0073), 0x5410);
              const uint32_t fail = (((b03 & 0x80808080u) * 0x00204081u) >> 28) |
                                    ((((b47 & 0x80808080u) * 0x00204081u) >> 28) << 4);
              const int left = np - c1;
              const uint32_t passbits =
                  ~fail & (valid ? (left >= 8 ? 0xFFu : (1u << left) - 1u) : 0u);
              uint32_t mine = 0;
              if (__any_sync(0xffffffffu, passbits != 0)) {  // else every word is 0
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const uint32_t mj = __ballot_sync(0xffffffffu, (passbits >> j) & 1u);
                  if (lane == j) mine = mj;
                }
              }
              // lane j writes pair c1 + j's mask word (none past the block's end)
              if (warp * 32 < m.nvec && lane < 8 && lane < left) mask[wr_s[c1 + lane] + word] = mine;
            }
          }
        }
      }
      // Every consumer has read this stage's meta and finished with its
      // buffers (and TMEM) before it is handed back to the producer.
      tc_fence_before();
      named_bar_consumers();
      if (tid == 0) mbar_expect_tx_arrive(empty, 0);
    }
    if (abort && tid == 0) flag_error(err, kErrMmaTimeout);
    if (mma_pending) {
      // The MMA whose wait ran out may still be in flight: give it a
      // bounded time to land before the TMEM is freed.
      mbar_wait_bounded(bar_mma, ph_mma, wait_ns);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(taddr, kTmemCols);
}

}  // namespace

bool mma_supported(const rq_index* ix) { return ix->dp == kMmaK; }

rq_status launch_scan_mma(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                          int sms, int withhold, bool window) {
  if (ix->dp != kMmaK) return fail(RQ_ERR_NOT_IMPLEMENTED, "tensor-core scan built for D_p = 128");
  const auto kern = window ? scan_mma_kernel<true> : scan_mma_kernel<false>;
  RQ_TRY(allow_dynamic_smem((const void*)kern, kSmAlloc));
  // Three blocks per SM (registers; ~69 KB of shared memory each); their
  // TMEM (128 columns each) stays within the SM's 512 columns.
  const unsigned grid = (unsigned)std::max(1, std::min(sms * 3, ix->n_items));
  const int64_t qstride = (sh.nq + 3) & ~int64_t(3);
  if (window) {
    kern<<<grid, kMmaThreads, kSmAlloc, st>>>(
        ix->items, ix->n_items, ws.wcount, ws.wcount + ix->nlist, sh.nq, ws.wqpb, ws.wqdig,
        ws.wdest, reinterpret_cast<const float*>(ws.wlim), qstride, ix->offsets, ix->codes,
        ix->fac, nullptr, reinterpret_cast<uint32_t*>(ws.keys), ix->d_err, kWaitLimitNs, 0);
  } else {
    kern<<<grid, kMmaThreads, kSmAlloc, st>>>(
        ix->items, ix->n_items, ws.list_count, nullptr, sh.nq, ws.qpb, ws.qdig, ws.qwrow,
        ws.qtau, qstride, ix->offsets, ix->codes, ix->fac, ws.mask, nullptr, ix->d_err,
        withhold ? kTestWaitLimitNs : kWaitLimitNs, withhold);
  }
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

}  // namespace rq
