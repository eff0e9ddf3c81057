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
// Pipeline of one block (persistent over work items = 256-vector blocks of a
// list): TMA bulk copies bring the item's packed codes, {r^2, f} factors,
// the B tile (the group's query digits, pre-swizzled in their per-list
// bucket) and the group's parameters into one of two shared-memory stages,
// completing on that stage's mbarrier, while the block works on the other
// stage. Thread t expands the codes of vector t of the item to an FP8 row of
// the A tile of its 128-vector half (128B swizzle); one thread issues four
// tcgen05.mma (K = 32 bytes each) per tile into that tile's TMEM accumulator
// (columns [64 tile, 64 tile + 64)); thread t then reads its own row back
// with tcgen05.ld (warp w: TMEM lanes 32 (w % 4) .. of tile w / 4) for the
// float32 estimator epilogue, so all eight warps share the epilogue.
#include <cuda_runtime.h>

#include "rq_common.cuh"
#include "rq_scan.cuh"

namespace rq {
namespace {

constexpr int kMmaM = 128;        // vectors per tile (TMEM lanes)
constexpr int kMmaNmax = 64;      // pairs per MMA group (TMEM columns)
constexpr int kMmaK = 128;        // D_p
constexpr int kItemV = kGroupVectors;  // 256 vectors per work item = 2 tiles
constexpr int kMmaThreads = 256;  // eight warps
constexpr uint64_t kWaitNs = 2000000000ull;  // an mbarrier wait gives up after 2 s
constexpr int kTmemCols = 2 * kMmaNmax;    // one accumulator per tile of the item

// Shared memory of one block (offsets from a 1024-byte aligned base).
constexpr int kSmA = 0;                                  // 2 tiles x 128 x 128 B (128B swizzle)
constexpr int kSmB = kSmA + 2 * kMmaM * kMmaK;           // 2 stages x 64 x 128 B
constexpr int kSmCode = kSmB + 2 * kMmaNmax * kMmaK;     // 2 stages x 256 x 16 B
constexpr int kFacBytes = (kItemV + 2) * 8;              // +1 for alignment, rounded
constexpr int kSmFac = kSmCode + 2 * kItemV * 16;        // 2 stages x 258 x 8 B
constexpr int kSmQp = kSmFac + 2 * kFacBytes;            // 2 stages x 64 x 16 B
constexpr int kSmTau = kSmQp + 2 * kMmaNmax * 16;        // 64 x uint32
constexpr int kSmQid = kSmTau + kMmaNmax * 4;            // 64 x int32
constexpr int kSmBar = kSmQid + kMmaNmax * 4;            // 3 mbarriers: load[2], mma
constexpr int kSmMeta = kSmBar + 3 * 8;                  // 2 stages x int4 meta
constexpr int kSmTmem = kSmMeta + 2 * 16;                // TMEM base address
constexpr int kSmNext = kSmTmem + 4;                     // next item index
constexpr int kSmBytes = kSmNext + 4;
constexpr int kSmAlloc = kSmBytes + 1024;                // room to align the base

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_arrive(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase with the given parity; false after kWaitNs (the block
// then stops and reports through the error word).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15u) == 15u && globaltimer_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// TMA bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completing on an mbarrier's transaction count.
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// Shared-memory matrix descriptor: K-major rows of 128 bytes with the 128B
// swizzle, 8-row groups 1024 bytes apart (start address and strides in units
// of 16 bytes, descriptor version 1 at bit 46, layout type 2 = 128B swizzle).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor of kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B =
// E4M3 (0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t idesc_e4m3_f32(uint32_t m, uint32_t n) {
  return (1u << 4) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of 16-byte chunk c of row r in a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_offset(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}
// Four code bits (a nibble) -> four FP8 bytes 0x38 (1.0) or 0x00: the
// multiply places bit i at bit 8i without carries (bit i + 7j lands on a
// multiple of 8 only for j = i).
__device__ __forceinline__ uint32_t nibble_to_e4m3(uint32_t n) {
  return ((n * 0x00204081u) & 0x01010101u) * 0x38u;
}

// Work item meta of one stage: {list, first slot, vectors, pairs}.
struct Meta {
  int l, lo, nvec, cnt;
};

// Thread 0: read item `it`, record its meta, and start the TMA copies of
// its codes, factors, first B tile and parameters into `stage`.
__device__ __forceinline__ void issue_item(int it, int stage, uint8_t* sm, uint32_t sbase,
                                           const int2* items, const int32_t* list_count,
                                           const int64_t* offsets, const uint8_t* codes,
                                           const float2* fac, const uint8_t* qdb,
                                           const float4* qpb, int64_t pair_stride) {
  const int2 w = items[it];
  const int l = w.x;
  const int cnt = list_count[l];
  const int64_t lo = offsets[l] + w.y;
  const int nvec = (int)min((int64_t)kItemV, offsets[l + 1] - lo);
  Meta* meta = reinterpret_cast<Meta*>(sm + kSmMeta) + stage;
  meta->l = l;
  meta->lo = (int)lo;
  meta->nvec = nvec;
  meta->cnt = cnt;
  const uint32_t bar = sbase + kSmBar + 8 * stage;
  if (cnt == 0) {
    mbar_expect_tx_arrive(bar, 0);
    return;
  }
  const int np = min(kMmaNmax, cnt);
  const int64_t lo_al = lo & ~(int64_t)1;
  const uint32_t fac_bytes = (uint32_t)((((lo - lo_al) + nvec) * 8 + 15) & ~15);
  const uint32_t code_bytes = (uint32_t)nvec * 16;
  const uint32_t b_bytes = (uint32_t)np * kMmaK;
  const uint32_t qp_bytes = (uint32_t)np * 16;
  mbar_expect_tx_arrive(bar, code_bytes + fac_bytes + b_bytes + qp_bytes);
  tma_load_1d(sbase + kSmCode + stage * kItemV * 16, codes + lo * 16, code_bytes, bar);
  tma_load_1d(sbase + kSmFac + stage * kFacBytes, fac + lo_al, fac_bytes, bar);
  tma_load_1d(sbase + kSmB + stage * kMmaNmax * kMmaK, qdb + (int64_t)l * pair_stride * kMmaK,
              b_bytes, bar);
  tma_load_1d(sbase + kSmQp + stage * kMmaNmax * 16, qpb + (int64_t)l * pair_stride, qp_bytes,
              bar);
}

__global__ void __launch_bounds__(kMmaThreads, 3)
scan_mma_kernel(const int2* __restrict__ items, int n_items, int32_t* __restrict__ work_counter,
                const int32_t* __restrict__ list_count, const int32_t* __restrict__ list_pairs,
                int64_t pair_stride, const float4* __restrict__ qpb,
                const uint8_t* __restrict__ qdb, int npmax, const int64_t* __restrict__ offsets,
                const uint8_t* __restrict__ codes, const float2* __restrict__ fac,
                const uint32_t* __restrict__ ids, const uint32_t* __restrict__ bound,
                int32_t* __restrict__ counts, uint64_t* __restrict__ cand, int64_t cap,
                int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sbase = smem_u32(sm);
  uint32_t* s_tau = reinterpret_cast<uint32_t*>(sm + kSmTau);
  int32_t* s_qid = reinterpret_cast<int32_t*>(sm + kSmQid);
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(sm + kSmTmem);
  volatile int* s_next = reinterpret_cast<volatile int*>(sm + kSmNext);
  const Meta* meta = reinterpret_cast<const Meta*>(sm + kSmMeta);
  const uint32_t bar_mma = sbase + kSmBar + 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(sbase + kSmBar, 1);
    mbar_init(sbase + kSmBar + 8, 1);
    mbar_init(bar_mma, 1);
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
  const uint64_t adesc = sdesc_sw128(sbase + kSmA);
  uint32_t ph_load[2] = {0u, 0u};
  uint32_t ph_mma = 0;
  bool abort = false;

  if (tid == 0) {
    const int it = atomicAdd(work_counter, 1);
    *s_next = it;
    if (it < n_items)
      issue_item(it, 0, sm, sbase, items, list_count, offsets, codes, fac, qdb, qpb, pair_stride);
  }
  __syncthreads();
  int cur = *s_next;
  int st = 0;
  while (cur < n_items && !abort) {
    __syncthreads();  // everyone has read s_next before it is overwritten
    if (tid == 0) {
      const int nx = atomicAdd(work_counter, 1);
      *s_next = nx;
      if (nx < n_items)
        issue_item(nx, st ^ 1, sm, sbase, items, list_count, offsets, codes, fac, qdb, qpb,
                   pair_stride);
    }
    const bool ok = mbar_wait_bounded(sbase + kSmBar + 8 * st, ph_load[st]);
    ph_load[st] ^= 1u;
    if (__syncthreads_or(!ok)) {
      abort = true;
      break;
    }
    const Meta m = meta[st];
    if (m.cnt > 0) {
      const uint8_t* code_s = sm + kSmCode + st * kItemV * 16;
      const float2* fac_s = reinterpret_cast<const float2*>(sm + kSmFac + st * kFacBytes) +
                            (m.lo & 1);
      const float4* qp_s = reinterpret_cast<const float4*>(sm + kSmQp + st * kMmaNmax * 16);
      const int32_t* lp = list_pairs + (int64_t)m.l * pair_stride;
      const uint64_t bdesc = sdesc_sw128(sbase + kSmB + st * kMmaNmax * kMmaK);
      for (int g0 = 0; g0 < m.cnt && !abort; g0 += kMmaNmax) {
        const int np = min(kMmaNmax, m.cnt - g0);
        const int n = max(16, (np + 15) & ~15);
        if (g0 > 0) {
          // Later groups of a list probed by more than kMmaNmax queries:
          // the B tile and parameters are reloaded in this stage.
          if (tid == 0) {
            const uint32_t bar = sbase + kSmBar + 8 * st;
            mbar_expect_tx_arrive(bar, (uint32_t)np * (kMmaK + 16));
            tma_load_1d(sbase + kSmB + st * kMmaNmax * kMmaK,
                        qdb + ((int64_t)m.l * pair_stride + g0) * kMmaK, (uint32_t)np * kMmaK,
                        bar);
            tma_load_1d(sbase + kSmQp + st * kMmaNmax * 16, qpb + (int64_t)m.l * pair_stride + g0,
                        (uint32_t)np * 16, bar);
          }
          const bool ok2 = mbar_wait_bounded(sbase + kSmBar + 8 * st, ph_load[st]);
          ph_load[st] ^= 1u;
          if (__syncthreads_or(!ok2)) {
            abort = true;
            break;
          }
        }
        for (int g = tid; g < np; g += kMmaThreads) {
          const int q = lp[g0 + g] / npmax;
          s_tau[g] = bound[q];
          s_qid[g] = q;
        }
        // A tiles: thread t expands vector t of the item (tile t / 128, row
        // t % 128); they are unchanged across the groups of the item.
        if (g0 == 0) {
          const int tile = tid >> 7, r = tid & (kMmaM - 1);
          uint4 cw = make_uint4(0, 0, 0, 0);
          if (tid < m.nvec) cw = *reinterpret_cast<const uint4*>(code_s + tid * 16);
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
        __syncthreads();
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
        const bool ok3 = mbar_wait_bounded(bar_mma, ph_mma);
        ph_mma ^= 1u;
        if (__syncthreads_or(!ok3)) {
          abort = true;
          break;
        }
        tc_fence_after();
        // Epilogue: thread t = vector t = TMEM lane 32 (w % 4) + lane of
        // tile w / 4; 16 pairs per TMEM load.
        {
          const int quarter = warp & 3, tile = warp >> 2;
          if (tile < ntiles) {
            const int v = tid;
            const bool valid = v < m.nvec;
            const int64_t s = (int64_t)m.lo + v;
            float2 f = make_float2(0.0f, 0.0f);
            int pc = 0;
            if (valid) {
              f = fac_s[v];
              const uint4 cw = *reinterpret_cast<const uint4*>(code_s + v * 16);
              pc = __popc(cw.x) + __popc(cw.y) + __popc(cw.z) + __popc(cw.w);
            }
            const float bterm = (float)(2 * pc - kMmaK);
            for (int c1 = 0; c1 < np; c1 += 16) {
              uint32_t r[16];
              tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) +
                            (uint32_t)(tile * kMmaNmax + c1), r);
              float d[16];
              uint32_t passbits = 0;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int g = c1 + j;
                d[j] = 0.0f;
                if (g < np) {
                  const float4 qp = qp_s[g];
                  const float ip = __uint_as_float(r[j]);
                  const float a = __fsub_rn(__fmul_rn(2.0f, ip), (float)__float_as_int(qp.w));
                  const float t = __fadd_rn(__fmul_rn(qp.y, a), __fmul_rn(qp.x, bterm));
                  float dd = __fsub_rn(__fadd_rn(qp.z, f.x), __fmul_rn(2.0f, __fmul_rn(f.y, t)));
                  dd = __fadd_rn(dd, 0.0f);
                  d[j] = dd;
                  if (valid && orderable(dd) <= s_tau[g]) passbits |= 1u << j;
                }
              }
              append_chunk<16>(passbits, d, s_qid + c1, s, ids, counts, cand, cap, lane, err);
            }
          }
        }
        tc_fence_before();
        __syncthreads();
      }
    }
    __syncthreads();
    cur = *s_next;
    st ^= 1;
  }
  if (abort) {
    if (tid == 0) flag_error(err, kErrMmaTimeout);
    // Copies or an MMA may still be in flight: give them a bounded time.
    mbar_wait_bounded(bar_mma, ph_mma);
    mbar_wait_bounded(sbase + kSmBar, ph_load[0]);
    mbar_wait_bounded(sbase + kSmBar + 8, ph_load[1]);
  } else if (cur >= n_items) {
    // The last issued prefetch (of an index past the end) loaded nothing.
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(taddr, kTmemCols);
}

}  // namespace

bool mma_supported(const rq_index* ix) { return ix->dp == kMmaK; }

rq_status launch_scan_mma(rq_index* ix, const SearchShape& sh, Workspace& ws, cudaStream_t st,
                          int sms) {
  if (ix->dp != kMmaK) return fail(RQ_ERR_NOT_IMPLEMENTED, "tensor-core scan built for D_p = 128");
  static bool attr_set = false;
  if (!attr_set) {
    RQ_CUDA(cudaFuncSetAttribute(scan_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmAlloc));
    attr_set = true;
  }
  // Three blocks per SM (registers; ~69 KB of shared memory each); their
  // TMEM (128 columns each) stays within the SM's 512 columns.
  scan_mma_kernel<<<(unsigned)(sms * 3), kMmaThreads, kSmAlloc, st>>>(
      ix->items, ix->n_items, ws.work_count, ws.list_count, ws.list_pairs, sh.nq, ws.qpb, ws.qdig,
      sh.npmax, ix->offsets, ix->codes, ix->fac, ix->ids, ws.bound, ws.counts, ws.cand, ws.cap,
      ix->d_err);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

}  // namespace rq
