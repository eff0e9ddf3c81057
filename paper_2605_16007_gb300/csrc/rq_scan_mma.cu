// Tensor-core form of the grouped code scan (Eqs. 4-5 with a 4-bit query,
// Section 3.3.2), for D_p = 128.
//
// The integer inner product ip = sum_d bit_d * q_u,d of a 128-vector tile
// with a group of up to 64 quantised (query, list) residuals is one
// [128 x 128] x [128 x N] product. Both operands are held exactly in FP8 E4M3
// (a code bit is 0 or 1.0, a query digit an integer 0..15), and the FP32
// accumulation of at most 128 products of integers <= 15 is exact, so ip is
// the same integer the popcount form computes. The tile is issued as four
// tcgen05.mma (K = 32 bytes each) by one thread, accumulated in tensor
// memory, and read back with tcgen05.ld by the four warps of the block, one
// TMEM lane (= one vector) per thread, for the float32 estimator epilogue.
#include <cuda_runtime.h>

#include "rq_common.cuh"
#include "rq_scan.cuh"

namespace rq {
namespace {

constexpr int kMmaM = 128;        // vectors per tile (TMEM lanes)
constexpr int kMmaNmax = 64;      // pairs per MMA group (TMEM columns)
constexpr int kMmaK = 128;        // D_p
constexpr int kMmaThreads = 128;  // four warps: one TMEM lane quarter each
constexpr uint64_t kWaitNs = 2000000000ull;  // an mbarrier wait gives up after 2 s

// Shared memory of one block (offsets from a 1024-byte aligned base).
constexpr int kSmA = 0;                             // 128 rows x 128 B, 128B swizzle
constexpr int kSmB = kSmA + kMmaM * kMmaK;          // 64 rows x 128 B, 128B swizzle
constexpr int kSmLut = kSmB + kMmaNmax * kMmaK;     // 256 x uint64: byte -> 8 FP8
constexpr int kSmQp = kSmLut + 256 * 8;             // 64 x float4
constexpr int kSmTau = kSmQp + kMmaNmax * 16;       // 64 x uint32
constexpr int kSmQid = kSmTau + kMmaNmax * 4;       // 64 x int32
constexpr int kSmBar = kSmQid + kMmaNmax * 4;       // mbarrier (8 B)
constexpr int kSmTmem = kSmBar + 8;                 // TMEM base address (4 B)
constexpr int kSmItem = kSmTmem + 4;                // item index (4 B)
constexpr int kSmFlag = kSmItem + 4;                // abort flag (4 B)
constexpr int kSmBytes = kSmFlag + 4;
constexpr int kSmAlloc = kSmBytes + 1024;           // room to align the base

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
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

// Waits for the phase with the given parity; false after kWaitNs (the
// caller then reports RQ_ERR_DEVICE through the error word).
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of 16-byte chunk c of row r in a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_offset(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

__global__ void __launch_bounds__(kMmaThreads)
scan_mma_kernel(const int2* __restrict__ items, int n_items, int32_t* __restrict__ work_counter,
                const int32_t* __restrict__ list_count, const int32_t* __restrict__ list_pairs,
                int64_t pair_stride, const float4* __restrict__ qparams,
                const uint8_t* __restrict__ qdig, int npmax, const int64_t* __restrict__ offsets,
                const uint8_t* __restrict__ codes, const float2* __restrict__ fac,
                const uint32_t* __restrict__ ids, const uint32_t* __restrict__ bound,
                int32_t* __restrict__ counts, uint64_t* __restrict__ cand, int64_t cap,
                int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  const uint32_t sbase = smem_u32(sm);
  uint64_t* lut = reinterpret_cast<uint64_t*>(sm + kSmLut);
  float4* s_qp = reinterpret_cast<float4*>(sm + kSmQp);
  uint32_t* s_tau = reinterpret_cast<uint32_t*>(sm + kSmTau);
  int32_t* s_qid = reinterpret_cast<int32_t*>(sm + kSmQid);
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(sm + kSmTmem);
  volatile int* s_item = reinterpret_cast<volatile int*>(sm + kSmItem);
  const uint32_t bar = sbase + kSmBar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 256; i += kMmaThreads) {
    uint64_t v = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if ((i >> b) & 1) v |= (uint64_t)0x38 << (8 * b);
    lut[i] = v;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(sbase + kSmTmem, kMmaNmax);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_tmem;
  const uint64_t adesc = sdesc_sw128(sbase + kSmA);
  const uint64_t bdesc = sdesc_sw128(sbase + kSmB);
  uint32_t phase = 0;
  bool abort = false;

  for (;;) {
    if (tid == 0) *s_item = atomicAdd(work_counter, 1);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    if (it >= n_items) break;
    const int2 w = items[it];
    const int l = w.x;
    const int cnt = list_count[l];
    if (cnt == 0) continue;
    const int64_t list_end = offsets[l + 1];
    const int64_t item_end = min(list_end, offsets[l] + w.y + kGroupVectors);
    const int32_t* lp = list_pairs + (int64_t)l * pair_stride;
    for (int64_t lo = offsets[l] + w.y; lo < item_end && !abort; lo += kMmaM) {
      // A tile: this thread's vector, expanded to FP8 in the swizzled layout.
      const int64_t s = lo + tid;
      const bool valid = s < item_end;
      uint4 code = make_uint4(0, 0, 0, 0);
      float2 f = make_float2(0.0f, 0.0f);
      if (valid) {
        code = __ldg(reinterpret_cast<const uint4*>(codes + s * 16));
        f = fac[s];
      }
      const int pc = __popc(code.x) + __popc(code.y) + __popc(code.z) + __popc(code.w);
      const float bterm = (float)(2 * pc - kMmaK);
      {
        const uint32_t wds[4] = {code.x, code.y, code.z, code.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t wd = wds[c >> 1];
          const int sh = (c & 1) * 16;
          const uint64_t lo8 = lut[(wd >> sh) & 255u];
          const uint64_t hi8 = lut[(wd >> (sh + 8)) & 255u];
          uint4 v = make_uint4((uint32_t)lo8, (uint32_t)(lo8 >> 32), (uint32_t)hi8,
                               (uint32_t)(hi8 >> 32));
          *reinterpret_cast<uint4*>(sm + kSmA + sw128_offset(tid, c)) = v;
        }
      }
      for (int g0 = 0; g0 < cnt && !abort; g0 += kMmaNmax) {
        const int np = min(kMmaNmax, cnt - g0);
        const int n = max(16, (np + 15) & ~15);
        // B tile: the group's query digits (rows past np are zero).
        for (int i = tid; i < n * 8; i += kMmaThreads) {
          const int g = i >> 3, c = i & 7;
          uint4 v = make_uint4(0, 0, 0, 0);
          if (g < np) v = __ldg(reinterpret_cast<const uint4*>(qdig + (int64_t)lp[g0 + g] * kMmaK) + c);
          *reinterpret_cast<uint4*>(sm + kSmB + sw128_offset(g, c)) = v;
        }
        for (int g = tid; g < np; g += kMmaThreads) {
          const int pair = lp[g0 + g];
          const int q = pair / npmax;
          s_qp[g] = qparams[pair];
          s_tau[g] = bound[q];
          s_qid[g] = q;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
          const uint32_t id = idesc_e4m3_f32(kMmaM, (uint32_t)n);
#pragma unroll
          for (int k = 0; k < kMmaK / 32; ++k)
            mma_e4m3(taddr, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), id, k > 0);
          mma_commit(bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        abort = __syncthreads_or(!ok) != 0;
        tc_fence_after();
        if (abort) break;
        // Epilogue: thread = TMEM lane = vector; 32 pairs per TMEM load.
        for (int c0 = 0; c0 < np; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int g = c0 + j;
            if (g >= np) break;
            const float4 qp = s_qp[g];
            const float ip = __uint_as_float(r[j]);
            const float a = __fsub_rn(__fmul_rn(2.0f, ip), (float)__float_as_int(qp.w));
            const float t = __fadd_rn(__fmul_rn(qp.y, a), __fmul_rn(qp.x, bterm));
            float d = __fsub_rn(__fadd_rn(qp.z, f.x), __fmul_rn(2.0f, __fmul_rn(f.y, t)));
            d = __fadd_rn(d, 0.0f);
            const bool pass = valid && orderable(d) <= s_tau[g];
            const int q = s_qid[g];
            append_candidates(pass, d, s, ids, counts + q, cand + (int64_t)q * cap, cap, lane, err);
          }
        }
        tc_fence_before();
        __syncthreads();
      }
    }
    if (abort) break;
  }
  if (abort) {
    if (tid == 0) flag_error(err, kErrMmaTimeout);
    // An MMA may still be in flight: give it a bounded time to land.
    mbar_wait_bounded(bar, phase);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(taddr, kMmaNmax);
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
  // At most seven blocks fit an SM by shared memory (~31 KB each), so their
  // TMEM (64 columns each) never exceeds the SM's 512 columns.
  scan_mma_kernel<<<(unsigned)(sms * 6), kMmaThreads, kSmAlloc, st>>>(
      ix->items, ix->n_items, ws.work_count, ws.list_count, ws.list_pairs, sh.nq, ws.qparams,
      ws.qdig, sh.npmax, ix->offsets, ix->codes, ix->fac, ix->ids, ws.bound, ws.counts, ws.cand,
      ws.cap, ix->d_err);
  RQ_CUDA(cudaGetLastError());
  return RQ_OK;
}

}  // namespace rq
