// Device helpers shared by the librq kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rq {

constexpr uint64_t kU64Max = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t kU32Max = 0xFFFFFFFFu;

// Device error codes written to the index error word.
enum DeviceError : int32_t {
  kErrNone = 0,
  kErrCandidateOverflow = 1,
  kErrBadProbe = 2,
  kErrSelectOverflow = 3,
  kErrMmaTimeout = 4,     // a bounded wait of the tensor-core scan ran out
  kErrScanTimeout = 5,    // a bounded wait of the streaming scan ran out
  kErrBadIndex = 6,       // (checked builds) an index fell outside its buffer
};


__device__ __forceinline__ void flag_error(int32_t* err, int32_t code) {
  if (err) atomicCAS(err, 0, code);
}

// Checked builds (-DRQ_CHECKS=1) test the indexes of the scan output and of
// the candidate slots against their buffers; a bad one sets kErrBadIndex in
// the error word and the access is skipped. Normal builds compile the checks
// away.
#ifndef RQ_CHECKS
#define RQ_CHECKS 0
#endif
__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int32_t* err) {
  if (!RQ_CHECKS) return true;
  if (i >= 0 && i < n) return true;
  flag_error(err, kErrBadIndex);
  return false;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies
// with a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t stream,
                                              uint64_t index) {
  return philox4x32_10(
      make_uint4((uint32_t)index, (uint32_t)(index >> 32), stream, 0u),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ---------------------------------------------------------------------------
// Order-preserving float -> uint32 map and (distance, id) keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t orderable(float d) {
  const uint32_t u = __float_as_uint(d);
  return u ^ ((u >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}

__device__ __forceinline__ float from_orderable(uint32_t o) {
  const uint32_t u = o ^ ((o >> 31) ? 0x80000000u : 0xFFFFFFFFu);
  return __uint_as_float(u);
}

__device__ __forceinline__ uint64_t make_key(float d, uint32_t id) {
  return ((uint64_t)orderable(d) << 32) | id;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
// Warp minimum / maximum of a float (no NaN): one reduction on the
// order-preserving integer image.
__device__ __forceinline__ float warp_min(float v) {
  return from_orderable(__reduce_min_sync(0xffffffffu, orderable(v)));
}
__device__ __forceinline__ float warp_max(float v) {
  return from_orderable(__reduce_max_sync(0xffffffffu, orderable(v)));
}
__device__ __forceinline__ int warp_sum_int(int v) { return __reduce_add_sync(0xffffffffu, v); }
// The 32-lane order: each lane holds its partial sum; combine with strides
// 16, 8, 4, 2, 1, each addition rounded once.
__device__ __forceinline__ float lane_tree_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Bitonic sort of m (power of two) uint64 keys in shared memory, ascending.
// All threads of the block must call it.
// ---------------------------------------------------------------------------
__device__ inline void block_bitonic_sort(uint64_t* s, int m) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t a = s[i], b = s[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            s[i] = b;
            s[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int next_pow2(int v) {
  int m = 1;
  while (m < v) m <<= 1;
  return m;
}

// ---------------------------------------------------------------------------
// Block radix select over keys in global memory: the rank-th smallest
// (1-based) of `count` uint64 keys, by 8-bit digits from the top. `hist` is
// 256 ints of shared memory, `bcast` two uint64 of shared memory.
// ---------------------------------------------------------------------------
__device__ inline uint64_t block_radix_select_u64(const uint64_t* keys,
                                                  int64_t count, int64_t rank,
                                                  int* hist, uint64_t* bcast) {
  uint64_t prefix = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    const uint64_t hi_mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
      const uint64_t k = keys[i];
      if ((k & hi_mask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t cum = 0;
      int b = 0;
      for (; b < 256; ++b) {
        if (cum + hist[b] >= rank) break;
        cum += hist[b];
      }
      if (b > 255) b = 255;
      bcast[0] = prefix | ((uint64_t)b << shift);
      bcast[1] = (uint64_t)(rank - cum);
    }
    __syncthreads();
    prefix = bcast[0];
    rank = (int64_t)bcast[1];
    __syncthreads();
  }
  return prefix;
}


}  // namespace rq

namespace rq {

// ---------------------------------------------------------------------------
// Helpers of the radix selections (8-bit digits): loops run in whole rounds
// of 32 so that warps stay converged.
// ---------------------------------------------------------------------------

// Adds 1 to hist[d] for every active lane (shared-memory atomics; lanes
// that hit the same bin are serialised by the hardware).
__device__ __forceinline__ void hist_add(int* hist, int d, bool active) {
  if (active) atomicAdd(&hist[d], 1);
}

// Sorts 32 uint64 keys held one per lane (ascending by lane) with a bitonic
// network of warp shuffles. All 32 lanes must call it.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      // keep the smaller of the pair on the lower lane of an ascending run
      v = (lower == up) ? (v < o ? v : o) : (v < o ? o : v);
    }
  }
  return v;
}

}  // namespace rq

namespace rq {

// ---------------------------------------------------------------------------
// Warp-level selection: one warp serves one query, synchronising with
// __syncwarp only. `hist` is 256 ints and `small` 32 keys of the warp's own
// shared memory. All 32 lanes call these functions.
// ---------------------------------------------------------------------------

// The bucket where the running count of hist reaches `rank` (1-based), as
// (b, count below b, hist[b]) in every lane.
__device__ __forceinline__ void warp_find_bucket(const int* hist, int rank, int& b, int& below,
                                                 int& cnt) {
  const int lane = threadIdx.x & 31;
  int h[8];
  int sum = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    h[i] = hist[lane * 8 + i];
    sum += h[i];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int excl = incl - sum;
  const unsigned m = __ballot_sync(0xffffffffu, excl < rank && rank <= incl);
  const int src = m ? __ffs(m) - 1 : 31;
  int bb = 7, cum = excl;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (cum + h[i] >= rank) {
      bb = i;
      break;
    }
    cum += h[i];
  }
  int hb = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (i == bb) hb = h[i];
  b = __shfl_sync(0xffffffffu, lane * 8 + bb, src);
  below = __shfl_sync(0xffffffffu, cum, src);
  cnt = __shfl_sync(0xffffffffu, hb, src);
}




// ---------------------------------------------------------------------------
// Block-level selection: every thread of the block takes part (histograms by
// shared-memory atomics, the bucket search by warp 0). `hist` is 256 ints,
// `small` 32 keys and `ctl` 8 ints of shared memory; src is shared memory.
// ---------------------------------------------------------------------------

// One narrowing step: histogram of the digit of `width` (<= 8) bits at
// `shift` over the keys whose bits under `mask` equal `prefix`, and the
// bucket holding the rank-th (1-based) of them, as (b, count below b, count
// in b) in every thread.
template <typename K>
__device__ inline void block_narrow(const K* src, int m, int shift, int width, K mask, K prefix,
                                    int rank, int* hist, int* ctl, int& b, int& below, int& cnt) {
  const K dmask = ((K)1 << width) - 1;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  // eight keys per thread per round, their loads issued together (src may
  // be global memory)
  const int stride = blockDim.x;
  for (int i0 = threadIdx.x; i0 < m; i0 += 8 * stride) {
    K k[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = i0 + j * stride < m ? src[i0 + j * stride] : (K)0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i0 + j * stride < m && (k[j] & mask) == prefix)
        atomicAdd(&hist[(int)((k[j] >> shift) & dmask)], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int bb, bl, bc;
    warp_find_bucket(hist, rank, bb, bl, bc);
    if (threadIdx.x == 0) {
      ctl[0] = bb;
      ctl[1] = bl;
      ctl[2] = bc;
    }
  }
  __syncthreads();
  b = ctl[0];
  below = ctl[1];
  cnt = ctl[2];
}

// Highest bit in which the m keys differ (-1 when all are equal): the radix
// passes start there, since the bits above it are common to every key (the
// leading bits of nearby float32 distances usually are). `red` holds 2 x 32
// keys of shared memory.
template <typename K>
__device__ inline int block_top_diff_bit(const K* src, int m, K* red) {
  const K k0 = src[0];
  K x = 0;
  const int stride = blockDim.x;
  for (int i0 = threadIdx.x; i0 < m; i0 += 8 * stride) {  // eight loads in flight
    K k[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = i0 + j * stride < m ? src[i0 + j * stride] : k0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x |= k[j] ^ k0;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  K all = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) all |= red[w];
  __syncthreads();
  if (all == 0) return -1;
  return (int)(sizeof(K) * 8) - 1 - (sizeof(K) == 8 ? __clzll((long long)all) : __clz((int)all));
}

// Sorts dst[0, n) ascending, dst[n, next_pow2(n)) holding all ones.
__device__ inline void block_sort_keys(uint64_t* dst, int n) {
  if (n <= 32) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const uint64_t v = warp_sort32(lane < n ? dst[lane] : kU64Max);
      if (lane < n) dst[lane] = v;
    }
    __syncthreads();
    return;
  }
  block_bitonic_sort(dst, next_pow2(n));
}

// The n smallest of m distinct uint64 keys into dst[0, n) (ascending if
// `sorted`, else in no fixed order), dst[n, next_pow2(n)) = all ones; dst
// holds next_pow2(max(n, 1)) keys. Returns min(n, m).
__device__ inline int block_select_smallest(const uint64_t* src, int m, int n, uint64_t* dst,
                                            int* hist, uint64_t* small, int* ctl, bool sorted) {
  const int tid = threadIdx.x;
  const int sel = min(n, m);
  const int mp = next_pow2(max(sel, 1));
  if (m <= n) {
    for (int i = tid; i < mp; i += blockDim.x) dst[i] = (i < m) ? src[i] : kU64Max;
    __syncthreads();
    if (sorted) block_sort_keys(dst, sel);
    return sel;
  }
  // Digits of up to 8 bits from the highest bit where the keys differ; the
  // bits above it are common and go into the prefix at once.
  const int top = block_top_diff_bit<uint64_t>(src, m, small);
  uint64_t mask = top < 0 ? ~0ull : (top >= 63 ? 0 : ~((2ull << top) - 1));
  uint64_t prefix = src[0] & mask;
  int rank = n, cnt = m;
  for (int hb = top; hb >= 0 && cnt > 32;) {
    const int shift = max(0, hb - 7), width = hb - shift + 1;
    int b, below;
    block_narrow<uint64_t>(src, m, shift, width, mask, prefix, rank, hist, ctl, b, below, cnt);
    prefix |= (uint64_t)b << shift;
    mask |= ((1ull << width) - 1) << shift;
    rank -= below;
    hb = shift - 1;
  }
  // Keys below the bucket go straight to dst; the bucket (at most 32 keys)
  // is sorted in one warp and its first `rank` keys complete the selection.
  if (tid == 0) {
    ctl[3] = 0;
    ctl[4] = 0;
  }
  __syncthreads();
  // eight keys per thread in flight; a warp reserves room for its keys
  // below the bucket with one atomic
  const int lane = tid & 31;
  for (int w0 = tid - lane; w0 < m; w0 += 8 * (int)blockDim.x) {  // warp-uniform
    uint64_t k[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = w0 + lane + j * (int)blockDim.x;
      k[j] = i < m ? src[i] : kU64Max;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool in = w0 + lane + j * (int)blockDim.x < m;
      const uint64_t km = k[j] & mask;
      const bool lo = in && km < prefix;
      const uint32_t mb = __ballot_sync(0xffffffffu, lo);
      int base = 0;
      if (lane == 0 && mb) base = atomicAdd(&ctl[3], __popc(mb));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (lo) dst[base + __popc(mb & ((1u << lane) - 1u))] = k[j];
      if (in && km == prefix) {
        const int p = atomicAdd(&ctl[4], 1);
        if (p < 32) small[p] = k[j];
      }
    }
  }
  __syncthreads();
  if (tid < 32) {
    const int ns = min(ctl[4], 32);
    const uint64_t v = warp_sort32(tid < ns ? small[tid] : kU64Max);
    if (tid < rank) dst[n - rank + tid] = v;
  }
  for (int i = n + tid; i < mp; i += blockDim.x) dst[i] = kU64Max;
  __syncthreads();
  if (sorted) block_sort_keys(dst, n);
  return sel;
}

// The rank-th smallest (1-based) of m uint32 values (duplicates allowed).
__device__ inline uint32_t block_kth_u32(const uint32_t* src, int m, int rank, int* hist,
                                         uint64_t* small, int* ctl) {
  const int top = block_top_diff_bit<uint32_t>(src, m, reinterpret_cast<uint32_t*>(small));
  if (top < 0) return src[0];
  uint32_t mask = top >= 31 ? 0u : ~((2u << top) - 1u);
  uint32_t prefix = src[0] & mask;
  int cnt = m;
  for (int hb = top; hb >= 0 && cnt > 32;) {
    const int shift = max(0, hb - 7), width = hb - shift + 1;
    int b, below;
    block_narrow<uint32_t>(src, m, shift, width, mask, prefix, rank, hist, ctl, b, below, cnt);
    prefix |= (uint32_t)b << shift;
    mask |= ((1u << width) - 1u) << shift;
    rank -= below;
    hb = shift - 1;
  }
  if (mask == 0xFFFFFFFFu) return prefix;
  // At most 32 values left in the bucket: sort them in one warp.
  if (threadIdx.x == 0) ctl[4] = 0;
  __syncthreads();
  for (int i0 = threadIdx.x; i0 < m; i0 += 8 * blockDim.x) {  // eight loads in flight
    uint32_t k[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = i0 + j * blockDim.x < m ? src[i0 + j * blockDim.x] : 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i0 + j * blockDim.x < m && (k[j] & mask) == prefix) {
        const int p = atomicAdd(&ctl[4], 1);
        if (p < 32) small[p] = k[j];
      }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int ns = min(ctl[4], 32);
    const uint64_t v = warp_sort32(threadIdx.x < ns ? small[threadIdx.x] : kU64Max);
    const uint64_t r = __shfl_sync(0xffffffffu, v, rank - 1);
    if (threadIdx.x == 0) ctl[5] = (int)(uint32_t)r;
  }
  __syncthreads();
  return (uint32_t)ctl[5];
}

// An upper bound on the rank-th smallest (1-based) of m uint32 values: the
// radix passes stop once the bucket holding it has at most `slack` values,
// and the bucket's upper edge is returned (the exact value when every bit
// got resolved). At most `slack` - 1 values lie above the rank-th and at or
// below the result, unless the values run out of bits first.
__device__ inline uint32_t block_kth_upper_u32(const uint32_t* src, int m, int rank, int slack,
                                               int* hist, uint64_t* small, int* ctl) {
  const int top = block_top_diff_bit<uint32_t>(src, m, reinterpret_cast<uint32_t*>(small));
  if (top < 0) return src[0];
  uint32_t mask = top >= 31 ? 0u : ~((2u << top) - 1u);
  uint32_t prefix = src[0] & mask;
  int cnt = m;
  for (int hb = top; hb >= 0 && cnt > slack;) {
    const int shift = max(0, hb - 7), width = hb - shift + 1;
    int b, below;
    block_narrow<uint32_t>(src, m, shift, width, mask, prefix, rank, hist, ctl, b, below, cnt);
    prefix |= (uint32_t)b << shift;
    mask |= ((1u << width) - 1u) << shift;
    rank -= below;
    hb = shift - 1;
  }
  return prefix | ~mask;  // the unresolved low bits all set
}

}  // namespace rq
