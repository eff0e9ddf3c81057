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
  kErrMmaTimeout = 4,
};

__device__ __forceinline__ void flag_error(int32_t* err, int32_t code) {
  if (err) atomicCAS(err, 0, code);
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
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
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

// Same over uint32 keys held in shared memory (4 digits of 8 bits).
__device__ inline uint32_t block_radix_select_u32(const uint32_t* keys,
                                                  int count, int rank,
                                                  int* hist, uint32_t* bcast) {
  uint32_t prefix = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    const uint32_t hi_mask = (shift == 24) ? 0u : (~0u << (shift + 8));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      const uint32_t k = keys[i];
      if ((k & hi_mask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int cum = 0, b = 0;
      for (; b < 256; ++b) {
        if (cum + hist[b] >= rank) break;
        cum += hist[b];
      }
      if (b > 255) b = 255;
      bcast[0] = prefix | ((uint32_t)b << shift);
      bcast[1] = (uint32_t)(rank - cum);
    }
    __syncthreads();
    prefix = bcast[0];
    rank = (int)bcast[1];
    __syncthreads();
  }
  return prefix;
}

}  // namespace rq

namespace rq {

// ---------------------------------------------------------------------------
// Block-wide radix selection with 8-bit digits. All threads of the block call
// these functions (loops run in whole rounds so that warps stay converged).
// `hist` is 256 ints and `res` 4 ints of shared memory.
// ---------------------------------------------------------------------------

// Adds 1 to hist[d] for every active lane, one atomic per distinct digit of
// the warp. All 32 lanes must call it.
__device__ __forceinline__ void hist_add(int* hist, int d, bool active) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  const unsigned peers = __match_any_sync(act, d);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[d], __popc(peers));
}

// Warp 0 finds the bucket b where the running count of hist reaches `rank`
// (1-based): res = {b, count below b, hist[b]}. rank must not exceed the
// total count.
__device__ __forceinline__ void find_bucket(const int* hist, int rank, int* res) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
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
  if (lane == src) {
    int cum = excl, b = 7;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (cum + h[i] >= rank) {
        b = i;
        break;
      }
      cum += h[i];
    }
    res[0] = lane * 8 + b;
    res[1] = cum;
    res[2] = h[b];
  }
}

// Appends the active lanes' values at dst[base + rank] with one atomic per
// warp on *counter; positions at or past `cap` are dropped.
template <typename T>
__device__ __forceinline__ void block_append(T* dst, int* counter, int cap, T v, bool active) {
  const unsigned m = __ballot_sync(0xffffffffu, active);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (active) {
    const int pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < cap) dst[pos] = v;
  }
}

// The n smallest of m distinct uint64 keys at src (shared or global memory),
// ascending in dst[0, n) and dst[n, next_pow2(n)) = all ones. Returns
// min(n, m). dst holds next_pow2(max(n, 1)) keys of shared memory; `small`
// holds kSelectSmall keys of shared memory. Radix passes (8-bit digits from
// the top) narrow the bucket holding the n-th key until it has at most
// kSelectSmall keys; the keys below it are taken whole and the bucket is
// sorted to supply the rest.
constexpr int kSelectSmall = 256;

__device__ inline int block_select_smallest(const uint64_t* src, int m, int n, uint64_t* dst,
                                            uint64_t* small, int* hist, int* res,
                                            bool sorted = true) {
  const int T = blockDim.x;
  const int sel = min(n, m);
  const int mp = next_pow2(max(sel, 1));
  if (m <= n) {
    for (int i = threadIdx.x; i < mp; i += T) dst[i] = (i < m) ? src[i] : kU64Max;
    __syncthreads();
    if (sorted) block_bitonic_sort(dst, mp);
    return sel;
  }
  uint64_t prefix = 0, mask = 0;
  int rank = n, cnt = m;
  for (int shift = 56; shift >= 0 && cnt > kSelectSmall; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += T) hist[i] = 0;
    __syncthreads();
    for (int base = 0; base < m; base += T) {
      const int i = base + threadIdx.x;
      uint64_t k = 0;
      bool act = false;
      if (i < m) {
        k = src[i];
        act = (k & mask) == prefix;
      }
      hist_add(hist, (int)((k >> shift) & 255), act);
    }
    __syncthreads();
    find_bucket(hist, rank, res);
    __syncthreads();
    const int b = res[0], below = res[1];
    cnt = res[2];
    __syncthreads();
    prefix |= (uint64_t)b << shift;
    mask |= 0xFFull << shift;
    rank -= below;
  }
  // Keys below the bucket all belong to the result (n - rank of them); the
  // bucket (cnt <= kSelectSmall keys, or one key after all eight digits)
  // gives its rank smallest.
  if (threadIdx.x == 0) {
    res[2] = 0;
    res[3] = 0;
  }
  __syncthreads();
  for (int base = 0; base < m; base += T) {
    const int i = base + threadIdx.x;
    uint64_t k = kU64Max;
    if (i < m) k = src[i];
    const uint64_t km = k & mask;
    block_append(dst, &res[3], n, k, i < m && km < prefix);
    block_append(small, &res[2], kSelectSmall, k, i < m && km == prefix);
  }
  __syncthreads();
  const int nb = min(res[2], kSelectSmall);
  const int sp = next_pow2(max(nb, 1));
  for (int i = nb + threadIdx.x; i < sp; i += T) small[i] = kU64Max;
  __syncthreads();
  block_bitonic_sort(small, sp);
  const int have = n - rank;
  for (int i = threadIdx.x; i < rank; i += T) dst[have + i] = small[i];
  for (int i = n + threadIdx.x; i < mp; i += T) dst[i] = kU64Max;
  __syncthreads();
  if (sorted) block_bitonic_sort(dst, mp);
  return sel;
}

// The rank-th smallest (1-based) of m uint32 values in shared memory
// (duplicates allowed): radix passes narrow the bucket holding it to at most
// kSelectSmall values, which are then sorted. `small` holds kSelectSmall
// uint64 of shared memory.
__device__ inline uint32_t block_kth_u32(const uint32_t* src, int m, int rank, uint64_t* small,
                                         int* hist, int* res) {
  const int T = blockDim.x;
  uint32_t prefix = 0, mask = 0;
  int cnt = m;
  for (int shift = 24; shift >= 0 && cnt > kSelectSmall; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += T) hist[i] = 0;
    __syncthreads();
    for (int base = 0; base < m; base += T) {
      const int i = base + threadIdx.x;
      uint32_t k = 0;
      bool act = false;
      if (i < m) {
        k = src[i];
        act = (k & mask) == prefix;
      }
      hist_add(hist, (int)((k >> shift) & 255), act);
    }
    __syncthreads();
    find_bucket(hist, rank, res);
    __syncthreads();
    const int b = res[0], below = res[1];
    cnt = res[2];
    __syncthreads();
    prefix |= (uint32_t)b << shift;
    mask |= 0xFFu << shift;
    rank -= below;
  }
  if (mask == 0xFFFFFFFFu) return prefix;
  if (threadIdx.x == 0) res[3] = 0;
  __syncthreads();
  for (int base = 0; base < m; base += T) {
    const int i = base + threadIdx.x;
    uint32_t k = 0;
    if (i < m) k = src[i];
    block_append(small, &res[3], kSelectSmall, (uint64_t)k, i < m && (k & mask) == prefix);
  }
  __syncthreads();
  const int nb = min(res[3], kSelectSmall);
  const int sp = next_pow2(max(nb, 1));
  for (int i = nb + threadIdx.x; i < sp; i += T) small[i] = kU64Max;
  __syncthreads();
  block_bitonic_sort(small, sp);
  const uint32_t v = (uint32_t)small[rank - 1];
  __syncthreads();
  return v;
}

}  // namespace rq
