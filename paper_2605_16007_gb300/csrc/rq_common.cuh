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
