// block_distinct.cuh -- the per-block distinct count behind the GPU cost
// (Definition 2, Eq. 1: a block loads each distinct data vertex it touches
// once).  Shared by cost_block_kernel (kernels.cu) and the no-allocation
// variant (noalloc.cu), which differ only in where the touched flags live and
// in the checks they make on their inputs.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

namespace ep {
namespace dev {

// Sorts keys[0, P) ascending in place: a bitonic network over a power of two
// P, every thread of the CUDA block taking part; ends with a block barrier.
__device__ __forceinline__ void block_bitonic_sort(int32_t* keys, int P) {
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const int32_t a = keys[i], b = keys[j];
          if ((a > b) == ((i & size) == 0)) {
            keys[i] = b;
            keys[j] = a;
          }
        }
      }
      __syncthreads();
    }
}

// Over the sorted keys[0, nk): calls on_distinct(key) once per distinct key
// (by the thread that finds its first occurrence) and returns the number of
// distinct keys this thread found.
template <typename OnDistinct>
__device__ __forceinline__ unsigned int count_distinct_sorted(const int32_t* keys, int nk,
                                                              OnDistinct on_distinct) {
  unsigned int cnt = 0;
  for (int i = threadIdx.x; i < nk; i += blockDim.x)
    if (i == 0 || keys[i] != keys[i - 1]) {
      ++cnt;
      on_distinct(keys[i]);
    }
  return cnt;
}

// Adds the per-thread values of the whole CUDA block (a multiple of 32 threads)
// to *total with one atomic.
__device__ __forceinline__ void block_sum_add(unsigned int v, unsigned long long* total) {
  __shared__ unsigned int warp_sum[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned int s = threadIdx.x < (blockDim.x >> 5) ? warp_sum[threadIdx.x] : 0u;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(total, (unsigned long long)s);
  }
}

// Sum of one-byte flags f[0, nd) added to *total (grid-stride, one atomic per warp).
__device__ __forceinline__ void sum_flags(const uint8_t* __restrict__ f, int64_t nd,
                                          unsigned long long* __restrict__ total) {
  unsigned int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    cnt += f[i];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(total, (unsigned long long)cnt);
}

}  // namespace dev
}  // namespace ep
