// noalloc.cu -- the load count of a schedule for callers that cannot
// allocate device memory.
//
// ep_cost() keeps its per-vertex "touched" flags in a workspace it allocates
// with cudaMalloc on first use.  Some callers cannot let a library do that:
// code running while a stream is being captured into a CUDA graph (cudaMalloc
// is not allowed there), applications that own all device memory through
// their own pool and forbid outside allocations, and latency-sensitive loops
// where an allocation's implicit device synchronisation is not acceptable.
// ep_cost_noalloc() gives them the same count with the flags in a fixed
// file-scope device array instead; the caller passes every input and output.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "epcache.h"

namespace {

// Scratch flags: one byte per data vertex.  Every GPU that loads this module
// keeps these EP_NOALLOC_MAX_VERTICES bytes until the process exits; all
// calls share them (the previous call's flags stay until cleared).
static __device__ __align__(256) uint8_t g_touched[EP_NOALLOC_MAX_VERTICES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_addr[kMaxDevices] = {};  // device address of g_touched, per device

thread_local char g_msg[256];

int fail(int code, const char* msg) {
  snprintf(g_msg, sizeof g_msg, "%s", msg);
  return code;
}

// One CUDA block per schedule block: sort the block's endpoint ids in shared
// memory (bitonic network over P = power of two >= 2 * tasks), count the
// distinct ids and flag them in `touched`.
__global__ void cost_noalloc_kernel(const int64_t* __restrict__ block_ptr,
                                    const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                    int P, int64_t nd, uint8_t* __restrict__ touched,
                                    unsigned long long* __restrict__ loads) {
  extern __shared__ int32_t keys[];
  __shared__ unsigned int part[32];
  const int64_t e0 = block_ptr[blockIdx.x];
  // a block larger than the caller's max_ne is cut to what shared memory holds
  const int ne = (int)min(block_ptr[blockIdx.x + 1] - e0, (int64_t)(P / 2));
  const int nk = 2 * ne;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    keys[i] = i < ne ? eu[e0 + i] : i < nk ? ev[e0 + i - ne] : INT_MAX;
  __syncthreads();
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
  unsigned int distinct = 0;
  for (int i = threadIdx.x; i < nk; i += blockDim.x)
    if (i == 0 || keys[i] != keys[i - 1]) {
      ++distinct;
      if ((uint64_t)(uint32_t)keys[i] < (uint64_t)nd) touched[keys[i]] = 1;  // ids outside [0, nd) are not flagged
    }
  for (int o = 16; o > 0; o >>= 1) distinct += __shfl_down_sync(0xffffffffu, distinct, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = distinct;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned int v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0u;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loads, (unsigned long long)v);
  }
}

__global__ void count_touched_kernel(const uint8_t* __restrict__ touched, int64_t nd,
                                     unsigned long long* __restrict__ total) {
  unsigned int c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    c += touched[i];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(total, (unsigned long long)c);
}

}  // namespace

extern "C" const char* ep_noalloc_last_error(void) { return g_msg; }

extern "C" int ep_cost_noalloc(const int64_t* block_ptr, const int32_t* eu, const int32_t* ev,
                               int64_t k, int64_t nd, int32_t max_ne, unsigned long long* counts,
                               void* stream) {
  g_msg[0] = 0;
  if (!block_ptr || !eu || !ev || !counts) return fail(EP_EINVAL, "null pointer argument");
  if (k < 1 || k > INT32_MAX) return fail(EP_EINVAL, "k out of range");
  if (nd < 1) return fail(EP_EINVAL, "nd must be positive");
  if (nd > (int64_t)EP_NOALLOC_MAX_VERTICES)
    return fail(EP_EINVAL,
                "nd exceeds EP_NOALLOC_MAX_VERTICES; use ep_cost(), which sizes its own workspace");
  if (max_ne < 1 || max_ne > EP_MAX_C) return fail(EP_EINVAL, "max_ne out of [1, EP_MAX_C]");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(EP_ENODEV, "no usable current CUDA device");
  }
  uint8_t* touched = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_touched);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(EP_ECUDA, "cudaGetSymbolAddress of the scratch flags failed");
      }
      g_addr[dev] = static_cast<uint8_t*>(p);
    }
    touched = g_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int P = 2;
  while (P < 2 * max_ne) P <<= 1;
  const size_t smem = (size_t)P * sizeof(int32_t);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(cost_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return fail(EP_ECUDA, "cannot raise the shared-memory limit of the cost kernel");
  // the flags keep the previous call's contents: clear the part this call uses
  if (cudaMemsetAsync(touched, 0, (size_t)nd, st) != cudaSuccess ||
      cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess)
    return fail(EP_ECUDA, "cudaMemsetAsync failed");
  const int tpb = P >= 1024 ? 1024 : (P < 32 ? 32 : P);
  cost_noalloc_kernel<<<(unsigned)k, tpb, smem, st>>>(block_ptr, eu, ev, P, nd, touched, counts);
  int64_t g = (nd + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  count_touched_kernel<<<(unsigned)g, 256, 0, st>>>(touched, nd, counts + 1);
  if (cudaGetLastError() != cudaSuccess) return fail(EP_ECUDA, "kernel launch failed");
  return EP_OK;
}
