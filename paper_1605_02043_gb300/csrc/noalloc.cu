// noalloc.cu -- the load count of a schedule for callers that cannot
// allocate device memory.
//
// ep_cost() keeps its per-vertex "touched" flags in a workspace it allocates
// with cudaMalloc on first use.  Some callers cannot let a library do that:
// applications that hand all device memory to their own pool or framework
// allocator and forbid allocations behind its back, and latency-bound loops
// that cannot take the implicit device synchronisation cudaMalloc and
// cudaFree may cause.  ep_cost_noalloc() gives them the same count with the
// flags in a fixed file-scope device array instead; the caller passes every
// input and output.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "block_distinct.cuh"
#include "epcache.h"

namespace {

// Scratch: one flag byte per data vertex, then a status word.  Every GPU that
// loads this module keeps these bytes until the process exits; all calls share
// them (the previous call's contents stay until cleared).
struct Scratch {
  uint8_t touched[EP_NOALLOC_MAX_VERTICES];
  unsigned int status;  // EP_NOALLOC_* bits of the current call
};
static __device__ __align__(256) Scratch g_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
Scratch* g_addr[kMaxDevices] = {};  // device address of g_scratch, per device

thread_local char g_msg[256];

int fail(int code, const char* msg) {
  snprintf(g_msg, sizeof g_msg, "%s", msg);
  return code;
}

// A CUDA runtime call of this entry point failed: record the message and clear
// the runtime's last-error slot, which that failure has just set, so that the
// next call on this thread does not see it.
int fail_cuda(cudaError_t e, const char* what) {
  snprintf(g_msg, sizeof g_msg, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return EP_ECUDA;
}

// One CUDA block per schedule block: sort the block's endpoint ids in shared
// memory (bitonic network over P = power of two >= 2 * max_ne), count the
// distinct ids and flag them.  A block with more than P / 2 tasks (or a
// negative length) cannot be sorted in the space the caller's max_ne gave:
// it is not counted and the call's status gets EP_NOALLOC_BAD_BLOCK.  An id
// outside [0, nd) is counted but not flagged, and sets EP_NOALLOC_BAD_ID.
__global__ void cost_noalloc_kernel(const int64_t* __restrict__ block_ptr,
                                    const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                    int P, int64_t nd, Scratch* __restrict__ s,
                                    unsigned long long* __restrict__ loads) {
  extern __shared__ int32_t keys[];
  const int64_t e0 = block_ptr[blockIdx.x];
  const int64_t len = block_ptr[blockIdx.x + 1] - e0;
  if (len < 0 || len > P / 2) {  // uniform over the CUDA block
    if (threadIdx.x == 0) atomicOr(&s->status, (unsigned int)EP_NOALLOC_BAD_BLOCK);
    return;
  }
  const int ne = (int)len, nk = 2 * ne;
  for (int i = threadIdx.x; i < P; i += blockDim.x)
    keys[i] = i < ne ? eu[e0 + i] : i < nk ? ev[e0 + i - ne] : INT_MAX;
  __syncthreads();
  ep::dev::block_bitonic_sort(keys, P);
  bool bad = false;
  const unsigned int distinct = ep::dev::count_distinct_sorted(keys, nk, [&](int32_t v) {
    if ((uint64_t)(uint32_t)v < (uint64_t)nd && v >= 0)
      s->touched[v] = 1;
    else
      bad = true;
  });
  if (bad) atomicOr(&s->status, (unsigned int)EP_NOALLOC_BAD_ID);
  ep::dev::block_sum_add(distinct, loads);
}

__global__ void count_touched_kernel(const Scratch* __restrict__ s, int64_t nd,
                                     unsigned long long* __restrict__ total) {
  ep::dev::sum_flags(s->touched, nd, total);
}

// Last launch of a call: a misused call overwrites both counts.
__global__ void finish_kernel(const Scratch* __restrict__ s, unsigned long long* __restrict__ counts) {
  const unsigned int st = s->status;
  if (st) {
    counts[0] = EP_NOALLOC_INVALID;
    counts[1] = st;
  }
}

template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                   cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
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
  Scratch* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name
    // g_scratch is not a device address, so look the address up
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) {
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress of the scratch array");
        return fail(EP_ECUDA, "cudaGetSymbolAddress of the scratch array gave no address");
      }
      g_addr[dev] = static_cast<Scratch*>(p);
    }
    scratch = g_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int P = 2;
  while (P < 2 * max_ne) P <<= 1;
  const size_t smem = (size_t)P * sizeof(int32_t);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(cost_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail_cuda(e, "raising the shared-memory limit of the cost kernel");
  }
  // the scratch keeps the previous call's contents: clear the flags this call
  // uses and the status word
  e = cudaMemsetAsync(scratch->touched, 0, (size_t)nd, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&scratch->status, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync");
  const int tpb = P >= 1024 ? 1024 : (P < 32 ? 32 : P);
  e = launch(cost_noalloc_kernel, (unsigned)k, (unsigned)tpb, smem, st, block_ptr, eu, ev, P, nd,
             scratch, counts);
  if (e != cudaSuccess) return fail_cuda(e, "launch of the cost kernel");
  int64_t g = (nd + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  e = launch(count_touched_kernel, (unsigned)g, 256u, 0, st, (const Scratch*)scratch, nd, counts + 1);
  if (e != cudaSuccess) return fail_cuda(e, "launch of the flag count");
  e = launch(finish_kernel, 1u, 1u, 0, st, (const Scratch*)scratch, counts);
  if (e != cudaSuccess) return fail_cuda(e, "launch of the status check");
  return EP_OK;
}
