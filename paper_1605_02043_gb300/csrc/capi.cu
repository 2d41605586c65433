// capi.cu -- the extern "C" boundary of libepcache (declared in epcache.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>

#include "epcache.h"
#include "internal.h"
#include "flux_common.cuh"
#include "kernels.h"

namespace {

thread_local std::string g_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, b ? b : 16);
    if (e == cudaSuccess) bytes = b ? b : 16;
    return e;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

template <typename T>
cudaError_t upload(DBuf& d, const std::vector<T>& v) {
  cudaError_t e = d.ensure(v.size() * sizeof(T));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(d.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Event pairs recorded around launches; resolved lazily in ep_timing_read.
struct EventTimer final : ep::dev::Timer {
  bool on = false;
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open = nullptr;
  double total[EP_T_CLASSES] = {};
  int64_t count[EP_T_CLASSES] = {};

  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  void begin(int, cudaStream_t st) override {
    if (!on) return;
    open = take();
    if (open) cudaEventRecord(open, st);
  }
  void end(int cls, cudaStream_t st) override {
    if (!on || !open) return;
    cudaEvent_t e = take();
    if (!e) return;
    cudaEventRecord(e, st);
    pending.push_back({cls, open, e});
    open = nullptr;
    if (pending.size() > 8192) collect();
  }
  void collect() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        total[p.cls] += ms;
        count[p.cls] += 1;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void clear() {
    collect();
    for (int i = 0; i < EP_T_CLASSES; ++i) {
      total[i] = 0;
      count[i] = 0;
    }
  }
  ~EventTimer() override {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct ep_schedule {
  ep::HostSchedule h;
  int device = -1;  // device holding the uploaded copy, -1 before upload
  int tpb = 192;      // consumer threads of the forward and SpMV kernels
  int tpb_adj = 352;  // consumer threads of the adjoint kernels
  bool bacc_dirty = true;
  // device copy of the schedule
  DBuf d_desc, d_flist, d_ylist, d_ent, d_perm, d_wmap, d_rec, d_xrec, d_yrec, d_bptr, d_eu,
      d_ev;
  DBuf d_sidx, d_soff, d_sid, d_gslot, d_frec, d_fsid;  // flux layout
  // workspace
  DBuf ws_x, ws_out, ws_w, ws_bacc, ws_lam, ws_gw, ws_hist, ws_flags, ws_cnt;
  DBuf ws_hx, ws_hw, ws_hout;
  // vertex-ordered maps for inputs read from host memory (built on first use):
  // records of every vertex (CSR) and the weight slots of every task (2 each)
  DBuf d_hptr, d_hrec, d_tslot;
  bool host_maps = false;
  // shard halo (ep_set_halo): shared id of every halo vertex here, -1 if untouched
  std::vector<int32_t> hmap;
  DBuf d_hmap;
  const void* zeroed_x = nullptr;  // workspace buffers last cleared whole (their
  const void* zeroed_w = nullptr;  // padding is never written by the scatter kernels)
  EventTimer timer;
  ep::dev::Timer* t() { return timer.on ? &timer : nullptr; }
  int stages = 3;  // pipelined kernels with this many stages; 0 = one CUDA block per schedule block
  int stall = -1;  // test hook of the bounded waits (ep_debug_stall)
  int cache = EP_CACHE_SMEM;  // forward flux kernel family (ep_set_cache)
  // [0] forward accumulator phase, [1] adjoint accumulator phase,
  // [2] error word, [3] CUDA blocks finished in the current launch
  DBuf ws_ctl;
  size_t ws_bacc_set = 0;  // floats of one accumulator buffer (6 buffers: 3 forward, 3 adjoint)
  int32_t bacc_D = 0;      // state width the accumulators were last used with
  bool pending[2] = {false, false};  // a state of this kind was left pending
  int sm_count = 0;
  // launch plans of the pipelined kernels, cached per (D, adjoint) so that
  // steps inside a stream capture only enqueue work
  ep::dev::TmaPlan plans[EP_MAX_D + 1][2];
  int plan_key[EP_MAX_D + 1][2] = {};
};

namespace {

bool bipartite(const ep_schedule* s) { return (s->h.flags & EP_BIPARTITE) != 0; }

constexpr int kCtlWords = 4;

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      s->bacc_dirty = true;                                                               \
      return fail(EP_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                     \
  } while (0)

// Makes sure a CUDA device exists and the schedule is uploaded to the current one.
int ensure_device(ep_schedule* s) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return fail(EP_ENODEV, "no CUDA device");
  }
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (s->device >= 0) {
    if (dev != s->device)
      return fail(EP_EINVAL, "schedule lives on device %d, current device is %d", s->device, dev);
    return EP_OK;
  }
  const ep::HostSchedule& h = s->h;
  std::vector<int32_t> eu(h.m), ev(h.m);
  for (int64_t i = 0; i < h.m; ++i) {
    const int32_t e = h.edge_perm[i];
    eu[i] = bipartite(s) ? (int32_t)(h.n + h.src[e]) : h.src[e];
    ev[i] = h.dst[e];
  }
  CU(upload(s->d_eu, eu));
  CU(upload(s->d_ev, ev));
  CU(upload(s->d_bptr, h.block_ptr));
  CU(upload(s->d_perm, h.edge_perm));
  if (bipartite(s)) {
    CU(upload(s->d_desc, h.sdesc));
    CU(upload(s->d_flist, h.xlist));
    CU(upload(s->d_ylist, h.ylist));
    CU(upload(s->d_ent, h.sent));
    CU(upload(s->d_wmap, h.wmap));
    CU(upload(s->d_xrec, h.xrec_of));
    CU(upload(s->d_yrec, h.yrec_of));
  } else {
    CU(upload(s->d_desc, h.fdesc));
    CU(upload(s->d_sidx, h.sidx));
    CU(upload(s->d_soff, h.soff));
    CU(upload(s->d_sid, h.sid_list));
    CU(upload(s->d_frec, h.fold_rec));
    CU(upload(s->d_fsid, h.fold_sid));
    CU(upload(s->d_gslot, h.gslot));
    CU(upload(s->d_wmap, h.wmap));
    CU(upload(s->d_rec, h.rec_of));
    if (!s->hmap.empty()) CU(upload(s->d_hmap, s->hmap));
  }
  s->device = dev;
  return EP_OK;
}

cudaStream_t as_stream(void* p) { return static_cast<cudaStream_t>(p); }

// The device address of p when it is host memory the GPU can read and write
// directly (pinned through CUDA), else null.
const void* host_mapped(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // an unregistered pointer is not an error here
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Maps for reading inputs in vertex / task order: every record of a vertex
// (CSR over the data vertices) and the weight slots of every task.
int ensure_host_maps(ep_schedule* s) {
  if (s->host_maps) return EP_OK;
  const ep::HostSchedule& h = s->h;
  std::vector<int32_t> tslot(2 * (size_t)h.m, -1);
  for (size_t j = 0; j < h.wmap.size(); ++j) {
    const int32_t t = h.wmap[j];
    if (t < 0) continue;
    int32_t* sl = &tslot[2 * (size_t)t];
    (sl[0] < 0 ? sl[0] : sl[1]) = (int32_t)j;
  }
  if (!bipartite(s)) {
    std::vector<int32_t> ptr(h.nd + 1, 0), rec;
    for (int32_t v : h.vrec)
      if (v >= 0) ++ptr[v + 1];
    for (int64_t v = 0; v < h.nd; ++v) ptr[v + 1] += ptr[v];
    rec.resize(ptr[h.nd]);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t r = 0; r < h.vrec.size(); ++r)
      if (h.vrec[r] >= 0) rec[fill[h.vrec[r]]++] = (int32_t)r;
    CU(upload(s->d_hptr, ptr));
    CU(upload(s->d_hrec, rec));
  }
  CU(upload(s->d_tslot, tslot));
  s->host_maps = true;
  return EP_OK;
}

// State from the caller's order into schedule layout: every vertex's values
// are read once, in vertex order, and written to each of its records (a
// gather by record would read each record's components from scattered
// 4-byte locations).  Records of no vertex are left as they are: no kernel
// reads them.
int layout_in_state(ep_schedule* s, int32_t D, const float* x, float* x_lay, cudaStream_t st) {
  if (int rc = ensure_host_maps(s)) return rc;
  CU(ep::dev::layout_in_csr(s->d_hptr.as<int32_t>(), s->d_hrec.as<int32_t>(), s->h.nd, s->h.n_rec, D, x, x_lay,
                            st, s->t()));
  return EP_OK;
}

// weight layout: flux schedules one weight per slot (two per task), SpMV
// schedules one per task, both padded per block (wmap: slot -> task)
const int32_t* wmap_of(ep_schedule* s) { return s->d_wmap.as<int32_t>(); }
int64_t wlen_of(const ep_schedule* s) { return s->h.w_pad; }

// accumulator sets: forward steps and adjoint steps rotate their own three
// buffers with their own phase word
constexpr int kFwd = 0, kAdj = 1;

ep::dev::FluxArgs flux_args(ep_schedule* s, int kind, const float* w, const float* x_in, float* x_out,
                            float* out, float tau) {
  ep::dev::FluxArgs a;
  a.desc = s->d_desc.as<ep::FluxDesc>();
  a.k = (int64_t)s->h.fdesc.size();  // kernel blocks (large schedule blocks are cut)
  a.sidx = s->d_sidx.as<uint16_t>();
  a.soff = s->d_soff.as<uint16_t>();
  a.sid = s->d_sid.as<int32_t>();
  a.w = w;
  a.x_in = x_in;
  a.x_out = x_out;
  a.bacc = s->ws_bacc.as<float>() + (size_t)kind * 3 * s->ws_bacc_set;
  a.phase = s->ws_ctl.as<int>() + kind;
  a.done = s->ws_ctl.as<int>() + 3;
  a.out = out;
  a.fold_rec = s->d_frec.as<int32_t>();
  a.fold_sid = s->d_fsid.as<int32_t>();
  a.n_copies = (int64_t)s->h.fold_rec.size();
  a.n_rec = s->h.n_rec;
  a.n_sh = s->h.n_sh;
  a.tau = tau;
  a.max_nv = s->h.max_nv;
  a.max_nslot = s->h.max_nslot;
  a.max_nsh = s->h.max_nsh;
  a.max_nsl = s->h.max_nsl;
  a.tpb = kind == kAdj ? s->tpb_adj : s->tpb;
  a.timer = s->t();
  return a;
}

int tma_plan_compute(ep_schedule* s, int32_t D, bool adjoint, ep::dev::TmaPlan& P);

// Stage layout and grid of the pipelined kernels for state width D (cached;
// recomputed when the stage count, thread count or stall hook changes).
int tma_plan(ep_schedule* s, int32_t D, bool adjoint, ep::dev::TmaPlan& P) {
  const int key = 1 + s->stages + 16 * (adjoint ? s->tpb_adj : s->tpb) + (1 << 16) * (s->stall + 1);
  if (s->plan_key[D][adjoint] != key) {
    if (int rc = tma_plan_compute(s, D, adjoint, s->plans[D][adjoint])) return rc;
    s->plan_key[D][adjoint] = key;
  }
  P = s->plans[D][adjoint];
  return EP_OK;
}

int tma_plan_compute(ep_schedule* s, int32_t D, bool adjoint, ep::dev::TmaPlan& P) {
  const ep::HostSchedule& h = s->h;
  ep::dev::TmaLayout& L = P.L;
  L = ep::dev::tma_layout(flux_args(s, kFwd, nullptr, nullptr, nullptr, nullptr, 0.f), D, adjoint);
  if (!s->sm_count) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev));
  }
  int optin = 0, dev = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  L.stages = std::min(s->stages, ep::dev::kMaxStages);
  L.stall = s->stall;
  optin -= 1024;  // room for the kernel's static shared memory
  while (L.stages > 2 && (int64_t)L.stages * L.stage_bytes > optin) --L.stages;
  P.fits = (int64_t)L.stages * L.stage_bytes <= optin;
  if (!P.fits) return EP_OK;  // the launch falls back to one CUDA block per schedule block
  P.smem = (size_t)L.stages * L.stage_bytes;
  // producer warp, fix-up warps, consumer warps
  const int tpb = adjoint ? s->tpb_adj : s->tpb;
  P.threads = 32 * (1 + ep::dev::kFixupWarps) + std::min(tpb, 1024 - 32 * (1 + ep::dev::kFixupWarps));
  const void* kern = ep::dev::flux_tma_kernel_ptr(D, adjoint);
  // the limit is a per-kernel attribute shared by every schedule: open it to
  // the device maximum (the launch still asks for P.smem)
  cudaFuncAttributes fa;
  CU(cudaFuncGetAttributes(&fa, kern));
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // the barriers are static shared memory
  if ((int64_t)P.smem > dyn_max)
    return fail(EP_EINVAL, "pipelined stages need %zu bytes of shared memory (limit %d)", P.smem, dyn_max);
  CU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  int per_sm = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P.threads, P.smem));
  if (per_sm < 1) return fail(EP_EINVAL, "pipelined kernel does not fit on an SM");
  P.per_sm = per_sm;
  P.grid = (int)std::min<int64_t>((int64_t)h.fdesc.size(), (int64_t)per_sm * s->sm_count);
  if (!s->ws_ctl.p) {
    CU(s->ws_ctl.ensure(kCtlWords * sizeof(int)));
    CU(cudaMemset(s->ws_ctl.p, 0, kCtlWords * sizeof(int)));
  }
  P.err = s->ws_ctl.as<int>() + 2;
  return EP_OK;
}

// accumulators of the shared vertices (two buffers, see acc_buffer) and the
// control words: allocated; both buffers zero and the phase reset after an
// allocation or an interrupted launch
int ensure_bacc(ep_schedule* s, int32_t D, cudaStream_t st) {
  // floats of one buffer, sized for the widest accumulator record
  const size_t set = std::max<size_t>((size_t)s->h.n_sh * ep::dev::acc_stride(D), s->ws_bacc_set);
  if (set != s->ws_bacc_set || !s->ws_bacc.p) {
    CU(s->ws_bacc.ensure(6 * set * sizeof(float)));
    s->ws_bacc_set = set;
    s->bacc_dirty = true;
  }
  if (D != s->bacc_D) {  // the accumulator records change shape
    s->bacc_D = D;
    s->bacc_dirty = true;
  }
  if (!s->ws_ctl.p) {
    CU(s->ws_ctl.ensure(kCtlWords * sizeof(int)));
    CU(cudaMemsetAsync(s->ws_ctl.p, 0, kCtlWords * sizeof(int), st));
  }
  if (s->bacc_dirty) {  // every control word but the error word
    CU(cudaMemsetAsync(s->ws_bacc.p, 0, s->ws_bacc.bytes, st));
    CU(cudaMemsetAsync(s->ws_ctl.p, 0, 2 * sizeof(int), st));
    CU(cudaMemsetAsync(s->ws_ctl.as<int>() + 3, 0, sizeof(int), st));
    s->bacc_dirty = false;
  }
  return EP_OK;
}

// The one-block kernels stage a whole schedule block in shared memory.
int block_fits(ep_schedule* s, size_t need) {
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (need + 1024 > (size_t)optin)
    return fail(EP_EINVAL,
                "a schedule block needs %zu bytes of shared memory (limit %d): use a smaller C",
                need, optin - 1024);
  return EP_OK;
}

// Finish of a pending state (flux_common.cuh, the accumulator rotation):
// every shared copy of x_out becomes x_in's + tau * the last step's sums.
int finish_any(ep_schedule* s, int kind, int32_t D, const float* x_in, float* x_out, float* out,
               float tau, cudaStream_t st) {
  ep::dev::FluxArgs a = flux_args(s, kind, nullptr, x_in, x_out, out, tau);
  CU(ep::dev::bnd_update(a, D, x_out, x_in, out, st));
  return EP_OK;
}

// A new state is about to start: sums still pending from an unfinished one
// must not reach it.
void fresh_state(ep_schedule* s) {
  if (s->pending[0] || s->pending[1]) s->bacc_dirty = true;
  s->pending[0] = s->pending[1] = false;
}

// One forward step in schedule layout.  The shared copies of x_out are left
// one step behind (pending) unless `finish`; the edge kernels bring pending
// copies of x_in up to date as they stage them.
int flux_step_any(ep_schedule* s, int32_t D, const float* w, const float* x_in, float* x_out,
                  float* out, float tau, bool finish, cudaStream_t st) {
  ep::dev::FluxArgs a = flux_args(s, kFwd, w, x_in, x_out, out, tau);
  if (s->cache == EP_CACHE_L1) {
    // the read-only-cache kernel reads x_in in place: finish a pending input first
    if (s->pending[kFwd])
      if (int rc = finish_any(s, kFwd, D, x_in, const_cast<float*>(x_in), nullptr, tau, st)) return rc;
    CU(ep::dev::flux_step_ldg(a, D, st));
  } else {
    ep::dev::TmaPlan P;
    if (s->stages != 0) {
      if (int rc = tma_plan(s, D, false, P)) return rc;
    }
    if (s->stages == 0 || !P.fits) {
      if (int rc = block_fits(s, ep::dev::flux_block_smem(a, D, false))) return rc;
      CU(ep::dev::flux_step(a, D, st));
    } else if (a.k > 0) {
      struct Scope {
        ep::dev::Timer* t;
        cudaStream_t st;
        Scope(ep::dev::Timer* t_, cudaStream_t s_) : t(t_), st(s_) {
          if (t) t->begin(ep::dev::T_EDGE_FWD, st);
        }
        ~Scope() {
          if (t) t->end(ep::dev::T_EDGE_FWD, st);
        }
      } sc(a.timer, st);
      CU(ep::dev::flux_fwd_tma(a, P, D, st));
    }
  }
  s->pending[kFwd] = !finish;
  if (finish) return finish_any(s, kFwd, D, x_out, x_out, out, tau, st);
  return EP_OK;
}

// One adjoint step in schedule layout (x finished; lam's shared copies left
// pending unless `finish`).
int flux_adj_any(ep_schedule* s, int32_t D, const float* w, const float* x, float* lam, float* gw,
                 float tau, bool finish, cudaStream_t st) {
  ep::dev::FluxArgs a = flux_args(s, kAdj, w, x, nullptr, nullptr, tau);
  ep::dev::TmaPlan P;
  if (s->stages != 0) {
    if (int rc = tma_plan(s, D, true, P)) return rc;
  }
  if (s->stages == 0 || !P.fits) {
    if (int rc = block_fits(s, ep::dev::flux_block_smem(a, D, true))) return rc;
    CU(ep::dev::flux_adjoint_step(a, D, lam, gw, st));
  } else if (a.k > 0) {
    struct Scope {
      ep::dev::Timer* t;
      cudaStream_t st;
      Scope(ep::dev::Timer* t_, cudaStream_t s_) : t(t_), st(s_) {
        if (t) t->begin(ep::dev::T_EDGE_ADJ, st);
      }
      ~Scope() {
        if (t) t->end(ep::dev::T_EDGE_ADJ, st);
      }
    } sc(a.timer, st);
    CU(ep::dev::flux_adj_tma(a, P, D, lam, gw, st));
  }
  s->pending[kAdj] = !finish;
  if (finish) return finish_any(s, kAdj, D, lam, lam, nullptr, tau, st);
  return EP_OK;
}

bool misaligned(const void* p) { return p && ((uintptr_t)p & 15u); }

int check_flux(ep_schedule* s, int32_t D) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (bipartite(s)) return fail(EP_EINVAL, "flux kernels need a non-bipartite schedule");
  if (D < 1 || D > EP_MAX_D) return fail(EP_EINVAL, "D = %d out of [1, %d]", D, EP_MAX_D);
  return EP_OK;
}

// SpMV kernel on schedule-layout buffers
int spmv_lay(ep_schedule* s, const float* x_lay, const float* w_lay, float* y_lay, cudaStream_t st) {
  const ep::HostSchedule& h = s->h;
  ep::dev::SpmvArgs a;
  a.desc = s->d_desc.as<ep::SpmvDesc>();
  a.k = h.k;
  a.xlist = s->d_flist.as<int32_t>();
  a.ylist = s->d_ylist.as<int32_t>();
  a.ent = s->d_ent.as<uint32_t>();
  a.w = w_lay;
  a.x = x_lay;
  a.y = y_lay;
  a.ny_int = h.ny_int;
  a.ny_zero = h.n - h.ny_int;
  a.max_nx = h.max_nx;
  a.max_ny = h.max_ny;
  a.max_nxy = h.max_nxy;
  a.u = h.spmv_u;
  a.tpb = s->tpb;
  a.readonly = s->cache == EP_CACHE_L1;
  a.timer = s->t();
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const ep::dev::SpmvPlan P = ep::dev::spmv_plan(a, optin);
  if (P.wpb == 0)
    return fail(EP_EINVAL,
                "a schedule block needs %zu bytes of shared memory (limit %d): use a smaller C",
                P.smem, optin - 1024);
  CU(ep::dev::spmv(a, st));
  return EP_OK;
}

// Workspace w in schedule layout from the caller's w.  from_host: w is read
// in task order (it lives in host memory and crosses the host link once,
// coalesced); the padding slots, never written then, are cleared with the
// buffer.
int weights_to_ws(ep_schedule* s, const float* w, bool from_host, cudaStream_t st) {
  CU(s->ws_w.ensure((size_t)wlen_of(s) * sizeof(float)));
  if (!from_host) {
    CU(ep::dev::gather(wmap_of(s), wlen_of(s), w, s->ws_w.as<float>(), st, s->t()));
    s->zeroed_w = nullptr;
    return EP_OK;
  }
  if (int rc = ensure_host_maps(s)) return rc;
  if (s->zeroed_w != s->ws_w.p) {
    CU(cudaMemsetAsync(s->ws_w.p, 0, s->ws_w.bytes, st));
    s->zeroed_w = s->ws_w.p;
  }
  CU(ep::dev::weights_scatter(s->d_tslot.as<int32_t>(), s->h.m, w, s->ws_w.as<float>(), st, s->t()));
  return EP_OK;
}

int run_spmv(ep_schedule* s, const float* x, const float* w, float* y, cudaStream_t st,
             bool from_host = false) {
  const ep::HostSchedule& h = s->h;
  CU(s->ws_x.ensure((size_t)h.n * sizeof(float)));
  CU(s->ws_out.ensure((size_t)h.n * sizeof(float)));
  CU(ep::dev::layout_in(s->d_xrec.as<int32_t>(), h.n, h.n, 1, x, s->ws_x.as<float>(), st, s->t()));
  if (int rc = weights_to_ws(s, w, from_host, st)) return rc;
  if (int rc = spmv_lay(s, s->ws_x.as<float>(), s->ws_w.as<float>(), s->ws_out.as<float>(), st))
    return rc;
  CU(ep::dev::layout_out(s->d_yrec.as<int32_t>(), h.n, h.n, 1, s->ws_out.as<float>(), y, st, s->t()));
  return EP_OK;
}

int new_schedule(ep_schedule** out, ep_schedule** holder) {
  ep_schedule* s = new (std::nothrow) ep_schedule();
  if (!s) return fail(EP_ENOMEM, "out of host memory");
  *holder = s;
  (void)out;
  return EP_OK;
}

int check_edges(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t C,
                uint32_t flags) {
  if (!src || !dst) return fail(EP_EINVAL, "null edge arrays");
  if (m <= 0 || m >= INT32_MAX) return fail(EP_EINVAL, "m = %lld out of range", (long long)m);
  if (n <= 0 || n >= INT32_MAX / 2) return fail(EP_EINVAL, "n = %lld out of range", (long long)n);
  if (C < 1 || C > EP_MAX_C) return fail(EP_EINVAL, "C = %d out of [1, %d]", C, EP_MAX_C);
  if (flags & ~(EP_BIPARTITE | EP_DEFAULT_ORDER | EP_PRESCREEN))
    return fail(EP_EINVAL, "unknown flags");
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
      return fail(EP_EINVAL, "task %lld uses a vertex outside [0, %lld)", (long long)e, (long long)n);
  return EP_OK;
}

// Partition (Section 3) and build the schedule into s.  A raised *stop ends
// the work early with EP_ECANCELED.
int fill_partition(ep_schedule* s, const int32_t* src, const int32_t* dst, int64_t m, int64_t n,
                   int32_t C, uint32_t flags, int threads, const std::atomic<int>* stop) {
  try {
    ep::HostSchedule& h = s->h;
    h.m = m;
    h.n = n;
    h.nd = (flags & EP_BIPARTITE) ? 2 * n : n;
    h.C = C;
    h.flags = flags & ~EP_PRESCREEN;
    h.k = (m + C - 1) / C;
    h.src.assign(src, src + m);
    h.dst.assign(dst, dst + m);
    h.part.resize(m);
    h.origin = (flags & EP_DEFAULT_ORDER) ? ep::kOriginDefault : ep::kOriginPartition;
    bool placed = false;
    if ((flags & EP_PRESCREEN) && !(flags & EP_DEFAULT_ORDER)) {
      const ep::PrescreenResult pr = ep::prescreen(src, dst, m, n, (flags & EP_BIPARTITE) != 0);
      h.origin = pr.origin;
      if (pr.origin == ep::kOriginPath) {
        for (int64_t i = 0; i < m; ++i) h.part[pr.order[i]] = (int32_t)(i / C);
        placed = true;
      } else if (pr.origin != ep::kOriginPartition) {
        for (int64_t e = 0; e < m; ++e) h.part[e] = (int32_t)(e / C);
        placed = true;
      }
    }
    if (!placed && !ep::partition_edges(src, dst, m, n, C, h.flags, threads, h.part.data(), stop))
      return fail(EP_ECANCELED, "partition cancelled");
    if (stop && stop->load()) return fail(EP_ECANCELED, "partition cancelled");
    std::string err = ep::build_schedule(h, threads);
    if (!err.empty()) return fail(EP_EINVAL, "%s", err.c_str());
  } catch (const std::bad_alloc&) {
    return fail(EP_ENOMEM, "out of host memory");
  }
  return EP_OK;
}

}  // namespace

// Asynchronous partition (the optimisation thread of Section 4.2).
struct ep_job {
  std::vector<int32_t> src, dst;  // private copies of the edge list
  int64_t m = 0, n = 0;
  int32_t C = 0, threads = 0;
  uint32_t flags = 0, test = 0;
  std::atomic<int> stop{0};
  std::mutex mu;
  std::condition_variable cv;
  bool done = false;  // guarded by mu, like the fields below
  int rc = EP_OK;
  std::string msg;
  ep_schedule* result = nullptr;
  double seconds = 0;
  std::thread th;
};

namespace {

constexpr int kHoldSeconds = 60;        // a held test job gives up after this long
constexpr int kLdgMaxPositions = 4096;  // 4 positions per thread, 1024 threads

void job_main(ep_job* j) {
  const auto t0 = std::chrono::steady_clock::now();
  int rc = EP_OK;
  std::string msg;
  ep_schedule* s = nullptr;
  if (j->test & EP_JOB_TEST_FAIL) {
    rc = EP_ENOMEM;
    msg = "injected failure";
  } else if (j->test & EP_JOB_TEST_HOLD) {
    std::unique_lock<std::mutex> lk(j->mu);
    const bool stop = j->cv.wait_for(lk, std::chrono::seconds(kHoldSeconds),
                                     [&] { return j->stop.load() != 0; });
    rc = stop ? EP_ECANCELED : EP_ETIMEOUT;
    msg = stop ? "partition cancelled" : "held test job timed out";
  } else if ((rc = new_schedule(nullptr, &s)) == EP_OK) {
    rc = fill_partition(s, j->src.data(), j->dst.data(), j->m, j->n, j->C, j->flags, j->threads,
                        &j->stop);
    if (rc != EP_OK) {
      delete s;
      s = nullptr;
    }
  }
  if (rc != EP_OK && msg.empty()) msg = g_error;
  {
    std::lock_guard<std::mutex> lk(j->mu);
    j->rc = rc;
    j->msg = msg;
    j->result = s;
    j->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    j->done = true;
  }
  j->cv.notify_all();
}

}  // namespace

extern "C" {

int ep_version(void) { return 100; }

const char* ep_last_error(void) { return g_error.c_str(); }

int ep_partition(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t C,
                 uint32_t flags, int32_t threads, ep_schedule** out) {
  g_error.clear();
  if (!out) return fail(EP_EINVAL, "null output pointer");
  *out = nullptr;
  if (int rc = check_edges(src, dst, m, n, C, flags)) return rc;
  ep_schedule* s = nullptr;
  if (int rc = new_schedule(out, &s)) return rc;
  if (int rc = fill_partition(s, src, dst, m, n, C, flags, threads, nullptr)) {
    delete s;
    return rc;
  }
  *out = s;
  return EP_OK;
}

int ep_partition_start(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, int32_t C,
                       uint32_t flags, int32_t threads, ep_job** out) {
  g_error.clear();
  if (!out) return fail(EP_EINVAL, "null output pointer");
  *out = nullptr;
  const uint32_t test = flags & (EP_JOB_TEST_FAIL | EP_JOB_TEST_HOLD);
  flags &= ~test;
  if (int rc = check_edges(src, dst, m, n, C, flags)) return rc;
  ep_job* j = new (std::nothrow) ep_job();
  if (!j) return fail(EP_ENOMEM, "out of host memory");
  try {
    j->src.assign(src, src + m);
    j->dst.assign(dst, dst + m);
    j->m = m;
    j->n = n;
    j->C = C;
    j->flags = flags;
    j->threads = threads;
    j->test = test;
    j->th = std::thread(job_main, j);
  } catch (const std::exception&) {
    delete j;
    return fail(EP_ENOMEM, "could not start the partition thread");
  }
  *out = j;
  return EP_OK;
}

int ep_job_wait(ep_job* j, int64_t timeout_ms, int32_t* done) {
  g_error.clear();
  if (!j || !done) return fail(EP_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(j->mu);
  if (timeout_ms < 0)
    j->cv.wait(lk, [&] { return j->done; });
  else if (timeout_ms > 0)
    j->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return j->done; });
  *done = j->done ? 1 : 0;
  return EP_OK;
}

int ep_job_take(ep_job* j, ep_schedule** out, double* seconds) {
  g_error.clear();
  if (!j || !out) return fail(EP_EINVAL, "null argument");
  *out = nullptr;
  std::lock_guard<std::mutex> lk(j->mu);
  if (!j->done) return fail(EP_EINVAL, "the partition job is still running");
  if (seconds) *seconds = j->seconds;
  if (j->rc != EP_OK) return fail(j->rc, "partition job: %s", j->msg.c_str());
  if (!j->result) return fail(EP_EINVAL, "the schedule was already taken");
  *out = j->result;
  j->result = nullptr;
  return EP_OK;
}

int ep_job_cancel(ep_job* j) {
  g_error.clear();
  if (!j) return fail(EP_EINVAL, "null job");
  {
    std::lock_guard<std::mutex> lk(j->mu);
    j->stop.store(1);
  }
  j->cv.notify_all();
  return EP_OK;
}

int ep_job_free(ep_job* j) {
  if (!j) return EP_OK;
  ep_job_cancel(j);
  if (j->th.joinable()) j->th.join();
  delete j->result;
  delete j;
  return EP_OK;
}

int ep_prescreen(const int32_t* src, const int32_t* dst, int64_t m, int64_t n, uint32_t flags,
                 ep_prescreen_info* out) {
  g_error.clear();
  if (!out) return fail(EP_EINVAL, "null output pointer");
  if (flags & ~EP_BIPARTITE) return fail(EP_EINVAL, "unknown flags");
  if (int rc = check_edges(src, dst, m, n, 1, flags)) return rc;
  try {
    const ep::PrescreenResult pr = ep::prescreen(src, dst, m, n, (flags & EP_BIPARTITE) != 0);
    out->touched = pr.touched;
    out->degree_sum = pr.degree_sum;
    out->max_degree = pr.max_degree;
    out->origin = pr.origin;
  } catch (const std::bad_alloc&) {
    return fail(EP_ENOMEM, "out of host memory");
  }
  return EP_OK;
}

int ep_schedule_origin(const ep_schedule* s, int32_t* origin) {
  g_error.clear();
  if (!s || !origin) return fail(EP_EINVAL, "null argument");
  *origin = s->h.origin;
  return EP_OK;
}

int ep_batch(ep_schedule* const* parts, int32_t count, ep_schedule** out) {
  g_error.clear();
  if (!out || !parts || count <= 0) return fail(EP_EINVAL, "bad batch arguments");
  *out = nullptr;
  int64_t m = 0, n = 0, k = 0;
  int32_t C = 0;
  const uint32_t flags = parts[0] ? parts[0]->h.flags : 0;
  for (int32_t i = 0; i < count; ++i) {
    if (!parts[i]) return fail(EP_EINVAL, "null part %d", i);
    if (parts[i]->h.flags != flags) return fail(EP_EINVAL, "parts differ in flags");
    m += parts[i]->h.m;
    n += parts[i]->h.n;
    k += parts[i]->h.k;
    C = std::max(C, parts[i]->h.C);
  }
  if (m >= INT32_MAX || n >= INT32_MAX / 2) return fail(EP_EINVAL, "batch too large");
  ep_schedule* s = nullptr;
  if (int rc = new_schedule(out, &s)) return rc;
  try {
    ep::HostSchedule& h = s->h;
    h.m = m;
    h.n = n;
    h.nd = (flags & EP_BIPARTITE) ? 2 * n : n;
    h.C = C;
    h.flags = flags & ~EP_DEFAULT_ORDER;
    h.k = k;
    h.src.reserve(m);
    h.dst.reserve(m);
    h.part.reserve(m);
    int64_t voff = 0, boff = 0;
    for (int32_t i = 0; i < count; ++i) {
      const ep::HostSchedule& p = parts[i]->h;
      for (int64_t e = 0; e < p.m; ++e) {
        h.src.push_back((int32_t)(p.src[e] + voff));
        h.dst.push_back((int32_t)(p.dst[e] + voff));
        h.part.push_back((int32_t)(p.part[e] + boff));
      }
      voff += p.n;
      boff += p.k;
    }
    std::string err = ep::build_schedule(h, 0);
    if (!err.empty()) {
      delete s;
      return fail(EP_EINVAL, "%s", err.c_str());
    }
  } catch (const std::bad_alloc&) {
    delete s;
    return fail(EP_ENOMEM, "out of host memory");
  }
  *out = s;
  return EP_OK;
}

void ep_schedule_free(ep_schedule* s) { delete s; }

int ep_schedule_info(const ep_schedule* s, int64_t* m, int64_t* n, int64_t* nd, int64_t* k,
                     int32_t* C, uint32_t* flags) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (m) *m = s->h.m;
  if (n) *n = s->h.n;
  if (nd) *nd = s->h.nd;
  if (k) *k = s->h.k;
  if (C) *C = s->h.C;
  if (flags) *flags = s->h.flags;
  return EP_OK;
}

int ep_schedule_arrays(const ep_schedule* s, const int64_t** block_ptr, const int32_t** edge_perm,
                       const int64_t** vert_ptr, const int32_t** vert_list, const int32_t** relabel) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (block_ptr) *block_ptr = s->h.block_ptr.data();
  if (edge_perm) *edge_perm = s->h.edge_perm.data();
  if (vert_ptr) *vert_ptr = s->h.vert_ptr.data();
  if (vert_list) *vert_list = s->h.vert_list.data();
  if (relabel) *relabel = s->h.relabel.data();
  return EP_OK;
}

int ep_cost_host(const ep_schedule* s, int64_t* loads, int64_t* vertex_cut) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (loads) *loads = s->h.loads;
  if (vertex_cut) *vertex_cut = s->h.loads - s->h.touched;
  return EP_OK;
}

int ep_cost(ep_schedule* s, int64_t* loads, int64_t* vertex_cut, void* stream) {
  g_error.clear();
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (int rc = ensure_device(s)) return rc;
  cudaStream_t st = as_stream(stream);
  CU(s->ws_flags.ensure((size_t)s->h.nd));
  CU(s->ws_cnt.ensure(2 * sizeof(unsigned long long)));
  ep::dev::CostArgs a;
  a.block_ptr = s->d_bptr.as<int64_t>();
  a.k = s->h.k;
  a.eu = s->d_eu.as<int32_t>();
  a.ev = s->d_ev.as<int32_t>();
  a.max_ne = s->h.max_ne;
  a.touched = s->ws_flags.as<uint8_t>();
  a.nd = s->h.nd;
  a.counters = s->ws_cnt.as<unsigned long long>();
  a.timer = s->t();
  CU(ep::dev::cost(a, st));
  unsigned long long c[2];
  CU(cudaMemcpyAsync(c, a.counters, sizeof c, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (loads) *loads = (int64_t)c[0];
  if (vertex_cut) *vertex_cut = (int64_t)c[0] - (int64_t)c[1];
  return EP_OK;
}

int32_t ep_record_floats(int32_t D) { return ep::record_floats(D); }

int64_t ep_layout_floats(const ep_schedule* s, int32_t D) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  return bipartite(s) ? s->h.n : s->h.n_rec * ep::record_floats(D);
}

int64_t ep_weights_floats(const ep_schedule* s) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  return wlen_of(s);
}

int ep_layout_in(ep_schedule* s, int32_t D, const float* x, float* x_lay, void* stream) {
  g_error.clear();
  if (int rc = check_flux(s, D)) return rc;
  if (!x || !x_lay) return fail(EP_EINVAL, "null argument");
  if (misaligned(x_lay)) return fail(EP_EINVAL, "schedule-layout buffers must be 16-byte aligned");
  if (int rc = ensure_device(s)) return rc;
  fresh_state(s);
  return layout_in_state(s, D, x, x_lay, as_stream(stream));
}

int ep_layout_out(ep_schedule* s, int32_t D, const float* x_lay, float* x, void* stream) {
  g_error.clear();
  if (int rc = check_flux(s, D)) return rc;
  if (!x || !x_lay) return fail(EP_EINVAL, "null argument");
  if (misaligned(x_lay)) return fail(EP_EINVAL, "schedule-layout buffers must be 16-byte aligned");
  if (int rc = ensure_device(s)) return rc;
  CU(ep::dev::layout_out(s->d_rec.as<int32_t>(), s->h.nd, s->h.n_rec, D, x_lay, x,
                         as_stream(stream), s->t()));
  return EP_OK;
}

int ep_weights_in(ep_schedule* s, const float* w, float* w_lay, void* stream) {
  g_error.clear();
  if (!s || !w || !w_lay) return fail(EP_EINVAL, "null argument");
  if (misaligned(w_lay)) return fail(EP_EINVAL, "schedule-layout buffers must be 16-byte aligned");
  if (int rc = ensure_device(s)) return rc;
  CU(ep::dev::gather(wmap_of(s), wlen_of(s), w, w_lay, as_stream(stream), s->t()));
  return EP_OK;
}

int ep_weights_out_add(ep_schedule* s, const float* w_lay, float* w, void* stream) {
  g_error.clear();
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (int rc = ensure_device(s)) return rc;
  if (bipartite(s))
    CU(ep::dev::scatter_add(wmap_of(s), wlen_of(s), w_lay, w, as_stream(stream), s->t()));
  else  // the source-side slot of every task holds its value
    CU(ep::dev::gather_add(s->d_gslot.as<int32_t>(), s->h.m, w_lay, w, as_stream(stream), s->t()));
  return EP_OK;
}

namespace {

int step_checks(ep_schedule* s, int32_t D, const void* a, const void* b, const void* c,
                const void* d) {
  if (int rc = check_flux(s, D)) return rc;
  if (!a || !b || !c) return fail(EP_EINVAL, "null argument");
  if (misaligned(a) || misaligned(b) || misaligned(c) || misaligned(d))
    return fail(EP_EINVAL, "schedule-layout buffers must be 16-byte aligned");
  return ensure_device(s);
}

// a forward step in schedule layout (ep_step, ep_step_pending)
int step_entry(ep_schedule* s, int32_t D, const float* x_in, float* x_out, const float* w_lay,
               float* out_lay, float tau, bool finish, cudaStream_t st) {
  if (int rc = ensure_bacc(s, D, st)) return rc;
  const int64_t t = s->h.n_run, nr = s->h.n_rec;
  if (nr > t) {
    // untouched records: zero flux, and the state carried over when out of place
    int32_t first[4], width[4];
    const int np = ep::planes_of(D, first, width);
    for (int k = 0; k < np; ++k) {
      const size_t off = (size_t)first[k] * nr + (size_t)t * width[k];
      const size_t bytes = (size_t)(nr - t) * width[k] * sizeof(float);
      if (out_lay) CU(cudaMemsetAsync(out_lay + off, 0, bytes, st));
      if (x_out != x_in)
        CU(cudaMemcpyAsync(x_out + off, x_in + off, bytes, cudaMemcpyDeviceToDevice, st));
    }
  }
  return flux_step_any(s, D, w_lay, x_in, x_out, out_lay, tau, finish, st);
}

}  // namespace

int ep_step(ep_schedule* s, int32_t D, const float* x_in, float* x_out, const float* w_lay,
            float* out_lay, float tau, void* stream) {
  g_error.clear();
  if (int rc = step_checks(s, D, x_in, x_out, w_lay, out_lay)) return rc;
  return step_entry(s, D, x_in, x_out, w_lay, out_lay, tau, true, as_stream(stream));
}

int ep_step_pending(ep_schedule* s, int32_t D, const float* x_in, float* x_out, const float* w_lay,
                    float tau, void* stream) {
  g_error.clear();
  if (int rc = step_checks(s, D, x_in, x_out, w_lay, nullptr)) return rc;
  return step_entry(s, D, x_in, x_out, w_lay, nullptr, tau, false, as_stream(stream));
}

int ep_finish(ep_schedule* s, int32_t D, float* x_lay, float tau, void* stream) {
  g_error.clear();
  if (int rc = step_checks(s, D, x_lay, x_lay, x_lay, nullptr)) return rc;
  cudaStream_t st = as_stream(stream);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  if (int rc = finish_any(s, kFwd, D, x_lay, x_lay, nullptr, tau, st)) return rc;
  s->pending[kFwd] = false;
  return EP_OK;
}

int ep_adjoint_step(ep_schedule* s, int32_t D, const float* x_lay, const float* w_lay, float* lam,
                    float* grad_w_lay, float tau, void* stream) {
  g_error.clear();
  if (int rc = step_checks(s, D, x_lay, w_lay, lam, grad_w_lay)) return rc;
  if (!grad_w_lay) return fail(EP_EINVAL, "null argument");
  cudaStream_t st = as_stream(stream);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  return flux_adj_any(s, D, w_lay, x_lay, lam, grad_w_lay, tau, true, st);
}

int ep_adjoint_step_pending(ep_schedule* s, int32_t D, const float* x_lay, const float* w_lay,
                            float* lam, float* grad_w_lay, float tau, void* stream) {
  g_error.clear();
  if (int rc = step_checks(s, D, x_lay, w_lay, lam, grad_w_lay)) return rc;
  if (!grad_w_lay) return fail(EP_EINVAL, "null argument");
  cudaStream_t st = as_stream(stream);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  return flux_adj_any(s, D, w_lay, x_lay, lam, grad_w_lay, tau, false, st);
}

int ep_adjoint_finish(ep_schedule* s, int32_t D, float* lam, float tau, void* stream) {
  g_error.clear();
  if (int rc = step_checks(s, D, lam, lam, lam, nullptr)) return rc;
  cudaStream_t st = as_stream(stream);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  if (int rc = finish_any(s, kAdj, D, lam, lam, nullptr, tau, st)) return rc;
  s->pending[kAdj] = false;
  return EP_OK;
}

namespace {
int run_flux(ep_schedule* s, int32_t D, int32_t steps, float tau, float* x, const float* w, float* out,
             bool from_host, cudaStream_t st);
}  // namespace

int ep_run(ep_schedule* s, int32_t kernel, float* x, const float* w, float* out, int32_t D,
           int32_t steps, float tau, void* stream) {
  g_error.clear();
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (!x || !w) return fail(EP_EINVAL, "null x or w");
  cudaStream_t st = as_stream(stream);
  if (kernel == EP_KERNEL_SPMV) {
    if (!bipartite(s)) return fail(EP_EINVAL, "SpMV needs a bipartite schedule");
    if (D != 1 || steps != 1) return fail(EP_EINVAL, "SpMV takes D = 1 and steps = 1");
    if (!out) return fail(EP_EINVAL, "SpMV needs an output vector");
    if (int rc = ensure_device(s)) return rc;
    return run_spmv(s, x, w, out, st);
  }
  if (kernel != EP_KERNEL_FLUX) return fail(EP_EINVAL, "unknown kernel %d", kernel);
  if (int rc = check_flux(s, D)) return rc;
  if (steps < 1) return fail(EP_EINVAL, "steps must be >= 1");
  if (int rc = ensure_device(s)) return rc;
  return run_flux(s, D, steps, tau, x, w, out, false, st);
}

namespace {

// ep_run's flux part: x, w and out in the caller's layout, device addresses.
// from_host: x and w are read in vertex / task order (host memory the GPU
// reads over the host link).
int run_flux(ep_schedule* s, int32_t D, int32_t steps, float tau, float* x, const float* w, float* out,
             bool from_host, cudaStream_t st) {
  const ep::HostSchedule& h = s->h;
  const int32_t R = ep::record_floats(D);
  const size_t lay = (size_t)h.n_rec * R * sizeof(float);
  CU(s->ws_x.ensure(lay));
  if (out) {
    CU(s->ws_out.ensure(lay));
  }
  fresh_state(s);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  if (s->zeroed_x != s->ws_x.p) {  // records of no vertex stay zero
    CU(cudaMemsetAsync(s->ws_x.p, 0, s->ws_x.bytes, st));
    s->zeroed_x = s->ws_x.p;
  }
  if (int rc = layout_in_state(s, D, x, s->ws_x.as<float>(), st)) return rc;
  if (int rc = weights_to_ws(s, w, from_host, st)) return rc;
  if (out) CU(cudaMemsetAsync(s->ws_out.p, 0, lay, st));
  // the shared copies stay pending between steps; the last step finishes them
  for (int32_t t = 0; t < steps; ++t) {
    const bool last = t == steps - 1;
    float* o = (out && last) ? s->ws_out.as<float>() : nullptr;
    if (int rc = flux_step_any(s, D, s->ws_w.as<float>(), s->ws_x.as<float>(), s->ws_x.as<float>(), o,
                               tau, last, st))
      return rc;
  }
  CU(ep::dev::layout_out(s->d_rec.as<int32_t>(), h.nd, h.n_rec, D, s->ws_x.as<float>(), x, st, s->t()));
  if (out) CU(ep::dev::layout_out(s->d_rec.as<int32_t>(), h.nd, h.n_rec, D, s->ws_out.as<float>(), out, st, s->t()));
  return EP_OK;
}

}  // namespace

int ep_run_host(ep_schedule* s, int32_t kernel, float* x, const float* w, float* out, int32_t D,
                int32_t steps, float tau, void* stream) {
  g_error.clear();
  if (!s || !x || !w) return fail(EP_EINVAL, "null argument");
  if (D < 1 || D > EP_MAX_D) return fail(EP_EINVAL, "D out of range");
  if (int rc = ensure_device(s)) return rc;
  cudaStream_t st = as_stream(stream);
  const ep::HostSchedule& h = s->h;
  // pinned host buffers: the layout kernels read x and w and write the
  // results over the host link themselves, with no staging copy in between
  float* dx = const_cast<float*>(static_cast<const float*>(host_mapped(x)));
  const float* dw = static_cast<const float*>(host_mapped(w));
  float* dout = out ? const_cast<float*>(static_cast<const float*>(host_mapped(out))) : nullptr;
  if (dx && dw && (!out || dout)) {
    int rc;
    if (kernel == EP_KERNEL_SPMV) {
      if (!bipartite(s)) return fail(EP_EINVAL, "SpMV needs a bipartite schedule");
      if (D != 1 || steps != 1) return fail(EP_EINVAL, "SpMV takes D = 1 and steps = 1");
      if (!out) return fail(EP_EINVAL, "SpMV needs an output vector");
      rc = run_spmv(s, dx, dw, dout, st, true);
    } else if (kernel == EP_KERNEL_FLUX) {
      if ((rc = check_flux(s, D))) return rc;
      if (steps < 1) return fail(EP_EINVAL, "steps must be >= 1");
      rc = run_flux(s, D, steps, tau, dx, dw, dout, true, st);
    } else {
      return fail(EP_EINVAL, "unknown kernel %d", kernel);
    }
    if (rc) return rc;
    CU(cudaStreamSynchronize(st));
    return EP_OK;
  }
  // other host memory: staged through device buffers by the copy engines
  const size_t xb = (size_t)(kernel == EP_KERNEL_SPMV ? h.n : h.n * D) * sizeof(float);
  CU(s->ws_hx.ensure(xb));
  CU(s->ws_hw.ensure((size_t)h.m * sizeof(float)));
  if (out) CU(s->ws_hout.ensure(xb));
  CU(cudaMemcpyAsync(s->ws_hx.p, x, xb, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(s->ws_hw.p, w, (size_t)h.m * sizeof(float), cudaMemcpyHostToDevice, st));
  int rc = ep_run(s, kernel, s->ws_hx.as<float>(), s->ws_hw.as<float>(),
                  out ? s->ws_hout.as<float>() : nullptr, D, steps, tau, stream);
  if (rc) return rc;
  if (kernel != EP_KERNEL_SPMV) CU(cudaMemcpyAsync(x, s->ws_hx.p, xb, cudaMemcpyDeviceToHost, st));
  if (out) CU(cudaMemcpyAsync(out, s->ws_hout.p, xb, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return EP_OK;
}

int ep_run_adjoint(ep_schedule* s, const float* x0, const float* w, float* lam, float* grad_w,
                   int32_t D, int32_t steps, float tau, void* stream) {
  g_error.clear();
  if (int rc = check_flux(s, D)) return rc;
  if (!x0 || !w || !lam || !grad_w) return fail(EP_EINVAL, "null argument");
  if (steps < 1) return fail(EP_EINVAL, "steps must be >= 1");
  if (int rc = ensure_device(s)) return rc;
  cudaStream_t st = as_stream(stream);
  const ep::HostSchedule& h = s->h;
  const int32_t R = ep::record_floats(D);
  const size_t lay = (size_t)h.n_rec * R;
  CU(s->ws_hist.ensure(lay * steps * sizeof(float)));
  CU(s->ws_lam.ensure(lay * sizeof(float)));
  CU(s->ws_w.ensure((size_t)wlen_of(s) * sizeof(float)));
  CU(s->ws_gw.ensure((size_t)wlen_of(s) * sizeof(float)));
  fresh_state(s);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  float* hist = s->ws_hist.as<float>();
  if (int rc = layout_in_state(s, D, x0, hist, st)) return rc;
  CU(ep::dev::gather(wmap_of(s), wlen_of(s), w, s->ws_w.as<float>(), st, s->t()));
  CU(cudaMemsetAsync(s->ws_gw.p, 0, (size_t)wlen_of(s) * sizeof(float), st));
  // the recomputed states are read whole by the adjoint: finish every one
  for (int32_t t = 0; t + 1 < steps; ++t)
    if (int rc = flux_step_any(s, D, s->ws_w.as<float>(), hist + lay * t, hist + lay * (t + 1), nullptr,
                               tau, true, st))
      return rc;
  if (int rc = layout_in_state(s, D, lam, s->ws_lam.as<float>(), st)) return rc;
  // the cotangent's shared copies stay pending between adjoint steps
  for (int32_t t = steps - 1; t >= 0; --t)
    if (int rc = flux_adj_any(s, D, s->ws_w.as<float>(), hist + lay * t, s->ws_lam.as<float>(),
                              s->ws_gw.as<float>(), tau, t == 0, st))
      return rc;
  CU(ep::dev::layout_out(s->d_rec.as<int32_t>(), h.nd, h.n_rec, D, s->ws_lam.as<float>(), lam, st, s->t()));
  CU(ep::dev::gather_add(s->d_gslot.as<int32_t>(), h.m, s->ws_gw.as<float>(), grad_w, st, s->t()));
  return EP_OK;
}

int ep_timing(ep_schedule* s, int32_t enable) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (enable == 2) s->timer.clear();
  s->timer.on = enable != 0;
  return EP_OK;
}

int ep_timing_read(ep_schedule* s, int32_t kernel_class, double* total_ms, int64_t* launches) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (kernel_class < 0 || kernel_class >= EP_T_CLASSES) return fail(EP_EINVAL, "bad kernel class");
  s->timer.collect();
  if (total_ms) *total_ms = s->timer.total[kernel_class];
  if (launches) *launches = s->timer.count[kernel_class];
  return EP_OK;
}

int check_spmv(ep_schedule* s) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (!bipartite(s)) return fail(EP_EINVAL, "SpMV needs a bipartite schedule");
  return ensure_device(s);
}

int ep_spmv_x_in(ep_schedule* s, const float* x, float* x_lay, void* stream) {
  g_error.clear();
  if (int rc = check_spmv(s)) return rc;
  if (!x || !x_lay) return fail(EP_EINVAL, "null argument");
  CU(ep::dev::layout_in(s->d_xrec.as<int32_t>(), s->h.n, s->h.n, 1, x, x_lay, as_stream(stream), s->t()));
  return EP_OK;
}

int ep_spmv_y_out(ep_schedule* s, const float* y_lay, float* y, void* stream) {
  g_error.clear();
  if (int rc = check_spmv(s)) return rc;
  if (!y || !y_lay) return fail(EP_EINVAL, "null argument");
  CU(ep::dev::layout_out(s->d_yrec.as<int32_t>(), s->h.n, s->h.n, 1, y_lay, y, as_stream(stream), s->t()));
  return EP_OK;
}

int ep_spmv(ep_schedule* s, const float* x_lay, const float* w_lay, float* y_lay, void* stream) {
  g_error.clear();
  if (int rc = check_spmv(s)) return rc;
  if (!x_lay || !w_lay || !y_lay) return fail(EP_EINVAL, "null argument");
  if (misaligned(x_lay) || misaligned(w_lay) || misaligned(y_lay))
    return fail(EP_EINVAL, "schedule-layout buffers must be 16-byte aligned");
  return spmv_lay(s, x_lay, w_lay, y_lay, as_stream(stream));
}

int ep_set_pipeline(ep_schedule* s, int32_t stages) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (stages < 0 || stages == 1 || stages > ep::dev::kMaxStages)
    return fail(EP_EINVAL, "stages = %d (0, or 2..%d)", stages, ep::dev::kMaxStages);
  s->stages = stages;
  return EP_OK;
}

int ep_pipeline_info(ep_schedule* s, int32_t D, int32_t adjoint, int32_t* grid, int32_t* per_sm,
                     int32_t* threads, int32_t* stages, int32_t* stage_bytes) {
  g_error.clear();
  if (int rc = check_flux(s, D)) return rc;
  if (int rc = ensure_device(s)) return rc;
  int32_t g = 0, p = 0, t = 0, st = 0, sb = 0;
  if (s->stages != 0) {
    ep::dev::TmaPlan P;
    if (int rc = tma_plan(s, D, adjoint != 0, P)) return rc;
    if (P.fits) g = P.grid, p = P.per_sm, t = P.threads, st = P.L.stages, sb = P.L.stage_bytes;
  }
  if (grid) *grid = g;
  if (per_sm) *per_sm = p;
  if (threads) *threads = t;
  if (stages) *stages = st;
  if (stage_bytes) *stage_bytes = sb;
  return EP_OK;
}

int ep_check_errors(ep_schedule* s, int32_t* code, void* stream) {
  g_error.clear();
  if (!s || !code) return fail(EP_EINVAL, "null argument");
  *code = 0;
  if (!s->ws_ctl.p) return EP_OK;
  int v = 0;
  cudaStream_t st = as_stream(stream);
  CU(cudaMemcpyAsync(&v, s->ws_ctl.as<int>() + 2, sizeof v, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *code = v;
  if (v) {
    CU(cudaMemsetAsync(s->ws_ctl.as<int>() + 2, 0, sizeof(int), st));
    s->bacc_dirty = true;  // an interrupted launch may have left partial sums
    return fail(EP_ETIMEOUT, "a pipelined kernel gave up waiting (code %d)", v);
  }
  return EP_OK;
}

int ep_set_cache(ep_schedule* s, int32_t mode) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (mode != EP_CACHE_SMEM && mode != EP_CACHE_L1) return fail(EP_EINVAL, "cache mode %d", mode);
  if (mode == EP_CACHE_L1 && !bipartite(s) && s->h.max_nv > kLdgMaxPositions)
    return fail(EP_EINVAL, "a block has %d positions; the read-only-cache kernel takes at most %d",
                s->h.max_nv, kLdgMaxPositions);
  s->cache = mode;
  return EP_OK;
}

int ep_debug_stall(ep_schedule* s, int32_t block_index) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (block_index < -1 || block_index > 255) return fail(EP_EINVAL, "block_index = %d", block_index);
  s->stall = block_index;
  return EP_OK;
}

int ep_set_threads(ep_schedule* s, int32_t threads) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (threads < 32 || threads > 1024 || threads % 32) return fail(EP_EINVAL, "threads = %d", threads);
  s->tpb = threads;
  return EP_OK;
}

int ep_set_halo(ep_schedule* s, const int32_t* halo, int64_t nh) {
  g_error.clear();
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (bipartite(s)) return fail(EP_EINVAL, "a halo applies to flux schedules only");
  if (nh < 0 || (nh > 0 && !halo)) return fail(EP_EINVAL, "null or negative halo list");
  ep::HostSchedule& h = s->h;
  for (int64_t i = 0; i < nh; ++i)
    if (halo[i] < 0 || halo[i] >= h.nd) return fail(EP_EINVAL, "halo vertex %d out of range", halo[i]);
  h.halo.assign(halo, halo + nh);
  const std::string err = ep::rebuild_flux_layout(h);
  if (!err.empty()) return fail(EP_EINVAL, "%s", err.c_str());
  // shared id of every shared vertex's data vertex, then of every halo vertex
  std::vector<int32_t> sid_of(h.nd, -1);
  for (int64_t sh = 0; sh < h.n_sh; ++sh) sid_of[h.vrec[h.crec[h.cptr[sh]]]] = (int32_t)sh;
  s->hmap.resize(nh);
  for (int64_t i = 0; i < nh; ++i) s->hmap[i] = sid_of[halo[i]];
  // the layout changed: upload again, new plans, new accumulators, new maps
  s->device = -1;
  for (auto& row : s->plan_key)
    for (int& k : row) k = 0;
  s->pending[0] = s->pending[1] = false;
  s->bacc_dirty = true;
  s->host_maps = false;
  s->zeroed_x = s->zeroed_w = nullptr;
  return EP_OK;
}

namespace {
int halo_move_entry(ep_schedule* s, int32_t D, float* buf, bool pack, void* stream) {
  g_error.clear();
  if (int rc = check_flux(s, D)) return rc;
  if (s->hmap.empty()) return EP_OK;
  if (!buf) return fail(EP_EINVAL, "null buffer");
  if (int rc = ensure_device(s)) return rc;
  cudaStream_t st = as_stream(stream);
  if (int rc = ensure_bacc(s, D, st)) return rc;
  ep::dev::FluxArgs a = flux_args(s, kFwd, nullptr, nullptr, nullptr, nullptr, 0.f);
  CU(ep::dev::halo_move(a, D, s->d_hmap.as<int32_t>(), (int64_t)s->hmap.size(), buf, pack, st));
  return EP_OK;
}
}  // namespace

int ep_halo_pack(ep_schedule* s, int32_t D, float* buf, void* stream) {
  return halo_move_entry(s, D, buf, true, stream);
}

int ep_halo_unpack(ep_schedule* s, int32_t D, const float* buf, void* stream) {
  return halo_move_entry(s, D, const_cast<float*>(buf), false, stream);
}

int ep_set_adjoint_threads(ep_schedule* s, int32_t threads) {
  if (!s) return fail(EP_EINVAL, "null schedule");
  if (threads < 32 || threads > 1024 || threads % 32) return fail(EP_EINVAL, "threads = %d", threads);
  s->tpb_adj = threads;
  return EP_OK;
}

}  // extern "C"
