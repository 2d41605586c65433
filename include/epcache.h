/*
 * epcache.h -- C ABI of libepcache: edge-partitioned gather/interact/scatter
 * kernels for GB300 (sm_103a).
 *
 * Method: "A Graph-based Model for GPU Caching Problems" (Li et al.).  Data
 * objects are vertices and tasks are edges of a data-affinity graph (Section
 * 3.1, Definition 1).  Tasks are split into blocks of capacity C so that the
 * number of distinct vertices each block touches, summed over blocks, is small
 * (Eq. 1), by the clone-and-connect transform, a balanced vertex partition and
 * the reconstruction of Definition 4 (Section 3.2).  Each CUDA thread block
 * then stages its block's distinct vertices in shared memory once (Section 4,
 * the software-cache kernel) and scatters its results back.
 *
 * Conventions for every call:
 *   - return value 0 (EP_OK) or a negative EP_E* code; ep_last_error() gives
 *     a message for the calling thread;
 *   - arrays named "host" are read during the call only and stay owned by the
 *     caller; device pointers are caller-owned CUDA global memory on the
 *     current device; the library never frees caller memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is enqueued on it and the call returns without
 *     synchronising unless stated otherwise.  The edge kernels and the
 *     finish of pending shared copies are launched with programmatic stream
 *     serialisation and wait for the preceding kernel's completion before
 *     touching memory; a caller kernel placed just before them that signals
 *     its dependents early (griddepcontrol.launch_dependents) must have
 *     written its results by then;
 *   - a schedule owns its host arrays, its device copy and its device
 *     workspace.  Calls on one schedule must not overlap in time (they share
 *     that workspace); distinct schedules are independent.
 *   - there is no CPU fallback: kernel calls return EP_ENODEV without a CUDA
 *     device.
 */
#ifndef EPCACHE_H
#define EPCACHE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EP_OK 0
#define EP_EINVAL (-1)   /* bad argument (sizes, ids out of range, flags) */
#define EP_ENOMEM (-2)   /* host or device allocation failed */
#define EP_ECUDA (-3)    /* a CUDA runtime call failed (message has details) */
#define EP_ETIMEOUT (-4) /* a bounded wait expired (device kernel or host thread) */
#define EP_ENODEV (-5)   /* no CUDA device */
#define EP_ECANCELED (-6) /* an asynchronous partition job was cancelled */

/* ep_partition flags */
#define EP_BIPARTITE 1u     /* SpMV graph: x_j -> vertex j, y_i -> vertex n+i */
#define EP_DEFAULT_ORDER 2u /* no partitioning: C consecutive tasks per block */
#define EP_PRESCREEN 4u     /* run ep_prescreen first and follow its outcome */

/* kernels */
#define EP_KERNEL_FLUX 0 /* f = w (x_v - x_u)/(1+|x_v - x_u|^2); out_u += f, out_v -= f */
#define EP_KERNEL_SPMV 1 /* y_u += w x_v on a bipartite schedule (u = row, v = col) */

#define EP_MAX_D 8       /* state width limit for the flux kernels */
#define EP_MAX_C 16384   /* block capacity limit (local indices are 16-bit) */

typedef struct ep_schedule ep_schedule; /* opaque, library-owned */
typedef struct ep_job ep_job;           /* opaque: an asynchronous partition */

/* Library version (major*10000 + minor*100 + patch). */
int ep_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *ep_last_error(void);

/*
 * Balanced edge partition (Section 3.1 Eq. 1; Section 3.2 Definitions 3-4).
 *   src, dst  host int32[m]: task e uses data objects src[e] and dst[e],
 *             both in [0, n).  Task id = position.  Self loops use one object;
 *             repeated pairs stay separate tasks.  With EP_BIPARTITE the task
 *             is the nonzero A[src[e]][dst[e]] of an n x n matrix and touches
 *             x_{dst[e]} (vertex dst[e]) and y_{src[e]} (vertex n + src[e]).
 *   C         block capacity in tasks, 1 <= C <= EP_MAX_C; k = ceil(m/C)
 *             blocks, every block holds exactly C tasks except the last.
 *   flags     EP_BIPARTITE, EP_DEFAULT_ORDER, EP_PRESCREEN.
 *   threads   host threads for the recursion (<= 0: all hardware threads).
 *   out       receives a new schedule; free it with ep_schedule_free().
 * The result is deterministic and independent of `threads`.  Host-only: runs
 * without a GPU.  EP_EINVAL for m <= 0, m >= 2^31, n <= 0, ids out of range or
 * C out of range.
 */
int ep_partition(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int32_t C,
                 uint32_t flags, int32_t threads, ep_schedule **out);

/*
 * Asynchronous partition: the optimisation thread of Section 4.2, which
 * partitions while the application keeps running its kernel under the
 * default schedule, and is stopped if the application ends first.
 * ep_partition_start checks its arguments like ep_partition, copies src and
 * dst (the caller may free them on return) and starts one host thread that
 * runs ep_partition on the copies; the result is bit-identical to
 * ep_partition's.  Test hooks (host-side fault injection, no GPU involved):
 * flags | EP_JOB_TEST_FAIL makes the job fail at once with EP_ENOMEM;
 * flags | EP_JOB_TEST_HOLD makes it do nothing until cancelled (after 60 s
 * it ends by itself with EP_ETIMEOUT).
 *   ep_job_wait    waits up to timeout_ms (0: poll, < 0: no limit); *done = 1
 *                  once the job has ended (finished, failed or cancelled).
 *   ep_job_take    after the end: hands over the schedule (*out, to be freed
 *                  with ep_schedule_free) and the job's wall time in seconds
 *                  (*seconds, may be NULL); returns the job's own error code
 *                  (EP_ECANCELED, EP_ENOMEM, ...) if it failed, EP_EINVAL if
 *                  it is still running or the schedule was already taken.
 *   ep_job_cancel  asks the job to stop; the partitioner checks the request
 *                  between coarsening levels and between bisections, so the
 *                  job ends soon after with EP_ECANCELED.
 *   ep_job_free    cancels, joins the thread and frees everything not taken.
 * A job may be waited on from several threads; ep_job_free must be the last
 * call on it.
 */
#define EP_JOB_TEST_FAIL 0x100u
#define EP_JOB_TEST_HOLD 0x200u
int ep_partition_start(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int32_t C,
                       uint32_t flags, int32_t threads, ep_job **out);
int ep_job_wait(ep_job *job, int64_t timeout_ms, int32_t *done);
int ep_job_take(ep_job *job, ep_schedule **out, double *seconds);
int ep_job_cancel(ep_job *job);
int ep_job_free(ep_job *job);

/*
 * Pre-screen (Section 4, the optimisation workflow): look at the graph before
 * partitioning it.  Host-only.  Degrees count the tasks that use a data
 * vertex (a self loop once).  The outcome, in this order:
 *   EP_ORIGIN_PATH      the tasks form one simple path: preset schedule that
 *                       walks the path from its smaller-id end and cuts it every
 *                       C tasks; it loads m + k vertices, the optimum of Eq. 1
 *                       (C path edges touch at least C + 1 vertices).
 *   EP_ORIGIN_STAR      every task uses one centre and a leaf of its own: every
 *                       schedule loads m + k, so the default order is kept.
 *   EP_ORIGIN_LOW_REUSE mean degree of the touched vertices <= 2 (little
 *                       data reuse): the default order is kept.
 *   EP_ORIGIN_PARTITION otherwise: partition.
 * The paper names the checks but neither their thresholds nor its preset
 * schedules; these are this library's (the path and star presets are
 * optimal, the reuse threshold is the paper's own remark that a mean degree
 * of at most 2 leaves little sharing).  flags: EP_BIPARTITE only.
 * ep_partition with EP_PRESCREEN applies the outcome; ep_schedule_origin()
 * tells how a schedule's order was chosen (EP_ORIGIN_DEFAULT: asked for with
 * EP_DEFAULT_ORDER).
 */
#define EP_ORIGIN_PARTITION 0
#define EP_ORIGIN_DEFAULT 1
#define EP_ORIGIN_PATH 2
#define EP_ORIGIN_STAR 3
#define EP_ORIGIN_LOW_REUSE 4
typedef struct {
  int64_t touched;    /* data vertices used by at least one task */
  int64_t degree_sum; /* sum of their degrees */
  int64_t max_degree;
  int32_t origin;     /* the outcome, EP_ORIGIN_* */
  int32_t pad;
} ep_prescreen_info;
int ep_prescreen(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, uint32_t flags,
                 ep_prescreen_info *out);
int ep_schedule_origin(const ep_schedule *s, int32_t *origin);

/* Sizes of a schedule.  nd = number of data vertices (n, or 2n if bipartite).
 * Any output pointer may be NULL. */
int ep_schedule_info(const ep_schedule *s, int64_t *m, int64_t *n, int64_t *nd, int64_t *k,
                     int32_t *C, uint32_t *flags);

/*
 * Borrowed host views of a schedule (valid until ep_schedule_free):
 *   block_ptr[k+1]   tasks of block b are edge_perm[block_ptr[b] .. block_ptr[b+1])
 *   edge_perm[m]     task ids grouped by block, ascending within a block (Def. 4)
 *   vert_ptr[k+1]    vertices of block b are vert_list[vert_ptr[b] .. vert_ptr[b+1])
 *   vert_list[L]     distinct vertices per block in first-touch order (task
 *                    order, endpoint src-side then dst-side); L = loads
 *   relabel[nd]      cpack id of every data vertex (Section 4.1): order of first
 *                    appearance over blocks 0..k-1, untouched vertices last
 * Any output pointer may be NULL.
 */
int ep_schedule_arrays(const ep_schedule *s, const int64_t **block_ptr, const int32_t **edge_perm,
                       const int64_t **vert_ptr, const int32_t **vert_list,
                       const int32_t **relabel);

/* Host-side cost (Eq. 1): loads = sum_b |V_b|, vertex_cut = sum_v (p_v - 1). */
int ep_cost_host(const ep_schedule *s, int64_t *loads, int64_t *vertex_cut);

/*
 * GPU cost (Section 3.1, Definition 2 and Eq. 1): one CUDA block per schedule
 * block sorts that block's 2|block| endpoint ids in shared memory, counts the
 * distinct ones and marks touched vertices; loads = sum_b |V_b| and
 * vertex_cut = loads - #touched.  Uploads the schedule on first use.
 * Synchronises `stream` (the results are host values).
 */
int ep_cost(ep_schedule *s, int64_t *loads, int64_t *vertex_cut, void *stream);

/*
 * Forward run in the caller's layout (device pointers).  The edge kernel is the
 * software-cache kernel of Section 4 (Fig. 7(d)) run under the schedule of
 * Section 3.2; the flux interaction is the particle kernel of the cfd example
 * of Section 1, SpMV the y = A x of Section 5.2 on the bipartite graph of
 * Definition 1.  The explicit time step x <- x + tau*flux has no counterpart
 * in the paper: it is this library's workload definition.
 *   EP_KERNEL_FLUX: x float[D][n] (in: x_0, out: x_T), w float[m] (task
 *     order), out float[D][n] or NULL (receives flux(x_{T-1})), 1 <= D <=
 *     EP_MAX_D, steps = T >= 1 explicit steps x_{t+1} = x_t + tau*flux(x_t).
 *     With tau = 0, x is unchanged and out = flux(x).
 *   EP_KERNEL_SPMV (bipartite schedule): x float[n] (read), w float[m],
 *     out float[n] = y (written), D = 1, steps = 1, tau ignored.
 * Uses schedule-owned device workspace (allocated on first use: make the
 * first call before any stream capture).  Every kernel stages a whole
 * schedule block in shared memory: EP_EINVAL (nothing launched) when the
 * largest block does not fit, i.e. C too large for the graph and D (for
 * D = 5 on mesh-like graphs, C up to a few thousand tasks fits).
 */
int ep_run(ep_schedule *s, int32_t kernel, float *x, const float *w, float *out, int32_t D,
           int32_t steps, float tau, void *stream);

/*
 * No counterpart in the paper (a host-buffer convenience of this library).
 * Same as ep_run with HOST pointers (x in/out, w in, out optional); returns
 * after the results are in host memory (synchronises the stream).  When all
 * of x, w (and out) are pinned through CUDA (cudaHostAlloc, cudaHostRegister,
 * a pinned torch tensor), the layout kernels read x in vertex order and w in
 * task order straight over the host link and write the results back the same
 * way, with no staging copy; any other host memory is staged through device
 * buffers with cudaMemcpyAsync.  The buffers must not be touched by the host
 * until the call returns.
 */
int ep_run_host(ep_schedule *s, int32_t kernel, float *x, const float *w, float *out, int32_t D,
                int32_t steps, float tau, void *stream);

/*
 * No counterpart in the paper: the reverse-mode derivative of the explicit
 * flux steps for a linear loss L = <g, x_T> (lam = g on entry), this library's
 * training pattern.  It runs over the same schedule and with the same access
 * pattern as the forward kernel of Section 4.
 * Reverse sweep of `steps` flux steps started from x0 (device, float[D][n],
 * caller layout): recomputes x_0..x_{T-1} into workspace, then for t = T-1..0
 *   gbar_e = lam_u - lam_v, d = x_v - x_u, s = |d|^2,
 *   grad_w[e] += tau <gbar_e, d>/(1+s),
 *   lam += tau * scatter(+h_e to v, -h_e to u),
 *   h_e = w_e (gbar_e/(1+s) - 2 d (d.gbar_e)/(1+s)^2).
 * lam float[D][n]: in dL/dx_T, out dL/dx_0.  grad_w float[m]: accumulated.
 */
int ep_run_adjoint(ep_schedule *s, const float *x0, const float *w, float *lam, float *grad_w,
                   int32_t D, int32_t steps, float tau, void *stream);

/* ----------------------------------------------------- schedule layout API
 * The kernels work on the schedule's own layout (the paper's opt_arrayA,
 * Section 4.1, rearranged for bulk copies): for every kernel block, in block
 * order, one contiguous run of state records holding first the vertices that
 * only this block uses, then the block's own copy of every shared vertex it
 * uses (a shared vertex has one record per block that uses it; all copies
 * hold the same value between calls); the untouched vertices follow.  The D
 * components of every record are split into planes of width 4, 2 and 1
 * (D = 4a + 2b + c): plane k is a contiguous array of n_rec records of its
 * width, so a buffer is n_rec * D floats.  Flux schedules (the forward
 * kernels read every task from both of its endpoints) keep one weight per
 * incidence slot, two per task; SpMV schedules one per task.  Keeping state
 * in this layout across calls avoids the permutations.
 */
int32_t ep_record_floats(int32_t D);
/* Floats needed for one state buffer in schedule layout (n_records * D). */
int64_t ep_layout_floats(const ep_schedule *s, int32_t D);
/* x_lay <- x (caller layout float[D][n]); every copy of a shared vertex is
 * written, padding records get 0. */
int ep_layout_in(ep_schedule *s, int32_t D, const float *x, float *x_lay, void *stream);
/* x <- x_lay (caller layout float[D][n]). */
int ep_layout_out(ep_schedule *s, int32_t D, const float *x_lay, float *x, void *stream);
/* Floats of a task-weight buffer in schedule layout: flux schedules one slot
 * per task endpoint (sliced per block, see ep_step), SpMV schedules the tasks
 * in edge_perm order; every block's run starts on a 16-byte boundary. */
int64_t ep_weights_floats(const ep_schedule *s);
/* w_lay <- w permuted into schedule layout: every slot of a task gets its
 * weight, padding slots get 0. */
int ep_weights_in(ep_schedule *s, const float *w, float *w_lay, void *stream);
/* w[task] += w_lay[slot] for every task, from one slot per task: its only
 * slot (SpMV), or the slot at its first endpoint (flux), which is where
 * ep_adjoint_step accumulates the weight gradient. */
int ep_weights_out_add(ep_schedule *s, const float *w_lay, float *w, void *stream);

/*
 * One explicit flux step in schedule layout: x_out = x_in + tau*flux(x_in)
 * (x_out may equal x_in), out_lay = flux(x_in) if not NULL.  Two kernel
 * launches: the edge kernel updates the vertices only one kernel block uses
 * in place and adds the partial flux of the shared ones into schedule-owned
 * accumulators; the finish then writes x + tau * flux to every copy of each
 * shared vertex.
 */
int ep_step(ep_schedule *s, int32_t D, const float *x_in, float *x_out, const float *w_lay,
            float *out_lay, float tau, void *stream);

/*
 * No counterpart in the paper (a launch-saving form of ep_step for loops of
 * many steps).  Between two steps only the vertices used by one kernel block
 * need their new value in memory; the copies of a shared vertex can wait:
 * ep_step_pending makes one explicit step like ep_step but leaves the shared
 * copies of x_out one step behind (pending) and launches only the edge kernel;
 * the next step (ep_step or ep_step_pending, which accept a pending input)
 * brings them up to date as it stages them, and ep_finish brings them up to
 * date in memory.  x_out is a valid state only after ep_finish (or after an
 * ep_step).  The pending sums live in the schedule's accumulators: finish a
 * pending state before starting another one on the same schedule
 * (ep_layout_in and ep_run discard sums still pending).  tau of ep_finish must
 * be the last step's.  Launches inside a stream capture replay correctly for
 * any number of steps.
 */
int ep_step_pending(ep_schedule *s, int32_t D, const float *x_in, float *x_out, const float *w_lay,
                    float tau, void *stream);
int ep_finish(ep_schedule *s, int32_t D, float *x_lay, float tau, void *stream);

/*
 * SpMV in schedule layout (bipartite schedules, Section 5.2): y_lay = A x_lay
 * with x_lay over column records and y_lay over row records (n floats each,
 * ep_spmv_x_in / ep_spmv_y_out permute), w_lay from ep_weights_in.  One
 * warp per schedule block: the block's x entries are staged in shared memory
 * (the software cache), its row-ranked entries are split into equal chunks,
 * one per lane, whatever the row lengths, and rows that cross chunk ends are
 * joined by a segmented scan over the warp.  Rows used by one block are
 * stored, rows shared by blocks accumulated with atomics after zeroing.
 * Buffers 16-byte aligned (EP_EINVAL otherwise); EP_EINVAL when one warp's
 * staged x and row totals of the largest block do not fit in shared memory.
 */
int ep_spmv_x_in(ep_schedule *s, const float *x, float *x_lay, void *stream);
int ep_spmv_y_out(ep_schedule *s, const float *y_lay, float *y, void *stream);
int ep_spmv(ep_schedule *s, const float *x_lay, const float *w_lay, float *y_lay, void *stream);

/*
 * One adjoint step in schedule layout: lam (in lam_{t+1}, out lam_t) and
 * grad_w_lay += per-task terms, evaluated at state x_lay = x_t.
 */
int ep_adjoint_step(ep_schedule *s, int32_t D, const float *x_lay, const float *w_lay, float *lam,
                    float *grad_w_lay, float tau, void *stream);

/*
 * No counterpart in the paper: ep_adjoint_step with the shared copies of lam
 * left pending, and their finish (the same scheme as ep_step_pending and
 * ep_finish, with accumulators of their own; x_lay must be a finished state).
 */
int ep_adjoint_step_pending(ep_schedule *s, int32_t D, const float *x_lay, const float *w_lay,
                            float *lam, float *grad_w_lay, float tau, void *stream);
int ep_adjoint_finish(ep_schedule *s, int32_t D, float *lam, float tau, void *stream);

/*
 * No counterpart in the paper (a build-side pattern of this library): the
 * union of balanced edge partitions of disjoint affinity graphs (Definition 1)
 * is an edge partition of their union, and its cost (Eq. 1) is the sum of the
 * parts' costs, so many small graphs can share one launch.
 * Merge independent schedules (disjoint graphs, e.g. many meshes) into one
 * schedule whose blocks run in a single launch.  Vertex ids of part i are
 * offset by the sum of the n of parts 0..i-1, task ids likewise by m.  The
 * parts must share flags and may differ in C.  The parts stay valid.
 */
int ep_batch(ep_schedule *const *parts, int32_t count, ep_schedule **out);

/*
 * Per-kernel timing (instrumentation, off by default).  When enabled, every
 * launch of the schedule's kernels is bracketed by CUDA events recorded on
 * its own stream; ep_timing_read() waits for the recorded events and returns
 * the summed device time and launch count of one kernel class since the last
 * reset:
 *   EP_T_EDGE_FWD  flux edge kernel (forward)      EP_T_BND   shared-vertex update
 *   EP_T_EDGE_ADJ  flux edge kernel (adjoint)      EP_T_SPMV  SpMV edge kernel
 *   EP_T_LAYOUT    layout / weight permutations    EP_T_COST  cost kernels
 * enable = 0 turns timing off; enable = 2 clears the totals and keeps it on.
 */
#define EP_T_EDGE_FWD 0
#define EP_T_BND 1
#define EP_T_EDGE_ADJ 2
#define EP_T_SPMV 3
#define EP_T_LAYOUT 4
#define EP_T_COST 5
#define EP_T_CLASSES 6
int ep_timing(ep_schedule *s, int32_t enable);
int ep_timing_read(ep_schedule *s, int32_t kernel_class, double *total_ms, int64_t *launches);

/* No counterpart in the paper (launch tuning): threads that compute per CUDA
 * block in the forward flux and SpMV kernels (32..1024, multiple of 32;
 * default 192), and in the adjoint flux kernels (default 352: the adjoint
 * stages twice the state per kernel block and does about twice the arithmetic
 * per task, so fewer CUDA blocks fit an SM and each wants more warps).
 * EP_EINVAL for a count out of range.  Does not change results beyond FP32
 * rounding order. */
int ep_set_threads(ep_schedule *s, int32_t threads);
int ep_set_adjoint_threads(ep_schedule *s, int32_t threads);

/*
 * No counterpart in the paper (multi-GPU sharding; the exchange volume is
 * bounded by the auxiliary-edge cut of Section 3, Theorem 1).  A schedule of
 * one shard (a contiguous range of another schedule's blocks) declares its
 * halo: the nh data vertices (ids in [0, nd); any order, duplicates allowed)
 * that other shards' tasks touch too.  Every halo vertex the shard touches
 * then takes the shared-vertex path of the flux layout, so its per-step sum
 * sits in an accumulator record instead of being applied in place.  Rebuilds
 * the flux layout (the schedule, its vertex lists and its cost are
 * unchanged), clears any pending state, and uploads again on the next call.
 * EP_EINVAL for a bipartite schedule or an id out of range.
 *
 * ep_halo_pack: after ep_step_pending, copies the sums of the last forward
 * edge kernel at the halo vertices into buf (device, nh x D floats, row i =
 * halo vertex i, zeros where this shard does not touch it).  ep_halo_unpack
 * writes buf back into those sums; between the two the caller sums buf over
 * all shards (an all-reduce across processes, or a sum of the shards'
 * buffers on one device).  The next step or ep_finish then applies the global
 * sums to every copy.  Both are no-ops without a halo; enqueued on `stream`.
 */
int ep_set_halo(ep_schedule *s, const int32_t *halo, int64_t nh);
int ep_halo_pack(ep_schedule *s, int32_t D, float *buf, void *stream);
int ep_halo_unpack(ep_schedule *s, int32_t D, const float *buf, void *stream);

/*
 * Edge-kernel organisation for flux steps (the software cache of Section 4).
 * stages = 0: one CUDA block per kernel block (stage, compute, write back).
 * stages = 2..8 (default 3): persistent CUDA blocks; a producer thread fills a
 * ring of that many shared-memory stages with 1-D TMA bulk copies of each
 * kernel block's contiguous pieces (its record run, slots, weights, shared
 * ids); consumer warps (ep_set_threads / ep_set_adjoint_threads, at most
 * 928 threads of them are used beside the producer and fix-up warps) take
 * whole slices of 32 positions and compute one stage while the next ones
 * load.  Results agree up to FP32 rounding order.  Fewer stages are used when
 * that many do not fit in shared memory; when two do not fit, launches use the
 * stages = 0 kernel instead.
 */
int ep_set_pipeline(ep_schedule *s, int32_t stages);

/*
 * No counterpart in the paper (instrumentation): the launch plan the
 * pipelined kernels use for state width D (adjoint != 0: the adjoint kernel)
 * on the current device: *grid CUDA blocks (*per_sm per SM) of *threads
 * threads, *stages shared-memory stages of *stage_bytes bytes each.
 * *stages = 0 when the schedule's blocks do not fit two stages (the one-block
 * kernel runs instead) or when ep_set_pipeline chose 0.  Any output may be
 * NULL.  Needs a device (EP_ENODEV otherwise).
 */
int ep_pipeline_info(ep_schedule *s, int32_t D, int32_t adjoint, int32_t *grid, int32_t *per_sm,
                     int32_t *threads, int32_t *stages, int32_t *stage_bytes);

/*
 * Reads and clears the error word of the pipelined kernels (synchronises
 * `stream`): every wait inside them is bounded, and an expired wait sets a
 * bit here instead of hanging (bit 0: waiting for data, bit 1: waiting for a
 * free stage).  *code = 0 and EP_OK when clean, else EP_ETIMEOUT.
 */
int ep_check_errors(ep_schedule *s, int32_t *code, void *stream);

/*
 * Where the forward flux and SpMV kernels read a block's data from (the
 * study of Section 5, Fig. 11 and Table 3: texture cache vs software cache).
 * EP_CACHE_SMEM (default): staged into shared memory (the flux kernels
 * chosen by ep_set_pipeline; SpMV stages x).  EP_CACHE_L1: nothing staged;
 * every read goes through the read-only data cache (ld.global.nc, which
 * replaces the texture binding of the paper's GPUs).  Flux: one CUDA block
 * per schedule block, one thread per vertex position (up to 4 per thread).
 * SpMV: x read through that cache, y written as before (EP-text of
 * Section 5).  The adjoint keeps its staged kernels.  Results agree up to
 * FP32 rounding order.  EP_EINVAL for another mode, or for EP_CACHE_L1 on a
 * flux schedule whose block has more than 4096 vertex positions.
 */
#define EP_CACHE_SMEM 0
#define EP_CACHE_L1 1
int ep_set_cache(ep_schedule *s, int32_t mode);

/*
 * Test hook for the bounded waits (no counterpart in the paper).  With
 * block_index >= 0, the producer of every persistent CUDA block leaves the
 * stage of its block_index-th schedule block unfilled (nothing copied,
 * nothing arrives), so the consumers' bounded wait for it expires: the
 * launch returns early with bit 0 set in the error word, its results are
 * invalid, and ep_check_errors() reports EP_ETIMEOUT and resets the
 * accumulators.  -1 (default) turns the hook off.
 */
int ep_debug_stall(ep_schedule *s, int32_t block_index);

/* No counterpart in the paper (resource release): frees a schedule, its host
 * arrays, its device copy and its workspace.  NULL is ignored.  The caller
 * must make sure no kernel enqueued on the schedule is still running. */
void ep_schedule_free(ep_schedule *s);

/* ---------------------------------------------------- no-allocation variant
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot let a library allocate device memory: applications that hand all
 * device memory to their own pool or framework allocator and forbid
 * allocations behind its back, and latency-bound loops that cannot take the
 * implicit device synchronisation that cudaMalloc and cudaFree may cause.  It
 * computes what ep_cost() computes, from caller-owned device arrays, and
 * allocates nothing:
 *   block_ptr  device int64[k+1]: tasks of block b are positions
 *              [block_ptr[b], block_ptr[b+1]) of eu/ev
 *   eu, ev     device int32[m]: the two data-vertex ids of every task, in
 *              schedule order (ids in [0, nd); a self loop repeats its id)
 *   max_ne     largest block_ptr[b+1] - block_ptr[b], 1..EP_MAX_C
 *   counts     device uint64[2], written: [0] = loads = sum_b |V_b|,
 *              [1] = number of distinct vertices (vertex cut = [0] - [1])
 * The device arrays cannot be checked on the host, so misuse is reported in
 * `counts` itself: if any block is longer than max_ne (or block_ptr
 * decreases), or any id lies outside [0, nd), counts[0] is set to
 * EP_NOALLOC_INVALID and counts[1] holds the reasons (EP_NOALLOC_BAD_BLOCK,
 * EP_NOALLOC_BAD_ID, or both); the return value is still EP_OK, because the
 * call does not wait for its kernels.
 * Its only scratch is a fixed array of EP_NOALLOC_MAX_VERTICES one-byte
 * flags plus a status word in the library's device memory, which every GPU
 * that loads this part of the library keeps until the process exits.  nd
 * above that limit gives EP_EINVAL.  The first call on a device looks up that
 * array's device address.  All calls share the array, so calls whose kernels
 * overlap on the GPU race with each other; each call clears the flags and the
 * status word it uses before counting.  Enqueued on `stream`, no
 * synchronisation.  Errors: EP_EINVAL, EP_ENODEV, EP_ECUDA, with a message
 * from ep_noalloc_last_error().
 */
#define EP_NOALLOC_MAX_VERTICES (1 << 24)
#define EP_NOALLOC_INVALID 0xffffffffffffffffull /* counts[0] of a misused call */
#define EP_NOALLOC_BAD_BLOCK 1u /* counts[1] bit: a block longer than max_ne */
#define EP_NOALLOC_BAD_ID 2u    /* counts[1] bit: an id outside [0, nd) */
int ep_cost_noalloc(const int64_t *block_ptr, const int32_t *eu, const int32_t *ev, int64_t k,
                    int64_t nd, int32_t max_ne, unsigned long long *counts, void *stream);
const char *ep_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EPCACHE_H */
