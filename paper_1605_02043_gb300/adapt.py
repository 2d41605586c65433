"""EP-adapt: switch to the partitioned schedule when it is ready (Section 4.2).

The paper's runtime starts the partitioner on a host thread as soon as the
application begins, keeps running the original kernel meanwhile, swaps the
optimised schedule in when the thread finishes, times the first optimised
run and goes back to the original if that run is slower, and stops the
thread if the application ends before it finishes.

Here the "original kernel" is the same edge kernel under the default
schedule (C consecutive tasks per block), the thread is the library's
ep_partition_start job, and a swap converts the resident state from one
schedule layout to the other through the caller's data order (two layout
kernels).  Every GPU call is timed with CUDA events on the launching stream;
timings are read back only once their end event has completed, so steady
state never blocks the host.  One difference from the paper: the first
`trial_skip` calls under the new schedule (default 1) are not used for the
decision, because the first launch of a kernel configuration also pays
one-time host set-up (launch plan, shared-memory limit) inside its events.

`Policy` holds the decisions and is plain host logic; `AdaptiveFlux`
applies them to repeated flux steps on the GPU.
"""
from __future__ import annotations

from . import EpError, PartitionJob, Schedule

DEFAULT, TRIAL, OPTIMISED, REVERTED, FAILED = "default", "trial", "optimised", "reverted", "failed"


class Policy:
    """Decisions of EP-adapt, fed with job events and per-step times (ms).

    Phases: DEFAULT until the job ends; then TRIAL if it produced a schedule
    (else FAILED, staying on the default schedule); after the first timed
    call under the new schedule, OPTIMISED if its time per step is at most
    (1 + margin) x the default schedule's (mean of the last `history` default
    calls), else REVERTED.  Without any default timing the trial is kept.
    """

    def __init__(self, margin: float = 0.0, history: int = 8):
        self.margin = margin
        self.history = history
        self.phase = DEFAULT
        self.default_ms: list[float] = []
        self.trial_ms: float | None = None
        self.error: str | None = None

    def add_default(self, ms_per_step: float):
        self.default_ms = (self.default_ms + [ms_per_step])[-self.history:]

    def job_ended(self, ok: bool, error: str | None = None) -> bool:
        """Returns True when the caller must swap the new schedule in."""
        if self.phase != DEFAULT:
            return False
        if ok:
            self.phase = TRIAL
            return True
        self.phase = FAILED
        self.error = error
        return False

    def reference_ms(self) -> float | None:
        if not self.default_ms:
            return None
        return sum(self.default_ms) / len(self.default_ms)

    def trial_done(self, ms_per_step: float) -> bool:
        """Returns True to keep the new schedule, False to go back."""
        if self.phase != TRIAL:
            raise RuntimeError(f"no trial in progress (phase {self.phase})")
        self.trial_ms = ms_per_step
        ref = self.reference_ms()
        keep = ref is None or ms_per_step <= (1.0 + self.margin) * ref
        self.phase = OPTIMISED if keep else REVERTED
        return keep


class AdaptiveFlux:
    """Repeated explicit flux steps (the cfd interaction of Section 1) under EP-adapt.

    x: CUDA float32 (D, n) initial state, w: CUDA float32 (m,) task weights,
    both in the caller's order.  The state stays resident in the current
    schedule's layout; `state(out)` copies it back to (D, n).
    `job_test` passes ep_partition_start's test hooks through.
    """

    def __init__(self, src, dst, n: int, C: int, x, w, *, threads: int = 0, stages: int = 3,
                 cuda_threads: int = 192, margin: float = 0.0, trial_skip: int = 1,
                 job_test: int = 0):
        import torch

        self._torch = torch
        self.D = int(x.shape[0])
        self.n = n
        self._w = w
        self._knobs = (stages, cuda_threads)
        self.policy = Policy(margin)
        self.default = self._ready(Schedule.partition(src, dst, n, C, default_order=True))
        self.job = PartitionJob(src, dst, n, C, threads=threads, test=job_test)
        self.optimised: Schedule | None = None
        self.cur = self.default
        self.xl, self.wl = self._load(self.default, x)
        self._pending = []  # (end event, start event, steps, schedule name)
        self.steps_done = 0
        self.switch_step: int | None = None
        self.partition_seconds: float | None = None
        self._skip = trial_skip

    def _ready(self, S: Schedule) -> Schedule:
        S.set_pipeline(self._knobs[0])
        S.set_threads(self._knobs[1])
        return S

    def _load(self, S: Schedule, x):
        xl = self._torch.empty(S.layout_floats(self.D), device=x.device)
        wl = self._torch.empty(S.weights_floats(), device=x.device)
        S.layout_in(x, xl)
        S.weights_in(self._w, wl)
        return xl, wl

    def _swap(self, S: Schedule):
        x = self._torch.empty(self.D, self.n, device=self.xl.device)
        self.cur.layout_out(self.xl, x)
        self.xl, self.wl = self._load(S, x)
        self.cur = S

    def step(self, tau: float = 1e-3, steps: int = 1):
        """Run `steps` steps as one timed call, then advance the policy."""
        torch = self._torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            self.cur.step(self.D, self.xl, self.xl, self.wl, None, tau)
        e1.record()
        self._pending.append((e1, e0, steps, "opt" if self.cur is self.optimised else "def"))
        self.steps_done += steps
        self._advance()

    def _advance(self):
        P = self.policy
        while self._pending and self._pending[0][0].query():
            e1, e0, steps, which = self._pending.pop(0)
            ms = e0.elapsed_time(e1) / steps
            if which == "def":
                P.add_default(ms)
            elif P.phase == TRIAL:
                if self._skip > 0:
                    self._skip -= 1
                elif not P.trial_done(ms):
                    self._swap(self.default)
        if P.phase == DEFAULT and self.job is not None and self.job.done():
            try:
                S = self._ready(self.job.take())
                ok, err = True, None
            except EpError as e:
                S, ok, err = None, False, str(e)
            self.partition_seconds = self.job.seconds
            if P.job_ended(ok, err):
                self.optimised = S
                self._swap(S)
                self.switch_step = self.steps_done

    def poll(self):
        """Advance the policy (read finished timings, check the job) without launching."""
        self._advance()

    def finish(self):
        """Wait for the outstanding timings and settle a pending trial."""
        self._torch.cuda.synchronize()
        self._advance()

    def state(self, x_out):
        self.cur.layout_out(self.xl, x_out)

    @property
    def phase(self) -> str:
        return self.policy.phase

    def close(self):
        """End of the application: stop the partition thread if still running."""
        if self.job is not None:
            self.job.close()
            self.job = None
