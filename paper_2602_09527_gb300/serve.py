"""Request loop over the batched engine (vrps_batch_*): continuous batching of reconstruction
jobs with admission by device-memory footprint.

Requests wait in arrival order.  Before every group of ticks the loop scans the waiting
requests in that order and admits each one whose geometry class has a free handle and whose
state fits the memory budget.  A request waiting for a handle of its own class does not hold
up requests of other classes behind it (handles are per class); a request waiting for memory
does (memory is shared: admitting later, smaller jobs past it could starve it), so the scan
stops there.  Admitted jobs join the running batch at the next tick, and a job's handle and
memory are released as soon as its last iteration has finished on the device.  All device
work (job setup, every tick, the result copy) happens in the library; this module only
schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import torch

from . import _binding as vb


@dataclass
class Request:
    """One reconstruction request: a geometry class, its data and the solver settings."""
    key: object                  # geometry class (requests of one class share handles)
    b: torch.Tensor              # device sinogram, natural angle order
    arrival: float               # seconds since the start of the run
    alpha: float
    gamma: float
    seed: int
    p: float = 0.1
    estimator: str = "SAGA"
    fgp_iters: int = 50
    max_iters: int = 100
    n_subsets: int = 0           # 0: the geometry's N
    storage: str = "FP32"
    correction_epochs: int = 0
    admitted: float | None = None
    finished: float | None = None
    report: dict | None = None
    x: torch.Tensor | None = None


@dataclass
class ServerStats:
    latencies: list = field(default_factory=list)
    queue_waits: list = field(default_factory=list)
    completed: int = 0
    ticks: int = 0
    peak_jobs: int = 0
    peak_bytes: int = 0
    wall: float = 0.0


class BatchServer:
    """Continuous batching of jobs on one GPU.

    pools: {key: [Geometry, ...]} handles per geometry class (each running job holds one);
    budget_bytes: upper bound on the summed footprint (vrps_job_footprint) of running jobs;
    ticks_per_step: ticks enqueued between two admission / completion checks;
    max_running: at most this many jobs advance together (None: no limit besides handles and
    memory) -- fewer concurrent jobs make each tick, and so each job, finish sooner;
    priority, grid_share: the batch's CUDA stream priority and the fraction of the GPU's
    resident thread-block slots its persistent launches take (vrps_batch_set_*)."""

    def __init__(self, pools: dict, budget_bytes: int, ticks_per_step: int = 2, graphs: bool = True,
                 max_running: int | None = None, priority: int | None = None, grid_share: float = 1.0):
        self.free = {k: list(v) for k, v in pools.items()}
        self.budget = int(budget_bytes)
        self.ticks_per_step = int(ticks_per_step)
        self.max_running = max_running
        self.batch = vb.Batch(graphs=graphs, priority=priority, grid_share=grid_share)
        self.running = {}            # job id -> (request, geometry, bytes)
        self.used = 0

    ADMITTED, NO_HANDLE, NO_MEMORY = 0, 1, 2

    def _try_admit(self, r: Request, now: float) -> int:
        pool = self.free.get(r.key)
        if not pool or (self.max_running is not None and len(self.running) >= self.max_running):
            return self.NO_HANDLE
        g = pool[-1]
        need = vb.job_footprint(g, max_iters=r.max_iters, storage=r.storage)
        if self.running and self.used + need > self.budget:
            return self.NO_MEMORY
        pool.pop()
        r.x = torch.empty(g.n, device=r.b.device, dtype=torch.float32)
        jid = self.batch.submit(g, r.b, alpha=r.alpha, p=r.p, gamma=r.gamma, seed=r.seed, estimator=r.estimator,
                                fgp_iters=r.fgp_iters, max_iters=r.max_iters, n_subsets=r.n_subsets,
                                storage=r.storage, correction_epochs=r.correction_epochs, x_out=r.x)
        r.admitted = now
        self.running[jid] = (r, g, need)
        self.used += need
        return self.ADMITTED

    def _admit_waiting(self, waiting: list, now: float):
        """Admits waiting requests in arrival order: past requests whose class has no free
        handle, up to the first that does not fit the memory budget."""
        keep = []
        for q, r in enumerate(waiting):
            got = self._try_admit(r, now)
            if got == self.NO_MEMORY:
                keep.extend(waiting[q:])
                break
            if got == self.NO_HANDLE:
                keep.append(r)
        waiting[:] = keep

    def run(self, requests: list, clock=time.perf_counter, t0: float | None = None) -> ServerStats:
        """Serves `requests` (sorted by arrival) in real time; returns latency statistics.
        t0: the clock reading that arrival times count from (default: now)."""
        st = ServerStats()
        waiting = []
        i = 0
        t0 = clock() if t0 is None else t0
        while i < len(requests) or waiting or self.running:
            now = clock() - t0
            while i < len(requests) and requests[i].arrival <= now:
                waiting.append(requests[i])
                i += 1
            if waiting:
                self._admit_waiting(waiting, now)
            st.peak_jobs = max(st.peak_jobs, len(self.running))
            st.peak_bytes = max(st.peak_bytes, self.used)
            if self.running:
                self.batch.step(self.ticks_per_step)
                st.ticks += self.ticks_per_step
            elif i < len(requests):
                time.sleep(max(0.0, min(requests[i].arrival - now, 0.002)))
            now = clock() - t0
            for jid in list(self.running):
                done, rep = self.batch.poll(jid)
                if not done:
                    continue
                r, g, need = self.running.pop(jid)
                r.finished = now
                r.report = rep
                self.batch.release(jid)
                self.free[r.key].append(g)
                self.used -= need
                st.completed += 1
                st.latencies.append(r.finished - r.arrival)
                st.queue_waits.append(r.admitted - r.arrival)
        st.wall = clock() - t0
        return st

    def close(self):
        self.batch.close()


class SequentialServer:
    """The per-job baseline: requests in arrival order, one vrps_solve at a time (on `stream`,
    default the current stream)."""

    def __init__(self, pools: dict, stream=None):
        self.geom = {k: v[0] for k, v in pools.items()}
        self.stream = stream

    def run(self, requests: list, clock=time.perf_counter, t0: float | None = None) -> ServerStats:
        st = ServerStats()
        t0 = clock() if t0 is None else t0
        for r in requests:
            now = clock() - t0
            if r.arrival > now:
                time.sleep(r.arrival - now)
            r.admitted = clock() - t0
            g = self.geom[r.key]
            x, rep, _ = vb.solve(r.b, g, r.alpha, "VR_PROXSKIP", p=r.p, gamma=r.gamma, seed=r.seed,
                                 estimator=r.estimator, fgp_iters=r.fgp_iters, max_iters=r.max_iters,
                                 n_subsets=r.n_subsets, storage=r.storage, correction_epochs=r.correction_epochs,
                                 stream=self.stream)
            r.finished = clock() - t0
            r.report, r.x = rep, x
            st.completed += 1
            st.latencies.append(r.finished - r.arrival)
            st.queue_waits.append(r.admitted - r.arrival)
        st.wall = clock() - t0
        return st


def percentile(values, q):
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    v = sorted(values)
    if not v:
        return float("nan")
    pos = (len(v) - 1) * q / 100.0
    lo = int(pos)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)


def merge_stats(parts: list, wall: float) -> ServerStats:
    st = ServerStats(wall=wall)
    for q in parts:
        st.latencies += q.latencies
        st.queue_waits += q.queue_waits
        st.completed += q.completed
        st.ticks += q.ticks
        st.peak_jobs += q.peak_jobs
        st.peak_bytes += q.peak_bytes
    return st


class MixedServer:
    """2D and 3D requests: a 2D BatchServer and, for the 3D requests, either a 3D BatchServer
    (mode3d "batch": its own batch, share of the memory budget and persistent grids taking
    grid_share3d of the GPU) or one vrps_solve at a time in arrival order (mode3d "solve":
    ordinary launches, so that the 2D batch's thread blocks interleave with them block by
    block).  Each side runs on its own CUDA stream, the 2D one with the highest priority (its
    short jobs wait least for SMs) and the 3D one with the lowest.  The 3D loop runs in a
    worker thread; the library releases the GIL in every call, so neither loop waits for the
    other's host blocking."""

    def __init__(self, pools: dict, pools3d: dict, budget_bytes: int, ticks_per_step: int = 2,
                 share3d: float = 0.5, ticks_per_step3d: int = 1, max_running: int | None = None,
                 max_running3d: int | None = None, grid_share3d: float = 1.0, mode3d: str = "batch"):
        self.s2 = BatchServer(pools, int(budget_bytes * (1.0 - share3d)), ticks_per_step, max_running=max_running,
                              priority=-1000)
        if mode3d == "solve":
            self.s3 = SequentialServer(pools3d, stream=torch.cuda.Stream(priority=0))   # 0: the lowest
        else:
            self.s3 = BatchServer(pools3d, int(budget_bytes * share3d), ticks_per_step3d, max_running=max_running3d,
                                  priority=0, grid_share=grid_share3d)
        self.keys3 = set(pools3d)

    def run(self, requests: list, clock=time.perf_counter) -> ServerStats:
        import threading
        r3 = [r for r in requests if r.key in self.keys3]
        r2 = [r for r in requests if r.key not in self.keys3]
        out = {}
        t0 = clock()

        def work3():
            out["3d"] = self.s3.run(r3, clock, t0)

        th = threading.Thread(target=work3)
        th.start()
        st2 = self.s2.run(r2, clock, t0)
        th.join()
        st = merge_stats([st2, out["3d"]], clock() - t0)
        st.ticks = st2.ticks
        return st

    def close(self):
        self.s2.close()
        if hasattr(self.s3, "close"):
            self.s3.close()
