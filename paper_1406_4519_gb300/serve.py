"""Serving many decompositions: continuous batching of CP-ALS jobs.

Jobs (sparse 3-way tensors with a rank) arrive over time.  The server keeps
every admitted job resident on the GPU (its flattened CSR copies and factors),
advances all admitted jobs together one ALS sweep (Algorithm 4) at a time
through a batch (dfacto_batch_*), and retires a job when its fit stops moving
(relative change |fit - previous fit| < tol |previous fit|, or absolute with
relative=False) or after max_iters sweeps; the job's result is its factors and
weights, copied to the host at retirement.

Admission is first come, first served under a device-memory budget: a job is
admitted when the estimated footprint of everything admitted stays within the
budget.  Membership changes take effect when the batch is rebuilt (its
concatenated CSR copies are rebuilt from the jobs', a cost that grows with
everything resident): admissions at most once per `rebuild_interval` seconds,
so that a burst of arrivals does not rebuild after every sweep; retirements
alone only once the finished jobs, which ride along until then, hold
`waste_limit` of the batch's nonzeros.

A request whose tensor cannot be built (invalid coordinates, duplicates, no
device memory) finishes at once with its error and no result; the others are
not affected.

The scheduling decisions live in `Scheduler` (pure Python, no GPU), the device
work in `GpuEngine`; `serve()` runs the loop in real time against a list of
arrival times.  `serve_sequential()` is the comparison: one job at a time, in
arrival order, each with its own single-tensor ALS loop.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

# Library statuses that concern one request only (include/dfacto.h): bad
# arguments, a coordinate outside dims, a duplicate coordinate, no device
# memory for this tensor.  Any other failure (ECUDA leaves the context unusable,
# EINTERNAL is a library fault) stops the server.
REQUEST_STATUSES = (1, 2, 3, 4)  # DFACTO_EINVAL, ERANGE, EDUP, ENOMEM


def is_request_failure(e: BaseException) -> bool:
    """True when building one request failed for a reason of its own (its
    tensor or its size), so that the request can fail alone."""
    status = getattr(e, "status", None)
    if status is not None:
        return status in REQUEST_STATUSES
    # input that cannot describe a tensor, or no host/device memory for it
    return isinstance(e, (ValueError, MemoryError)) or type(e).__name__ == "OutOfMemoryError"


@dataclass
class JobSpec:
    """One request: a tensor (COO on the device), its rank and start factors."""
    job_id: int
    arrival: float                 # seconds from the start of the run
    dims: Sequence[int]
    nnz: int
    rank: int
    make: Callable                 # () -> (idx, val, factors): device tensors


@dataclass
class JobState:
    spec: JobSpec
    admitted_at: Optional[float] = None
    finished_at: Optional[float] = None
    iters: int = 0
    fits: List[float] = field(default_factory=list)
    footprint: int = 0
    result: Optional[dict] = None
    error: Optional[str] = None    # set when the request could not be served

    @property
    def latency(self) -> Optional[float]:
        if self.finished_at is None:
            return None
        return self.finished_at - self.spec.arrival


def footprint_bytes(dims: Sequence[int], nnz: int, rank: int, factor_bytes: int) -> int:
    """Upper estimate of the device bytes a job holds while it is served: the
    CSR copies of its three modes twice (the job's own and the batch's
    concatenated copy; per mode 8 bytes per nonzero for (index, value), at most
    one fiber per nonzero at 16 bytes, 8 bytes per row pointer, end bits), the
    factors (own and pooled), the MTTKRP outputs, and the row-pass buffers."""
    sd = sum(int(d) for d in dims)
    csr = 3 * (8 * nnz + 16 * nnz + nnz // 8 + 4 * nnz // 32) + 8 * (sd + 3)
    factors = factor_bytes * rank * sd
    rows = 4 * rank * sd + 2 * 4 * rank * max(dims)
    return 2 * csr + 2 * factors + rows + (1 << 20)


def converged(fits: Sequence[float], tol: float, relative: bool = True) -> bool:
    """|fit_k - fit_{k-1}| < tol * |fit_{k-1}| (relative) or < tol (absolute),
    tested from the second sweep on."""
    if len(fits) < 2:
        return False
    change = abs(fits[-1] - fits[-2])
    return change < (tol * abs(fits[-2]) if relative else tol)


class Scheduler:
    """Admission, retirement and rebuild decisions; no device work."""

    def __init__(self, budget_bytes: float, max_iters: int = 50, tol: float = 1e-4,
                 rebuild_interval: float = 0.005, factor_bytes: int = 2, relative: bool = True,
                 waste_limit: float = 0.5):
        self.budget = float(budget_bytes)
        self.max_iters = int(max_iters)
        self.tol = float(tol)
        self.relative = bool(relative)
        self.waste_limit = float(waste_limit)
        self.rebuild_interval = float(rebuild_interval)
        self.factor_bytes = int(factor_bytes)
        self.pending: List[JobState] = []    # arrived, not admitted (FIFO)
        self.active: Dict[int, JobState] = {}  # admitted, not finished
        self.done: List[JobState] = []
        self.used = 0
        self.last_rebuild = -1e30

    def arrive(self, job: JobState) -> None:
        job.footprint = footprint_bytes(job.spec.dims, job.spec.nnz, job.spec.rank, self.factor_bytes)
        self.pending.append(job)

    def admissible(self) -> List[JobState]:
        """Pending jobs to admit now, first come first served: stop at the first
        job that does not fit (no overtaking).  A job larger than the whole
        budget is admitted alone once nothing else is resident."""
        out = []
        used = self.used
        for job in self.pending:
            if used + job.footprint <= self.budget or (used == 0 and not out):
                out.append(job)
                used += job.footprint
            else:
                break
        return out

    def reject(self, job: JobState, now: float, error: str) -> None:
        """A pending job that cannot be served (its tensor failed to build): it
        leaves the queue finished, with the error and no result."""
        self.pending.remove(job)
        job.error = error
        job.finished_at = now
        self.done.append(job)

    def admit(self, jobs: Sequence[JobState], now: float) -> None:
        for job in jobs:
            self.pending.remove(job)
            job.admitted_at = now
            self.active[job.spec.job_id] = job
            self.used += job.footprint

    def record_sweep(self, fits: Dict[int, float]) -> List[JobState]:
        """Record one sweep's fits; return the jobs that are now finished
        (fit change below tolerance, or max_iters sweeps)."""
        finished = []
        for jid, fit in fits.items():
            job = self.active[jid]
            job.iters += 1
            job.fits.append(float(fit))
            if converged(job.fits, self.tol, self.relative) or job.iters >= self.max_iters:
                finished.append(job)
        return finished

    def retire(self, job: JobState, now: float) -> None:
        job.finished_at = now
        del self.active[job.spec.job_id]
        self.used -= job.footprint
        self.done.append(job)

    def should_rebuild(self, now: float, admitted_waiting: bool, waste: float,
                       have_batch: bool) -> bool:
        """admitted_waiting: admitted jobs not yet in the batch; waste: the
        fraction of the batch's nonzeros that belong to finished jobs."""
        if not have_batch:
            return admitted_waiting
        if not self.active:
            return True  # everything in the batch has finished
        if admitted_waiting and now - self.last_rebuild >= self.rebuild_interval:
            return True
        return waste >= self.waste_limit


class GpuEngine:
    """Device side of the server: builds jobs, keeps one batch of the admitted
    jobs, runs sweeps, reads results."""

    def __init__(self, factor_dtype: int, use_graph: bool = False):
        from . import dfacto
        self.dfacto = dfacto
        self.factor_dtype = factor_dtype
        # A batch lives from one membership change to the next (a few sweeps),
        # too short for a captured graph to pay for its capture by default.
        self.use_graph = use_graph
        self.tensors: Dict[int, "dfacto.Tensor"] = {}
        self.batch = None
        self.members: List[int] = []

    def build(self, job: JobState) -> None:
        idx, val, F = job.spec.make()
        t = self.dfacto.Tensor(idx, val, job.spec.dims, rank=job.spec.rank,
                               factor_dtype=self.factor_dtype)
        t.set_factors(F)
        self.tensors[job.spec.job_id] = t

    def rebuild(self, members: Sequence[int]) -> None:
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        self.members = list(members)
        if self.members:
            self.batch = self.dfacto.Batch([self.tensors[j] for j in self.members], autotune=False,
                                           use_graph=self.use_graph)

    def sweep(self) -> Dict[int, float]:
        st, fits = self.batch.als_iter(want_fits=True)
        return dict(zip(self.members, fits))

    def result(self, jid: int) -> dict:
        import torch
        t = self.tensors[jid]
        return {"factors": [f.cpu() for f in t.factors(dtype=torch.float32)], "lambda": t.lam()}

    def release(self, jid: int) -> None:
        t = self.tensors.pop(jid)
        if self.batch is not None and jid in self.members:
            return  # still in the batch: dropped at the next rebuild
        del t

    def close(self) -> None:
        if self.batch is not None:
            self.batch.close()
            self.batch = None


def serve(jobs: Sequence[JobSpec], budget_bytes: float = 120e9, max_iters: int = 50,
          tol: float = 1e-4, rebuild_interval: float = 0.005, factor_dtype: Optional[int] = None,
          engine=None, clock: Callable[[], float] = time.perf_counter,
          sleep: Callable[[float], None] = time.sleep, relative: bool = True) -> List[JobState]:
    """Serve `jobs` (sorted by arrival) in real time; returns the finished jobs
    with their latencies (arrival -> factors on the host)."""
    if engine is None:
        from . import dfacto
        engine = GpuEngine(dfacto.BF16 if factor_dtype is None else factor_dtype)
    fbytes = 4 if factor_dtype == 0 else 2
    sch = Scheduler(budget_bytes, max_iters, tol, rebuild_interval, fbytes, relative)
    order = sorted(jobs, key=lambda j: j.arrival)
    nxt = 0
    sch_done_nnz: Dict[int, int] = {}
    t0 = clock()
    retired_in_batch = set()   # finished jobs whose handles still sit in the batch
    in_batch_nnz = 0           # nonzeros of the jobs in the current batch
    changed = False            # admitted jobs not yet in the batch
    while nxt < len(order) or sch.pending or sch.active:
        now = clock() - t0
        while nxt < len(order) and order[nxt].arrival <= now:
            sch.arrive(JobState(order[nxt]))
            nxt += 1
        adm = sch.admissible()
        if adm:
            built = []
            for job in adm:
                try:
                    engine.build(job)
                    built.append(job)
                except Exception as e:
                    if not is_request_failure(e):
                        raise  # the device or the library is at fault: stop serving
                    sch.reject(job, clock() - t0, "%s: %s" % (type(e).__name__, e))
            if built:
                sch.admit(built, clock() - t0)
                changed = True
        now = clock() - t0
        waste = (sum(sch_done_nnz[j] for j in retired_in_batch) / in_batch_nnz
                 if in_batch_nnz else 0.0)
        if sch.should_rebuild(now, changed, waste, engine.batch is not None):
            members = sorted(sch.active)
            engine.rebuild(members)
            for jid in retired_in_batch:
                engine.release(jid)
            retired_in_batch.clear()
            in_batch_nnz = sum(sch.active[j].spec.nnz for j in members)
            sch.last_rebuild = now
            changed = False
        if engine.batch is None or not sch.active:
            if nxt < len(order):
                sleep(max(0.0, min(order[nxt].arrival - (clock() - t0), 0.01)))
            continue
        fits = engine.sweep()
        fits = {j: f for j, f in fits.items() if j in sch.active}
        for job in sch.record_sweep(fits):
            job.result = engine.result(job.spec.job_id)
            sch.retire(job, clock() - t0)
            retired_in_batch.add(job.spec.job_id)
            sch_done_nnz[job.spec.job_id] = job.spec.nnz
    engine.close()
    return sch.done


def serve_sequential(jobs: Sequence[JobSpec], max_iters: int = 50, tol: float = 1e-4,
                     factor_dtype: int = 0, clock: Callable[[], float] = time.perf_counter,
                     sleep: Callable[[float], None] = time.sleep,
                     relative: bool = True) -> List[JobState]:
    """The comparison server: one job at a time in arrival order, each run to
    convergence with the single-tensor ALS entry point."""
    import torch

    from . import dfacto
    order = sorted(jobs, key=lambda j: j.arrival)
    done = []
    t0 = clock()
    for spec in order:
        now = clock() - t0
        if spec.arrival > now:
            sleep(spec.arrival - now)
        job = JobState(spec, admitted_at=clock() - t0)
        idx, val, F = spec.make()
        t = dfacto.Tensor(idx, val, spec.dims, rank=spec.rank, factor_dtype=factor_dtype)
        t.set_factors(F)
        while True:
            st, fit = t.als_iter(want_fit=True)
            job.iters += 1
            job.fits.append(fit)
            if converged(job.fits, tol, relative) or job.iters >= max_iters:
                break
        job.result = {"factors": [f.cpu() for f in t.factors(dtype=torch.float32)], "lambda": t.lam()}
        job.finished_at = clock() - t0
        del t
        done.append(job)
    return done


def latency_stats(done: Sequence[JobState]) -> dict:
    """p50 / p99 latency and throughput of the jobs that finished with a
    result (requests that failed are counted apart)."""
    failed = sum(1 for j in done if j.error is not None)
    done = [j for j in done if j.error is None]
    lat = sorted(j.latency for j in done if j.latency is not None)
    if not lat:
        return {"jobs": 0, "failed": failed}

    def pct(p):
        k = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
        return lat[k]

    first = min(j.spec.arrival for j in done)
    last = max(j.finished_at for j in done)
    return {"jobs": len(lat), "failed": failed, "p50_s": pct(50), "p99_s": pct(99),
            "mean_s": sum(lat) / len(lat),
            "jobs_per_s": len(lat) / max(last - first, 1e-9),
            "mean_iters": sum(j.iters for j in done) / len(done),
            "mean_final_fit": sum(j.fits[-1] for j in done if j.fits) / max(1, len(done))}
