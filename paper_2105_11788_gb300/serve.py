"""Serving loop: continuous batching of bisimulation-reduction requests.

Requests (an LTS each) arrive over time. The loop keeps `workers` batches in
flight, each on its own CUDA stream: whenever a worker is free it takes every
request that has arrived so far (up to `max_batch` and up to the device-memory
budget), plans them as one batch (bisim_batch_plan) and refines them in one
launch (bisim_batch_refine). Requests that arrive while batches run are
admitted as soon as a worker and memory free up, and their kernels overlap the
running ones on the device (the batch kernel is an ordinary, non-cooperative
launch). A request whose footprint alone exceeds the budget is admitted only
when nothing else is in flight.

With a large-request lane (`big_executor`, `big_states`), an LTS of at least
`big_states` states that arrives while the lane holds fewer than `big_backlog`
requests skips the batches and is reduced alone on its own stream by the
single-LTS path, which spreads one LTS over the whole GPU, one such request
at a time; inside a batch a large LTS runs on a single CTA and holds its
batch back. When the lane is backed up, large requests join the batches, so
that under heavy load they are reduced side by side instead of in a line.

Results are canonical block ids, identical to what the one-at-a-time path
returns for the same LTS. Latency is measured from a request's arrival to the
moment its batch's results are on the host.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Callable, List, Optional, Sequence

import numpy as np


def footprint_bytes(n: int, m: int, num_act: int = 1) -> int:
    """Device bytes one LTS needs at most during a batched reduction, from the
    sizes of what the path allocates per transition and per state:
      transitions: the inputs on the device (src, act, dst: 12 B), their copy
        in the batch's union (12 B), the incoming-transition index (8 B) and
        per mark slot (at most one per transition) its owner, label and mark
        (12 B): 44 B; with more than 128 labels the sort by (source, label)
        adds 32 B of temporaries;
      states: initial labels and output (8 B), their union copy (4 B), the
        plan's per-state arrays (29 B), the frontier state with the 32 worklist
        rings (228 B), the label sets and the set-up and output temporaries
        (at most 40 B): 309 B;
    plus 1 MiB for the small per-batch arrays."""
    per_t = 44 + (32 if num_act > 128 else 0)
    return per_t * int(m) + 309 * int(n) + (1 << 20)


def gpu_trim(keep_bytes: int = 0) -> None:
    """Give the memory that finished plans left in the device's memory pool
    back to the device (the library keeps freed plan memory for reuse while a
    process serves, so that later plans need no new mappings)."""
    from . import bisim

    bisim.bisim_pool_trim(keep_bytes)


@dataclasses.dataclass
class Request:
    rid: int
    lts: object
    arrival: float  # seconds after the start of serving


@dataclasses.dataclass
class Result:
    rid: int
    labels: np.ndarray
    arrival: float
    dispatch: float
    done: float
    batch: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def gpu_executor(opts=None, device: str = "cuda"):
    """Executor running a batch on the calling thread's own CUDA stream."""
    import torch

    from . import bisim

    local = threading.local()

    def run(ltss: Sequence) -> List[np.ndarray]:
        if not hasattr(local, "stream"):
            local.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(local.stream):
            parts = bisim.reduce_batch(list(ltss), opts, device=device, stream=local.stream)
        return parts

    return run


def gpu_single_executor(opts=None, device: str = "cuda"):
    """Executor reducing one LTS with the single-LTS path on the calling
    thread's own CUDA stream."""
    import torch

    from . import bisim

    local = threading.local()

    def run(lts) -> np.ndarray:
        if not hasattr(local, "stream"):
            local.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(local.stream):
            return bisim.reduce(lts, opts, device=device, stream=local.stream)

    return run


class BatchServer:
    def __init__(self, executor: Callable[[Sequence], List[np.ndarray]], mem_budget: int,
                 workers: int = 2, max_batch: int = 1024,
                 footprint: Callable[[object], int] = lambda l: footprint_bytes(l.n, l.m, l.num_act),
                 big_executor: Optional[Callable[[object], np.ndarray]] = None, big_states: int = 0,
                 big_backlog: int = 2, on_idle: Optional[Callable[[], None]] = None):
        self.executor = executor
        self.big_executor = big_executor
        self.big_states = int(big_states)
        self.big_backlog = int(big_backlog)
        self.big_served = 0
        self.mem_budget = int(mem_budget)
        self.workers = int(workers)
        self.max_batch = int(max_batch)
        self.footprint = footprint
        self.on_idle = on_idle  # called when serve() has drained every request (e.g. gpu_trim)
        self.max_inflight_bytes = 0
        self.batches = 0
        self.max_concurrent = 0

    def _big(self, req: Request) -> bool:
        return self.big_executor is not None and req.lts.n >= self.big_states

    def serve(self, requests: Sequence[Request], clock=time.perf_counter) -> List[Result]:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        big_queue: collections.deque = collections.deque()
        inflight = {}  # future -> (batch id, [requests], bytes, dispatch time)
        big = None  # (future, request, bytes, dispatch time, batch id) of the large-request lane
        inflight_bytes = 0
        results: List[Result] = []
        t0 = clock()
        with cf.ThreadPoolExecutor(max_workers=self.workers) as pool, \
                cf.ThreadPoolExecutor(max_workers=1) as big_pool:
            while pending or queue or big_queue or inflight or big:
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    r = pending.popleft()
                    lane = self._big(r) and len(big_queue) + (big is not None) < self.big_backlog
                    (big_queue if lane else queue).append(r)
                # retire finished batches and the finished large request
                for fut in [f for f in inflight if f.done()]:
                    bid, reqs, nbytes, tdisp = inflight.pop(fut)
                    parts = fut.result()
                    tdone = clock() - t0
                    for r, lab in zip(reqs, parts):
                        results.append(Result(r.rid, lab, r.arrival, tdisp, tdone, bid))
                    inflight_bytes -= nbytes
                if big is not None and big[0].done():
                    fut, r, nbytes, tdisp, bid = big
                    results.append(Result(r.rid, fut.result(), r.arrival, tdisp, clock() - t0, bid))
                    inflight_bytes -= nbytes
                    big = None
                # the large-request lane: one at a time, within the memory budget
                if big is None and big_queue:
                    fp = self.footprint(big_queue[0].lts)
                    if inflight_bytes + fp <= self.mem_budget or not inflight:
                        r = big_queue.popleft()
                        big = (big_pool.submit(self.big_executor, r.lts), r, fp, clock() - t0, self.batches)
                        self.batches += 1
                        self.big_served += 1
                        inflight_bytes += fp
                        self.max_inflight_bytes = max(self.max_inflight_bytes, inflight_bytes)
                # admit: every arrived request that fits, while a worker is free
                while queue and len(inflight) < self.workers:
                    batch, nbytes = [], 0
                    while queue and len(batch) < self.max_batch:
                        fp = self.footprint(queue[0].lts)
                        fits = inflight_bytes + nbytes + fp <= self.mem_budget
                        alone = not batch and not inflight and big is None
                        if not (fits or alone):
                            break
                        batch.append(queue.popleft())
                        nbytes += fp
                    if not batch:
                        break  # memory full: wait for a batch to finish
                    tdisp = clock() - t0
                    fut = pool.submit(self.executor, [r.lts for r in batch])
                    inflight[fut] = (self.batches, batch, nbytes, tdisp)
                    self.batches += 1
                    inflight_bytes += nbytes
                    self.max_inflight_bytes = max(self.max_inflight_bytes, inflight_bytes)
                    self.max_concurrent = max(self.max_concurrent, len(inflight) + (big is not None))
                # sleep until the next arrival or a completion
                timeout = 0.002
                if pending:
                    timeout = max(0.0, min(timeout, pending[0].arrival - (clock() - t0)))
                waiting = list(inflight) + ([big[0]] if big is not None else [])
                if waiting:
                    cf.wait(waiting, timeout=timeout, return_when=cf.FIRST_COMPLETED)
                elif timeout > 0:
                    time.sleep(timeout)
        results.sort(key=lambda r: r.rid)
        if self.on_idle is not None:
            self.on_idle()
        return results


def latency_summary(results: Sequence[Result]) -> dict:
    lat = np.array([r.latency for r in results], dtype=np.float64)
    span = max(r.done for r in results) - min(r.arrival for r in results) if results else 0.0
    return {
        "requests": len(results),
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
        "mean_ms": float(lat.mean() * 1e3) if len(lat) else None,
        "throughput_lts_per_s": len(results) / span if span > 0 else None,
        "batches": len({r.batch for r in results}),
    }


def poisson_requests(ltss: Sequence, rate_per_s: float, seed: int = 0,
                     arrivals: Optional[np.ndarray] = None) -> List[Request]:
    """Requests with Poisson arrivals at `rate_per_s` (or given arrival times)."""
    if arrivals is None:
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, len(ltss)))
    return [Request(i, l, float(t)) for i, (l, t) in enumerate(zip(ltss, arrivals))]
