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


def footprint_bytes(n: int, m: int) -> int:
    """Device bytes one LTS needs during a batched reduction: inputs, plan
    arrays and sort temporaries (about 80 B per transition) and refinement
    state with the bucketed worklist (about 256 B per state)."""
    return 80 * int(m) + 256 * int(n) + (1 << 20)


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


class BatchServer:
    def __init__(self, executor: Callable[[Sequence], List[np.ndarray]], mem_budget: int,
                 workers: int = 2, max_batch: int = 1024,
                 footprint: Callable[[object], int] = lambda l: footprint_bytes(l.n, l.m)):
        self.executor = executor
        self.mem_budget = int(mem_budget)
        self.workers = int(workers)
        self.max_batch = int(max_batch)
        self.footprint = footprint
        self.max_inflight_bytes = 0
        self.batches = 0
        self.max_concurrent = 0

    def serve(self, requests: Sequence[Request], clock=time.perf_counter) -> List[Result]:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        inflight = {}  # future -> (batch id, [requests], bytes, dispatch time)
        inflight_bytes = 0
        results: List[Result] = []
        t0 = clock()
        with cf.ThreadPoolExecutor(max_workers=self.workers) as pool:
            while pending or queue or inflight:
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    queue.append(pending.popleft())
                # retire finished batches
                for fut in [f for f in inflight if f.done()]:
                    bid, reqs, nbytes, tdisp = inflight.pop(fut)
                    parts = fut.result()
                    tdone = clock() - t0
                    for r, lab in zip(reqs, parts):
                        results.append(Result(r.rid, lab, r.arrival, tdisp, tdone, bid))
                    inflight_bytes -= nbytes
                # admit: every arrived request that fits, while a worker is free
                while queue and len(inflight) < self.workers:
                    batch, nbytes = [], 0
                    while queue and len(batch) < self.max_batch:
                        fp = self.footprint(queue[0].lts)
                        fits = inflight_bytes + nbytes + fp <= self.mem_budget
                        alone = not batch and not inflight
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
                    self.max_concurrent = max(self.max_concurrent, len(inflight))
                # sleep until the next arrival or a completion
                timeout = 0.002
                if pending:
                    timeout = max(0.0, min(timeout, pending[0].arrival - (clock() - t0)))
                if inflight:
                    cf.wait(list(inflight), timeout=timeout, return_when=cf.FIRST_COMPLETED)
                elif timeout > 0:
                    time.sleep(timeout)
        results.sort(key=lambda r: r.rid)
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
