"""Host logic of the serving loop (no GPU): admission by memory footprint,
continuous batching across workers, latency bookkeeping. The executor is a
fake that runs the CPU oracle and sleeps in proportion to the work."""
import time

import numpy as np

import oracle
from paper_2105_11788_gb300 import lts_gen, serve


def _fake_executor(calls):
    def run(ltss):
        calls.append(len(ltss))
        time.sleep(0.002 + 1e-7 * sum(l.m for l in ltss))
        return [oracle.ks_lts(l) for l in ltss]
    return run


def _stream(k, seed=3):
    rng = np.random.default_rng(seed)
    return [lts_gen.stream_instance(rng, n_lo=50, n_hi=2000, idx=i) for i in range(k)]


def test_every_request_served_with_the_oracle_result():
    ltss = _stream(40)
    reqs = serve.poisson_requests(ltss, rate_per_s=2000.0, seed=1)
    calls = []
    srv = serve.BatchServer(_fake_executor(calls), mem_budget=1 << 40, workers=2)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(40))
    for r, l in zip(res, ltss):
        assert r.labels.tolist() == oracle.ks_lts(l).tolist()
        assert r.done >= r.dispatch >= r.arrival - 1e-9
    assert sum(calls) == 40
    assert srv.max_concurrent == 2  # arrivals outpace service: both workers busy
    s = serve.latency_summary(res)
    assert s["requests"] == 40 and s["p99_ms"] >= s["p50_ms"] > 0


def test_memory_budget_limits_what_is_in_flight():
    ltss = _stream(30, seed=5)
    fps = [serve.footprint_bytes(l.n, l.m) for l in ltss]
    budget = 3 * max(fps)
    reqs = [serve.Request(i, l, 0.0) for i, l in enumerate(ltss)]
    srv = serve.BatchServer(_fake_executor([]), mem_budget=budget, workers=3)
    res = srv.serve(reqs)
    assert len(res) == 30
    assert srv.max_inflight_bytes <= budget
    assert srv.batches > 1


def test_oversize_request_runs_alone():
    ltss = _stream(5, seed=7)
    reqs = [serve.Request(i, l, 0.0) for i, l in enumerate(ltss)]
    calls = []
    srv = serve.BatchServer(_fake_executor(calls), mem_budget=1, workers=2)
    res = srv.serve(reqs)
    assert len(res) == 5 and calls == [1, 1, 1, 1, 1]


def test_max_batch_is_respected():
    ltss = _stream(25, seed=8)
    reqs = [serve.Request(i, l, 0.0) for i, l in enumerate(ltss)]
    calls = []
    srv = serve.BatchServer(_fake_executor(calls), mem_budget=1 << 40, workers=1, max_batch=7)
    srv.serve(reqs)
    assert max(calls) <= 7 and sum(calls) == 25


def test_large_requests_take_their_own_lane():
    ltss = _stream(30, seed=9)
    thr = sorted(l.n for l in ltss)[20]  # the ten largest (ties included) go to the lane
    big_calls, calls = [], []

    def big(lts):
        big_calls.append(lts.n)
        time.sleep(0.001)
        return oracle.ks_lts(lts)

    srv = serve.BatchServer(_fake_executor(calls), mem_budget=1 << 40, workers=2, big_executor=big,
                            big_states=thr, big_backlog=1 << 30)
    res = srv.serve(serve.poisson_requests(ltss, rate_per_s=1000.0, seed=2))
    assert [r.rid for r in res] == list(range(30))
    for r, l in zip(res, ltss):
        assert r.labels.tolist() == oracle.ks_lts(l).tolist()
    assert sorted(big_calls) == sorted(l.n for l in ltss if l.n >= thr)
    assert sum(calls) == sum(1 for l in ltss if l.n < thr)
    assert srv.big_served == len(big_calls)


def test_backed_up_lane_sends_large_requests_to_the_batches():
    ltss = _stream(30, seed=9)
    thr = sorted(l.n for l in ltss)[20]
    big_calls, calls = [], []

    def big(lts):
        big_calls.append(lts.n)
        time.sleep(0.05)  # slow lane: arrivals back it up
        return oracle.ks_lts(lts)

    srv = serve.BatchServer(_fake_executor(calls), mem_budget=1 << 40, workers=2, big_executor=big,
                            big_states=thr, big_backlog=1)
    res = srv.serve([serve.Request(i, l, 0.0) for i, l in enumerate(ltss)])
    assert [r.rid for r in res] == list(range(30))
    for r, l in zip(res, ltss):
        assert r.labels.tolist() == oracle.ks_lts(l).tolist()
    assert len(big_calls) == 1 and sum(calls) == 29  # one lane slot, the rest batched
