"""Serving loop on the GPU: requests arriving while batches run are admitted
into overlapping batches, and every result is bit-identical to the same LTS
reduced alone through the one-at-a-time path."""
import numpy as np
import pytest

from paper_2105_11788_gb300 import bisim, lts_gen, serve

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    import torch

    assert torch.cuda.is_available()
    bisim.load(build_if_missing=True)
    rng = np.random.default_rng(21)
    ltss = [lts_gen.stream_instance(rng, n_lo=100, n_hi=30000, idx=i) for i in range(60)]
    alone = [bisim.reduce(l) for l in ltss]
    reqs = serve.poisson_requests(ltss, rate_per_s=400.0, seed=2)
    srv = serve.BatchServer(serve.gpu_executor(), mem_budget=8 << 30, workers=3, max_batch=16)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(60))
    for r, a in zip(res, alone):
        assert np.array_equal(r.labels, a)
    assert srv.batches > 1
    s = serve.latency_summary(res)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_large_request_lane_overlaps_the_batches():
    """Large LTSs reduced alone by the single-LTS path (a cooperative launch)
    while batches of small ones run on other streams: results unchanged."""
    rng = np.random.default_rng(22)
    ltss = [lts_gen.stream_instance(rng, n_lo=100, n_hi=60000, idx=i) for i in range(60)]
    alone = [bisim.reduce(l) for l in ltss]
    thr = 20000
    srv = serve.BatchServer(serve.gpu_executor(), mem_budget=8 << 30, workers=3, max_batch=16,
                            big_executor=serve.gpu_single_executor(), big_states=thr, big_backlog=1 << 30)
    res = srv.serve(serve.poisson_requests(ltss, rate_per_s=400.0, seed=3))
    assert [r.rid for r in res] == list(range(60))
    for r, a in zip(res, alone):
        assert np.array_equal(r.labels, a)
    assert srv.big_served == sum(1 for l in ltss if l.n >= thr) > 0
