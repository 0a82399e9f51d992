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


def test_footprint_covers_what_the_library_allocates():
    """Admission counts footprint_bytes per request. The library's own
    allocations (the device pool's high-water mark over a batched and a
    single-LTS reduction; the inputs on the device come from torch's
    allocator and footprint_bytes counts them too) stay within it, and not
    far below it; trimming gives the pool's unused memory back."""
    rng = np.random.default_rng(23)
    ltss = [lts_gen.stream_instance(rng, n_lo=1000, n_hi=100000, idx=i) for i in range(48)]
    cases = [("batch", ltss, lambda: bisim.reduce_batch(ltss)),
             ("single", [ltss[0]], lambda: bisim.reduce(ltss[0]))]
    for name, group, run in cases:
        import torch

        torch.cuda.synchronize()
        before = bisim.bisim_pool_usage()["used"]
        bisim.bisim_pool_reset_high()
        run()
        torch.cuda.synchronize()
        peak = bisim.bisim_pool_usage()["used_high"] - before
        budget = sum(serve.footprint_bytes(l.n, l.m, l.num_act) for l in group)
        assert 0 < peak <= budget, (name, peak, budget)
        assert peak >= budget // 4, (name, peak, budget)
    serve.gpu_trim()
    u = bisim.bisim_pool_usage()
    assert u["reserved"] - u["used"] <= 64 << 20
