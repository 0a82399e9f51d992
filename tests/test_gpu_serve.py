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
