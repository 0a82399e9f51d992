"""Full-size parity of the batched and served stream (4,096 LTSs with n
log-uniform in [100, 200,000], 107,689,033 states and 538,565,985
transitions in all): every LTS of the one-launch batch equals the oracle,
every LTS of at least 100,000 states also equals the one-at-a-time path, and
a serving run whose requests include such LTSs - in the batch lane and in the
large-request lane - returns the one-at-a-time results. The oracle runs in a
pool of spawned worker processes (about 100 s of CPU in all)."""
import numpy as np
import pytest

import oracle
from paper_2105_11788_gb300 import autotune, bisim, lts_gen, serve

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BIG = 100_000


@pytest.fixture(scope="module")
def stream():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    bisim.load(build_if_missing=True)
    ltss, _ = lts_gen.batch_stream(seed=4, k=4096)
    assert sum(l.n for l in ltss) == 107_689_033 and sum(l.m for l in ltss) == 538_565_985
    return ltss


@pytest.fixture(scope="module")
def want(stream):
    return oracle.ks_many(stream)


def _check_all(parts, want):
    bad = [i for i, (g, w) in enumerate(zip(parts, want)) if not np.array_equal(g, w)]
    assert not bad, f"{len(bad)} LTSs differ from the oracle, first {bad[:5]}"


def test_full_stream_batch_matches_oracle(stream, want):
    """One batch plan and one launch over all 4,096 LTSs: default launch shape."""
    parts, st, inst = bisim.reduce_batch(stream, return_stats=True)
    _check_all(parts, want)
    for i, (l, w) in enumerate(zip(stream, want)):
        B = int(w.max()) + 1
        assert B + 1 <= inst[i].rounds <= 3 * l.n + l.num_act + 2, i


def test_full_stream_batch_in_the_tuned_launch_shape(stream, want, tmp_path):
    """The launch shape the benchmark's autotuner picks for this batch."""
    tuner = autotune.BatchTuner(cache_path=str(tmp_path / "tune.json"), repeats=1)
    opts, rec = tuner.tune(stream)
    parts = bisim.reduce_batch(stream, opts)
    _check_all(parts, want)


def test_large_stream_lts_equal_the_one_at_a_time_path(stream, want):
    big = [i for i, l in enumerate(stream) if l.n >= BIG]
    assert len(big) > 300
    for i in big:
        got = bisim.reduce(stream[i])
        assert np.array_equal(got, want[i]), i


@pytest.mark.parametrize("lane", ["batch", "large"])
def test_serving_with_large_requests(stream, want, lane):
    """Requests of at least 100,000 states served in the batch lane or in the
    large-request lane, mixed with small ones: the oracle's partitions."""
    big = [i for i, l in enumerate(stream) if l.n >= BIG][:8]
    small = [i for i, l in enumerate(stream) if l.n < 20_000][:24]
    idx = sorted(big + small)
    reqs = serve.poisson_requests([stream[i] for i in idx], rate_per_s=200.0, seed=5)
    kw = {}
    if lane == "large":
        kw = dict(big_executor=serve.gpu_single_executor(), big_states=BIG, big_backlog=1 << 30)
    srv = serve.BatchServer(serve.gpu_executor(), mem_budget=32 << 30, workers=3, max_batch=16, **kw)
    res = srv.serve(reqs)
    assert [r.rid for r in res] == list(range(len(idx)))
    for r, i in zip(res, idx):
        assert np.array_equal(r.labels, want[i]), i
    if lane == "large":
        assert srv.big_served == len(big)
    else:
        assert srv.big_served == 0
