"""Randomised GPU stress of the frontier schedules: many LTS shapes, every
launch shape and splitter setting, each result against the oracle; and the
same LTS reduced many times in a row (the schedules race by design, the
partition may not change)."""
import numpy as np
import pytest

import oracle
from paper_2105_11788_gb300 import bisim, lts_gen

pytestmark = pytest.mark.gpu

SETTINGS = [dict(threads=t, splitters=k, light_edges=le, split_budget=bud, local_states=-1)
            for t in (128, 512, 1024) for k in (2, 16, 0) for le in (0, -1, 1 << 30) for bud in (0, 3)
            if not (le == -1 and k != 0)]
# the whole LTS on one CTA, or one CTA until a splitter exceeds 8 / 100 states
SETTINGS += [dict(threads=t, splitters=k, split_budget=bud, local_states=lo)
             for t in (128, 1024) for k in (1, 16, 0) for bud in (0, 3) for lo in (1 << 30, 8, 100)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    bisim.load(build_if_missing=True)


def _case(seed):
    rng = np.random.default_rng(9000 + seed)
    kind = seed % 4
    if kind == 0:
        return lts_gen.random_small(seed, int(rng.integers(20, 600)), int(rng.integers(1, 7)),
                                    int(rng.integers(10, 2400)), blocks=int(rng.integers(1, 5)))
    if kind == 1:
        return lts_gen.quotient_expansion(seed=seed, classes=int(rng.integers(20, 300)),
                                          trans=int(rng.integers(50, 3000)), num_act=int(rng.integers(1, 9)),
                                          copies_hi=int(rng.integers(2, 30)))
    if kind == 2:
        return lts_gen.powerlaw(seed=seed, n=int(rng.integers(200, 5000)), num_act=int(rng.integers(1, 12)))
    return lts_gen.stream_instance(rng, n_lo=100, n_hi=4000, idx=seed)


@pytest.mark.parametrize("chunk", range(8))
def test_random_shapes_all_settings(chunk):
    for seed in range(chunk * 12, chunk * 12 + 12):
        lts = _case(seed)
        want = oracle.ks_lts(lts).tolist()
        for kw in SETTINGS:
            got = bisim.reduce(lts, bisim.make_opts(engine=bisim.ENGINE_FRONTIER, **kw))
            assert got.tolist() == want, (lts.name, kw)


def test_repeated_runs_give_the_same_partition():
    lts = lts_gen.quotient_expansion(seed=17, classes=400, trans=4000, copies_hi=40)
    want = oracle.ks_lts(lts).tolist()
    rounds = set()
    for _ in range(25):
        got, st = bisim.reduce(lts, return_stats=True)
        assert got.tolist() == want
        rounds.add(st.rounds)
    assert all(r >= int(max(want)) + 2 for r in rounds)
