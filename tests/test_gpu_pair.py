"""GPU parity of the (C, a)-pair engine: Algorithm 2 one label at a time under
the priority rule, against oracle.pair (identical leader labels and iteration
counts) and against oracle.ks (the partition)."""
import numpy as np
import pytest

import oracle
from oracle import defs
from paper_2105_11788_gb300 import bisim, lts_gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    bisim.load(build_if_missing=True)


def run(lts, **kw):
    return bisim.reduce(lts, bisim.make_opts(engine=bisim.ENGINE_PAIR, **kw), return_stats=True)


def _bounds(lts, want, st):
    B = defs.num_blocks(want)
    pi0 = defs.num_blocks(lts.init) if lts.init is not None and lts.n else min(lts.n, 1)
    nl = max(1, len(set(lts.act.tolist())))
    assert B * nl + 1 <= st.rounds <= (2 * B - pi0) * nl + 1, lts.name


def test_leaders_and_iterations_equal_the_oracle():
    cases = [lts_gen.random_small(s, 30, 1 + s % 4, 80, blocks=1 + s % 3) for s in range(60)]
    cases += [lts_gen.kripke_uniform(), lts_gen.chain(n=400), lts_gen.fan_out(60),
              lts_gen.quotient_expansion(seed=4, classes=60, trans=500, num_act=5, copies_hi=8)]
    for lts in cases:
        labels, rounds = oracle.pair_lts(lts)
        got, st = run(lts, raw_labels=True)
        assert got.tolist() == labels.tolist(), lts.name
        assert st.rounds == rounds and st.pre_rounds == 0, lts.name


def test_one_label_is_algorithm_2():
    for lts in (lts_gen.kripke_uniform(seed=2), lts_gen.chain(n=500)):
        labels, rounds, _ = oracle.pram_lts(lts, alg2=True, skip_preprocess=True)
        got, st = run(lts, raw_labels=True)
        assert got.tolist() == labels.tolist() and st.rounds == rounds


@pytest.mark.parametrize("make", [lambda: lts_gen.quotient_expansion(seed=1),
                                  lambda: lts_gen.chain(seed=2, n=50000),
                                  lambda: lts_gen.powerlaw(seed=3, n=20000)],
                         ids=["qexp-full", "chain-full", "powerlaw-20k"])
def test_larger_workloads_match_ks(make):
    lts = make()
    want = oracle.ks_lts(lts)
    got, st = run(lts)
    assert got.tolist() == want.tolist()
    _bounds(lts, want, st)


def test_edge_cases():
    e = np.zeros(0, dtype=np.int32)
    init = np.array([3, 3, 0, 1, 0, 3], dtype=np.int32)
    lts = lts_gen.LTS("empty", 6, 1, e, e, e, init)
    got, st = run(lts)
    assert got.tolist() == defs.canonical(init).tolist()
    assert st.rounds == 3 + 1  # three selections without labels, then the empty one
    got, _ = run(lts_gen.from_triples(1, 1, [(0, 0, 0)]))
    assert got.tolist() == [0]
    # many labels, most unused; duplicated transitions
    lts = lts_gen.random_small(7, 50, 3, 200)
    lts.num_act = 1000
    lts.act = (lts.act * 300).astype(np.int32)
    dup = lts_gen.LTS("dup", lts.n, lts.num_act, np.concatenate([lts.src, lts.src]),
                      np.concatenate([lts.act, lts.act]), np.concatenate([lts.dst, lts.dst]))
    got, st = run(dup)
    assert got.tolist() == oracle.ks_lts(dup).tolist()
    labels, rounds = oracle.pair_lts(dup)
    assert st.rounds == rounds


def test_round_cap_and_timeout():
    lts = lts_gen.chain(n=200)
    with pytest.raises(bisim.BisimError) as ei:
        run(lts, round_cap=5)
    assert ei.value.code == bisim.BISIM_EROUNDS
    with pytest.raises(bisim.BisimError) as ei:
        run(lts_gen.kripke_uniform(n=500, m=2000), test_hook=1, timeout_ms=200)
    assert ei.value.code == bisim.BISIM_ETIMEOUT
    got, _ = run(lts)
    assert np.array_equal(got, np.arange(200))


def test_batch_path_rejects_the_pair_engine():
    ltss = [lts_gen.random_small(1, 10, 2, 20), lts_gen.random_small(2, 12, 2, 30)]
    with pytest.raises(bisim.BisimError) as ei:
        bisim.reduce_batch(ltss, bisim.make_opts(engine=bisim.ENGINE_PAIR))
    assert ei.value.code == bisim.BISIM_ENOTSUP
