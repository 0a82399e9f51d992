"""GPU parity of the batch path (bisim_batch_plan / bisim_batch_refine): every
LTS of a batch gets exactly the oracle's partition, and exactly what the
one-at-a-time path returns."""
import numpy as np
import pytest

import oracle
from paper_2105_11788_gb300 import bisim, lts_gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    bisim.load(build_if_missing=True)


def _random_batch(seed, k):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(1, 60))
        A = int(rng.integers(1, 6))
        m = int(rng.integers(0, 5 * n))
        out.append(lts_gen.random_small(seed * 1000 + i, n, A, m, blocks=int(rng.integers(1, 4))))
    return out


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_random_batch_vs_oracle(threads):
    ltss = _random_batch(7, 300)
    parts, st, inst = bisim.reduce_batch(ltss, bisim.make_opts(threads=threads), return_stats=True)
    for i, (l, got) in enumerate(zip(ltss, parts)):
        want = oracle.ks_lts(l)
        assert got.tolist() == want.tolist(), i
        assert inst[i].num_blocks == int(want.max()) + 1
        B = int(want.max()) + 1
        assert B + 1 <= inst[i].rounds <= 3 * l.n + l.num_act + 2


def test_stream_instances_match_single_path_and_oracle():
    rng = np.random.default_rng(44)
    ltss = [lts_gen.stream_instance(rng, n_lo=100, n_hi=20000, idx=i) for i in range(48)]
    parts = bisim.reduce_batch(ltss)
    for l, got in zip(ltss, parts):
        assert got.tolist() == oracle.ks_lts(l).tolist()
        assert got.tolist() == bisim.reduce(l).tolist()


def test_mixed_workloads_in_one_batch():
    ltss = [lts_gen.kripke_uniform(seed=0), lts_gen.chain(n=3000), lts_gen.fan_out(300),
            lts_gen.quotient_expansion(seed=5, classes=300, trans=3000, copies_hi=30)]
    parts = bisim.reduce_batch(ltss)
    for l, got in zip(ltss, parts):
        assert got.tolist() == oracle.ks_lts(l).tolist()


def test_batch_edge_cases():
    e = np.zeros(0, dtype=np.int32)
    ltss = [lts_gen.LTS("empty", 4, 1, e, e, e, np.array([0, 0, 3, 3], np.int32)),
            lts_gen.from_triples(1, 1, [(0, 0, 0)]),
            lts_gen.LTS("none", 0, 1, e, e, e),
            lts_gen.from_triples(3, 2, [(0, 1, 1), (1, 1, 2)])]
    parts = bisim.reduce_batch(ltss)
    assert parts[0].tolist() == [0, 0, 1, 1]
    assert parts[1].tolist() == [0]
    assert parts[2].tolist() == []
    assert parts[3].tolist() == oracle.ks_lts(ltss[3]).tolist()


def test_batch_rejects_out_of_range_local_ids():
    bad = [lts_gen.from_triples(3, 1, [(0, 0, 1)]), lts_gen.from_triples(2, 1, [(0, 0, 2)])]
    with pytest.raises(bisim.BisimError) as ei:
        bisim.reduce_batch(bad)
    assert ei.value.code == bisim.BISIM_EINVAL
    bad = [lts_gen.from_triples(3, 2, [(0, 1, 1)]), lts_gen.from_triples(2, 1, [(0, 1, 1)])]
    with pytest.raises(bisim.BisimError) as ei:
        bisim.reduce_batch(bad)
    assert ei.value.code == bisim.BISIM_EINVAL


def test_batch_refine_twice_on_one_plan():
    import torch

    ltss = _random_batch(9, 50)
    so, to, na, src, act, dst, init = bisim.pack_batch(ltss)
    d = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    tsrc, tact, tdst, tinit = d(src), d(act), d(dst), d(init)
    N = int(so[-1])
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    h = bisim.bisim_batch_plan(len(ltss), so, to, na, tsrc.data_ptr(), tact.data_ptr(), tdst.data_ptr(),
                               tinit.data_ptr())
    try:
        bisim.bisim_batch_refine(h, out.data_ptr(), len(ltss))
        first = out.cpu().numpy().copy()
        bisim.bisim_batch_refine(h, out.data_ptr(), len(ltss))
        second = out.cpu().numpy()
    finally:
        bisim.bisim_plan_destroy(h)
    assert np.array_equal(first, second)
    for i, l in enumerate(ltss):
        assert first[so[i]:so[i + 1]].tolist() == oracle.ks_lts(l).tolist()


def test_split_schedule_matches_single_launch():
    """Largest LTSs in a concurrent wide launch: same results."""
    rng = np.random.default_rng(31)
    ltss = [lts_gen.stream_instance(rng, n_lo=100, n_hi=30000, idx=i) for i in range(64)]
    want = bisim.reduce_batch(ltss)
    for wthr, wmin in ((1024, 5000), (512, 1), (256, 1 << 30)):
        got = bisim.reduce_batch(ltss, bisim.make_opts(threads=128, wide_threads=wthr, wide_min_states=wmin))
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
    for l, g in zip(ltss[:16], want[:16]):
        assert g.tolist() == oracle.ks_lts(l).tolist()


@pytest.mark.parametrize("splitters,multi_min", [(1, 0), (4, 0), (0, 0), (16, 3000)],
                         ids=["one", "four", "default", "large-only"])
def test_batch_several_splitters_per_round(splitters, multi_min):
    """CTA rounds with several splitters: oracle partitions, identical to one
    splitter per round, and the per-LTS iteration bounds hold."""
    rng = np.random.default_rng(77)
    ltss = [lts_gen.stream_instance(rng, n_lo=100, n_hi=8000, idx=i) for i in range(40)]
    ltss += _random_batch(12, 60)
    parts, st, inst = bisim.reduce_batch(ltss, bisim.make_opts(splitters=splitters, split_budget=8 if multi_min else 0,
                                                               multi_min_states=multi_min), return_stats=True)
    for i, (l, got) in enumerate(zip(ltss, parts)):
        want = oracle.ks_lts(l)
        assert got.tolist() == want.tolist(), i
        B = int(want.max()) + 1 if l.n else 0
        assert B + 1 <= inst[i].rounds <= 3 * l.n + l.num_act + 2
    assert st.steps <= st.rounds
