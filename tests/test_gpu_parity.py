"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit-exact on canonical block ids, plus the PRAM round counts and leader
labels of the dense engine under the priority rule."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import defs
from paper_2105_11788_gb300 import bisim, lts_gen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# the frontier engine twice: the hybrid/grid schedule, and one CTA for the whole LTS
FRONTIER_GRID = dict(engine=bisim.ENGINE_FRONTIER, local_states=-1)
FRONTIER_LOCAL = dict(engine=bisim.ENGINE_FRONTIER, local_states=1 << 30)
ENGINES = [dict(engine=bisim.ENGINE_DENSE), FRONTIER_GRID, FRONTIER_LOCAL]
ENGINE_IDS = ["dense", "frontier", "frontier-local"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    bisim.load(build_if_missing=True)


def run(lts, engine=bisim.ENGINE_AUTO, **kw):
    kw = {**engine, **kw} if isinstance(engine, dict) else {"engine": engine, **kw}
    return bisim.reduce(lts, bisim.make_opts(**kw), return_stats=True)


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _lts_from_golden(g, init=None):
    return lts_gen.from_triples(g["n"], g["num_act"], g["transitions"], init)


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_paper_examples(engine):
    g1 = _golden("fig1_iteration.json")
    lts = _lts_from_golden(g1, g1["block_before"])
    got, st = run(lts, engine)
    assert got.tolist() == [0, 1, 2, 3, 3]
    g3 = _golden("fig3_preprocessing.json")
    got, st = run(_lts_from_golden(g3), engine)
    assert got.tolist() == [0, 1, 2]
    assert st.mark_length == 6 and st.pre_rounds == 3


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_random_small_vs_oracle(engine):
    for seed in range(150):
        rng = np.random.default_rng(5000 + seed)
        n = int(rng.integers(1, 40))
        A = int(rng.integers(1, 5))
        m = int(rng.integers(0, 4 * n))
        lts = lts_gen.random_small(seed, n, A, m, blocks=int(rng.integers(1, 4)))
        want = oracle.ks_lts(lts)
        got, st = run(lts, engine)
        assert got.tolist() == want.tolist(), (seed, n, A, m)
        assert st.num_blocks == defs.num_blocks(want)


@pytest.mark.slow
def test_dense_matches_pram_on_the_full_chain():
    """The 50,000-state chain (99,999 iterations): the dense engine's leader
    labels and iteration count equal the lock-step PRAM simulation exactly,
    with Algorithm 3 and with Algorithm 2 (one label)."""
    lts = lts_gen.chain(seed=2, n=50000)
    for alg2 in (False, True):
        labels, rounds, pre = oracle.pram_lts(lts, alg2=alg2)
        got, st = run(lts, bisim.ENGINE_DENSE, raw_labels=True, rcpp_alg2=alg2)
        assert got.tolist() == labels.tolist()
        assert st.rounds == rounds and st.pre_rounds == pre


def test_dense_matches_pram_rounds_and_leaders():
    """Priority rule on both sides: identical leader labels and iteration
    counts (Algorithm 3, and Algorithm 2 for one label)."""
    cases = [lts_gen.random_small(s, 30, 1 + s % 3, 70, blocks=2) for s in range(40)]
    cases.append(lts_gen.kripke_uniform())
    cases.append(lts_gen.chain(n=300))
    cases.append(lts_gen.fan_out(40))
    for lts in cases:
        for alg2 in ([False, True] if lts.num_act == 1 else [False]):
            labels, rounds, pre = oracle.pram_lts(lts, alg2=alg2)
            got, st = run(lts, bisim.ENGINE_DENSE, raw_labels=True, rcpp_alg2=alg2)
            assert got.tolist() == labels.tolist(), lts.name
            assert st.rounds == rounds and st.pre_rounds == pre, lts.name


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_kripke_1000(engine):
    lts = lts_gen.kripke_uniform(seed=0)
    got, st = run(lts, engine)
    want = oracle.ks_lts(lts)
    assert got.tolist() == want.tolist()
    B = defs.num_blocks(want)
    assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_quotient_expansion_full_size(engine):
    """~100k states, ~1.1M transitions, 8 Zipf labels: equal to the oracle
    and to the quotient's partition pulled back through the class map."""
    lts = lts_gen.quotient_expansion(seed=1)
    got, st = run(lts, engine)
    want = oracle.ks_lts(lts)
    assert got.tolist() == want.tolist()
    assert got.tolist() == defs.pullback(lts.cls, oracle.ks_lts(lts.quotient)).tolist()
    B = defs.num_blocks(want)
    assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1
    # the definitions, checked on the GPU's output directly
    assert defs.is_stable(lts.n, lts.src, lts.act, lts.dst, got)
    assert defs.refines(got, np.zeros(lts.n, dtype=np.int32))


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_chain_full_size(engine):
    """Closed form: the 50,000-state chain is discrete; B+1 <= rounds <= 3n-2+1."""
    n = 50000
    lts = lts_gen.chain(seed=2, n=n)
    got, st = run(lts, engine)
    assert np.array_equal(got, np.arange(n, dtype=np.int32))
    assert n + 1 <= st.rounds <= 3 * n - 2 + 1


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_fan_out(engine):
    for n in (3, 10, 100, 700):
        got, _ = run(lts_gen.fan_out(n), engine)
        assert got.tolist() == [0, 0] + list(range(1, n - 1))


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_edge_cases(engine):
    e = np.zeros(0, dtype=np.int32)
    # no transitions: the initial partition itself
    init = np.array([3, 3, 0, 1, 0, 3], dtype=np.int32)
    got, st = run(lts_gen.LTS("empty", 6, 1, e, e, e, init), engine)
    assert got.tolist() == defs.canonical(init).tolist()
    assert st.rounds == 3 + 1
    # one state, self loop
    got, _ = run(lts_gen.from_triples(1, 1, [(0, 0, 0)]), engine)
    assert got.tolist() == [0]
    # many labels, most unused; duplicates
    lts = lts_gen.random_small(7, 50, 3, 200)
    lts.num_act = 1000
    lts.act = (lts.act * 300).astype(np.int32)
    src = np.concatenate([lts.src, lts.src]); act = np.concatenate([lts.act, lts.act])
    dst = np.concatenate([lts.dst, lts.dst])
    dup = lts_gen.LTS("dup", lts.n, lts.num_act, src, act, dst)
    got, st = run(dup, engine)
    assert got.tolist() == oracle.ks_lts(dup).tolist()
    assert st.pre_rounds == 3


def test_invalid_inputs_are_rejected():
    bad = lts_gen.from_triples(3, 2, [(0, 0, 1), (2, 1, 3)])
    with pytest.raises(bisim.BisimError) as ei:
        run(bad)
    assert ei.value.code == bisim.BISIM_EINVAL
    bad = lts_gen.from_triples(3, 2, [(0, 2, 1)])
    with pytest.raises(bisim.BisimError) as ei:
        run(bad)
    assert ei.value.code == bisim.BISIM_EINVAL
    bad = lts_gen.from_triples(3, 1, [(0, 0, 1)], init=[0, 5, 0])
    with pytest.raises(bisim.BisimError) as ei:
        run(bad)
    assert ei.value.code == bisim.BISIM_EINVAL
    # still usable afterwards (states 1 and 2 are both deadlocked)
    got, _ = run(lts_gen.from_triples(3, 1, [(0, 0, 1)]))
    assert got.tolist() == [0, 1, 1]


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_round_cap_reports_error(engine):
    lts = lts_gen.chain(n=200)
    with pytest.raises(bisim.BisimError) as ei:
        run(lts, engine, round_cap=5)
    assert ei.value.code == bisim.BISIM_EROUNDS
    got, _ = run(lts, engine)
    assert np.array_equal(got, np.arange(200))


@pytest.mark.parametrize("engine", ENGINES[:2], ids=ENGINE_IDS[:2])
def test_barrier_wait_times_out_and_context_survives(engine):
    """CTA 0 never arrives at its first barrier (a flag nothing sets); the
    other CTAs give up after the time limit and the call reports it."""
    lts = lts_gen.kripke_uniform(n=500, m=2000)
    with pytest.raises(bisim.BisimError) as ei:
        run(lts, engine, test_hook=1, timeout_ms=200)
    assert ei.value.code == bisim.BISIM_ETIMEOUT
    got, _ = run(lts, engine)
    assert got.tolist() == oracle.ks_lts(lts).tolist()


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_refine_twice_same_plan(engine):
    import torch

    lts = lts_gen.quotient_expansion(seed=9, classes=300, trans=3000, copies_hi=20)
    d = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    with bisim.Plan(lts.n, lts.num_act, d(lts.src), d(lts.act), d(lts.dst), None,
                    bisim.make_opts(**engine)) as p:
        a, s1 = p.refine()
        a = a.cpu().numpy()
        b, s2 = p.refine()
        b = b.cpu().numpy()
    assert np.array_equal(a, b)
    assert a.tolist() == oracle.ks_lts(lts).tolist()


def test_host_buffer_entry_point():
    lts = lts_gen.quotient_expansion(seed=3, classes=200, trans=2000, copies_hi=10)
    out = np.empty(lts.n, dtype=np.int32)
    p = lambda a: a.ctypes.data  # noqa: E731
    st = bisim.bisim_reduce_host(lts.n, lts.m, lts.num_act, p(lts.src), p(lts.act), p(lts.dst),
                                 None, p(out))
    assert out.tolist() == oracle.ks_lts(lts).tolist()
    assert st.num_blocks == defs.num_blocks(out)


def test_host_buffer_entry_point_with_initial_partition():
    """All four input arrays from host memory (copied on separate streams
    before the plan), pageable and pinned, with and without the labels."""
    import torch

    lts = lts_gen.kripke_uniform(seed=5, n=20000, m=80000)
    want = oracle.ks_lts(lts).tolist()
    for pinned in (False, True):
        conv = (lambda a: torch.from_numpy(a).pin_memory()) if pinned else torch.from_numpy
        src, act, dst, init = conv(lts.src), conv(lts.act), conv(lts.dst), conv(lts.init)
        out = torch.empty(lts.n, dtype=torch.int32)
        if pinned:
            out = out.pin_memory()
        for with_act in (True, False):
            bisim.bisim_reduce_host(lts.n, lts.m, lts.num_act, src.data_ptr(),
                                    act.data_ptr() if with_act else None, dst.data_ptr(), init.data_ptr(),
                                    out.data_ptr())
            if with_act or lts.num_act == 1:
                assert out.tolist() == want


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_launch_shapes(engine):
    lts = lts_gen.quotient_expansion(seed=4, classes=400, trans=4000, copies_hi=30)
    want = oracle.ks_lts(lts)
    for threads, per_sm in ((128, 1), (256, 2), (1024, 1)):
        got, _ = run(lts, engine, threads=threads, ctas_per_sm=per_sm)
        assert got.tolist() == want.tolist(), (threads, per_sm)


@pytest.mark.parametrize("light_edges,local", [(-1, 0), (0, -1), (1 << 30, -1), (0, 1 << 30)],
                         ids=["grid", "hybrid", "all-light", "one-cta"])
def test_frontier_schedules(light_edges, local):
    """Frontier rounds on the whole grid, hybrid (light rounds on one CTA),
    every eligible round light, and the whole LTS on one CTA: same
    partitions."""
    cases = [lts_gen.random_small(100 + s, 40, 1 + s % 3, 120, blocks=2) for s in range(30)]
    cases += [lts_gen.kripke_uniform(), lts_gen.chain(n=2000), lts_gen.fan_out(200),
              lts_gen.quotient_expansion(seed=6, classes=500, trans=5000, copies_hi=40)]
    for lts in cases:
        got, st = run(lts, bisim.ENGINE_FRONTIER, light_edges=light_edges, local_states=local)
        assert got.tolist() == oracle.ks_lts(lts).tolist(), lts.name
        assert (st.grid_ctas == 1) == (local > 0), lts.name


def test_one_cta_start_and_hand_off():
    """A sparse LTS (m <= 4n) starts on one CTA; a denser one takes the hybrid
    schedule. A round whose splitter holds more than local_states states, or
    (by default) a run of rounds in which most splitters win, hands the rest
    of the refinement to the grid: same partition."""
    n = 8192
    got, st = run(lts_gen.fan_out(n), bisim.ENGINE_FRONTIER)
    assert st.grid_ctas == 1 and got.tolist() == [0, 0] + list(range(1, n - 1))
    assert st.local_steps == st.steps
    dense = lts_gen.quotient_expansion(seed=4, classes=400, trans=4000, copies_hi=30)
    assert dense.m > 4 * dense.n
    got, st = run(dense, bisim.ENGINE_FRONTIER)
    assert st.grid_ctas > 1 and got.tolist() == oracle.ks_lts(dense).tolist()
    assert st.local_steps == 0
    # 100 singleton blocks on a chain, then a 1,900-state cycle that no
    # singleton splits: its round (1,900 > 512 states) goes to the grid
    big, small = 1900, 100
    trip = [(i, 0, (i + 1) % big) for i in range(big)]
    trip += [(big + i, 0, big + i + 1) for i in range(small - 1)]
    init = [0] * big + list(range(1, small + 1))
    lts = lts_gen.from_triples(big + small, 1, trip, init)
    got, st = run(lts, bisim.ENGINE_FRONTIER, local_states=512)
    assert got.tolist() == defs.canonical(np.array(init, dtype=np.int32)).tolist()
    assert st.grid_ctas > 1 and st.rounds >= small + 1
    assert 0 < st.local_steps < st.steps  # the singletons' rounds ran on one CTA
    got, st = run(lts, bisim.ENGINE_FRONTIER, local_states=4096)
    assert st.grid_ctas == 1 and got.tolist() == defs.canonical(np.array(init, dtype=np.int32)).tolist()
    # a sparse power-law LTS: thousands of independent small splitters
    lts = lts_gen.powerlaw(seed=3, n=20000, mean_deg=3.0)
    assert lts.m <= 4 * lts.n
    got, st = run(lts, bisim.ENGINE_FRONTIER)
    assert st.grid_ctas > 1 and got.tolist() == oracle.ks_lts(lts).tolist()
    # one splitter per round on one CTA
    lts = lts_gen.kripke_uniform()
    got, st = run(lts, bisim.ENGINE_FRONTIER, splitters=1, threads=256)
    assert got.tolist() == oracle.ks_lts(lts).tolist()
    assert st.grid_ctas == 1 and st.steps == st.rounds


@pytest.mark.parametrize("local", [16, 64, 300])
def test_hand_off_at_random_points(local):
    """Hand-offs from one CTA to the grid wherever a splitter first exceeds
    the threshold: every partition equals the oracle's, and the splitter
    iterations obey the bounds."""
    cases = [lts_gen.random_small(700 + s, 200, 1 + s % 3, 500, blocks=1 + s % 4) for s in range(20)]
    cases += [lts_gen.kripke_uniform(seed=5), lts_gen.chain(n=3000), lts_gen.fan_out(500),
              lts_gen.quotient_expansion(seed=6, classes=500, trans=5000, copies_hi=40)]
    for lts in cases:
        want = oracle.ks_lts(lts)
        got, st = run(lts, bisim.ENGINE_FRONTIER, local_states=local)
        assert got.tolist() == want.tolist(), lts.name
        B = defs.num_blocks(want)
        assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1, lts.name
        assert st.steps <= st.rounds


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_preprocessing_rounds_and_direct_grouping_agree(engine):
    """Algorithm 5 one label at a time and the direct grouping by (initial
    block, label set) give the same partition and the same |pi_0'|."""
    cases = [lts_gen.random_small(300 + s, 60, 1 + s % 5, 200, blocks=1 + s % 3) for s in range(25)]
    cases += [lts_gen.quotient_expansion(seed=8, classes=400, trans=4000, num_act=20, copies_hi=20),
              lts_gen.kripke_uniform(seed=3)]
    for lts in cases:
        want = oracle.ks_lts(lts).tolist()
        got1, st1 = run(lts, engine, preprocess=1)
        got2, st2 = run(lts, engine, preprocess=2)
        assert got1.tolist() == want and got2.tolist() == want, lts.name
        assert st1.initial_blocks == st2.initial_blocks
        assert st1.pre_rounds == st2.pre_rounds


@pytest.mark.parametrize("local", [-1, 1 << 30], ids=["grid", "one-cta"])
@pytest.mark.parametrize("splitters", [1, 2, 7, 0], ids=["one", "two", "seven", "default"])
def test_several_splitters_per_round(splitters, local):
    """Rounds that take several splitters at once (deferring those whose
    touched blocks overlap) give the oracle's partition; the splitter
    iterations still obey B + 1 <= rounds <= 3B - |pi_0'| + 1, and there are
    never more barrier rounds than splitter iterations."""
    cases = [lts_gen.random_small(500 + s, 50, 1 + s % 4, 160, blocks=1 + s % 3) for s in range(30)]
    cases += [lts_gen.kripke_uniform(), lts_gen.chain(n=3000), lts_gen.fan_out(150),
              lts_gen.quotient_expansion(seed=6, classes=500, trans=5000, copies_hi=40),
              lts_gen.powerlaw(seed=3, n=20000)]
    for lts in cases:
        got, st = run(lts, bisim.ENGINE_FRONTIER, splitters=splitters, local_states=local)
        want = oracle.ks_lts(lts)
        assert got.tolist() == want.tolist(), lts.name
        B = defs.num_blocks(want)
        assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1, lts.name
        assert st.steps <= st.rounds
        if splitters == 1:
            assert st.steps == st.rounds


def test_several_splitters_large_worklist():
    """A power-law LTS whose refinement keeps thousands of small blocks
    unstable at once: rounds with up to 1024 splitters on the whole grid."""
    lts = lts_gen.powerlaw(seed=3, n=200000)
    got, st = run(lts, bisim.ENGINE_FRONTIER)
    assert got.tolist() == oracle.ks_lts(lts).tolist()
    assert st.steps * 4 < st.rounds  # many splitters per barrier round


def _hub_lts(seed, n, hubs, hub_deg, deg=6, num_act=2):
    """A few states with very many successors (hubs) among states of small
    out-degree, two initial blocks: the hubs share label sets and initial
    blocks, so their blocks are split state by state by many splitters."""
    rng = np.random.default_rng(seed)
    src = [np.repeat(np.arange(n, dtype=np.int64), deg)]
    src.append(np.repeat(np.arange(hubs, dtype=np.int64), hub_deg))
    src = np.concatenate(src)
    dst = rng.integers(0, n, src.size)
    act = rng.integers(0, num_act, src.size)
    init = rng.integers(0, 2, n).astype(np.int32)
    init[:hubs] = 0
    perm = rng.permutation(src.size)
    return lts_gen.LTS(f"hubs_s{seed}_n{n}", n, num_act, src[perm].astype(np.int32), act[perm].astype(np.int32),
                       dst[perm].astype(np.int32), init)


@pytest.mark.parametrize("peel,items", [(0, 0), (0, 1), (0, 8), (0, 24), (0, 64), (-1, 0)],
                         ids=["default", "one-per-warp", "8-per-warp", "24-per-warp", "64-per-warp",
                              "exclusive-only"])
def test_peel_rounds(peel, items):
    """Grid rounds where several splitters of one state may split the same
    block (each marking one member of it, not its leader): the oracle's
    partition, the iteration bounds of Theorem 3, and - with the default - far
    fewer barrier rounds than iterations on LTSs with hub blocks."""
    cases = [_hub_lts(1, 5000, 50, 400), _hub_lts(2, 20000, 200, 2000, num_act=3),
             _hub_lts(3, 3000, 3, 3000, deg=2, num_act=1),
             lts_gen.powerlaw(seed=3, n=200000), lts_gen.powerlaw(seed=8, n=50000, num_act=4),
             lts_gen.kripke_uniform(seed=3, n=20000, m=80000),
             lts_gen.quotient_expansion(seed=6, classes=500, trans=5000, copies_hi=40),
             lts_gen.fan_out(300), lts_gen.chain(n=2000)]
    cases += [lts_gen.random_small(700 + s, 60, 1 + s % 3, 240, blocks=1 + s % 3) for s in range(20)]
    for lts in cases:
        got, st = run(lts, bisim.ENGINE_FRONTIER, local_states=-1, peel=peel, peel_items=items)
        want = oracle.ks_lts(lts)
        assert got.tolist() == want.tolist(), lts.name
        B = defs.num_blocks(want)
        assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1, lts.name
        assert st.steps <= st.rounds
    if peel == 0 and items == 0:
        _, st = run(lts_gen.powerlaw(seed=3, n=200000), bisim.ENGINE_FRONTIER, local_states=-1)
        assert st.steps * 20 < st.rounds


@pytest.mark.parametrize("n,local", [(10_000, 0), (10_000, 1 << 30), (200_000, 0)])
def test_fan_out_large_closed_form(n, local):
    """Fan_out_n far beyond the paper's sizes: states 0 and 1 together, every
    other state alone (n - 1 blocks)."""
    got, st = run(lts_gen.fan_out(n), bisim.ENGINE_FRONTIER, local_states=local)
    assert np.array_equal(got, np.concatenate([[0, 0], np.arange(1, n - 1)]).astype(np.int32))
    assert st.num_blocks == n - 1


def test_vector_and_unaligned_input_paths():
    """Transition arrays are read four at a time when they start on a 16-byte
    boundary: a bad entry inside that part is caught, and arrays that start
    4 bytes past a boundary (read one by one) give the same partition."""
    import torch

    lts = lts_gen.random_small(61, 300, 3, 1000, blocks=2)
    bad = lts_gen.LTS("bad", lts.n, lts.num_act, lts.src.copy(), lts.act.copy(), lts.dst.copy(), lts.init)
    bad.dst[501] = lts.n  # out of range, inside the int4 part
    with pytest.raises(bisim.BisimError) as ei:
        run(bad)
    assert ei.value.code == bisim.BISIM_EINVAL
    bad = lts_gen.LTS("bad", lts.n, lts.num_act, lts.src.copy(), lts.act.copy(), lts.dst.copy(), lts.init)
    bad.act[502] = lts.num_act
    with pytest.raises(bisim.BisimError) as ei:
        run(bad)
    assert ei.value.code == bisim.BISIM_EINVAL
    pad = lambda a: torch.from_numpy(np.concatenate([[0], a]).astype(np.int32)).cuda()[1:]  # noqa: E731
    src, act, dst = pad(lts.src), pad(lts.act), pad(lts.dst)
    assert src.data_ptr() % 16 != 0
    with bisim.Plan(lts.n, lts.num_act, src, act, dst, torch.from_numpy(lts.init).cuda()) as p:
        got, _ = p.refine()
    assert got.cpu().numpy().tolist() == oracle.ks_lts(lts).tolist()


def _plan_arrays(lts, **kw):
    import torch

    d = lambda a: None if a is None else torch.from_numpy(a).cuda()  # noqa: E731
    with bisim.Plan(lts.n, lts.num_act, d(lts.src), d(lts.act), d(lts.dst), d(lts.init),
                    bisim.make_opts(**kw)) as p:
        return bisim.bisim_plan_arrays(p.handle, lts.n, lts.m)


@pytest.mark.parametrize("slots", [0, 1], ids=["label-sets", "sort"])
def test_plan_arrays_equal_algorithm4(slots):
    """The plan's mark-slot layout and incoming-transition index against the
    oracle's Algorithm 4 (sort by (source, label), order, nr_marks, off as
    start offsets): off, the owner and label of every slot, in_ptr, and per
    target the multiset of (source, slot) entries. Both routes (label sets;
    the sort) give the same arrays."""
    g = _golden("fig3_preprocessing.json")
    cases = [_lts_from_golden(g)]
    cases += [lts_gen.random_small(900 + s, 40, a, 200, blocks=2) for s, a in enumerate((1, 3, 32, 33, 70, 128))]
    cases += [lts_gen.random_small(950, 30, 200, 150), lts_gen.fan_out(50),
              lts_gen.quotient_expansion(seed=6, classes=300, trans=3000, copies_hi=20),
              lts_gen.powerlaw(seed=3, n=20000)]
    for lts in cases:
        got = _plan_arrays(lts, slots=slots, small=-1)  # the grid plan (a small LTS keeps no such arrays)
        ref = oracle.plan(lts.n, lts.num_act, lts.src, lts.act, lts.dst)
        off = ref["off"].astype(np.int64)
        L = ref["mark_length"]
        assert got["mark_length"] == L, lts.name
        assert got["off"][:lts.n].tolist() == off.tolist() and got["off"][lts.n] == L, lts.name
        s_sorted = lts.src[ref["perm"]].astype(np.int64)
        a_sorted = lts.act[ref["perm"]].astype(np.int64)
        slot_sorted = off[s_sorted] + ref["order"]
        want_src = np.zeros(L, np.int64)
        want_act = np.zeros(L, np.int64)
        want_src[slot_sorted] = s_sorted
        want_act[slot_sorted] = a_sorted
        assert got["slot_src"].tolist() == want_src.tolist(), lts.name
        assert got["slot_act"].tolist() == want_act.tolist(), lts.name
        indeg = np.bincount(lts.dst, minlength=lts.n)
        assert got["in_ptr"].tolist() == np.concatenate([[0], np.cumsum(indeg)]).tolist(), lts.name
        # per target, the multiset of (source << 32 | slot)
        d_sorted = lts.dst[ref["perm"]].astype(np.int64)
        want = np.sort((d_sorted << 40) | (s_sorted << 20) | slot_sorted) if lts.n < (1 << 20) else None
        ie = got["in_edge"]
        tgt = np.repeat(np.arange(lts.n, dtype=np.int64), indeg)
        have = np.sort((tgt << 40) | ((ie >> 32) << 20) | (ie & 0xffffffff))
        if want is not None:
            assert have.tolist() == want.tolist(), lts.name


def _small_cases():
    cases = [lts_gen.random_small(1200 + s, int(5 + 7 * s), 1 + s % 4, int(20 + 25 * s), blocks=1 + s % 3)
             for s in range(40)]
    cases += [lts_gen.kripke_uniform(), lts_gen.kripke_uniform(seed=7, n=600, m=4000), lts_gen.fan_out(300),
              lts_gen.chain(n=1500), lts_gen.quotient_expansion(seed=8, classes=40, trans=300, num_act=5, copies_hi=12),
              _hub_lts(4, 700, 10, 300, deg=3, num_act=2), lts_gen.powerlaw(seed=3, n=600, num_act=32)]
    e = np.zeros(0, dtype=np.int32)
    cases += [lts_gen.LTS("no-transitions", 7, 1, e, e, e, np.array([0, 0, 3, 3, 6, 6, 0], np.int32)),
              lts_gen.from_triples(1, 1, [(0, 0, 0)]), lts_gen.from_triples(2, 3, [(0, 2, 1), (0, 2, 1), (1, 2, 1)]),
              lts_gen.from_triples(4, 32, [(0, 31, 1), (1, 0, 2), (2, 31, 3), (3, 0, 0)])]
    return cases


def test_small_ltss_on_one_cta_in_shared_memory():
    """LTSs that fit in one CTA's shared memory are reduced by one launch
    (stats.engine = BISIM_ENGINE_SMALL): the oracle's partition, the same as
    with the path off, and Theorem 3's iteration bounds."""
    for lts in _small_cases():
        want = oracle.ks_lts(lts)
        got, st = run(lts, bisim.ENGINE_AUTO)
        assert st.engine == bisim.ENGINE_SMALL, lts.name
        assert got.tolist() == want.tolist(), lts.name
        assert st.num_blocks == defs.num_blocks(want)
        B = defs.num_blocks(want)
        assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1, lts.name
        off, st2 = run(lts, bisim.ENGINE_AUTO, small=-1)
        assert st2.engine != bisim.ENGINE_SMALL and off.tolist() == want.tolist(), lts.name
        assert st.pre_rounds == st2.pre_rounds and st.initial_blocks == st2.initial_blocks, lts.name
        assert st.mark_length == st2.mark_length, lts.name


@pytest.mark.parametrize("kw", [dict(splitters=1), dict(splitters=2, split_budget=1), dict(rcpp_alg2=True)],
                         ids=["one-splitter", "two-splitters", "algorithm-2"])
def test_small_path_settings(kw):
    for lts in _small_cases()[:30] + [lts_gen.kripke_uniform(), lts_gen.chain(n=1000)]:
        got, st = run(lts, bisim.ENGINE_FRONTIER, **kw)
        assert st.engine == bisim.ENGINE_SMALL
        assert got.tolist() == oracle.ks_lts(lts).tolist(), lts.name
        if kw.get("splitters") == 1:
            assert st.steps == st.rounds


def test_small_path_errors_and_replanning():
    """Out-of-range entries are rejected by bisim_plan; the round cap gives
    BISIM_EROUNDS; a plan refines twice with the same result."""
    import torch

    bad = lts_gen.from_triples(3, 2, [(0, 1, 1), (1, 2, 2)])
    with pytest.raises(bisim.BisimError) as ei:
        run(bad, bisim.ENGINE_AUTO)
    assert ei.value.code == bisim.BISIM_EINVAL
    with pytest.raises(bisim.BisimError) as ei:
        run(lts_gen.chain(n=500), bisim.ENGINE_AUTO, round_cap=10)
    assert ei.value.code == bisim.BISIM_EROUNDS
    lts = lts_gen.kripke_uniform(seed=2)
    d = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    with bisim.Plan(lts.n, lts.num_act, d(lts.src), d(lts.act), d(lts.dst), d(lts.init)) as p:
        a, st1 = p.refine()
        a = a.cpu().numpy().copy()
        b, st2 = p.refine()
        b = b.cpu().numpy()
    assert st1.engine == bisim.ENGINE_SMALL
    assert np.array_equal(a, b) and a.tolist() == oracle.ks_lts(lts).tolist()
