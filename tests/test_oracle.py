"""Pins for the CPU oracle (no GPU): the paper's worked examples, the
definitions of Section 2.2 by brute force, closed forms, and the round
bounds of Theorems 2 and 3."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import defs
from paper_2105_11788_gb300 import lts_gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _arrays(tr):
    t = np.asarray(tr, dtype=np.int32).reshape(-1, 3)
    return t[:, 0].copy(), t[:, 1].copy(), t[:, 2].copy()


def action_set_partition(n, src, act, init=None):
    """pi_0' of Section 4.1.1 from its definition: states grouped by
    (initial block, set of outgoing labels)."""
    sets = [set() for _ in range(n)]
    for s, a in zip(src, act):
        sets[int(s)].add(int(a))
    keys = [(0 if init is None else int(init[s]), tuple(sorted(sets[s]))) for s in range(n)]
    ids = {}
    return defs.canonical(np.array([ids.setdefault(k, len(ids)) for k in keys]))


# --------------------------------------------------------------------- Fig. 3


def test_fig3_preprocessing_arrays():
    g = _golden("fig3_preprocessing.json")
    src, act, dst = _arrays(g["transitions"])
    p = oracle.plan(g["n"], g["num_act"], src, act, dst)
    assert src[p["perm"]].tolist() == g["sorted_source"]
    assert act[p["perm"]].tolist() == g["sorted_label"]
    assert p["action_switch"].tolist() == g["action_switch"]
    assert p["order"].tolist() == g["order"]
    assert p["nr_marks"].tolist() == g["nr_marks"]
    # printed off = running totals of nr_marks; the start offsets used to
    # index mark_{off(s)+order} are the exclusive sums
    assert (p["off"] + p["nr_marks"]).tolist() == g["off_printed"]
    assert p["off"].tolist() == [0, 2, 5]
    assert p["mark_length"] == g["off_printed"][-1] == 6


def test_fig3_final_partition_is_discrete():
    g = _golden("fig3_preprocessing.json")
    src, act, dst = _arrays(g["transitions"])
    # s0, s1, s2 have different outgoing label sets, so no two are bisimilar
    assert oracle.ks(3, 3, src, act, dst).tolist() == [0, 1, 2]
    assert defs.brute_gfp(3, src, act, dst).tolist() == [0, 1, 2]
    labels, rounds, pre = oracle.pram(3, 3, src, act, dst)
    assert defs.canonical(labels).tolist() == [0, 1, 2]
    assert pre == 3
    assert rounds == 3 + 1  # three singleton splitters, then the empty iteration


def test_fig3_marks_index_by_off_plus_order():
    """mark_{off(s)+order_i}: with C = {s2} (after preprocessing every state is
    a singleton), the marked (state, label) pairs are exactly those with a
    transition into s2."""
    g = _golden("fig3_preprocessing.json")
    src, act, dst = _arrays(g["transitions"])
    block = np.array([0, 1, 2], dtype=np.int32)
    _, _, marks = oracle.pram_step(3, 3, src, act, dst, block, [True, True, True], C=2)
    # pairs in (source, label) order: (0,a) (0,c) (1,a) (1,b) (1,c) (2,c)
    assert marks.tolist() == [True, True, False, True, False, True]


# --------------------------------------------------------------------- Fig. 1


def test_fig1_one_iteration():
    g = _golden("fig1_iteration.json")
    src, act, dst = _arrays(g["transitions"])
    blk, uns, marks = oracle.pram_step(g["n"], 1, src, act, dst, g["block_before"],
                                       g["unstable_before"], g["splitter"], alg2=True)
    assert np.flatnonzero(marks).tolist() == g["marked_states"]
    assert blk.tolist() == g["block_after"]
    assert uns.tolist() == g["unstable_after"]


def test_fig1_one_iteration_alg3_keeps_splitter_unstable():
    """Algorithm 3 sets unstable_C again when any block split."""
    g = _golden("fig1_iteration.json")
    src, act, dst = _arrays(g["transitions"])
    blk, uns, _ = oracle.pram_step(g["n"], 1, src, act, dst, g["block_before"],
                                   g["unstable_before"], g["splitter"], alg2=False)
    assert blk.tolist() == g["block_after"]
    assert uns.tolist() == [True, False, True, True, False]


def test_fig1_final_partition():
    g = _golden("fig1_iteration.json")
    src, act, dst = _arrays(g["transitions"])
    init = g["block_before"]
    want = defs.brute_gfp(5, src, act, dst, init)
    assert want.tolist() == [0, 1, 2, 3, 3]  # s1 reaches B_s3 through nothing, s2 does
    assert oracle.ks(5, 1, src, act, dst, init).tolist() == want.tolist()
    assert defs.coarsest_by_enumeration(5, src, act, dst, init).tolist() == want.tolist()
    for alg2 in (False, True):
        labels, _, _ = oracle.pram(5, 1, src, act, dst, init, alg2=alg2)
        assert defs.canonical(labels).tolist() == want.tolist()
    labels, _ = oracle.pair(5, 1, src, act, dst, init)
    assert defs.canonical(labels).tolist() == want.tolist()


# ------------------------------------------------------------ brute force


def _check_all(n, A, src, act, dst, init, enum=True):
    want = defs.brute_gfp(n, src, act, dst, init)
    if enum:
        assert defs.coarsest_by_enumeration(n, src, act, dst, init).tolist() == want.tolist()
    assert defs.sigfix(n, src, act, dst, init).tolist() == want.tolist()
    assert oracle.ks(n, A, src, act, dst, init).tolist() == want.tolist()
    labels, rounds, pre = oracle.pram(n, A, src, act, dst, init)
    assert defs.canonical(labels).tolist() == want.tolist()
    B = defs.num_blocks(want)
    p0 = defs.num_blocks(action_set_partition(n, src, act, init))
    assert B + 1 <= rounds <= 3 * B - p0 + 1  # Theorem 3 plus the empty iteration
    assert pre == len(set(np.asarray(act).tolist()))
    # leader invariant: every label is a member of its own block
    assert all(labels[labels[s]] == labels[s] for s in range(n))
    if A == 1:
        labels2, rounds2, _ = oracle.pram(n, A, src, act, dst, init, alg2=True)
        assert defs.canonical(labels2).tolist() == want.tolist()
        assert B + 1 <= rounds2 <= 2 * B - p0 + 1  # Theorem 2 plus the empty iteration
    _check_pair(n, A, src, act, dst, init, want)
    return want


def _check_pair(n, A, src, act, dst, init, want):
    """(C, a)-pair splitters: the same partition; every final block is
    selected at least once and a label becomes unstable only when it is
    created or its block splits, so B * nl + 1 <= iterations <=
    (2B - |pi_0|) * nl + 1 with nl = max(1, labels that occur); with one
    label it is Algorithm 2 without preprocessing, iteration for iteration."""
    labels, rounds = oracle.pair(n, A, src, act, dst, init)
    assert defs.canonical(labels).tolist() == want.tolist()
    assert all(labels[labels[s]] == labels[s] for s in range(n))
    B = defs.num_blocks(want)
    pi0 = defs.num_blocks(init) if init is not None and n else min(n, 1)
    nl = max(1, len(set(np.asarray(act).tolist())))
    assert B * nl + 1 <= rounds <= (2 * B - pi0) * nl + 1
    if A == 1:
        labels2, rounds2, pre2 = oracle.pram(n, A, src, act, dst, init, alg2=True, skip_preprocess=True)
        assert pre2 == 0
        assert labels.tolist() == labels2.tolist() and rounds == rounds2


@pytest.mark.parametrize("n,A", [(1, 1), (1, 2), (2, 1), (2, 2), (3, 1)])
def test_exhaustive_tiny(n, A):
    for rel in defs.all_relations(n, A):
        src, act, dst = _arrays(rel) if rel else (np.zeros(0, np.int32),) * 3
        for init in defs.all_initial_partitions(n):
            _check_all(n, A, src, act, dst, init)


def test_sampled_n3_two_labels():
    rng = np.random.default_rng(11)
    triples = [(s, a, t) for s in range(3) for a in range(2) for t in range(3)]
    for _ in range(400):
        mask = rng.integers(0, 2, len(triples))
        rel = [triples[i] for i in range(len(triples)) if mask[i]]
        src, act, dst = _arrays(rel) if rel else (np.zeros(0, np.int32),) * 3
        init = rng.integers(0, 3, 3).astype(np.int32)
        _check_all(3, 2, src, act, dst, init)


@pytest.mark.parametrize("seed", range(60))
def test_random_small(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 9))
    A = int(rng.integers(1, 4))
    m = int(rng.integers(0, 3 * n))
    lts = lts_gen.random_small(seed, n, A, m, blocks=int(rng.integers(1, 3)))
    _check_all(n, A, lts.src, lts.act, lts.dst, lts.init, enum=n <= 6)


def test_random_medium_ks_vs_sigfix_and_pram():
    for seed in range(8):
        lts = lts_gen.random_small(seed, 300, 3, 700, blocks=3)
        want = defs.sigfix(lts.n, lts.src, lts.act, lts.dst, lts.init)
        got = oracle.ks_lts(lts)
        assert got.tolist() == want.tolist()
        labels, rounds, _ = oracle.pram_lts(lts)
        assert defs.canonical(labels).tolist() == want.tolist()
        assert defs.is_stable(lts.n, lts.src, lts.act, lts.dst, got)
        assert defs.refines(got, lts.init)


# ------------------------------------------------------------ closed forms


@pytest.mark.parametrize("n", [3, 4, 5, 10, 57, 200])
def test_fan_out(n):
    """Fan_out_n (Section 5.1): 0 and 1 are bisimilar, every other state is a
    singleton, n-1 blocks, 3n-3 transitions."""
    lts = lts_gen.fan_out(n)
    assert lts.m == 3 * n - 3
    want = [0, 0] + list(range(1, n - 1))
    assert oracle.ks_lts(lts).tolist() == want
    labels, rounds, pre = oracle.pram_lts(lts)
    assert defs.canonical(labels).tolist() == want


@pytest.mark.parametrize("n", [2, 3, 50, 400])
def test_chain(n):
    """i -> i+1 with a deadlocked last state: all states have different
    distances to the deadlock, so the result is discrete."""
    lts = lts_gen.chain(seed=5, n=n)
    assert oracle.ks_lts(lts).tolist() == list(range(n))
    for alg2 in (False, True):
        labels, rounds, pre = oracle.pram_lts(lts, alg2=alg2)
        assert defs.canonical(labels).tolist() == list(range(n))
        bound = (2 if alg2 else 3) * n - min(n, 2) + 1
        assert n + 1 <= rounds <= bound


def test_distinct_action_sets_take_n_plus_one_rounds():
    """When preprocessing already yields singletons, each state is popped
    once and nothing splits: n iterations plus the empty one (the shape of
    the Vasy_25_25 row of Table 1)."""
    n, A = 30, 5
    tr = [(s, a, 0) for s in range(n) for a in range(A) if ((s + 1) >> a) & 1]
    src, act, dst = _arrays(tr)
    labels, rounds, pre = oracle.pram(n, A, src, act, dst)
    assert defs.canonical(labels).tolist() == list(range(n))
    assert rounds == n + 1


def test_no_transitions_returns_initial_partition():
    init = np.array([3, 3, 0, 1, 0, 3], dtype=np.int32)
    e = np.zeros(0, dtype=np.int32)
    assert oracle.ks(6, 1, e, e, e, init).tolist() == defs.canonical(init).tolist()
    labels, rounds, pre = oracle.pram(6, 1, e, e, e, init)
    assert defs.canonical(labels).tolist() == defs.canonical(init).tolist()
    assert pre == 0 and rounds == 3 + 1
    # priority rule: each initial block is led by its smallest member
    assert labels.tolist() == [0, 0, 2, 3, 2, 0]


def test_quotient_pullback():
    """h (copy -> class) is a functional bisimulation onto the quotient, so
    the partition of the expansion is the quotient's partition pulled back."""
    for seed in range(4):
        rng = np.random.default_rng(seed)
        q = lts_gen.random_quotient(rng, 60, 240, 3)
        e = lts_gen.expand_quotient(rng, q, 1, 6, 0.1)
        qpart = oracle.ks_lts(q)
        assert defs.sigfix(q.n, q.src, q.act, q.dst).tolist() == qpart.tolist()
        want = defs.pullback(e.cls, qpart)
        assert oracle.ks_lts(e).tolist() == want.tolist()
        labels, _, _ = oracle.pram_lts(e)
        assert defs.canonical(labels).tolist() == want.tolist()


def test_duplicates_do_not_matter():
    lts = lts_gen.random_small(3, 40, 2, 90)
    base = oracle.ks_lts(lts)
    src = np.concatenate([lts.src, lts.src[:30]])
    act = np.concatenate([lts.act, lts.act[:30]])
    dst = np.concatenate([lts.dst, lts.dst[:30]])
    assert oracle.ks(lts.n, 2, src, act, dst).tolist() == base.tolist()


# --------------------------------------------------------- planted mistakes


def test_skipping_preprocessing_breaks_algorithm3():
    """Algorithm 3 compares mark_{off(s)+order} with the leader's slot at the
    same order, which only names the same label when both states have the
    same label set (the preprocessing invariant). Without the preprocessing
    rounds some LTS gets a wrong partition."""
    wrong = 0
    for seed in range(200):
        lts = lts_gen.random_small(seed, 5, 2, 7)
        want = oracle.ks_lts(lts)
        labels, _, _ = oracle.pram_lts(lts, skip_preprocess=True)
        if defs.canonical(labels).tolist() != want.tolist():
            wrong += 1
    assert wrong > 0


def test_stability_checker_detects_unstable():
    g = _golden("fig1_iteration.json")
    src, act, dst = _arrays(g["transitions"])
    assert not defs.is_stable(5, src, act, dst, [0, 0, 1, 2, 2])
    assert defs.is_stable(5, src, act, dst, [0, 1, 2, 3, 3])
    # merging two blocks of the result breaks stability
    assert not defs.is_stable(5, src, act, dst, [0, 0, 2, 3, 3])


def test_packed_and_row_wise_checks_agree(monkeypatch):
    """The stability and refinement checks pack each row into one int64 when
    the column ranges allow it; on random LTSs and random, coarsest and
    perturbed partitions both paths give the same answers."""
    rng = np.random.default_rng(123)
    answers = []
    for seed in range(60):
        n = int(rng.integers(1, 30))
        lts = lts_gen.random_small(seed, n, int(rng.integers(1, 4)), int(rng.integers(0, 4 * n)), blocks=2)
        coarsest = oracle.ks_lts(lts)
        parts = [coarsest, rng.integers(0, 3, n), np.arange(n), np.zeros(n, np.int64)]
        if n > 1:
            bad = coarsest.copy()
            bad[0] = bad[1]
            parts.append(bad)
        for part in parts:
            got = []
            for disabled in (False, True):
                monkeypatch.setattr(defs, "packed_disabled", disabled)
                got.append((defs.is_stable(lts.n, lts.src, lts.act, lts.dst, part),
                            defs.refines(part, coarsest), defs.refines(coarsest, part)))
            assert got[0] == got[1], (seed, list(part))
            answers.append(got[0])
    # both outcomes occur, so the comparison is not vacuous
    assert {a[0] for a in answers} == {True, False}
    assert {a[1] for a in answers} == {True, False}


def test_invalid_inputs_rejected():
    s = np.array([0, 5], dtype=np.int32)
    z = np.zeros(2, dtype=np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.ks(3, 1, s, z, z)
    with pytest.raises(oracle.OracleError):
        oracle.ks(3, 1, z, np.array([0, 1], np.int32), z)
    with pytest.raises(oracle.OracleError):
        oracle.ks(3, 1, z, z, z, np.array([0, 0, 9], np.int32))


def test_pair_splitters_one_label_at_a_time():
    """Two labels that separate states only together: s0 -a-> s2, s1 -b-> s2,
    s2 without transitions. The (C, a)-pair rounds must use each label on its
    own: the result is discrete (s0 and s1 have different action sets)."""
    src, act, dst = _arrays([(0, 0, 2), (1, 1, 2)])
    labels, rounds = oracle.pair(3, 2, src, act, dst)
    assert defs.canonical(labels).tolist() == [0, 1, 2]
    # selections, two iterations each: C = 0 ({0,1,2}; a splits off {1,2}
    # led by 1, b splits nothing: s1's b-target s2 left block 0), C = 0 again
    # ({0}, re-marked by its split), C = 1 ({1,2}; b splits off {2}), C = 1
    # ({1}), C = 2 ({2}); then the empty iteration
    assert rounds == 5 * 2 + 1


def test_pair_random_medium_matches_ks():
    for seed in range(6):
        lts = lts_gen.random_small(40 + seed, 200, 4, 600, blocks=2)
        labels, rounds = oracle.pair_lts(lts)
        assert defs.canonical(labels).tolist() == oracle.ks_lts(lts).tolist()
