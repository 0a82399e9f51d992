"""Seeded synthetic labelled transition systems (LTSs).

This module only draws random inputs; it holds none of the refinement
arithmetic, so both the CUDA path and the CPU oracle can consume its output.
Every generator takes an explicit seed and uses numpy's PCG64 stream, so the
same call on the same numpy version yields the same arrays.

The shapes follow the workloads of the paper's experiments (Section 5): LTSs
with n states, m transitions given as int32 (source, action, target) triples
in arbitrary order, and an optional initial block label per state (the input
I_i of Algorithm 2, a label in [0, n)).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class LTS:
    """An LTS as flat int32 arrays.

    n        number of states, states are 0..n-1
    num_act  number of action labels, labels are 0..num_act-1
    src, act, dst  int32 [m] transition triples (duplicates allowed)
    init     int32 [n] initial block label per state (values in [0, n)),
             or None for the single initial block {S}
    cls      int32 [n] class map h(s) for LTSs built by quotient expansion
             (h is a functional bisimulation onto `quotient`), else None
    quotient the small LTS the instance was expanded from, else None
    """

    name: str
    n: int
    num_act: int
    src: np.ndarray
    act: np.ndarray
    dst: np.ndarray
    init: Optional[np.ndarray] = None
    cls: Optional[np.ndarray] = None
    quotient: Optional["LTS"] = None

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def nbytes(self) -> int:
        b = self.src.nbytes + self.act.nbytes + self.dst.nbytes
        if self.init is not None:
            b += self.init.nbytes
        return b


def _i32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _shuffle(rng: np.random.Generator, src, act, dst):
    perm = rng.permutation(src.shape[0])
    return _i32(src[perm]), _i32(act[perm]), _i32(dst[perm])


def _ap_partition(rng: np.random.Generator, n: int) -> np.ndarray:
    """Initial partition from two Bernoulli(1/2) atomic propositions p, q per
    state: I = 2p + q (at most 4 initial blocks)."""
    p = rng.integers(0, 2, n, dtype=np.int32)
    q = rng.integers(0, 2, n, dtype=np.int32)
    return _i32(2 * p + q)


def zipf_labels(rng: np.random.Generator, size: int, num_act: int,
                s: float = 1.1) -> np.ndarray:
    """Finite Zipf labels on {0..num_act-1}: P(k) proportional to (k+1)^-s."""
    w = (np.arange(num_act, dtype=np.float64) + 1.0) ** (-s)
    w /= w.sum()
    return _i32(rng.choice(num_act, size=size, p=w))


def kripke_uniform(seed: int = 0, n: int = 1000, m: int = 4000) -> LTS:
    """Unlabelled Kripke structure: m transitions with source and target
    uniform over the n states, one action, initial partition from two random
    atomic propositions (4 blocks)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m, dtype=np.int32)
    dst = rng.integers(0, n, m, dtype=np.int32)
    act = np.zeros(m, dtype=np.int32)
    init = _ap_partition(rng, n)
    src, act, dst = _shuffle(rng, src, act, dst)
    return LTS(f"kripke_n{n}_m{m}_s{seed}", n, 1, src, act, dst, init)


def random_quotient(rng: np.random.Generator, classes: int, trans: int,
                    num_act: int, zipf_s: float = 1.1) -> LTS:
    qs = rng.integers(0, classes, trans, dtype=np.int32)
    qd = rng.integers(0, classes, trans, dtype=np.int32)
    qa = zipf_labels(rng, trans, num_act, zipf_s)
    return LTS(f"quotient_k{classes}_t{trans}", classes, num_act, _i32(qs), qa, _i32(qd))


def expand_quotient(rng: np.random.Generator, q: LTS, copies_lo: int, copies_hi: int,
                    dup_frac: float = 0.1, name: str = "expanded") -> LTS:
    """Replicate each class of quotient `q` into U{copies_lo..copies_hi} states.
    Every copy of class u receives every transition u -a-> v of the quotient,
    redirected to a uniformly random copy of v; then floor(dup_frac * m) exact
    duplicates of uniformly chosen transitions are appended and the transition
    order is shuffled. State numbers are a random permutation, so the members
    of a class are scattered. The class map h is returned in `cls`."""
    K = q.n
    copies = rng.integers(copies_lo, copies_hi + 1, K).astype(np.int64)
    n = int(copies.sum())
    start = np.concatenate([[0], np.cumsum(copies)[:-1]]).astype(np.int64)
    perm = rng.permutation(n).astype(np.int64)  # (class k, copy j) -> state perm[start[k]+j]
    cls = np.empty(n, dtype=np.int32)
    cls[perm] = np.repeat(np.arange(K, dtype=np.int32), copies)
    reps = copies[q.src]
    total = int(reps.sum())
    grp_start = np.repeat(np.cumsum(reps) - reps, reps)
    j = np.arange(total, dtype=np.int64) - grp_start
    src = perm[np.repeat(start[q.src], reps) + j]
    tgt_cls = np.repeat(q.dst.astype(np.int64), reps)
    pick = np.floor(rng.random(total) * copies[tgt_cls]).astype(np.int64)
    dst = perm[start[tgt_cls] + pick]
    act = np.repeat(q.act, reps)
    ndup = int(np.floor(dup_frac * total))
    if ndup > 0:
        d = rng.integers(0, total, ndup)
        src = np.concatenate([src, src[d]])
        dst = np.concatenate([dst, dst[d]])
        act = np.concatenate([act, act[d]])
    src, act, dst = _shuffle(rng, src, act, dst)
    return LTS(name, n, q.num_act, src, act, dst, None, cls, q)


def quotient_expansion(seed: int = 1, classes: int = 2000, trans: int = 20000,
                       num_act: int = 8, zipf_s: float = 1.1, copies_lo: int = 1,
                       copies_hi: int = 100, dup_frac: float = 0.1) -> LTS:
    """Labelled LTS by quotient expansion (about 100k states and 1.1M
    transitions at the defaults): a random quotient of `classes` classes and
    `trans` transitions with Zipf labels, each class replicated 1..100 times,
    plus 10% duplicated transitions; single initial block."""
    rng = np.random.default_rng(seed)
    q = random_quotient(rng, classes, trans, num_act, zipf_s)
    return expand_quotient(rng, q, copies_lo, copies_hi, dup_frac,
                           name=f"qexp_k{classes}_t{trans}_a{num_act}_s{seed}")


def chain(seed: int = 2, n: int = 50000) -> LTS:
    """Deep-refinement chain i -> i+1 (one action), last state deadlocked,
    single initial block; forces Theta(n) refinement rounds. The seed only
    shuffles the transition order."""
    rng = np.random.default_rng(seed)
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    act = np.zeros(n - 1, dtype=np.int32)
    src, act, dst = _shuffle(rng, src, act, dst)
    return LTS(f"chain_n{n}_s{seed}", n, 1, src, act, dst, None)


def powerlaw(seed: int = 3, n: int = 10_000_000, alpha: float = 2.1, mean_deg: float = 10.0,
             cap: int = 10_000, num_act: int = 32) -> LTS:
    """Large power-law LTS: out-degree min(cap, floor(x_m * U^(-1/alpha) + 1/2))
    with x_m = mean_deg * (alpha-1)/alpha (Pareto with the given mean), targets
    uniform, labels uniform on num_act, initial partition from two atomic
    propositions."""
    rng = np.random.default_rng(seed)
    xm = mean_deg * (alpha - 1.0) / alpha
    u = rng.random(n)
    u = np.maximum(u, np.finfo(np.float64).tiny)
    deg = np.minimum(float(cap), np.floor(xm * u ** (-1.0 / alpha) + 0.5)).astype(np.int64)
    m = int(deg.sum())
    src = np.repeat(np.arange(n, dtype=np.int32), deg)
    dst = rng.integers(0, n, m, dtype=np.int32)
    act = rng.integers(0, num_act, m, dtype=np.int32)
    init = _ap_partition(rng, n)
    src, act, dst = _shuffle(rng, src, act, dst)
    return LTS(f"powerlaw_n{n}_a{num_act}_s{seed}", n, num_act, src, act, dst, init)


def stream_instance(rng: np.random.Generator, n_lo: int = 100, n_hi: int = 200_000,
                    act_hi: int = 32, mean_deg: float = 5.0, dup_frac: float = 0.1,
                    zipf_s: float = 1.1, idx: int = 0) -> LTS:
    """One instance of the batched stream: n_target log-uniform in
    [n_lo, n_hi], |Act| uniform in [1, act_hi], quotient of
    max(1, round(n_target/20)) classes with Poisson(mean_deg/(1+dup_frac))
    out-degree and Zipf labels, each class copied U{1..39} times (mean 20),
    plus dup_frac duplicated transitions."""
    nt = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
    A = int(rng.integers(1, act_hi + 1))
    K = max(1, int(round(nt / 20)))
    deg = rng.poisson(mean_deg / (1.0 + dup_frac), K).astype(np.int64)
    T = int(deg.sum())
    qs = np.repeat(np.arange(K, dtype=np.int32), deg)
    qd = rng.integers(0, K, T, dtype=np.int32)
    qa = zipf_labels(rng, T, A, zipf_s)
    q = LTS(f"q{idx}", K, A, _i32(qs), qa, _i32(qd))
    return expand_quotient(rng, q, 1, 39, dup_frac, name=f"stream{idx}_n{nt}_a{A}")


def batch_stream(seed: int = 4, k: int = 4096, rate_per_s: float = 1000.0, **kw) -> tuple:
    """k stream instances plus Poisson arrival times (seconds) at `rate_per_s`."""
    rng = np.random.default_rng(seed)
    inst: List[LTS] = [stream_instance(rng, idx=i, **kw) for i in range(k)]
    arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, k))
    return inst, arrivals


def fan_out(n: int) -> LTS:
    """Fan_out_n of Section 5.1: states 0..n-1, i -a-> i+1 for 1 < i < n-1,
    and 0 -b-> i, 1 -b-> i for every state i (a = 0, b = 1)."""
    chain = np.arange(2, max(n - 1, 2), dtype=np.int64)
    every = np.arange(n, dtype=np.int64)
    s = np.concatenate([chain, np.stack([np.zeros(n, np.int64), np.ones(n, np.int64)], axis=1).ravel()])
    a = np.concatenate([np.zeros(chain.size, np.int64), np.ones(2 * n, np.int64)])
    d = np.concatenate([chain + 1, np.repeat(every, 2)])
    return LTS(f"fan_out_{n}", n, 2, _i32(s), _i32(a), _i32(d), None)


def random_small(seed: int, n: int, num_act: int, m: int, blocks: int = 1) -> LTS:
    """Small random LTS with `blocks` random initial labels (for brute-force
    cross-checks)."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m, dtype=np.int32)
    dst = rng.integers(0, n, m, dtype=np.int32)
    act = rng.integers(0, num_act, m, dtype=np.int32)
    init = None
    if blocks > 1:
        init = _i32(rng.integers(0, min(blocks, n), n))
    return LTS(f"small_s{seed}_n{n}_a{num_act}_m{m}", n, num_act, _i32(src), _i32(act), _i32(dst), init)


def from_triples(n: int, num_act: int, triples, init=None, name: str = "lts") -> LTS:
    t = np.asarray(list(triples), dtype=np.int32).reshape(-1, 3)
    return LTS(name, n, num_act, _i32(t[:, 0]), _i32(t[:, 1]), _i32(t[:, 2]),
               None if init is None else _i32(init))


def config(k: int, **overrides) -> LTS:
    """The five benchmark workloads by number (1-based); 5 returns a tuple
    (instances, arrival_times)."""
    if k == 1:
        return kripke_uniform(**overrides)
    if k == 2:
        return quotient_expansion(**overrides)
    if k == 3:
        return chain(**overrides)
    if k == 4:
        return powerlaw(**overrides)
    if k == 5:
        return batch_stream(**overrides)
    raise ValueError(f"no workload {k}")
