"""Definitions of Section 2.2 written out directly (numpy / pure Python).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* stability of a partition under its own blocks, per action (Section 2.2);
* refinement of one partition by another;
* canonical numbering (block ids in order of their first state);
* `sigfix`: the partition refined by signatures {(a, block(t)) | s -a-> t}
  until the number of blocks stops growing - the coarsest stable refinement
  restated without splitters;
* `brute_gfp`: the largest bisimulation inside the initial partition, as the
  greatest fixed point of the transfer condition of Definition 1 (small n);
* `coarsest_by_enumeration`: all set partitions refining pi_0 are tried and
  the stable one with the fewest blocks is returned (n <= 7).
"""
from __future__ import annotations

import numpy as np


def canonical(labels) -> np.ndarray:
    """Renumber blocks 0, 1, 2, ... in order of their first state."""
    labels = np.asarray(labels)
    n = labels.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int32)
    _, first, inv = np.unique(labels, return_index=True, return_inverse=True)
    rank = np.empty(first.shape[0], dtype=np.int32)
    rank[np.argsort(first, kind="stable")] = np.arange(first.shape[0], dtype=np.int32)
    return rank[inv.reshape(-1)].astype(np.int32)


def num_blocks(part) -> int:
    return int(np.unique(np.asarray(part)).shape[0])


def _unique_rows(cols, return_counts=False):
    """np.unique over the rows formed by the non-negative int64 columns
    `cols`. When the product of the column ranges fits in 63 bits each row is
    packed into one int64 (mixed radix, first column most significant) and
    the unique keys are unpacked again; otherwise the rows are compared as
    rows. Both give the same rows in the same (lexicographic) order."""
    cols = [np.asarray(c, dtype=np.int64) for c in cols]
    radix = [int(c.max()) + 1 if c.size else 1 for c in cols]
    span = 1
    for r in radix:
        span *= r
    if span < (1 << 63) and not packed_disabled:
        key = np.zeros(cols[0].shape[0], dtype=np.int64)
        for c, r in zip(cols, radix):
            key = key * r + c
        key = np.sort(key)
        first = np.ones(key.shape[0], dtype=bool)
        first[1:] = key[1:] != key[:-1]
        starts = np.flatnonzero(first)
        uk = key[starts]
        out = []
        for r in reversed(radix):
            out.append(uk % r)
            uk = uk // r
        rows = np.stack(out[::-1], axis=1)
        if return_counts:
            return rows, np.diff(np.append(starts, key.shape[0]))
        return rows
    return np.unique(np.stack(cols, axis=1), axis=0, return_counts=return_counts)


# tests set this to check that the packed and the row-wise paths agree
packed_disabled = False


def refines(fine, coarse) -> bool:
    """True iff every block of `fine` lies inside one block of `coarse`."""
    fine = np.asarray(fine, dtype=np.int64)
    coarse = np.asarray(coarse, dtype=np.int64)
    if fine.size == 0:
        return True
    pairs = _unique_rows([fine, coarse])
    return pairs.shape[0] == _unique_rows([fine]).shape[0]


def is_stable(n, src, act, dst, part) -> bool:
    """A partition is stable iff for every pair of blocks V, U and action a,
    either all states of V reach U with a or none does."""
    part = np.asarray(part, dtype=np.int64)
    if len(src) == 0:
        return True
    src = np.asarray(src, dtype=np.int64)
    act = np.asarray(act, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    reach = _unique_rows([src, act, part[dst]])  # s reaches U with a
    ukeys, counts = _unique_rows([part[reach[:, 0]], reach[:, 1], reach[:, 2]], return_counts=True)
    size = np.bincount(part, minlength=int(part.max()) + 1)
    return bool(np.all(counts == size[ukeys[:, 0]]))


def sigfix(n, src, act, dst, init=None) -> np.ndarray:
    """Refine by signatures sig(s) = (block(s), {(a, block(t)) | s -a-> t})
    until the block count is unchanged; canonical ids."""
    p = canonical(np.zeros(n, dtype=np.int32) if init is None else init)
    src = np.asarray(src, dtype=np.int64)
    act = np.asarray(act, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    nb = num_blocks(p) if n else 0
    while True:
        if len(src):
            trip = np.unique(np.stack([src, act, p[dst].astype(np.int64)], axis=1), axis=0)
            bounds = np.searchsorted(trip[:, 0], np.arange(n + 1))
        sigs = {}
        newp = np.empty(n, dtype=np.int64)
        for s in range(n):
            if len(src):
                rows = trip[bounds[s]:bounds[s + 1], 1:]
                key = (int(p[s]), tuple(map(tuple, rows.tolist())))
            else:
                key = (int(p[s]), ())
            newp[s] = sigs.setdefault(key, len(sigs))
        newp = canonical(newp)
        nb2 = num_blocks(newp) if n else 0
        if nb2 == nb:
            return newp
        p, nb = newp, nb2


def brute_gfp(n, src, act, dst, init=None) -> np.ndarray:
    """Largest bisimulation contained in the initial equivalence: start from
    all pairs in the same initial block and delete pairs violating the
    transfer condition of Definition 1 in either direction, until nothing
    changes. Canonical ids of the resulting equivalence classes."""
    init = [0] * n if init is None else [int(x) for x in init]
    succ = {}
    for s, a, t in zip(src, act, dst):
        succ.setdefault((int(s), int(a)), set()).add(int(t))
    acts = sorted({int(a) for a in act})
    R = {(s, t) for s in range(n) for t in range(n) if init[s] == init[t]}

    def transfer(s, t):
        for a in acts:
            for s2 in succ.get((s, a), ()):
                if not any((s2, t2) in R for t2 in succ.get((t, a), ())):
                    return False
        return True

    changed = True
    while changed:
        changed = False
        for (s, t) in sorted(R):
            if (s, t) in R and not (transfer(s, t) and transfer(t, s)):
                R.discard((s, t))
                R.discard((t, s))
                changed = True
    label = [min(t for t in range(n) if (s, t) in R) for s in range(n)]
    return canonical(np.array(label, dtype=np.int32)) if n else np.zeros(0, dtype=np.int32)


def _set_partitions(n):
    """All set partitions of {0..n-1} as restricted growth strings."""
    if n == 0:
        yield ()
        return

    def rec(i, cur, mx):
        if i == n:
            yield tuple(cur)
            return
        for v in range(mx + 2):
            cur.append(v)
            yield from rec(i + 1, cur, max(mx, v))
            cur.pop()

    yield from rec(1, [0], 0)


def coarsest_by_enumeration(n, src, act, dst, init=None) -> np.ndarray:
    """Among all set partitions refining pi_0, the stable one with the fewest
    blocks (it is unique: every stable refinement refines it)."""
    assert n <= 7
    p0 = np.zeros(n, dtype=np.int32) if init is None else np.asarray(init, dtype=np.int32)
    best = None
    for rgs in _set_partitions(n):
        part = np.array(rgs, dtype=np.int32)
        if not refines(part, p0):
            continue
        if not is_stable(n, src, act, dst, part):
            continue
        nb = num_blocks(part)
        if best is None or nb < best[0]:
            best = (nb, part)
    return canonical(best[1])


def pullback(cls, qpart) -> np.ndarray:
    """Partition of an expanded LTS induced by a partition of its quotient
    through the class map h: s and t share a block iff h(s) and h(t) do."""
    return canonical(np.asarray(qpart)[np.asarray(cls)])


def all_relations(n, num_act):
    """Every transition relation over n states and num_act labels (as lists
    of (s, a, t) triples); 2^(n*n*num_act) relations."""
    triples = [(s, a, t) for s in range(n) for a in range(num_act) for t in range(n)]
    for mask in range(1 << len(triples)):
        yield [triples[i] for i in range(len(triples)) if (mask >> i) & 1]


def all_initial_partitions(n):
    for rgs in _set_partitions(n):
        yield np.array(rgs, dtype=np.int32)


__all__ = [
    "canonical", "num_blocks", "refines", "is_stable", "sigfix", "brute_gfp",
    "coarsest_by_enumeration", "pullback", "all_relations", "all_initial_partitions",
]
