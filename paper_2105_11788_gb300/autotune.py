"""Autotuner for the launch shape of the batched refinement.

The batch kernel runs one LTS per CTA at a time; its best block size depends
on the batch: small LTSs want many small CTAs (more LTSs in flight), large
ones want wide CTAs (a round's touched blocks spread over more warps), and a
batch with both can use the split schedule (the largest LTSs in a concurrent
launch of wide CTAs). The tuner times `bisim_batch_refine` on the batch for
each candidate (threads per CTA, CTAs per SM, wide-launch threads and
threshold, splitters per round and their state budget), keeps the fastest, and caches the choice in a JSON file keyed by
the batch's shape bucket:

    (log2 of the LTS count, log2 of the largest LTS's states, log2 of the mean
     out-degree)

so later batches of the same shape reuse it without timing.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

from . import bisim

# (threads, ctas_per_sm, wide_threads, wide_min_states, splitters, split_budget, multi_min_states)
CANDIDATES: Tuple[Tuple[int, int, int, int, int, int, int], ...] = (
    (128, 0, 0, 0, 1, 0, 0), (256, 0, 0, 0, 1, 0, 0), (512, 0, 0, 0, 1, 0, 0),
    (256, 0, 1024, 1 << 15, 1, 0, 0),
    (256, 0, 0, 0, 16, 1, 0), (256, 0, 0, 0, 64, 2, 0),
    (512, 0, 0, 0, 16, 8, 50000), (256, 0, 0, 0, 16, 4, 20000),
)
KEYS = ("threads", "ctas_per_sm", "wide_threads", "wide_min_states", "splitters", "split_budget",
        "multi_min_states")


def _name(c) -> str:
    return "t{}x{}+w{}@{}+s{}b{}m{}".format(*c)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "bisim_gb300_autotune.json")


def shape_key(ltss: Sequence) -> str:
    k = len(ltss)
    nmax = max((l.n for l in ltss), default=1)
    deg = sum(l.m for l in ltss) / max(1, sum(l.n for l in ltss))
    return f"k{int(math.log2(max(k, 1)))}_n{int(math.log2(max(nmax, 1)))}_d{int(math.log2(max(deg, 1)))}"


class BatchTuner:
    def __init__(self, cache_path: Optional[str] = None, candidates=CANDIDATES, repeats: int = 2):
        self.cache_path = cache_path or DEFAULT_CACHE
        self.candidates = tuple(candidates)
        self.repeats = repeats
        self.cache: Dict[str, dict] = {}
        if os.path.exists(self.cache_path):
            try:
                with open(self.cache_path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def save(self):
        os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def lookup(self, ltss: Sequence) -> Optional[bisim.bisim_opts]:
        rec = self.cache.get(shape_key(ltss))
        if rec is None:
            return None
        return bisim.make_opts(**{k: rec.get(k, 0) for k in KEYS})

    def tune(self, ltss: Sequence, device: str = "cuda") -> Tuple[bisim.bisim_opts, dict]:
        """Time every candidate on this batch; record and return the best."""
        import torch

        so, to, na, src, act, dst, init = bisim.pack_batch(list(ltss))
        d = lambda a: None if a is None else torch.from_numpy(a).to(device)  # noqa: E731
        tsrc, tact, tdst, tinit = d(src), d(act), d(dst), d(init)
        n_total = int(so[-1])
        out = torch.empty(max(n_total, 1), dtype=torch.int32, device=device)
        stream = int(torch.cuda.current_stream().cuda_stream)
        timings = {}
        for cand in self.candidates:
            # the options (and with them the launch shape) belong to a plan,
            # so every candidate gets its own plan of the same batch
            best = math.inf
            opts = bisim.make_opts(**dict(zip(KEYS, cand)))
            hc = bisim.bisim_batch_plan(len(ltss), so, to, na, tsrc.data_ptr(), tact.data_ptr(), tdst.data_ptr(),
                                        tinit.data_ptr() if tinit is not None else None, opts, stream)
            try:
                for _ in range(self.repeats):
                    st, _ = bisim.bisim_batch_refine(hc, out.data_ptr(), len(ltss))
                    best = min(best, st.t_refine_ms)
            finally:
                bisim.bisim_plan_destroy(hc)
            timings[_name(cand)] = (best, cand)
        name = min(timings, key=lambda k: timings[k][0])
        ms, cand = timings[name]
        rec = dict(zip(KEYS, cand))
        rec.update({"refine_ms": ms, "timings_ms": {k: v[0] for k, v in timings.items()},
                    "when": time.strftime("%Y-%m-%dT%H:%M:%S")})
        self.cache[shape_key(ltss)] = rec
        self.save()
        return bisim.make_opts(**dict(zip(KEYS, cand))), rec

    def opts_for(self, ltss: Sequence, device: str = "cuda") -> bisim.bisim_opts:
        """Cached choice for this batch shape, tuning on a miss."""
        o = self.lookup(ltss)
        if o is not None:
            return o
        o, _ = self.tune(ltss, device)
        return o


def sample_for_tuning(ltss: Sequence, max_lts: int = 512, seed: int = 0):
    """A random subset that keeps the largest LTS (it sets the batch's span)."""
    if len(ltss) <= max_lts:
        return list(ltss)
    rng = np.random.default_rng(seed)
    big = int(np.argmax([l.n for l in ltss]))
    idx = set(rng.choice(len(ltss), size=max_lts - 1, replace=False).tolist())
    idx.add(big)
    return [ltss[i] for i in sorted(idx)]
