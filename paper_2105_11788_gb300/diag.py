"""Diagnostics on the GPU behind reported numbers: the grid-barrier cost and
the paper's bandwidth-bound rounds.

    python -m paper_2105_11788_gb300.diag barrier        # ns per grid barrier
    python -m paper_2105_11788_gb300.diag hbm [n]        # HBM-bound rounds (label, dense) vs peak

Each prints JSON lines.
"""
from __future__ import annotations

import json
import sys

from . import bisim, lts_gen

def barrier(iters: int = 20000, repeats: int = 3):
    res = {}
    for threads in (256, 512, 1024):
        for ctas in (1, 8, 16, 38, 76, 152, 304):
            try:
                res[f"{ctas}x{threads}"] = min(bisim.bisim_barrier_cost(ctas, threads, iters)
                                               for _ in range(repeats))
            except bisim.BisimError as e:
                res[f"{ctas}x{threads}"] = str(e)
    print(json.dumps({"barrier_ns": res}), flush=True)


def _hbm_peak():
    import os

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def paper_rounds(lts, src, act, dst, init, window: int = 200, peak: float = None, peak_kind: str = None) -> dict:
    """The bandwidth-bound rounds of the paper's method on one LTS (device
    tensors src/act/dst/init): the literal action-set preprocessing rounds
    (one pass over the states per label) and a window of `window` dense main
    rounds (every round scans all states and mark slots; the window ends with
    the round cap, BISIM_EROUNDS, when the whole dense run is longer). Achieved
    GB/s of algorithmic bytes against the HBM peak:
      label round: 14 B per state (block, own and leader's label-set word,
                   split flag written and read);
      dense round: 30 B per state + 8 B per mark slot, plus 12 B per walked
                   incoming transition."""
    import ctypes

    import torch

    if peak is None:
        peak, peak_kind = _hbm_peak()
    out = torch.empty(max(lts.n, 1), dtype=torch.int32, device=src.device)
    lib = bisim.load()
    opts = bisim.make_opts(engine=bisim.ENGINE_DENSE, preprocess=1, round_cap=window)
    with bisim.Plan(lts.n, lts.num_act, src, act, dst, init, opts) as p:
        st = bisim.bisim_stats()
        rc = lib.bisim_refine(p.handle, out.data_ptr(), ctypes.byref(st))
    label_bytes = 14.0 * st.n * st.pre_rounds
    dense_bytes = st.rounds * (30.0 * st.n + 8.0 * st.mark_length) + 12.0 * st.edges_visited
    lab_gbs = label_bytes / (st.t_pre_ms * 1e6) if st.t_pre_ms > 0 else 0.0
    den_gbs = dense_bytes / (st.t_main_ms * 1e6) if st.t_main_ms > 0 else 0.0
    return {"peak_gbs": peak, "peak_kind": peak_kind,
            "label_rounds": {"kernel": "k_label_rounds", "rounds": st.pre_rounds, "ms": st.t_pre_ms,
                             "bytes": label_bytes, "gbs": lab_gbs, "frac": lab_gbs / peak},
            "dense_window": {"kernel": "k_dense_main", "rounds": st.rounds, "ms": st.t_main_ms,
                             "bytes": dense_bytes, "gbs": den_gbs, "frac": den_gbs / peak,
                             "us_per_round": 1e3 * st.t_main_ms / max(st.rounds, 1),
                             "ended_by_round_cap": rc == bisim.BISIM_EROUNDS}}


def hbm(window: int = 200, repeats: int = 3, n: int = 10_000_000):
    """paper_rounds on the 10^7-state power-law LTS, `repeats` times."""
    import torch

    lts = lts_gen.powerlaw(seed=3, n=n)
    d = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    src, act, dst, init = d(lts.src), d(lts.act), d(lts.dst), d(lts.init)
    for rep in range(repeats):
        print(json.dumps({"workload": f"powerlaw n={n}", "rep": rep,
                          **paper_rounds(lts, src, act, dst, init, window)}), flush=True)


def main(argv):
    import torch

    torch.cuda.init()
    what = argv[1] if len(argv) > 1 else "barrier"
    bisim.load(build_if_missing=True)
    if what == "barrier":
        barrier()
    elif what == "hbm":
        hbm(n=int(argv[2]) if len(argv) > 2 else 10_000_000)
    else:
        raise SystemExit(f"unknown diagnostic {what}")


if __name__ == "__main__":
    main(sys.argv)
