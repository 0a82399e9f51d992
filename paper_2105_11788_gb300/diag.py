"""Diagnostics on the GPU: grid-barrier cost and launch-shape sweeps.

    python -m paper_2105_11788_gb300.diag barrier        # ns per grid barrier
    python -m paper_2105_11788_gb300.diag shapes         # main-loop time per launch shape
    python -m paper_2105_11788_gb300.diag splitters      # splitters per round / state budget sweep
    python -m paper_2105_11788_gb300.diag fanout         # Fan_out_n scaling, closed form checked
    python -m paper_2105_11788_gb300.diag hbm [n]        # HBM-bound rounds (label, dense) vs peak
    python -m paper_2105_11788_gb300.diag phases         # per-phase time of the hybrid rounds
                                                         # (builds the phase-timer library)

Each prints JSON lines.
"""
from __future__ import annotations

import json
import sys

import numpy as np

from . import bisim, lts_gen

WORKLOADS = {
    "kripke": lambda: lts_gen.kripke_uniform(seed=0),
    "qexp": lambda: lts_gen.quotient_expansion(seed=1),
    "chain": lambda: lts_gen.chain(seed=2, n=50000),
    "powerlaw2m": lambda: lts_gen.powerlaw(seed=3, n=2_000_000),
}


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


def shapes(workloads=("kripke", "qexp", "chain"), repeats: int = 3):
    for wl in workloads:
        lts = WORKLOADS[wl]()
        for eng in (bisim.ENGINE_FRONTIER, bisim.ENGINE_DENSE):
            for threads, mc in ((512, 0), (512, 76), (512, 38), (512, 16), (256, 152), (1024, 152)):
                best, st = None, None
                for _ in range(repeats):
                    _, st = bisim.reduce(lts, bisim.make_opts(engine=eng, threads=threads, max_ctas=mc),
                                         return_stats=True)
                    best = st.t_main_ms if best is None else min(best, st.t_main_ms)
                print(json.dumps({"workload": wl, "engine": eng, "threads": threads, "max_ctas": mc,
                                  "main_ms": best, "rounds": st.rounds,
                                  "us_per_round": 1000 * best / max(st.rounds, 1)}), flush=True)


def splitters(workloads=("qexp", "powerlaw2m"), repeats: int = 2):
    """Main-loop time against the splitters-per-round cap and the per-warp
    state budget of rounds with several splitters."""
    for wl in workloads:
        lts = WORKLOADS[wl]()
        for threads in (512, 1024):
            for kmax in (1, 64, 1024, 4096, 8192):
                for budget in ((1,) if kmax == 1 else (1, 2, 4)):
                    best, st = None, None
                    for _ in range(repeats):
                        _, st = bisim.reduce(lts, bisim.make_opts(engine=bisim.ENGINE_FRONTIER, threads=threads,
                                                                  splitters=kmax, split_budget=budget),
                                             return_stats=True)
                        best = st.t_main_ms if best is None else min(best, st.t_main_ms)
                    print(json.dumps({"workload": wl, "threads": threads, "splitters": kmax, "budget": budget,
                                      "main_ms": best, "rounds": st.rounds, "steps": st.steps}), flush=True)


def fanout(sizes=(10, 100, 200, 300, 400, 500, 600, 700, 10_000, 100_000, 1_000_000), repeats: int = 3):
    """Fan_out_n (Section 5.1): reduction time (plan + refinement, device) per
    engine against n, with the closed form checked (states 0 and 1 together,
    every other state alone)."""
    for n in sizes:
        lts = lts_gen.fan_out(n)
        want = np.concatenate([[0, 0], np.arange(1, n - 1)]).astype(np.int32)
        for eng in (bisim.ENGINE_FRONTIER, bisim.ENGINE_DENSE, bisim.ENGINE_PAIR):
            if eng != bisim.ENGINE_FRONTIER and n > 100_000:
                continue
            best, st = None, None
            for _ in range(repeats):
                got, st = bisim.reduce(lts, bisim.make_opts(engine=eng), return_stats=True)
                t = st.t_plan_ms + st.t_refine_ms
                best = t if best is None else min(best, t)
            print(json.dumps({"workload": "fanout", "n": n, "engine": eng, "ms": best, "rounds": st.rounds,
                              "steps": st.steps, "closed_form": bool(np.array_equal(got, want))}), flush=True)


def phases(workloads=("qexp", "powerlaw2m", "kripke"), repeats: int = 2):
    """Per-phase time of the hybrid rounds (phase-timer build of the library):
    microseconds per multi-splitter round for each phase, and the counts."""
    o = bisim.make_opts(local_states=-1)  # the hybrid schedule from the first round
    for wl in workloads:
        lts = WORKLOADS[wl]()
        bisim.reduce(lts, o)  # warm-up
        bisim.bisim_phase_reset()
        best = None
        for _ in range(repeats):
            _, st = bisim.reduce(lts, o, return_stats=True)
            best = st.t_main_ms if best is None else min(best, st.t_main_ms)
        ph = bisim.bisim_phase_times()
        rounds = max(ph["multi_rounds"], 1)
        per_round = {k: ph[k] / 1e3 / rounds for k in ("select", "publish", "claim", "barrier_claim", "mark",
                                                        "barrier_mark", "split", "barrier_split")}
        print(json.dumps({"workload": wl, "main_ms": best, "rounds": st.rounds, "steps": st.steps,
                          "us_per_multi_round": per_round, "counts_over_runs": {
                              k: ph[k] for k in ("multi_rounds", "single_rounds", "cta0_rounds", "splitters",
                                                 "splitter_states", "touched_blocks")}}), flush=True)


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
    if what == "phases":
        from . import _build

        bisim.load(path=_build.build_phase())
        phases(tuple(argv[2:]) or ("qexp", "powerlaw2m", "kripke"))
        return
    bisim.load(build_if_missing=True)
    if what == "barrier":
        barrier()
    elif what == "shapes":
        shapes(tuple(argv[2:]) or ("kripke", "qexp", "chain"))
    elif what == "fanout":
        fanout()
    elif what == "hbm":
        hbm(n=int(argv[2]) if len(argv) > 2 else 10_000_000)
    elif what == "splitters":
        splitters(tuple(argv[2:]) or ("qexp", "powerlaw2m"))
    else:
        raise SystemExit(f"unknown diagnostic {what}")


if __name__ == "__main__":
    main(sys.argv)
