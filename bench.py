"""Benchmark: strong-bisimulation reduction of one synthetic LTS per step.

A step is one whole reduction through the C ABI: bisim_plan (validation,
the mark-slot layout of the (source, label) pairs, incoming-transition CSR,
initial leaders, action-set preprocessing) and bisim_refine (the main loop
and the canonical output) on inputs already resident in device memory. The default
workload is the large power-law LTS (seed 3: 10,000,000 states, 99,917,783
transitions, out-degree Pareto alpha = 2.1 with mean 10, 32 uniform labels,
4 initial blocks from two atomic propositions). Single-LTS throughput is
reported in transitions of the LTS reduced per second (m / reduction time),
which stays comparable when the CPU oracle of the reference arm reduces a
smaller member of the same family.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle
(Kanellakis-Smolka, single thread) on the same workload instead (on a
bounded sample where a full reduction takes the oracle more than a few
seconds).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2105_11788_gb300 import lts_gen  # noqa: E402

WORKLOADS = {
    "powerlaw": ("large power-law LTS (seed 3, n=10,000,000, m=99,917,783, out-degree Pareto alpha=2.1 "
                 "mean 10 capped at 10,000, uniform targets, |Act|=32 uniform, 4 initial blocks from 2 "
                 "atomic propositions)", lambda: lts_gen.powerlaw(seed=3)),
    "qexp": ("labelled LTS by quotient expansion (seed 1, ~101.7k states, ~1.11M transitions, "
             "|Act|=8 Zipf, single initial block)", lambda: lts_gen.quotient_expansion(seed=1)),
    "kripke": ("Kripke structure (seed 0, n=1000, m=4000, 4 AP blocks)",
               lambda: lts_gen.kripke_uniform(seed=0)),
    "chain": ("deep-refinement chain (seed 2, n=50000)", lambda: lts_gen.chain(seed=2, n=50000)),
    "powerlaw2m": ("power-law LTS (seed 3, n=2M, m~20M, |Act|=32, 4 AP blocks)",
                   lambda: lts_gen.powerlaw(seed=3, n=2_000_000)),
}

# Fan_out_n (Section 5.1): the paper's Par-BCRP run times in ms (Titan RTX)
PAPER_FANOUT_MS = {10: 1, 100: 5, 200: 9, 300: 13, 400: 18, 500: 22, 600: 26, 700: 30}


def workload(args):
    """(description, generator) of the chosen single-LTS workload."""
    if args.workload == "fanout":
        n = args.fanout_n
        return (f"Fan_out_n of Section 5.1 (n={n}, 3n-3 transitions, labels a/b, single initial block)",
                lambda: lts_gen.fan_out(n))
    return WORKLOADS[args.workload]


# the reference arm's oracle reduces this smaller member of the same family
# per step where a full reduction of the workload takes it tens of seconds
REF_SAMPLE = {
    "powerlaw": ("the power-law LTS of the same generator and seed with n=1,000,000 (m~10M), one full "
                 "reduction per step", lambda: lts_gen.powerlaw(seed=3, n=1_000_000)),
}

SINGLE_METRIC = "LTS reduction throughput (transitions of the LTS reduced per second)"
SINGLE_UNIT = "transitions/s"


def vs_paper(args, value):
    """value / the paper's number for this exact workload and metric
    (transitions/s of Fan_out_n at the paper's run time), else None."""
    if args.workload == "fanout" and args.fanout_n in PAPER_FANOUT_MS:
        n = args.fanout_n
        return value / ((3 * n - 3) * 1000.0 / PAPER_FANOUT_MS[n])
    return None


L2_BYTES = 129 * 1024 * 1024
SERVE_BIG_STATES = 20000  # serving: LTSs with at least this many states are reduced alone


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.device_id:
                cmd += ["-i", self.device_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def source_digest(path):
    """sha256 of a CUDA source with comments removed and whitespace runs
    collapsed: it changes when the code changes, not when a comment does."""
    import hashlib
    import re

    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = re.sub(r"\s+", " ", text).strip()
    return hashlib.sha256(text.encode()).hexdigest()


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    record (profiles/ncu_traffic.json), or None when there is none or the
    kernel's source code has changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(f"{kernel}@{workload}")
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or source_digest(src) != rec.get("source_digest"):
        return None
    return rec["dram_bytes_per_launch"]


def dense_bytes_per_launch(st):
    """Algorithmic bytes of one main-loop launch of the dense engine: per round
    4n (unstable scan) + 4n (block, mark scan) + 4n (block, compare) + 8n (own
    off pair) + 8n (leader off pair) + 2n (split flag write and read) + 8L (own
    and leader mark slots); plus 12 B per incoming transition walked (8 B
    record + 4 B mark store)."""
    n, L = st.n, st.mark_length
    return st.rounds * (30 * n + 8 * L) + 12 * st.edges_visited


def frontier_bytes_per_launch(st):
    """Algorithmic bytes of one main-loop launch of the frontier engine: 20 B
    per incoming transition walked (8 B record, 4 B mark stamp, 4 B source
    block, 4 B touched stamp) and 24 B per state whose marks were compared
    (member id, block label, off pair, leader mark slots amortised, move and
    relabel)."""
    return 20 * st.edges_visited + 24 * st.states_visited


def run_reference(args, world, rank):
    """CPU oracle (Kanellakis-Smolka, one thread) on the same workload, or on
    its bounded sample (REF_SAMPLE); throughput in transitions reduced per
    second, like the GPU arm."""
    import oracle

    if world > 1 and rank != 0:
        return
    if args.workload == "stream":
        run_reference_stream(args, world)
        return
    desc, make = workload(args)
    if args.workload in REF_SAMPLE:
        sample_desc, make_sample = REF_SAMPLE[args.workload]
        lts = make_sample()
        sample = f"{sample_desc} by oracle_ks (single-threaded C), {args.steps} timed steps"
    else:
        lts = make()
        sample = f"{args.steps} full reductions of the workload (oracle_ks, single-threaded C)"
    for _ in range(args.warmup):
        oracle.ks_lts(lts)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.ks_lts(lts)
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = lts.m * 1000.0 / ms
    line = {
        "impl": "reference", "metric": SINGLE_METRIC, "value": value,
        "unit": SINGLE_UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": vs_paper(args, value),
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": desc, "sample_n": lts.n, "sample_m": lts.m, "num_act": lts.num_act,
                   "l2": "CPU run"},
        "cpu_baseline": {"value": value, "unit": SINGLE_UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "ms_per_reduction": ms},
        "e2e": {"value": value, "unit": SINGLE_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


STREAM_DESC = ("batched stream (seed 4): LTSs with n log-uniform in [100, 200000], m = 5n, |Act| in "
               "[1, 32], quotient expansion with n/20 classes")


def stream_sample(ltss, k):
    """k LTSs of the stream spread evenly over its size order (every
    (len/k)-th by state count), so the sample follows the stream's size mix."""
    order = sorted(range(len(ltss)), key=lambda i: (ltss[i].n, i))
    k = max(1, min(k, len(order)))
    return [order[int((j + 0.5) * len(order) / k)] for j in range(k)]


def run_reference_stream(args, world):
    """CPU oracle on the stream: every step reduces the same bounded sample
    (`--ref-sample` LTSs spread evenly over the stream's size order) one after
    the other; LTS/s = sample size / step time."""
    import oracle

    ltss_all, _ = lts_gen.batch_stream(seed=4, k=args.stream_k)
    idx = stream_sample(ltss_all, args.ref_sample)
    ltss = [ltss_all[i] for i in idx]
    k = len(ltss)
    for _ in range(args.warmup):
        for lts in ltss:
            oracle.ks_lts(lts)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for lts in ltss:
            oracle.ks_lts(lts)
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = k * 1000.0 / ms
    n_sample = sum(l.n for l in ltss)
    mean_stream = sum(l.n for l in ltss_all) / len(ltss_all)
    sample = (f"{k} LTSs spread evenly over the size order of the {args.stream_k}-LTS stream "
              f"(mean {n_sample / k:.0f} states against {mean_stream:.0f} for the whole stream), reduced one "
              f"after the other by oracle_ks (single-threaded C), {args.steps} times")
    line = {
        "impl": "reference", "metric": "batched LTS reduction throughput", "value": value,
        "unit": "LTS/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": STREAM_DESC, "k": args.stream_k, "sample": k, "l2": "CPU run"},
        "cpu_baseline": {"value": value, "unit": "LTS/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "states_per_s": n_sample * 1000.0 / ms, "sample_mean_n": n_sample / k,
                         "stream_mean_n": mean_stream},
        "e2e": {"value": value, "unit": "LTS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_stream(args, world, rank, local):
    """Stream workload: one step = batch plan + batch refine of all LTSs
    (inputs resident); plus the one-at-a-time rate on a sample, the serving
    loop at 0.5x / 1x / 2x that rate, and the oracle on a sample."""
    import torch

    from paper_2105_11788_gb300 import bisim, serve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bisim.load(build_if_missing=True)
    t_gen = time.perf_counter()
    ltss, _ = lts_gen.batch_stream(seed=4, k=args.stream_k)
    t_gen = time.perf_counter() - t_gen
    k = len(ltss)
    so, to, na, src, act, dst, init = bisim.pack_batch(ltss)
    N, M = int(so[-1]), int(to[-1])
    tuned = None
    if args.threads == 0 and not args.no_autotune:
        # launch shape picked by the autotuner, timed on this batch
        from paper_2105_11788_gb300 import autotune

        tuner = autotune.BatchTuner(cache_path=os.path.join(tempfile.gettempdir(), "bisim_bench_autotune.json"), repeats=1)
        opts, tuned = tuner.tune(ltss, device=str(dev))
    else:
        opts = bisim.make_opts(threads=args.threads, max_ctas=args.max_ctas)
    d = lambda a: torch.from_numpy(a).to(dev)  # noqa: E731
    tsrc, tact, tdst = d(src), d(act), d(dst)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = int(stream.cuda_stream)

    def step():
        h = bisim.bisim_batch_plan(k, so, to, na, tsrc.data_ptr(), tact.data_ptr(), tdst.data_ptr(), None,
                                   opts, sp)
        try:
            return bisim.bisim_batch_refine(h, out.data_ptr(), k)
        finally:
            bisim.bisim_plan_destroy(h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0])
    clocks.start()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    total_ms, kern_ms, stats = 0.0, [], []
    for _ in range(args.steps):
        e0.record(stream)
        st, inst = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        kern_ms.append(st.t_main_ms)
        stats.append(st)
    barrier(world)
    clk = clocks.stop()
    ms_step = max_over_ranks(total_ms / args.steps, world, dev)
    value = world * k * 1000.0 / ms_step
    st = stats[-1]
    # end to end from pinned host buffers (copies inside the timed region)
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    hsrc, hact, hdst = pin(src), pin(act), pin(dst)
    hout = torch.empty(N, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tsrc.copy_(hsrc, non_blocking=True)
    tact.copy_(hact, non_blocking=True)
    tdst.copy_(hdst, non_blocking=True)
    step()
    hout.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = 1000 * (time.perf_counter() - t0)
    # one at a time on a sample
    rng = np.random.default_rng(0)
    sample = rng.choice(k, size=min(args.plain_sample, k), replace=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        bisim.reduce(ltss[i], device=dev)
    plain_s = time.perf_counter() - t0
    plain_rate = len(sample) / plain_s
    # serving loop at 0.5x to 20x the one-at-a-time rate; LTSs of at least
    # SERVE_BIG_STATES states take the large-request lane (the single-LTS path)
    serving = {}
    if args.serve_requests > 0:
        sub = [ltss[i] for i in rng.choice(k, size=min(args.serve_requests, k), replace=False)]
        for mult in (0.5, 1.0, 2.0, 5.0, 20.0):
            reqs = serve.poisson_requests(sub, rate_per_s=mult * plain_rate, seed=int(mult * 10))
            srv = serve.BatchServer(serve.gpu_executor(device=str(dev)), mem_budget=64 << 30, workers=3,
                                    max_batch=256, big_executor=serve.gpu_single_executor(device=str(dev)),
                                    big_states=SERVE_BIG_STATES)
            res = srv.serve(reqs)
            serving[f"{mult}x"] = dict(serve.latency_summary(res), rate_per_s=mult * plain_rate,
                                       large_lane=srv.big_served)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        t0 = time.perf_counter()
        cnt = 0
        for i in rng.permutation(k):
            oracle.ks_lts(ltss[i])
            cnt += 1
            if time.perf_counter() - t0 > args.cpu_budget:
                break
        el = time.perf_counter() - t0
        cpu = {"value": cnt / el, "unit": "LTS/s", "cores": 1, "kind": "oracle",
               "sample": f"{cnt} LTSs of the stream in random order reduced by oracle_ks "
                         f"(single-threaded C), {el:.1f} s"}
    hbm, peak_kind = read_peaks()
    bytes_launch = frontier_bytes_per_launch(st)
    km = sum(kern_ms) / len(kern_ms)
    achieved = bytes_launch / (km * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": "batched LTS reduction throughput", "value": value, "unit": "LTS/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": STREAM_DESC, "k": k, "n_total": N, "m_total": M,
                       "threads": opts.threads, "ctas_per_sm": opts.ctas_per_sm,
                       "wide_threads": opts.wide_threads, "wide_min_states": opts.wide_min_states,
                       "splitters": opts.splitters, "split_budget": opts.split_budget,
                       "multi_min_states": opts.multi_min_states,
                       "autotune": tuned,
                       "l2": "inputs larger than L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": "k_frontier_batch", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                         "traffic": recorded_traffic("k_frontier_batch", f"stream{k}"),
                         "kernel_ms": km, "bytes_per_launch": bytes_launch},
            "e2e": {"value": world * k * 1000.0 / e2e_ms, "unit": "LTS/s",
                    "h2d_bytes_per_step": int(src.nbytes + act.nbytes + dst.nbytes),
                    "d2h_bytes_per_step": int(4 * N), "ms_per_step": e2e_ms},
            "cpu_baseline": cpu,
            "gpu_launches": int(sum(s.launches for s in stats)),
            "clocks": clk,
            "detail": {"plain_one_at_a_time_lts_per_s": plain_rate, "plain_sample": int(len(sample)),
                       "batched_over_plain": value / plain_rate, "serving": serving,
                       "t_plan_ms": st.t_plan_ms, "t_refine_ms": st.t_refine_ms, "t_main_ms": st.t_main_ms,
                       "rounds_total": st.rounds, "edges_visited": st.edges_visited,
                       "states_visited": st.states_visited, "grid_ctas": st.grid_ctas,
                       "generation_s": t_gen},
        }
        print(json.dumps(line), flush=True)


def cpu_baseline(lts, budget_s):
    import oracle

    t0 = time.perf_counter()
    k = 0
    while True:
        oracle.ks_lts(lts)
        k += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": k * lts.m / el, "unit": SINGLE_UNIT, "cores": 1, "kind": "oracle",
            "ms_per_reduction": 1000.0 * el / k,
            "sample": f"{k} full reductions of the same workload by oracle_ks (single-threaded C), "
                      f"{el:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="powerlaw", choices=sorted(WORKLOADS) + ["fanout", "stream"])
    ap.add_argument("--fanout-n", type=int, default=700, help="fanout: states of Fan_out_n")
    ap.add_argument("--stream-k", type=int, default=4096, help="LTSs in the stream workload")
    ap.add_argument("--plain-sample", type=int, default=128,
                    help="stream: LTSs reduced one at a time to estimate the plain rate")
    ap.add_argument("--ref-sample", type=int, default=24,
                    help="stream, --impl reference: LTSs of the stream the oracle reduces per step")
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="stream: requests per arrival rate in the serving run")
    ap.add_argument("--engine", default="auto", choices=["auto", "dense", "frontier", "pair"])
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0 = library default)")
    ap.add_argument("--max-ctas", type=int, default=0, help="cap on persistent-kernel CTAs")
    ap.add_argument("--local-states", type=int, default=0,
                    help="frontier: LTSs up to this many states on one CTA (0 = library rule, -1 = never)")
    ap.add_argument("--light-edges", type=int, default=0,
                    help="frontier: light-round threshold (0 = library default, <0 = grid only)")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="stream: skip the launch-shape tuner")
    ap.add_argument("--hbm-rounds", type=int, default=-1,
                    help="also time the paper's bandwidth-bound rounds (literal label rounds and a "
                         "window of this many dense rounds); -1 = 200 for the power-law workload, else off")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "stream":
        run_stream(args, world, rank, local)
        return

    import torch

    from paper_2105_11788_gb300 import bisim

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bisim.load(build_if_missing=True)
    engine = {"auto": bisim.ENGINE_AUTO, "dense": bisim.ENGINE_DENSE,
              "frontier": bisim.ENGINE_FRONTIER, "pair": bisim.ENGINE_PAIR}[args.engine]
    opts = bisim.make_opts(engine=engine, threads=args.threads, max_ctas=args.max_ctas,
                           light_edges=args.light_edges, local_states=args.local_states)
    desc, make = workload(args)
    lts = make()
    src = torch.from_numpy(lts.src).to(dev)
    act = torch.from_numpy(lts.act).to(dev)
    dst = torch.from_numpy(lts.dst).to(dev)
    init = torch.from_numpy(lts.init).to(dev) if lts.init is not None else None
    out = torch.empty(max(lts.n, 1), dtype=torch.int32, device=dev)
    in_bytes = lts.nbytes()
    flush = None
    if in_bytes < 2 * L2_BYTES:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = int(stream.cuda_stream)

    def step():
        h = bisim.bisim_plan(lts.n, lts.m, lts.num_act, src.data_ptr(), act.data_ptr(),
                             dst.data_ptr(), init.data_ptr() if init is not None else None, opts, sp)
        try:
            st = bisim.bisim_refine(h, out.data_ptr())
        finally:
            bisim.bisim_plan_destroy(h)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dev_id = ""
    try:
        dev_id = str(torch.cuda.get_device_properties(dev).uuid)
        if dev_id and not dev_id.startswith("GPU-"):
            dev_id = "GPU-" + dev_id
    except Exception:
        dev_id = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    clocks = ClockSampler(dev_id)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    total_ms = 0.0
    kernel_ms, kernel_bytes, stats = [], [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        if flush is not None:
            flush.fill_(1)  # untimed: evicts L2 between steps
        e0.record(stream)
        st = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        stats.append(st)
        kernel_ms.append(st.t_main_ms)
        kernel_bytes.append(dense_bytes_per_launch(st) if st.engine == bisim.ENGINE_DENSE
                            else frontier_bytes_per_launch(st))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_step = max_over_ranks(total_ms / args.steps, world, dev)
    value = world * lts.m * 1000.0 / ms_step
    st = stats[-1]
    hbm, peak_kind = read_peaks()
    achieved = (sum(kernel_bytes) / len(kernel_bytes)) / (sum(kernel_ms) / len(kernel_ms) * 1e-3) / 1e9
    if st.engine == bisim.ENGINE_DENSE:
        kname, schedule = "k_dense_main", "dense rounds on the whole grid"
    elif st.engine == bisim.ENGINE_PAIR:
        kname, schedule = "k_pair_main", "pair rounds on the whole grid"
    elif st.engine == bisim.ENGINE_SMALL:
        kname, schedule = "k_small", "one CTA in shared memory (the whole reduction in one launch)"
    elif st.grid_ctas == 1:
        kname, schedule = "k_frontier_batch", "one CTA (sparse LTS)"
    elif st.local_steps > 0:
        # started on one CTA, handed to the hybrid: the main loop is two
        # launches, whose bytes and time the achieved figure sums
        kname = "k_frontier_batch+k_frontier_hybrid"
        schedule = f"one CTA for {st.local_steps} of {st.steps} rounds, then hybrid"
    elif args.light_edges < 0:
        kname, schedule = "k_frontier_main", "every round on the whole grid"
    else:
        kname, schedule = "k_frontier_hybrid", "hybrid (light rounds on one CTA)"
    km_avg = sum(kernel_ms) / len(kernel_ms)
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_kind": peak_kind,
            "traffic": None if "+" in kname else recorded_traffic(kname, args.workload),
            "kernel_ms": km_avg,
            "bytes_per_launch": sum(kernel_bytes) / len(kernel_bytes)}
    # the rounds' other bound: barriers and dependent loads. Measured grid
    # barrier cost at this launch's grid size, beside the time per round
    latency = None
    if st.engine not in (bisim.ENGINE_DENSE, bisim.ENGINE_SMALL) and st.steps > 0:
        bar_ns = None
        try:
            ctas = max(1, st.grid_ctas)
            thr = args.threads or (1024 if ctas == 1 else 512)
            bar_ns = min(bisim.bisim_barrier_cost(ctas, thr, 5000, sp) for _ in range(3))
        except bisim.BisimError:
            pass
        per_round = 2 if st.rounds - 1 <= st.steps else 3  # one splitter per round: mark, split
        us_step = 1000.0 * st.t_main_ms / st.steps
        latency = {"us_per_round": us_step, "rounds": st.steps,
                   "barrier_us": None if bar_ns is None else bar_ns / 1000.0,
                   "barriers_per_round": per_round,
                   "barrier_share": None if bar_ns is None else per_round * bar_ns / 1000.0 / us_step,
                   "splitter_iterations_per_round": (st.rounds - 1) / st.steps}

    # end to end through the host-buffer entry point
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    hs, ha, hd = pin(lts.src), pin(lts.act), pin(lts.dst)
    hi = pin(lts.init) if lts.init is not None else None
    ho = torch.empty(max(lts.n, 1), dtype=torch.int32).pin_memory()
    e2e_ms = []
    for i in range(max(3, args.steps // 2) + 1):
        if flush is not None:
            flush.fill_(1)  # untimed: evicts L2, as between the device-timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bisim.bisim_reduce_host(lts.n, lts.m, lts.num_act, hs.data_ptr(), ha.data_ptr(),
                                hd.data_ptr(), hi.data_ptr() if hi is not None else None,
                                ho.data_ptr(), opts, sp)
        if i:
            e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_step = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, dev)
    h2d = lts.nbytes()
    paper_hbm = None
    hbm_window = args.hbm_rounds if args.hbm_rounds >= 0 else (200 if args.workload == "powerlaw" else 0)
    if hbm_window > 0:
        from paper_2105_11788_gb300 import diag

        diag.paper_rounds(lts, src, act, dst, init, window=min(hbm_window, 20))  # warm-up
        paper_hbm = diag.paper_rounds(lts, src, act, dst, init, window=hbm_window, peak=hbm,
                                      peak_kind=peak_kind)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lts, args.cpu_budget)
    if rank == 0:
        visits = (st.pre_rounds + st.rounds) * lts.m
        line = {
            "metric": SINGLE_METRIC, "value": value, "unit": SINGLE_UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": vs_paper(args, value),
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "n": lts.n, "m": lts.m, "num_act": lts.num_act,
                       "engine": args.engine, "schedule": schedule, "threads": args.threads,
                       "max_ctas": args.max_ctas,
                       "l2": "flushed between steps (256 MiB write)" if flush is not None
                             else "inputs larger than L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof,
            "latency": latency,
            "hbm_rounds": paper_hbm,
            "e2e": {"value": world * lts.m * 1000.0 / e2e_step, "unit": SINGLE_UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4 * lts.n,
                    "ms_per_step": e2e_step},
            "cpu_baseline": cpu,
            "gpu_launches": int(sum(s.launches for s in stats)),
            "clocks": clk,
            "detail": {"rounds": st.rounds, "steps": st.steps, "local_steps": st.local_steps,
                       "pre_rounds": st.pre_rounds,
                       "initial_blocks": st.initial_blocks, "num_blocks": st.num_blocks,
                       "mark_length": st.mark_length, "t_plan_ms": st.t_plan_ms,
                       "t_refine_ms": st.t_refine_ms, "t_pre_ms": st.t_pre_ms,
                       "t_main_ms": st.t_main_ms, "reduction_ms": ms_step,
                       "lts_per_s": world * 1000.0 / ms_step,
                       "us_per_round": 1000 * st.t_main_ms / max(st.steps, 1),
                       "us_per_iteration": 1000 * st.t_main_ms / max(st.rounds, 1),
                       "edges_visited": st.edges_visited, "states_visited": st.states_visited,
                       "grid_ctas": st.grid_ctas,
                       # incoming transitions the main loop's kernels walked, per second of main loop
                       "transition_visits_per_s": st.edges_visited / (st.t_main_ms * 1e-3)
                       if st.t_main_ms > 0 else None,
                       # (pre_rounds + rounds) * m / step time: the visits of the paper's
                       # m-thread rounds, which touch every transition every iteration
                       "pram_transition_visits_per_s": visits / (ms_step * 1e-3)},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
