"""Host logic of bench.py that needs no GPU: the comment-insensitive source
digest, the staleness rule of the committed DRAM-traffic record, the
algorithmic byte counts and the ratio to the paper's Fan_out_n times."""
import json
import os
import types

import bench


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_source_digest_ignores_comments_and_whitespace(tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    _write(a, "int f(int x) {\n  return x + 1;  // one more\n}\n")
    _write(b, "/* header */\nint f(int x) { return x + 1; }\n// trailing note\n")
    _write(c, "int f(int x) { return x + 2; }\n")
    assert bench.source_digest(a) == bench.source_digest(b)
    assert bench.source_digest(a) != bench.source_digest(c)


def test_recorded_traffic_is_dropped_when_the_kernel_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    _write(src, "__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"k@w": {"dram_bytes_per_launch": 1234, "source": "k.cu",
                   "source_digest": bench.source_digest(src)}}
    _write(tmp_path / "profiles" / "ncu_traffic.json", json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k", "w") == 1234
    assert bench.recorded_traffic("k", "other") is None
    _write(src, "// a comment does not matter\n__global__ void k() {}\n")
    assert bench.recorded_traffic("k", "w") == 1234
    _write(src, "__global__ void k() { int x = 0; }\n")
    assert bench.recorded_traffic("k", "w") is None


def test_committed_traffic_record_is_well_formed():
    path = os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")
    with open(path) as f:
        rec = json.load(f)
    for key, v in rec.items():
        if key.startswith("_"):
            continue
        kernel, workload = key.split("@")
        assert kernel.startswith("k_") and workload
        assert v["dram_bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(bench.ROOT, v["source"]))
        assert os.path.exists(os.path.join(bench.ROOT, v["summary"]))
        assert len(v["source_digest"]) == 64


def test_algorithmic_bytes():
    st = types.SimpleNamespace(n=10, mark_length=7, rounds=3, edges_visited=5, states_visited=4)
    assert bench.dense_bytes_per_launch(st) == 3 * (30 * 10 + 8 * 7) + 12 * 5
    assert bench.frontier_bytes_per_launch(st) == 20 * 5 + 24 * 4


def test_ratio_to_the_paper_fan_out_time():
    args = types.SimpleNamespace(workload="fanout", fanout_n=700)
    ms = bench.PAPER_FANOUT_MS[700]
    # the paper's run time as transitions of Fan_out_700 (3n - 3) reduced per second
    assert abs(bench.vs_paper(args, (3 * 700 - 3) * 1000.0 / ms) - 1.0) < 1e-12
    assert bench.vs_paper(types.SimpleNamespace(workload="qexp", fanout_n=700), 5.0) is None


def test_default_workload_is_the_large_power_law_lts():
    import inspect

    src = inspect.getsource(bench.main)
    assert 'default="powerlaw"' in src
    assert "n=10,000,000" in bench.WORKLOADS["powerlaw"][0]
    # the reference arm reduces a smaller member of the same family per step
    assert "powerlaw" in bench.REF_SAMPLE


def test_stream_sample_follows_the_size_mix():
    ltss = [types.SimpleNamespace(n=n) for n in [5, 1, 9, 3, 7, 2, 8, 4, 6, 10]]
    idx = bench.stream_sample(ltss, 5)
    assert len(set(idx)) == 5
    sizes = sorted(ltss[i].n for i in idx)
    assert sizes == [2, 4, 6, 8, 10]
    assert len(bench.stream_sample(ltss, 50)) == 10


def test_reference_arm_lines():
    """`bench.py --impl reference` times the oracle on the host and prints the
    contract's line, for a single-LTS workload and for the stream."""
    import subprocess
    import sys

    for extra in (["--workload", "kripke"], ["--workload", "stream", "--stream-k", "64", "--ref-sample", "4"]):
        r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                            "--steps", "1", "--warmup", "0", *extra],
                           capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
        assert r.returncode == 0, r.stderr
        line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
        unit = "LTS/s" if "stream" in extra else "transitions/s"
        assert line["impl"] == "reference" and line["unit"] == unit and line["value"] > 0
        assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
        assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
