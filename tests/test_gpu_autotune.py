"""The tuner picks a launch shape on the GPU and the tuned batch still
matches the one-at-a-time results."""
import numpy as np
import pytest

from paper_2105_11788_gb300 import autotune, bisim, lts_gen

pytestmark = pytest.mark.gpu


def test_tune_and_use(tmp_path):
    bisim.load(build_if_missing=True)
    rng = np.random.default_rng(17)
    ltss = [lts_gen.stream_instance(rng, n_lo=100, n_hi=8000, idx=i) for i in range(40)]
    t = autotune.BatchTuner(cache_path=str(tmp_path / "t.json"), repeats=1)
    opts, rec = t.tune(ltss)
    assert rec["threads"] in (128, 256, 512, 1024) and len(rec["timings_ms"]) == len(autotune.CANDIDATES)
    assert t.lookup(ltss).threads == rec["threads"]
    parts = bisim.reduce_batch(ltss, opts)
    for l, got in zip(ltss, parts):
        assert np.array_equal(got, bisim.reduce(l))
