"""Autotuner bookkeeping without a GPU: shape keys and the JSON cache."""
import numpy as np

from paper_2105_11788_gb300 import autotune, lts_gen


def _stream(k, seed=1):
    rng = np.random.default_rng(seed)
    return [lts_gen.stream_instance(rng, n_lo=50, n_hi=5000, idx=i) for i in range(k)]


def test_shape_key_buckets():
    a = _stream(16)
    assert autotune.shape_key(a) == autotune.shape_key(list(a))
    assert autotune.shape_key(a).startswith("k4_")
    assert autotune.shape_key(a[:1]).startswith("k0_")


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "tune.json")
    t = autotune.BatchTuner(cache_path=path)
    ltss = _stream(8)
    assert t.lookup(ltss) is None
    t.cache[autotune.shape_key(ltss)] = {"threads": 512, "ctas_per_sm": 1, "refine_ms": 1.0}
    t.save()
    t2 = autotune.BatchTuner(cache_path=path)
    o = t2.lookup(ltss)
    assert o.threads == 512 and o.ctas_per_sm == 1


def test_sample_keeps_largest():
    ltss = _stream(40, seed=4)
    big = max(l.n for l in ltss)
    sub = autotune.sample_for_tuning(ltss, max_lts=10)
    assert len(sub) == 10 and max(l.n for l in sub) == big
