"""Full-size parity on the large power-law LTS (10^7 states, ~10^8
transitions, 32 labels, 4 initial blocks), in the launch configuration the
benchmark uses: bit-exact canonical partition against the oracle, the round
bounds of Theorem 3, and the definitions themselves checked on the GPU's
output (it refines the initial partition and is stable for every block and
label), which share nothing with the oracle's refinable-partition design.
Takes a few minutes (the oracle alone ~50 s, the stability check ~20 s)."""
import numpy as np
import pytest

import oracle
from oracle import defs
from paper_2105_11788_gb300 import bisim, lts_gen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_powerlaw_full_size_matches_oracle():
    import torch

    assert torch.cuda.is_available()
    bisim.load(build_if_missing=True)
    lts = lts_gen.powerlaw(seed=3)
    got, st = bisim.reduce(lts, bisim.make_opts(), return_stats=True)
    want = oracle.ks_lts(lts)
    assert np.array_equal(got, want)
    B = int(want.max()) + 1
    assert st.num_blocks == B
    assert B + 1 <= st.rounds <= 3 * B - st.initial_blocks + 1
    assert st.pre_rounds == 32
    assert defs.refines(got, lts.init)
    assert defs.is_stable(lts.n, lts.src, lts.act, lts.dst, got)
