"""The allocation-free entry point bisim_canonical_ids_noalloc, for callers
that cannot allocate device memory (their device budget is owned by another
allocator, or an allocation would synchronise a latency-critical loop). Its
scratch is a fixed array inside the library, shared by every call, so the
test makes two calls in a row and checks that the second one is not affected
by what the first left behind.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_2105_11788_gb300 import bisim, lts_gen

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _raw_and_canonical(lts):
    """Leader labels and canonical ids from the existing entry point
    (bisim_refine with and without raw_labels)."""
    src, act, dst = _dev(lts.src), _dev(lts.act), _dev(lts.dst)
    init = _dev(lts.init) if lts.init is not None else None
    with bisim.Plan(lts.n, lts.num_act, src, act, dst, init, bisim.make_opts(raw_labels=True)) as p:
        raw, _ = p.refine()
        raw = raw.clone()
    with bisim.Plan(lts.n, lts.num_act, src, act, dst, init) as p:
        ids, st = p.refine()
        ids = ids.clone()
    return raw, ids, st.num_blocks


def test_noalloc_matches_bisim_refine_on_two_calls_in_a_row():
    import torch

    torch.cuda.init()
    big = lts_gen.quotient_expansion(seed=1)
    small = lts_gen.kripke_uniform(seed=0)
    cases = [_raw_and_canonical(big), _raw_and_canonical(small)]
    stream = int(torch.cuda.current_stream().cuda_stream)
    for raw, want, want_nb in cases + cases:  # every case twice, alternating sizes
        n = raw.shape[0]
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        for _ in range(2):
            nb = bisim.bisim_canonical_ids_noalloc(raw.data_ptr(), n, out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert nb == want_nb
            assert torch.equal(out, want)
            out.fill_(-7)


def test_noalloc_rejects_sizes_beyond_its_capacity():
    import torch

    n = bisim.BISIM_NOALLOC_MAX_N + 1
    lab = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bisim.BisimError) as ei:
        bisim.bisim_canonical_ids_noalloc(lab.data_ptr(), n, out.data_ptr())
    assert ei.value.code == bisim.BISIM_EINVAL
    # a label outside [0, n) is rejected as well, and the next call still works
    bad = torch.tensor([0, 1, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(bisim.BisimError) as ei:
        bisim.bisim_canonical_ids_noalloc(bad.data_ptr(), 3, out.data_ptr())
    assert ei.value.code == bisim.BISIM_EINVAL
    ok = torch.tensor([2, 2, 0], dtype=torch.int32, device="cuda")
    assert bisim.bisim_canonical_ids_noalloc(ok.data_ptr(), 3, out.data_ptr()) == 2
    torch.cuda.synchronize()
    assert out[:3].tolist() == [0, 0, 1]
