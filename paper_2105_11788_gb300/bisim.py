"""Thin ctypes binding of the C ABI in include/bisim.h.

The functions named like the C entry points (`bisim_plan`, `bisim_refine`,
`bisim_plan_destroy`, `bisim_reduce_host`, ...) only marshal arguments: raw
device or host addresses and sizes go in, error codes come out as
`BisimError`. Every step of the computation runs in libbisim.so's CUDA
kernels; there is no CPU fallback, and loading fails loudly when the
library has not been built.

`reduce()` and `Plan` are conveniences over torch tensors (torch is used for
device memory and streams only).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

from . import _build

BISIM_OK = 0
BISIM_EINVAL = -1
BISIM_ENOMEM = -2
BISIM_ECUDA = -3
BISIM_EROUNDS = -4
BISIM_ETIMEOUT = -5
BISIM_ENOTSUP = -6

ENGINE_AUTO = 0
ENGINE_DENSE = 1
ENGINE_FRONTIER = 2
ENGINE_PAIR = 3
ENGINE_SMALL = 4  # reported in stats only: a small LTS on one CTA in shared memory


class bisim_opts(ctypes.Structure):
    _fields_ = [
        ("engine", ctypes.c_int32),
        ("rcpp_alg2", ctypes.c_int32),
        ("raw_labels", ctypes.c_int32),
        ("threads", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("test_hook", ctypes.c_int32),
        ("round_cap", ctypes.c_int64),
        ("timeout_ms", ctypes.c_int64),
        ("max_ctas", ctypes.c_int32),
        ("light_edges", ctypes.c_int32),
        ("preprocess", ctypes.c_int32),
        ("wide_threads", ctypes.c_int32),
        ("wide_min_states", ctypes.c_int32),
        ("splitters", ctypes.c_int32),
        ("split_budget", ctypes.c_int32),
        ("multi_min_states", ctypes.c_int32),
        ("local_states", ctypes.c_int32),
        ("peel", ctypes.c_int32),
        ("peel_items", ctypes.c_int32),
        ("small", ctypes.c_int32),
        ("slots", ctypes.c_int32),
    ]


class bisim_stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("num_act", ctypes.c_int64),
        ("mark_length", ctypes.c_int64),
        ("pre_rounds", ctypes.c_int64),
        ("initial_blocks", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("num_blocks", ctypes.c_int64),
        ("edges_visited", ctypes.c_int64),
        ("states_visited", ctypes.c_int64),
        ("t_plan_ms", ctypes.c_double),
        ("t_refine_ms", ctypes.c_double),
        ("t_pre_ms", ctypes.c_double),
        ("t_main_ms", ctypes.c_double),
        ("launches", ctypes.c_int64),
        ("engine", ctypes.c_int32),
        ("grid_ctas", ctypes.c_int32),
        ("steps", ctypes.c_int64),
        ("local_steps", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = [
    "bisim_plan",
    "bisim_refine",
    "bisim_plan_destroy",
    "bisim_reduce_host",
    "bisim_strerror",
    "bisim_last_error",
    "bisim_version",
]


class BisimError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code}){': ' + detail if detail else ''}")


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False, path: Optional[str] = None):
    """Load libbisim.so (raises if it is missing and build_if_missing is False).
    `path` selects another build of the same library (the phase-timer build)."""
    global _lib
    if _lib is not None:
        if path is not None and getattr(_lib, "_path", None) != path:
            raise RuntimeError("another build of libbisim is already loaded in this process")
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        if not build_if_missing or path != _build.LIB:
            raise RuntimeError(f"libbisim not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    lib._path = path
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.bisim_plan.argtypes = [i32, i64, i32, P, P, P, P, ctypes.POINTER(bisim_opts), P,
                               ctypes.POINTER(P)]
    lib.bisim_plan.restype = ctypes.c_int
    lib.bisim_refine.argtypes = [P, P, ctypes.POINTER(bisim_stats)]
    lib.bisim_refine.restype = ctypes.c_int
    lib.bisim_plan_destroy.argtypes = [P]
    lib.bisim_plan_destroy.restype = None
    lib.bisim_reduce_host.argtypes = [i32, i64, i32, P, P, P, P, P, ctypes.POINTER(bisim_opts), P,
                                      ctypes.POINTER(bisim_stats)]
    lib.bisim_reduce_host.restype = ctypes.c_int
    lib.bisim_strerror.argtypes = [ctypes.c_int]
    lib.bisim_strerror.restype = ctypes.c_char_p
    lib.bisim_last_error.argtypes = []
    lib.bisim_last_error.restype = ctypes.c_char_p
    lib.bisim_version.argtypes = []
    lib.bisim_version.restype = i32
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().bisim_strerror(code).decode()
    except Exception:  # library missing: still describe the code
        return str(code)


def _check(code: int, where: str):
    if code != BISIM_OK:
        raise BisimError(code, where, load().bisim_last_error().decode())


def make_opts(engine: int = ENGINE_AUTO, rcpp_alg2: bool = False, raw_labels: bool = False,
              threads: int = 0, ctas_per_sm: int = 0, round_cap: int = 0, timeout_ms: int = 0,
              test_hook: int = 0, max_ctas: int = 0, light_edges: int = 0,
              preprocess: int = 0, wide_threads: int = 0, wide_min_states: int = 0,
              splitters: int = 0, split_budget: int = 0, multi_min_states: int = 0,
              local_states: int = 0, peel: int = 0, peel_items: int = 0, small: int = 0,
              slots: int = 0) -> bisim_opts:
    return bisim_opts(engine, int(rcpp_alg2), int(raw_labels), threads, ctas_per_sm, test_hook,
                      round_cap, timeout_ms, max_ctas, light_edges, preprocess, wide_threads,
                      wide_min_states, splitters, split_budget, multi_min_states, local_states, peel,
                      peel_items, small, slots)


# ----------------------------------------------------------- C-ABI mirrors


def bisim_plan(n: int, m: int, num_act: int, src: int, act: Optional[int], dst: int,
               init_block: Optional[int], opts: Optional[bisim_opts] = None,
               stream: int = 0) -> int:
    """Device addresses in, plan handle out (see include/bisim.h)."""
    lib = load()
    out = ctypes.c_void_p()
    rc = lib.bisim_plan(n, m, num_act, src or None, act or None, dst or None, init_block or None,
                        ctypes.byref(opts) if opts is not None else None, stream or None,
                        ctypes.byref(out))
    _check(rc, "bisim_plan")
    return out.value


def bisim_refine(plan: int, out_block: int) -> bisim_stats:
    st = bisim_stats()
    rc = load().bisim_refine(plan, out_block or None, ctypes.byref(st))
    _check(rc, "bisim_refine")
    return st


def bisim_plan_destroy(plan: Optional[int]) -> None:
    if plan:
        load().bisim_plan_destroy(plan)


def bisim_reduce_host(n: int, m: int, num_act: int, src_h: int, act_h: Optional[int], dst_h: int,
                      init_h: Optional[int], out_h: int, opts: Optional[bisim_opts] = None,
                      stream: int = 0) -> bisim_stats:
    st = bisim_stats()
    rc = load().bisim_reduce_host(n, m, num_act, src_h or None, act_h or None, dst_h or None,
                                  init_h or None, out_h or None,
                                  ctypes.byref(opts) if opts is not None else None, stream or None,
                                  ctypes.byref(st))
    _check(rc, "bisim_reduce_host")
    return st


def bisim_version() -> int:
    return int(load().bisim_version())


def bisim_barrier_cost(ctas: int, threads: int, iters: int, stream: int = 0) -> float:
    """Average device time of one grid-wide barrier, in nanoseconds."""
    f = load().bisim_barrier_cost
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    ns = ctypes.c_double(0)
    _check(f(ctas, threads, iters, stream or None, ctypes.byref(ns)), "bisim_barrier_cost")
    return float(ns.value)


# --------------------------------------------------- torch conveniences


def _stream_ptr(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A plan over device tensors (int32, contiguous, on the current device)."""

    def __init__(self, n, num_act, src, act, dst, init=None, opts=None, stream=None):
        import torch

        for t in (src, act, dst, init):
            if t is not None:
                assert t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()
        self.n = int(n)
        self.m = int(src.shape[0])
        self.num_act = int(num_act)
        self.opts = opts if opts is not None else make_opts()
        self.stream = stream
        self._keep = (src, act, dst, init)
        self.handle = bisim_plan(self.n, self.m, self.num_act, src.data_ptr(),
                                 act.data_ptr() if act is not None else None, dst.data_ptr(),
                                 init.data_ptr() if init is not None else None, self.opts,
                                 _stream_ptr(stream))
        self._keep = None  # inputs are only read during planning

    def refine(self, out=None):
        import torch

        if out is None:
            out = torch.empty(max(self.n, 1), dtype=torch.int32, device="cuda")
        st = bisim_refine(self.handle, out.data_ptr())
        return out[: self.n], st

    def close(self):
        bisim_plan_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.handle:
                self.close()
        except Exception:
            pass


def reduce(lts, opts=None, device="cuda", return_stats=False, stream=None):
    """Coarsest bisimulation partition of an `lts_gen.LTS` on the GPU;
    returns a numpy int32 array of canonical block ids."""
    import torch

    def dev(a):
        return None if a is None else torch.from_numpy(a).to(device)

    src, act, dst, init = dev(lts.src), dev(lts.act), dev(lts.dst), dev(lts.init)
    with Plan(lts.n, lts.num_act, src, act, dst, init, opts, stream=stream) as p:
        out, st = p.refine()
        res = out.cpu().numpy()
    return (res, st) if return_stats else res


PHASE_NAMES = ("select", "publish", "claim", "barrier_claim", "mark", "barrier_mark", "split",
               "barrier_split", "single_rounds_ns", "multi_rounds", "single_rounds", "cta0_rounds",
               "splitters", "splitter_states", "touched_blocks", "between_rounds")


def bisim_phase_reset():
    f = load().bisim_phase_reset
    f.argtypes = []
    f.restype = ctypes.c_int
    _check(f(), "bisim_phase_reset")


def bisim_phase_times() -> dict:
    """Accumulated phase slots of a phase-timer build (see include/bisim.h)."""
    f = load().bisim_phase_times
    f.argtypes = [ctypes.c_void_p]
    f.restype = ctypes.c_int
    buf = (ctypes.c_uint64 * 16)()
    _check(f(ctypes.addressof(buf)), "bisim_phase_times")
    return {k: int(v) for k, v in zip(PHASE_NAMES, buf)}


def bisim_pool_usage() -> dict:
    """Bytes of the device's default memory pool: in use, most in use since
    the last reset, reserved from the device."""
    f = load().bisim_pool_usage
    U = ctypes.POINTER(ctypes.c_uint64)
    f.argtypes = [U, U, U]
    f.restype = ctypes.c_int
    u, h, r = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(f(ctypes.byref(u), ctypes.byref(h), ctypes.byref(r)), "bisim_pool_usage")
    return {"used": int(u.value), "used_high": int(h.value), "reserved": int(r.value)}


def bisim_pool_reset_high() -> None:
    f = load().bisim_pool_reset_high
    f.argtypes = []
    f.restype = ctypes.c_int
    _check(f(), "bisim_pool_reset_high")


def bisim_pool_trim(keep_bytes: int = 0) -> None:
    """Return the pool's unused memory to the device (keeping keep_bytes)."""
    f = load().bisim_pool_trim
    f.argtypes = [ctypes.c_uint64]
    f.restype = ctypes.c_int
    _check(f(int(keep_bytes)), "bisim_pool_trim")


def bisim_plan_arrays(handle: int, n: int, m: int) -> dict:
    """The plan's mark-slot layout and incoming-transition index on the host."""
    import numpy as np

    f = load().bisim_plan_arrays
    P = ctypes.c_void_p
    f.argtypes = [P, P, P, P, P, P, ctypes.POINTER(ctypes.c_int64)]
    f.restype = ctypes.c_int
    L = ctypes.c_int64(0)
    _check(f(handle, None, None, None, None, None, ctypes.byref(L)), "bisim_plan_arrays")
    off = np.zeros(n + 1, np.int32)
    in_ptr = np.zeros(n + 1, np.int32)
    ss = np.zeros(max(L.value, 1), np.int32)
    sa = np.zeros(max(L.value, 1), np.int32)
    ie = np.zeros(max(m, 1), np.int64)
    ptr = lambda a: a.ctypes.data_as(P)  # noqa: E731
    _check(f(handle, ptr(off), ptr(ss), ptr(sa), ptr(in_ptr), ptr(ie), ctypes.byref(L)), "bisim_plan_arrays")
    return {"off": off, "slot_src": ss[:L.value], "slot_act": sa[:L.value], "in_ptr": in_ptr, "in_edge": ie[:m],
            "mark_length": int(L.value)}


def bisim_phase_trace(max_rounds: int = 1 << 16):
    """Per-round trace of a phase-timer build: a list of (selected, worklist,
    touched, carried out, ns, on CTA 0 alone) per recorded round."""
    f = load().bisim_phase_trace
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    f.restype = ctypes.c_int
    buf = (ctypes.c_uint32 * (6 * max_rounds))()
    _check(f(ctypes.addressof(buf), max_rounds), "bisim_phase_trace")
    v = list(buf)
    return [tuple(v[6 * i:6 * i + 6]) for i in range(max_rounds)]


def bisim_canonical_ids_noalloc(labels: int, n: int, out_ids: int, stream: int = 0) -> int:
    """Allocation-free canonical renumbering (device addresses in); returns
    the number of blocks. For callers that cannot allocate device memory: its
    scratch is a fixed array of the library, so n is limited to
    BISIM_NOALLOC_MAX_N and overlapping calls must be serialised."""
    f = load().bisim_canonical_ids_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    nb = ctypes.c_int32(0)
    rc = f(labels or None, n, out_ids or None, ctypes.byref(nb), stream or None)
    if rc != BISIM_OK:
        raise BisimError(rc, "bisim_canonical_ids_noalloc")
    return int(nb.value)


BISIM_NOALLOC_MAX_N = 1 << 20


class bisim_batch_inst(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("num_blocks", ctypes.c_int64)]


def bisim_batch_plan(k: int, state_off_h, trans_off_h, num_act_h, src: int, act: Optional[int], dst: int,
                     init_block: Optional[int], opts: Optional[bisim_opts] = None, stream: int = 0) -> int:
    """Batch plan (host offset arrays as numpy int64/int32, device addresses
    for the concatenated local arrays); returns the plan handle."""
    import numpy as np

    f = load().bisim_batch_plan
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, P, P, P, P, P, P, P, ctypes.POINTER(bisim_opts), P, ctypes.POINTER(P)]
    f.restype = ctypes.c_int
    so = np.ascontiguousarray(state_off_h, dtype=np.int64)
    to = np.ascontiguousarray(trans_off_h, dtype=np.int64)
    na = np.ascontiguousarray(num_act_h, dtype=np.int32)
    out = ctypes.c_void_p()
    rc = f(k, so.ctypes.data, to.ctypes.data, na.ctypes.data, src or None, act or None, dst or None,
           init_block or None, ctypes.byref(opts) if opts is not None else None, stream or None,
           ctypes.byref(out))
    _check(rc, "bisim_batch_plan")
    return out.value


def bisim_batch_refine(plan: int, out_block: int, k: int):
    """Returns (aggregate bisim_stats, array of k bisim_batch_inst)."""
    f = load().bisim_batch_refine
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(bisim_stats),
                  ctypes.POINTER(bisim_batch_inst)]
    f.restype = ctypes.c_int
    st = bisim_stats()
    inst = (bisim_batch_inst * k)()
    _check(f(plan, out_block or None, ctypes.byref(st), inst), "bisim_batch_refine")
    return st, inst


def pack_batch(ltss):
    """Concatenate LTSs (local ids) into the arrays bisim_batch_plan takes."""
    import numpy as np

    so = np.zeros(len(ltss) + 1, dtype=np.int64)
    to = np.zeros(len(ltss) + 1, dtype=np.int64)
    for i, l in enumerate(ltss):
        so[i + 1] = so[i] + l.n
        to[i + 1] = to[i] + l.m
    na = np.array([l.num_act for l in ltss], dtype=np.int32)
    cat = lambda xs: np.ascontiguousarray(np.concatenate(xs) if xs else np.zeros(0), dtype=np.int32)  # noqa
    src = cat([l.src for l in ltss])
    act = cat([l.act for l in ltss])
    dst = cat([l.dst for l in ltss])
    init = None
    if any(l.init is not None for l in ltss):
        init = cat([l.init if l.init is not None else np.zeros(l.n, np.int32) for l in ltss])
    return so, to, na, src, act, dst, init


def reduce_batch(ltss, opts=None, device="cuda", stream=None, return_stats=False):
    """Coarsest bisimulation partitions of many LTSs in one batched plan and
    one refinement launch; returns a list of numpy arrays (canonical ids)."""
    import torch

    so, to, na, src, act, dst, init = pack_batch(ltss)
    d = lambda a: None if a is None else torch.from_numpy(a).to(device)  # noqa: E731
    tsrc, tact, tdst, tinit = d(src), d(act), d(dst), d(init)
    N = int(so[-1])
    out = torch.empty(max(N, 1), dtype=torch.int32, device=device)
    sp = _stream_ptr(stream)
    h = bisim_batch_plan(len(ltss), so, to, na, tsrc.data_ptr() if tsrc.numel() else 0,
                         tact.data_ptr() if tact.numel() else 0, tdst.data_ptr() if tdst.numel() else 0,
                         tinit.data_ptr() if tinit is not None else None, opts, sp)
    try:
        st, inst = bisim_batch_refine(h, out.data_ptr(), len(ltss))
    finally:
        bisim_plan_destroy(h)
    res = out[:N].cpu().numpy()
    parts = [res[so[i]:so[i + 1]] for i in range(len(ltss))]
    return (parts, st, inst) if return_stats else parts
