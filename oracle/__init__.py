"""CPU oracle for strong-bisimulation partition refinement.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this package to check and time the CUDA path; the
library never imports it. It shares no code with the CUDA sources.

Two layers:

* `oracle.c` (compiled with gcc into `_build/liboracle.so`, loaded with
  ctypes): Kanellakis-Smolka refinement (Algorithm 1 with labels), the
  preprocessing arrays of Section 4.1.1 (Algorithm 4 and its scans), and a
  lock-step simulation of the PRAM program (Algorithms 2/3/5) under the
  priority write rule.
* `defs.py` (numpy / pure Python): the definitions themselves - stability,
  canonical numbering, the signature fixed point, the greatest-fixed-point
  bisimulation of Definition 1 and exhaustive search over partitions - used
  to pin the C functions on small inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .defs import (  # noqa: F401
    brute_gfp,
    canonical,
    coarsest_by_enumeration,
    is_stable,
    num_blocks,
    pullback,
    refines,
    sigfix,
)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_EROUNDS = -4


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into _build/liboracle.so (plain C, -O2)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.oracle_ks.argtypes = [i32, i64, i32, P, P, P, P, P, P]
            lib.oracle_plan.argtypes = [i32, i64, i32, P, P, P, P, P, P, P, P, P]
            lib.oracle_pram.argtypes = [i32, i64, i32, P, P, P, P, i32, i32, i64, P, P, P]
            lib.oracle_pram_step.argtypes = [i32, i64, i32, P, P, P, P, P, i32, i32, P, P]
            lib.oracle_pair.argtypes = [i32, i64, i32, P, P, P, P, i64, P, P]
            for f in (lib.oracle_ks, lib.oracle_plan, lib.oracle_pram, lib.oracle_pram_step, lib.oracle_pair):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


class OracleError(RuntimeError):
    pass


def ks(n, num_act, src, act, dst, init=None, return_stats=False):
    """Coarsest stable refinement of the initial partition (canonical ids)
    by Kanellakis-Smolka refinement (Algorithm 1, labels via pre_a)."""
    lib = _load()
    src, act, dst, init = _c32(src), _c32(act), _c32(dst), _c32(init)
    out = np.empty(max(n, 1), dtype=np.int32)
    st = np.zeros(3, dtype=np.int64)
    rc = lib.oracle_ks(n, src.shape[0], num_act, _ptr(src), _ptr(act), _ptr(dst), _ptr(init),
                       _ptr(out), _ptr(st))
    if rc:
        raise OracleError(f"oracle_ks failed: {rc}")
    out = out[:n]
    if return_stats:
        return out, {"pops": int(st[0]), "splits": int(st[1])}
    return out


def plan(n, num_act, src, act, dst):
    """Preprocessing arrays of Section 4.1.1 for the transitions sorted by
    (source, a): perm, action_switch, order (per sorted transition),
    nr_marks, off (per state), mark_length."""
    lib = _load()
    src, act, dst = _c32(src), _c32(act), _c32(dst)
    m = src.shape[0]
    perm = np.empty(max(m, 1), dtype=np.int64)
    sw = np.empty(max(m, 1), dtype=np.int32)
    order = np.empty(max(m, 1), dtype=np.int32)
    nr = np.empty(max(n, 1), dtype=np.int32)
    off = np.empty(max(n, 1), dtype=np.int64)
    L = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_plan(n, m, num_act, _ptr(src), _ptr(act), _ptr(dst), _ptr(perm), _ptr(sw),
                         _ptr(order), _ptr(nr), _ptr(off), _ptr(L))
    if rc:
        raise OracleError(f"oracle_plan failed: {rc}")
    return {"perm": perm[:m], "action_switch": sw[:m], "order": order[:m], "nr_marks": nr[:n],
            "off": off[:n], "mark_length": int(L[0])}


def pram(n, num_act, src, act, dst, init=None, alg2=False, skip_preprocess=False, round_cap=0):
    """Lock-step PRAM run under the priority rule. Returns (raw leader labels,
    rounds counting the final empty iteration, preprocessing rounds)."""
    lib = _load()
    src, act, dst, init = _c32(src), _c32(act), _c32(dst), _c32(init)
    out = np.empty(max(n, 1), dtype=np.int32)
    r = np.zeros(1, dtype=np.int64)
    pr = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_pram(n, src.shape[0], num_act, _ptr(src), _ptr(act), _ptr(dst), _ptr(init),
                         int(bool(alg2)), int(bool(skip_preprocess)), int(round_cap), _ptr(out),
                         _ptr(r), _ptr(pr))
    if rc:
        raise OracleError(f"oracle_pram failed: {rc}")
    return out[:n], int(r[0]), int(pr[0])


def pram_step(n, num_act, src, act, dst, block, unstable, C, alg2=False):
    """One main-loop iteration with splitter C from the given partition
    (leader labels) and unstable flags. Returns (block, unstable, marks)."""
    lib = _load()
    src, act, dst = _c32(src), _c32(act), _c32(dst)
    blk = np.array(block, dtype=np.int32)
    uns = np.array(unstable, dtype=np.int8)
    marks = np.zeros(max(src.shape[0], n, 1), dtype=np.int8)
    L = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_pram_step(n, src.shape[0], num_act, _ptr(src), _ptr(act), _ptr(dst),
                              _ptr(blk), _ptr(uns), int(C), int(bool(alg2)), _ptr(marks), _ptr(L))
    if rc:
        raise OracleError(f"oracle_pram_step failed: {rc}")
    nm = n if alg2 else int(L[0])
    return blk, uns.astype(bool), marks[:nm].astype(bool)


def pair(n, num_act, src, act, dst, init=None, round_cap=0):
    """(C, a)-pair splitters (Algorithm 2 one label at a time) under the
    priority rule. Returns (raw leader labels, iterations counting the final
    empty one)."""
    lib = _load()
    src, act, dst, init = _c32(src), _c32(act), _c32(dst), _c32(init)
    out = np.empty(max(n, 1), dtype=np.int32)
    r = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_pair(n, src.shape[0], num_act, _ptr(src), _ptr(act), _ptr(dst), _ptr(init),
                         int(round_cap), _ptr(out), _ptr(r))
    if rc:
        raise OracleError(f"oracle_pair failed: {rc}")
    return out[:n], int(r[0])


def ks_lts(lts, **kw):
    return ks(lts.n, lts.num_act, lts.src, lts.act, lts.dst, lts.init, **kw)


def _ks_job(job):
    return ks(*job)


def ks_many(ltss, processes=None):
    """oracle_ks on many LTSs, in a pool of worker processes started with
    'spawn' (safe in a process that has already initialised CUDA). Each job
    carries plain arrays, so the workers import only this package."""
    import multiprocessing as mp

    jobs = [(l.n, l.num_act, l.src, l.act, l.dst, l.init) for l in ltss]
    processes = processes or min(16, os.cpu_count() or 1)
    if processes <= 1 or len(jobs) < 2:
        return [_ks_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(processes) as pool:
        return pool.map(_ks_job, jobs, chunksize=max(1, len(jobs) // (8 * processes)))


def pram_lts(lts, **kw):
    return pram(lts.n, lts.num_act, lts.src, lts.act, lts.dst, lts.init, **kw)


def pair_lts(lts, **kw):
    return pair(lts.n, lts.num_act, lts.src, lts.act, lts.dst, lts.init, **kw)
