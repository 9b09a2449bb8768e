"""CPU oracle for the fused-BPT sampler (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library
(``paper_2311_10201_gb300``) and never imports it; the only module both sides
use is ``synth`` (seeded graphs and thresholds, none of the method's
arithmetic).

Functions (each cites the passage it follows in ``oracle.c`` / ``mlp.py``):
  philox, edge_draw, live, start          Philox4x32-10 and the liveness rule
  rr_sets                                 Definition 2, one BFS per sample
  rr_sets_fused                           Listing 1 (Section 3), colour masks
  greedy                                  max-k-cover greedy (Section 2)
  mlp (module)                            schedule-policy network, FP64
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None

U64P = ctypes.POINTER(ctypes.c_uint64)
U32P = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", _SO]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_philox.argtypes = [U32P, U32P, U32P]
        lib.oracle_edge_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_edge_draw.restype = ctypes.c_uint32
        lib.oracle_live.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.oracle_live.restype = ctypes.c_int
        lib.oracle_start.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.oracle_start.restype = ctypes.c_uint32
        lib.oracle_rr.argtypes = [ctypes.c_uint32, U64P, U32P, U32P, ctypes.c_uint64, ctypes.c_uint64, U64P,
                                  ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(U64P), ctypes.POINTER(U32P), U32P]
        lib.oracle_rr.restype = ctypes.c_int
        lib.oracle_rr_lt.argtypes = lib.oracle_rr.argtypes
        lib.oracle_rr_lt.restype = ctypes.c_int
        lib.oracle_vertex_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.oracle_vertex_draw.restype = ctypes.c_uint32
        lib.oracle_lt_choice.argtypes = [U64P, U32P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.oracle_lt_choice.restype = ctypes.c_int64
        lib.oracle_rr_fused.argtypes = [ctypes.c_uint32, U64P, U32P, U32P, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(U64P),
                                        ctypes.POINTER(U32P), U64P]
        lib.oracle_rr_fused.restype = ctypes.c_int
        lib.oracle_greedy.argtypes = [ctypes.c_uint32, ctypes.c_uint64, U64P, U32P, ctypes.c_uint32, U32P, U64P]
        lib.oracle_greedy.restype = ctypes.c_int
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def threads() -> int:
    return int(_load().oracle_threads())


def philox(ctr, key) -> list[int]:
    """Philox4x32-10 of a 4-word counter under a 2-word key."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _load().oracle_philox(c, k, o)
    return list(o)


def edge_draw(seed: int, s: int, e: int) -> int:
    return int(_load().oracle_edge_draw(seed, s, e))


def live(seed: int, s: int, e: int, thr: int) -> bool:
    return bool(_load().oracle_live(seed, s, e, thr))


def start(seed: int, s: int, n: int) -> int:
    return int(_load().oracle_start(seed, s, n))


class RRSets:
    """RR sets as CSR: row j (sample id first_id + j, or ids[j]) is
    verts[offsets[j]:offsets[j+1]], ascending."""

    def __init__(self, offsets, verts, starts=None):
        self.offsets = offsets
        self.verts = verts
        self.starts = starts

    def __len__(self):
        return self.offsets.size - 1

    def row(self, j):
        return self.verts[self.offsets[j]:self.offsets[j + 1]]


def _take(offp, vertp, count):
    lib = _load()
    off = np.ctypeslib.as_array(offp, shape=(count + 1,)).copy()
    total = int(off[-1])
    verts = np.ctypeslib.as_array(vertp, shape=(max(total, 1),))[:total].copy()
    lib.oracle_free(ctypes.cast(offp, ctypes.c_void_p))
    lib.oracle_free(ctypes.cast(vertp, ctypes.c_void_p))
    return off, verts


def rr_sets(g, seed: int, first_id: int = 0, count: int | None = None, ids=None, nthreads: int = 0,
            model: str = "ic") -> RRSets:
    """Definition 2: one BFS per sample over in-edges with hashed liveness
    (model "ic"), or one reverse walk over the kept in-edges (model "lt")."""
    lib = _load()
    fn = {"ic": lib.oracle_rr, "lt": lib.oracle_rr_lt}[model]
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        count = ids.size
    offp, vertp = U64P(), U32P()
    starts = np.zeros(max(count, 1), np.uint32)
    rc = fn(g.n, _p(g.row_ptr, ctypes.c_uint64), _p(g.col, ctypes.c_uint32), _p(g.thr, ctypes.c_uint32),
            seed, first_id, _p(ids, ctypes.c_uint64) if ids is not None else None, count, nthreads,
            ctypes.byref(offp), ctypes.byref(vertp), _p(starts, ctypes.c_uint32))
    if rc != 0:
        raise MemoryError("oracle_rr failed")
    off, verts = _take(offp, vertp, count)
    return RRSets(off, verts, starts[:count])


def vertex_draw(seed: int, s: int, v: int) -> int:
    """The LT model's draw of vertex v for sample s."""
    return int(_load().oracle_vertex_draw(seed, s, v))


def lt_choice(g, seed: int, s: int, v: int) -> int:
    """The in-edge v keeps for sample s under LT, or -1."""
    return int(_load().oracle_lt_choice(_p(g.row_ptr, ctypes.c_uint64), _p(g.thr, ctypes.c_uint32), seed, s, v))


def rr_sets_fused(g, seed: int, first_id: int, count: int, W: int = 1):
    """Listing 1 with 64*W colours per group; returns (RRSets, edge_accesses)."""
    lib = _load()
    offp, vertp = U64P(), U32P()
    acc = ctypes.c_uint64()
    rc = lib.oracle_rr_fused(g.n, _p(g.row_ptr, ctypes.c_uint64), _p(g.col, ctypes.c_uint32),
                             _p(g.thr, ctypes.c_uint32), seed, first_id, count, W, ctypes.byref(offp),
                             ctypes.byref(vertp), ctypes.byref(acc))
    if rc != 0:
        raise MemoryError("oracle_rr_fused failed")
    off, verts = _take(offp, vertp, count)
    return RRSets(off, verts), int(acc.value)


def greedy(n: int, rr: RRSets, k: int):
    """Greedy max-k-cover; returns (seeds[k], newly covered per pick[k])."""
    lib = _load()
    seeds = np.zeros(max(k, 1), np.uint32)
    gains = np.zeros(max(k, 1), np.uint64)
    off = np.ascontiguousarray(rr.offsets, np.uint64)
    verts = np.ascontiguousarray(rr.verts, np.uint32)
    if verts.size == 0:
        verts = np.zeros(1, np.uint32)
    rc = lib.oracle_greedy(n, len(rr), _p(off, ctypes.c_uint64), _p(verts, ctypes.c_uint32), k,
                           _p(seeds, ctypes.c_uint32), _p(gains, ctypes.c_uint64))
    if rc == -1:
        raise ValueError("k > n")
    if rc != 0:
        raise MemoryError("oracle_greedy failed")
    return seeds[:k], gains[:k]
