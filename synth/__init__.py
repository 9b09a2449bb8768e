"""Seeded synthetic inputs for the fused-BPT sampler: graphs, edge thresholds and
the five workload recipes.

This module is shared by the tests, the oracle's test inputs and the benchmark.
It contains none of the sampling method's arithmetic (no Philox, no liveness
test, no traversal): it only builds in-edge CSR graphs and the per-edge
threshold arrays that both the CUDA library and the oracle take as inputs.

The paper evaluates on SNAP social and web graphs (Table 1: 0.69M-4.8M
vertices, 5.1M-117M edges, average degree 11.7-76.3) that are not available
here; seeded R-MAT graphs of scale 20-24 with edge factor 16 stand in for them.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lib = None

U64P = ctypes.POINTER(ctypes.c_uint64)
U32P = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile gen.c into _synth.so (OpenMP when the compiler has it)."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", src, "-o", _SO]
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
        lib.synth_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, U64P, U32P]
        lib.synth_er.restype = ctypes.c_int
        lib.synth_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_int, U64P, U32P]
        lib.synth_rmat.restype = ctypes.c_uint64
        lib.synth_thr_uniform.argtypes = [ctypes.c_uint64, ctypes.c_double, U32P]
        lib.synth_thr_wc.argtypes = [ctypes.c_uint32, U64P, U32P]
        lib.synth_thr_choice.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), ctypes.c_uint32,
                                         ctypes.c_uint64, U32P]
        lib.synth_thr_of.argtypes = [ctypes.c_double]
        lib.synth_thr_of.restype = ctypes.c_uint32
        lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_draw.restype = ctypes.c_uint64
        lib.synth_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


@dataclass
class Graph:
    """In-edge CSR: row v lists the sources w of edges w -> v (ascending).
    Edge id e is the index into col/thr; thr[e] = floor(p(e) * 2^32), with
    0xFFFFFFFF meaning p = 1."""
    n: int
    row_ptr: np.ndarray  # uint64[n+1]
    col: np.ndarray      # uint32[m]
    thr: np.ndarray      # uint32[m]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def indeg(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def threshold(p: float) -> int:
    """floor(p * 2^32) clamped, with the always-live marker for p = 1."""
    return int(_load().synth_thr_of(float(p)))


def draw(seed: int, stream: int, i: int) -> int:
    return int(_load().synth_draw(seed, stream, i))


def er_graph(n: int, m: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    row_ptr = np.zeros(n + 1, np.uint64)
    col = np.zeros(m, np.uint32)
    rc = lib.synth_er(n, m, seed, _p(row_ptr, ctypes.c_uint64), _p(col, ctypes.c_uint32))
    if rc != 0:
        raise ValueError(f"synth_er failed ({rc})")
    return row_ptr, col


def rmat_graph(scale: int, ef: int, seed: int, a=0.57, b=0.19, c=0.19, permute=True):
    lib = _load()
    n = 1 << scale
    row_ptr = np.zeros(n + 1, np.uint64)
    col = np.zeros(ef * n, np.uint32)
    m = lib.synth_rmat(scale, ef, a, b, c, seed, int(permute), _p(row_ptr, ctypes.c_uint64),
                       _p(col, ctypes.c_uint32))
    if m == 2**64 - 1:
        raise ValueError("synth_rmat failed")
    return row_ptr, col[:m]


def thr_uniform(m: int, p: float) -> np.ndarray:
    thr = np.empty(m, np.uint32)
    _load().synth_thr_uniform(m, p, _p(thr, ctypes.c_uint32))
    return thr


def thr_wc(row_ptr: np.ndarray) -> np.ndarray:
    n = row_ptr.size - 1
    thr = np.empty(int(row_ptr[-1]), np.uint32)
    _load().synth_thr_wc(n, _p(row_ptr, ctypes.c_uint64), _p(thr, ctypes.c_uint32))
    return thr


def thr_choice(m: int, ps, seed: int) -> np.ndarray:
    thr = np.empty(m, np.uint32)
    arr = (ctypes.c_double * len(ps))(*ps)
    _load().synth_thr_choice(m, arr, len(ps), seed, _p(thr, ctypes.c_uint32))
    return thr


# ---------------------------------------------------------------------------
# Workload recipes (fixed seeds).  Each returns graphs plus sampling parameters.
# ---------------------------------------------------------------------------

GRAPH_SEED = 20231117
SAMPLE_SEED = 0x5EED_F00D_2311_1020


@dataclass
class Workload:
    name: str
    graphs: list
    S: list            # samples per graph
    seeds: list        # sampling seed per graph
    words: list        # candidate colour widths W
    k: int             # greedy budget (0 = none)


def er_1k() -> Workload:
    """Directed ER graph, 1,024 vertices, 8,192 edges, uniform p = 0.1,
    64 samples in one 64-colour word, greedy k = 4."""
    rp, col = er_graph(1024, 8192, GRAPH_SEED)
    g = Graph(1024, rp, col, thr_uniform(col.size, 0.1), "er-1k-8k-p0.1")
    return Workload("er_1k", [g], [64], [SAMPLE_SEED], [1], 4)


def rmat_wc(scale: int, ef: int = 16, seed: int = GRAPH_SEED) -> Graph:
    rp, col = rmat_graph(scale, ef, seed + scale)
    return Graph(1 << scale, rp, col, thr_wc(rp), f"rmat-s{scale}-ef{ef}-wc")


def rmat_s20_wc() -> Workload:
    """R-MAT scale 20, edge factor 16, weighted cascade, 65,536 samples,
    W in {1, 2, 4, 8}, fused and unfused."""
    return Workload("rmat_s20_wc", [rmat_wc(20)], [65536], [SAMPLE_SEED], [1, 2, 4, 8], 0)


def batched_32(max_scale: int = 20, count: int = 32) -> Workload:
    """32 independent R-MAT graphs: scale uniform in [12, max_scale], edge
    factor uniform in [8, 32], uniform p drawn per graph from [0.01, 0.1],
    samples per graph log-uniform in [4,096, 262,144]."""
    gs, Ss, seeds = [], [], []
    base = GRAPH_SEED ^ 0x3333
    for g in range(count):
        r = [draw(base, 21, 4 * g + j) for j in range(4)]
        scale = 12 + r[0] % (max_scale - 12 + 1)
        ef = 8 + r[1] % 25
        p = 0.01 + 0.09 * ((r[2] >> 11) / float(1 << 53))
        lo, hi = math.log(4096), math.log(262144)
        S = int(round(math.exp(lo + (hi - lo) * ((r[3] >> 11) / float(1 << 53)))))
        rp, col = rmat_graph(scale, ef, base + 97 * g)
        gs.append(Graph(1 << scale, rp, col, thr_uniform(col.size, p), f"rmat-s{scale}-ef{ef}-p{p:.4f}",
                        {"scale": scale, "ef": ef, "p": p}))
        Ss.append(S)
        seeds.append(SAMPLE_SEED + g)
    return Workload("batched_32", gs, Ss, seeds, [1, 2, 4, 8], 0)


def rmat_s22_wc() -> Workload:
    """R-MAT scale 22, edge factor 16, weighted cascade, 1,048,576 samples, k = 100."""
    return Workload("rmat_s22_wc", [rmat_wc(22)], [1 << 20], [SAMPLE_SEED], [1, 2, 4, 8], 100)


def rmat_s24_tri() -> Workload:
    """R-MAT scale 24, edge factor 16, trivalency p in {0.1, 0.01, 0.001} per
    edge, 4,194,304 samples, k = 200."""
    rp, col = rmat_graph(24, 16, GRAPH_SEED + 24)
    g = Graph(1 << 24, rp, col, thr_choice(col.size, [0.1, 0.01, 0.001], GRAPH_SEED ^ 0x24),
              "rmat-s24-ef16-tri")
    return Workload("rmat_s24_tri", [g], [1 << 22], [SAMPLE_SEED], [1, 2, 4, 8], 200)


WORKLOADS = {
    "er_1k": er_1k,
    "rmat_s20_wc": rmat_s20_wc,
    "batched_32": batched_32,
    "rmat_s22_wc": rmat_s22_wc,
    "rmat_s24_tri": rmat_s24_tri,
}
