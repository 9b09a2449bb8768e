"""fbpt: fused breadth-first probabilistic traversals on one GB300 GPU.

Thin ctypes binding over libfbpt (include/fbpt.h): argument marshalling only.
Every step of sampling and seed selection runs in the library's CUDA kernels;
there is no CPU path.  If libfbpt.so has not been built, importing the
binding's entry points raises.

    import paper_2311_10201_gb300 as fbpt
    g = fbpt.Graph(n, row_ptr, col, thr)                 # in-edge CSR + thresholds
    rr = fbpt.sample(g, seed, first_id, S, words=8)      # RR sets, device CSR
    offsets, verts, starts, vcount = rr.to_host()
    seeds, gains = fbpt.select_seeds(rr, k)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfbpt.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fbpt.h")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EDEVICE = 0, -1, -2, -3, -4, -5, -6
SCHED = {"push": 0, "pull": 1, "heuristic": 2, "learned": 3, "filtered": 4}
LAUNCH = {"host": 0, "graph": 1, "persistent": 2}
COMPACTION = {"queue": 0, "scan": 1}

U64P = ctypes.POINTER(ctypes.c_uint64)
U32P = ctypes.POINTER(ctypes.c_uint32)


class Opts(ctypes.Structure):
    _fields_ = [("words", ctypes.c_uint32), ("slots", ctypes.c_uint32), ("schedule", ctypes.c_uint32),
                ("launch", ctypes.c_uint32), ("unfused", ctypes.c_uint32), ("refill", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("model", ctypes.c_uint32),
                ("policy", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("spin_limit", ctypes.c_uint64),
                ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_uint64),
                ("compaction", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("words", ctypes.c_uint32), ("slots", ctypes.c_uint32), ("refill", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("candidates", ctypes.c_uint32), ("schedule", ctypes.c_uint32),
                ("probe_samples", ctypes.c_uint64), ("probe_rate", ctypes.c_double),
                ("rr_per_sample", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["schedule"] = {v: k for k, v in SCHED.items()}.get(d["schedule"], d["schedule"])
        return d


class ImmResult(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_uint64), ("samples", ctypes.c_uint64), ("first_final_id", ctypes.c_uint64),
                ("lower_bound", ctypes.c_double),
                ("coverage", ctypes.c_double), ("lambda_prime", ctypes.c_double), ("lambda_star", ctypes.c_double),
                ("rounds", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class RRSetsC(ctypes.Structure):
    _fields_ = [("S", ctypes.c_uint64), ("total", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("offsets", ctypes.c_void_p), ("verts", ctypes.c_void_p), ("starts", ctypes.c_void_p),
                ("vcount", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("internal", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("levels", "batches", "push_levels", "pull_levels", "units_expanded", "edge_accesses",
                 "philox_calls", "colour_edge_visits", "rr_total", "overflow_reruns", "mask_words", "trace_rows",
                 "groups_expanded")] + \
               [("ms_total", ctypes.c_double), ("ms_expand", ctypes.c_double), ("ms_commit", ctypes.c_double),
                ("ms_sweep", ctypes.c_double), ("ms_expand_events", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TRACE_DTYPE = np.dtype([(k, np.uint64) for k in
                        ("level", "units", "groups", "colours", "pending", "active_lanes", "finished_lanes",
                         "started_lanes", "expand_ns", "commit_ns", "sweep_ns")] +
                       [("direction", np.uint32), ("frontier_lanes", np.uint32),
                        ("features", np.float32, (6,)), ("outputs", np.float32, (8,)),
                        ("compaction", np.uint32), ("reserved", np.uint32)])


class FbptError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfbpt status {code}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes); every function the header declares
_SIGS = {
    "fbpt_graph_create": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "fbpt_graph_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fbpt_graph_info": (ctypes.c_int, [ctypes.c_void_p, U32P, U64P, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "fbpt_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.POINTER(Opts), ctypes.POINTER(RRSetsC), ctypes.POINTER(Stats)]),
    "fbpt_sample_batched": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p), U64P, U64P, U64P,
                                           ctypes.POINTER(Opts), ctypes.POINTER(RRSetsC), ctypes.POINTER(Stats)]),
    "fbpt_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(Opts),
                                     ctypes.POINTER(Tuning)]),
    "fbpt_graph_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Tuning)]),
    "fbpt_graph_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Tuning)]),
    "fbpt_policy_width": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(Opts),
                                         U32P, ctypes.POINTER(ctypes.c_float)]),
    "fbpt_imm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                ctypes.c_uint64, ctypes.POINTER(Opts), U32P, U64P, ctypes.POINTER(ImmResult),
                                ctypes.POINTER(Stats)]),
    "fbpt_rrsets_copy_rows": (ctypes.c_int, [ctypes.POINTER(RRSetsC), ctypes.c_uint64, ctypes.c_uint64, U64P, U32P,
                                             ctypes.c_uint64]),
    "fbpt_rrsets_free": (ctypes.c_int, [ctypes.POINTER(RRSetsC)]),
    "fbpt_rrsets_copy_to_host": (ctypes.c_int, [ctypes.POINTER(RRSetsC), ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "fbpt_select_seeds": (ctypes.c_int, [ctypes.POINTER(RRSetsC), ctypes.c_uint32, U32P, U64P]),
    "fbpt_select_seeds_noalloc": (ctypes.c_int, [ctypes.POINTER(RRSetsC), ctypes.c_uint32, U32P, U64P]),
    "fbpt_edge_draws": (ctypes.c_int, [ctypes.c_uint64, U64P, U64P, ctypes.c_uint64, U32P]),
    "fbpt_start_vertices": (ctypes.c_int, [ctypes.c_uint64, U64P, ctypes.c_uint64, ctypes.c_uint32, U32P]),
    "fbpt_abi_sizes": (ctypes.c_int, [U64P, ctypes.c_int]),
    "fbpt_philox_rate": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_double)]),
    "fbpt_policy_param_count": (ctypes.c_int, []),
    "fbpt_policy_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "fbpt_policy_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fbpt_policy_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_float)]),
    "fbpt_policy_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_uint64, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "fbpt_policy_adam_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p]),
    "fbpt_policy_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_uint64]),
    "fbpt_policy_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "fbpt_policy_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    "fbpt_order_compute": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, U64P, U32P, ctypes.c_uint32,
                                          ctypes.c_uint64, U32P]),
    "fbpt_graph_set_order": (ctypes.c_int, [ctypes.c_void_p, U32P, ctypes.c_uint32]),
    "fbpt_graph_get_order": (ctypes.c_int, [ctypes.c_void_p, U32P, U32P]),
    "fbpt_last_error": (ctypes.c_char_p, []),
    "fbpt_version": (ctypes.c_int, []),
}


def lib():
    """The loaded libfbpt; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfbpt.so not built ({LIB_PATH}); run paper_2311_10201_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        sizes = (ctypes.c_uint64 * 6)()
        L.fbpt_abi_sizes(sizes, 6)
        want = [ctypes.sizeof(Opts), ctypes.sizeof(RRSetsC), ctypes.sizeof(Stats), ctypes.sizeof(Tuning),
                ctypes.sizeof(ImmResult), TRACE_DTYPE.itemsize]
        if list(sizes) != want:
            raise RuntimeError(f"libfbpt struct layout mismatch: library {list(sizes)} vs binding {want}")
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise FbptError(rc, lib().fbpt_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream")


def _ptr_u64(a):
    return a.ctypes.data_as(U64P)


def _ptr_u32(a):
    return a.ctypes.data_as(U32P)


class Graph:
    """Library-owned device copy of an in-edge CSR with per-edge thresholds.

    row_ptr/col/thr: numpy arrays (host) or torch CUDA tensors (device)."""

    def __init__(self, n, row_ptr, col, thr, stream=None):
        self.n = int(n)
        self._h = ctypes.c_void_p()
        dev = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
        if dev:
            args = (row_ptr.data_ptr(), col.data_ptr(), thr.data_ptr(), 1)
            m = int(col.numel())
        else:
            row_ptr = np.ascontiguousarray(row_ptr, np.uint64)
            col = np.ascontiguousarray(col, np.uint32)
            thr = np.ascontiguousarray(thr, np.uint32)
            args = (row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                    thr.ctypes.data if thr.size else None, 0)
            m = int(col.size)
        self.m = m
        self.stream = _stream_handle(stream)
        _check(lib().fbpt_graph_create(self.n, m, args[0], args[1], args[2], args[3], self.stream,
                                       ctypes.byref(self._h)))

    @classmethod
    def from_synth(cls, g, stream=None):
        return cls(g.n, g.row_ptr, g.col, g.thr, stream)

    def set_order(self, perm=None, sorted_starts=False):
        """Relabel the sampler's vertex state by perm (perm[v] = new label;
        None = identity); sorted_starts: samples take lanes by start vertex.
        Results are unchanged."""
        p = None
        if perm is not None:
            p = np.ascontiguousarray(perm, np.uint32)
            if p.size != self.n:
                raise ValueError("perm must have n entries")
            self._perm = p
        _check(lib().fbpt_graph_set_order(self._h, _ptr_u32(p) if p is not None else None, int(bool(sorted_starts))))

    def get_order(self):
        """(perm, sorted_starts) currently set on the graph."""
        p = np.zeros(self.n, np.uint32)
        ss = ctypes.c_uint32()
        _check(lib().fbpt_graph_get_order(self._h, _ptr_u32(p), ctypes.byref(ss)))
        return p, bool(ss.value)

    def close(self):
        if self._h:
            lib().fbpt_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RRSets:
    """RR sets in library-owned device memory (CSR over samples)."""

    def __init__(self, c: RRSetsC, stats: Stats):
        self.c = c
        self.stats = stats

    @property
    def S(self):
        return int(self.c.S)

    @property
    def total(self):
        return int(self.c.total)

    def to_host(self):
        S, total, n = self.S, self.total, int(self.c.n)
        off = np.empty(S + 1, np.uint64)
        verts = np.empty(max(total, 1), np.uint32)
        starts = np.empty(S, np.uint32)
        vcount = np.empty(n, np.uint32)
        _check(lib().fbpt_rrsets_copy_to_host(ctypes.byref(self.c), off.ctypes.data, verts.ctypes.data,
                                              starts.ctypes.data, vcount.ctypes.data))
        return off, verts[:total], starts, vcount

    def index_to_host(self):
        """(offsets[S+1], starts[S], vcount[n]) without the vertex array."""
        S, n = self.S, int(self.c.n)
        off = np.empty(S + 1, np.uint64)
        starts = np.empty(S, np.uint32)
        vcount = np.empty(n, np.uint32)
        _check(lib().fbpt_rrsets_copy_to_host(ctypes.byref(self.c), off.ctypes.data, None, starts.ctypes.data,
                                              vcount.ctypes.data))
        return off, starts, vcount

    def rows(self, first, count):
        """Host copy of rows first .. first+count-1 only (fbpt_rrsets_copy_rows):
        (offsets[count+1] relative to the whole set, their vertices)."""
        off = np.empty(count + 1, np.uint64)
        cp = lib().fbpt_rrsets_copy_rows
        # the first and the last offset size the vertex buffer
        _check(cp(ctypes.byref(self.c), first, 0, off[:1].ctypes.data_as(U64P), None, 0))
        _check(cp(ctypes.byref(self.c), first + count, 0, off[count:].ctypes.data_as(U64P), None, 0))
        n = int(off[count] - off[0])
        verts = np.empty(max(n, 1), np.uint32)
        _check(cp(ctypes.byref(self.c), first, count, off.ctypes.data_as(U64P), verts.ctypes.data_as(U32P),
                  verts.size))
        return off, verts[:n]

    def free(self):
        if self.c.offsets:
            lib().fbpt_rrsets_free(ctypes.byref(self.c))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


REFILL = {"lane": 0, "batch": 1}


MODEL = {"ic": 0, "lt": 1}


def make_opts(words=0, slots=0, schedule="push", launch="persistent", unfused=False, stream=None, policy=None,
              spin_limit=0, refill="lane", blocks=0, model="ic", compaction="queue"):
    o = Opts()
    o.compaction = COMPACTION[compaction] if isinstance(compaction, str) else int(compaction)
    o.blocks = int(blocks)
    o.model = MODEL[model] if isinstance(model, str) else int(model)
    o.refill = REFILL[refill] if isinstance(refill, str) else int(refill)
    o.spin_limit = int(spin_limit)
    o.words, o.slots = int(words), int(slots)
    o.schedule = SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    o.launch = LAUNCH[launch] if isinstance(launch, str) else int(launch)
    o.unfused = int(bool(unfused))
    if policy is None and o.schedule == SCHED["learned"]:
        policy = default_policy()
    o.policy = policy._h.value if isinstance(policy, Policy) else policy
    o.stream = stream
    return o


def sample(g: Graph, seed: int, first_id: int, S: int, stream=None, trace_cap: int = 0, **kw) -> RRSets:
    """RR sets of samples first_id .. first_id+S-1 (fbpt_sample).  With
    trace_cap > 0 the per-level trace is returned as rr.trace."""
    o = make_opts(stream=_stream_handle(stream) if stream is not None else g.stream, **kw)
    trace = None
    if trace_cap:
        trace = np.zeros(trace_cap, TRACE_DTYPE)
        o.trace = trace.ctypes.data
        o.trace_cap = trace_cap
    c = RRSetsC()
    st = Stats()
    _check(lib().fbpt_sample(g._h, seed, first_id, S, ctypes.byref(o), ctypes.byref(c), ctypes.byref(st)))
    rr = RRSets(c, st)
    rr.trace = trace[:st.trace_rows] if trace is not None else None
    return rr


def sample_batched(graphs, seeds, first_ids, Ss, stream=None, **kw):
    G = len(graphs)
    o = make_opts(stream=_stream_handle(stream) if stream is not None else graphs[0].stream, **kw)
    hs = (ctypes.c_void_p * G)(*[g._h.value for g in graphs])
    arr = lambda xs: np.ascontiguousarray(xs, np.uint64)
    sd, fi, ss = arr(seeds), arr(first_ids), arr(Ss)
    outs = (RRSetsC * G)()
    st = Stats()
    _check(lib().fbpt_sample_batched(G, hs, _ptr_u64(sd), _ptr_u64(fi), _ptr_u64(ss), ctypes.byref(o), outs,
                                     ctypes.byref(st)))
    res = []
    for i in range(G):
        c = RRSetsC()
        ctypes.pointer(c)[0] = outs[i]
        res.append(RRSets(c, st))
    return res, st


def autotune(g: Graph, seed: int, S: int, **kw) -> dict:
    """Measure launch shapes of g (fbpt_autotune) and store the best on it; kw
    gives the schedule (and policy) the probes run with."""
    o = make_opts(stream=g.stream, **kw)
    t = Tuning()
    _check(lib().fbpt_autotune(g._h, seed, S, ctypes.byref(o), ctypes.byref(t)))
    return t.as_dict()


def policy_width(g: Graph, seed: int, S: int, policy=None, stream=None, launch="graph"):
    """Row width (words) the policy network picks for g (fbpt_policy_width),
    and its three scores (predicted log2 ns per sample at 4, 16, 64 words)."""
    o = make_opts(schedule="learned", launch=launch, stream=_stream_handle(stream), policy=policy)
    words = ctypes.c_uint32(0)
    scores = (ctypes.c_float * 3)()
    _check(lib().fbpt_policy_width(g._h, seed, S, ctypes.byref(o), ctypes.byref(words), scores))
    return int(words.value), [float(x) for x in scores]


def set_tuning(g: Graph, words, slots, refill="lane", blocks=0, schedule="push"):
    """Store a launch shape on g (fbpt_graph_set_tuning), used by the batched
    call when words == 0."""
    t = Tuning()
    t.words, t.slots, t.blocks = int(words), int(slots), int(blocks)
    t.refill = REFILL[refill] if isinstance(refill, str) else int(refill)
    t.schedule = SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    _check(lib().fbpt_graph_set_tuning(g._h, ctypes.byref(t)))


def tuning(g: Graph) -> dict:
    """The shape fbpt_autotune stored on g."""
    t = Tuning()
    _check(lib().fbpt_graph_tuning(g._h, ctypes.byref(t)))
    return t.as_dict()


def imm(g: Graph, k: int, epsilon: float, ell: float, seed: int, max_samples: int = 0, **kw):
    """IMM seed selection (fbpt_imm): (seeds[k], gains[k], result dict, Stats)."""
    o = make_opts(stream=g.stream, **kw)
    seeds = np.zeros(max(k, 1), np.uint32)
    gains = np.zeros(max(k, 1), np.uint64)
    res = ImmResult()
    st = Stats()
    _check(lib().fbpt_imm(g._h, k, float(epsilon), float(ell), seed, max_samples, ctypes.byref(o),
                          _ptr_u32(seeds), _ptr_u64(gains), ctypes.byref(res), ctypes.byref(st)))
    return seeds[:k], gains[:k], res.as_dict(), st


ORDER = {"identity": 0, "rcm": 1, "degree": 2, "random": 3, "cluster": 4}


def order_compute(n, row_ptr, col, method="rcm", seed=0):
    """Host-side vertex order of an in-edge CSR (numpy arrays): perm[v] = new
    label of v.  Needs no GPU."""
    rp = np.ascontiguousarray(row_ptr, np.uint64)
    c = np.ascontiguousarray(col, np.uint32)
    perm = np.zeros(int(n), np.uint32)
    meth = ORDER[method] if isinstance(method, str) else int(method)
    _check(lib().fbpt_order_compute(int(n), int(c.size), _ptr_u64(rp), _ptr_u32(c) if c.size else None, meth,
                                    int(seed), _ptr_u32(perm)))
    return perm


def select_seeds(rr: RRSets, k: int):
    """Greedy max-k-cover (fbpt_select_seeds): (seeds[k], newly covered rows per pick[k])."""
    seeds = np.zeros(max(k, 1), np.uint32)
    gains = np.zeros(max(k, 1), np.uint64)
    _check(lib().fbpt_select_seeds(ctypes.byref(rr.c), k, _ptr_u32(seeds), _ptr_u64(gains)))
    return seeds[:k], gains[:k]


def select_seeds_noalloc(rr: RRSets, k: int):
    """Greedy max-k-cover like select_seeds, but with the library's fixed
    device array as working memory (fbpt_select_seeds_noalloc): no device
    allocation, for callers that cannot allocate.  Calls must not overlap."""
    seeds = np.zeros(max(k, 1), np.uint32)
    gains = np.zeros(max(k, 1), np.uint64)
    _check(lib().fbpt_select_seeds_noalloc(ctypes.byref(rr.c), k, _ptr_u32(seeds), _ptr_u64(gains)))
    return seeds[:k], gains[:k]


class Policy:
    """Schedule-policy network parameters on the device (fbpt_policy)."""

    def __init__(self, params):
        params = np.ascontiguousarray(params, np.float32)
        self._h = ctypes.c_void_p()
        _check(lib().fbpt_policy_create(params.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), params.size,
                                        ctypes.byref(self._h)))

    def params(self):
        out = np.zeros(lib().fbpt_policy_param_count(), np.float32)
        _check(lib().fbpt_policy_get(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def save(self, path):
        """Write the parameters as text (fbpt_policy_save)."""
        _check(lib().fbpt_policy_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path):
        """A policy read from a text file (fbpt_policy_load)."""
        obj = cls.__new__(cls)
        obj._h = ctypes.c_void_p()
        _check(lib().fbpt_policy_load(os.fsencode(path), ctypes.byref(obj._h)))
        return obj

    def close(self):
        if self._h:
            lib().fbpt_policy_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


DEFAULT_POLICY_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy_default.txt")
_default_policy = None


def default_policy():
    """The network shipped with the package (trained by train_policy.py on
    per-level traces); the "learned" schedule uses it unless given another."""
    global _default_policy
    if _default_policy is None:
        _default_policy = Policy(np.loadtxt(DEFAULT_POLICY_FILE, dtype=np.float64).astype(np.float32))
    return _default_policy


class TrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p)]


def _train_arrays(features, actions, targets):
    X = np.ascontiguousarray(features, np.float32).reshape(-1, 6)
    A = np.ascontiguousarray(actions, np.uint32)
    Y = np.ascontiguousarray(targets, np.float32)
    if not (X.shape[0] == A.size == Y.size):
        raise ValueError("features, actions and targets must have the same rows")
    return X, A, Y


def policy_train(features, actions, targets, steps=2000, lr=3e-3, seed=0, init=None, stream=None):
    """Train the schedule network on the GPU (fbpt_policy_train); returns (Policy, loss)."""
    X, A, Y = _train_arrays(features, actions, targets)
    o = TrainOpts(steps, lr, seed, _stream_handle(stream))
    h = ctypes.c_void_p()
    loss = ctypes.c_float()
    init_arr = None if init is None else np.ascontiguousarray(init, np.float32)
    _check(lib().fbpt_policy_train(X.ctypes.data, A.ctypes.data, Y.ctypes.data, X.shape[0], ctypes.addressof(o),
                                   init_arr.ctypes.data if init_arr is not None else None, ctypes.byref(h),
                                   ctypes.byref(loss)))
    p = Policy.__new__(Policy)
    p._h = h
    return p, float(loss.value)


def policy_loss_grad(params, features, actions, targets, stream=None):
    """(loss, gradient) of the parameters on the rows, from the GPU kernel."""
    X, A, Y = _train_arrays(features, actions, targets)
    P = np.ascontiguousarray(params, np.float32)
    g = np.zeros(P.size, np.float32)
    loss = ctypes.c_float()
    _check(lib().fbpt_policy_loss_grad(P.ctypes.data, X.ctypes.data, A.ctypes.data, Y.ctypes.data, X.shape[0],
                                       ctypes.byref(loss), g.ctypes.data, _stream_handle(stream)))
    return float(loss.value), g


def policy_adam_step(params, grad, m, v, t, lr, stream=None):
    """One Adam update by the library's training kernel (fbpt_policy_adam_step);
    returns the new (params, m, v) as float32 arrays."""
    P = np.array(params, np.float32)
    G = np.ascontiguousarray(grad, np.float32)
    M = np.array(m, np.float32)
    V = np.array(v, np.float32)
    if not (P.size == G.size == M.size == V.size == lib().fbpt_policy_param_count()):
        raise ValueError("params, grad, m and v must each hold fbpt_policy_param_count() floats")
    _check(lib().fbpt_policy_adam_step(P.ctypes.data, G.ctypes.data, M.ctypes.data, V.ctypes.data, t, lr,
                                       _stream_handle(stream)))
    return P, M, V


def edge_draws(seed: int, s, e):
    s = np.ascontiguousarray(s, np.uint64)
    e = np.ascontiguousarray(e, np.uint64)
    out = np.zeros(max(s.size, 1), np.uint32)
    _check(lib().fbpt_edge_draws(seed, _ptr_u64(s), _ptr_u64(e), s.size, _ptr_u32(out)))
    return out[:s.size]


def philox_rate(seed: int = 1, calls_per_thread: int = 4096, stream=None) -> float:
    """Philox4x32-10 evaluations per second of a draw-only kernel (fbpt_philox_rate)."""
    out = ctypes.c_double(0.0)
    _check(lib().fbpt_philox_rate(seed, calls_per_thread, _stream_handle(stream), ctypes.byref(out)))
    return out.value


def start_vertices(seed: int, s, n: int):
    s = np.ascontiguousarray(s, np.uint64)
    out = np.zeros(max(s.size, 1), np.uint32)
    _check(lib().fbpt_start_vertices(seed, _ptr_u64(s), s.size, n, _ptr_u32(out)))
    return out[:s.size]


def build(force: bool = False):
    from . import builder
    return builder.build(force=force)
