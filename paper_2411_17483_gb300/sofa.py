"""Thin ctypes binding of the C ABI in include/sofa.h (argument marshalling only).

Every step of the search runs in libsofa.so's CUDA kernels; this module only
passes pointers, sizes and streams.  Tensors may live on the GPU or (for the
build and for host-buffer queries) on the host.  There is no CPU fallback:
if the library is missing, load() raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsofa.so")

SOFA_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "NOT_TRAINED", -6: "TIE_OVERFLOW", -7: "INTERNAL"}
MAX_K = 64
MAX_WORD = 32
MAX_WINDOW = 96

_lib = None


class SofaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sofa error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class BuildOpts(ctypes.Structure):
    _fields_ = [("sample_ratio", ctypes.c_float), ("binning", ctypes.c_int32), ("select", ctypes.c_int32),
                ("pool_coeffs", ctypes.c_int32), ("leaf_tiles", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("user_sel", ctypes.POINTER(ctypes.c_int32)), ("user_nsel", ctypes.c_int32),
                ("user_beta", ctypes.POINTER(ctypes.c_float))]


class TrainOpts(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_int64), ("n_classes", ctypes.c_int32), ("epochs", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("train_queries", ctypes.c_void_p), ("top_m", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("cand_cap", ctypes.c_int32), ("seed_count", ctypes.c_int32),
                ("seed_window", ctypes.c_int32), ("bound_precision", ctypes.c_int32), ("pool_cap", ctypes.c_int64),
                ("refine_filter", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("cand_budget", ctypes.c_int64),
                ("dense", ctypes.c_int32), ("approximate", ctypes.c_int32), ("series_bound", ctypes.c_int32),
                ("tile_checks", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("queries", "leaf_pairs", "tile_pairs", "candidates", "refined", "overflow_passes",
                 "n_leaves", "n_tiles", "filtered", "graph_replays", "graphs_recorded")] + [
                    ("seed_dist_sum", ctypes.c_double),
                                                        ("final_dist_sum", ctypes.c_double),
                                                        ("value_filtered", ctypes.c_int64),
                                                        ("dense_pairs", ctypes.c_int64),
                                                        ("dense_passes", ctypes.c_int64)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8),
                ("scan_tile_loads", ctypes.c_int64), ("scan_tile_checks", ctypes.c_int64)]


PHASES = ("qprep", "seed", "route", "scan", "refine", "final", "proposal", "pool")


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("n", ctypes.c_int32), ("l", ctypes.c_int32),
                ("alphabet", ctypes.c_int32), ("nsel", ctypes.c_int32), ("word_bytes", ctypes.c_int32),
                ("nyquist_first", ctypes.c_int32), ("leaf_tiles", ctypes.c_int32),
                ("n_leaves", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("delta_data", ctypes.c_double), ("delta_query", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("proposal_classes", ctypes.c_int64),
                ("proposal_train", ctypes.c_int64), ("proposal_loss", ctypes.c_double),
                ("proposal_top1", ctypes.c_double), ("proposal_topm", ctypes.c_double),
                ("appended", ctypes.c_int64)]


def load():
    """Load libsofa.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sig = {
        "sofa_build": (P, [P, i64, i32, i32, i32]),
        "sofa_build_ex": (P, [P, i64, i32, i32, i32, ctypes.POINTER(BuildOpts), P]),
        "sofa_insert": (ctypes.c_int, [P, P, i64, P]),
        "sofa_query": (ctypes.c_int, [P, P, i64, i32, P, P, P]),
        "sofa_query_multi": (ctypes.c_int, [P, i32, P, P, P, P, i64, P, P, P, P]),
        "sofa_query_window": (ctypes.c_int, [P, P, i64, i32, i32, P, P, P, P]),
        "sofa_train_proposal": (ctypes.c_int, [P, ctypes.POINTER(TrainOpts), P]),
        "sofa_set_seed_mode": (ctypes.c_int, [P, i32]),
        "sofa_mlp_grad": (ctypes.c_int, [i32, i32, i32, P, P, P, i32, P, ctypes.POINTER(ctypes.c_float), P]),
        "sofa_set_tuning": (ctypes.c_int, [P, ctypes.POINTER(Tuning)]),
        "sofa_autotune": (ctypes.c_int, [P, P, i64, i32, ctypes.c_char_p, ctypes.POINTER(Tuning), P]),
        "sofa_query_status": (ctypes.c_int, [P]),
        "sofa_stats": (ctypes.c_int, [P, ctypes.POINTER(Stats), i32]),
        "sofa_info": (ctypes.c_int, [P, ctypes.POINTER(Info)]),
        "sofa_set_profiling": (ctypes.c_int, [P, i32]),
        "sofa_profile": (ctypes.c_int, [P, ctypes.POINTER(Profile), i32]),
        "sofa_export_summary": (ctypes.c_int, [P, P, P, P]),
        "sofa_export_words": (ctypes.c_int, [P, P]),
        "sofa_export_perm": (ctypes.c_int, [P, P]),
        "sofa_lower_bounds": (ctypes.c_int, [P, P, i64, P, P]),
        "sofa_lower_bounds_noalloc": (ctypes.c_int, [P, P, i64, P, P]),
        "sofa_dense_sqdist": (ctypes.c_int, [P, P, i64, P, ctypes.POINTER(ctypes.c_float), P]),
        "sofa_value_bounds": (ctypes.c_int, [P, P, i64, P, ctypes.POINTER(ctypes.c_float), P]),
        "sofa_wait_selftest": (ctypes.c_int, [i32, P]),
        "sofa_save": (ctypes.c_int, [P, ctypes.c_char_p]),
        "sofa_load": (P, [ctypes.c_char_p, P]),
        "sofa_znorm": (ctypes.c_int, [P, i64, i32, P, P]),
        "sofa_free": (None, [P]),
        "sofa_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != SOFA_OK:
        raise SofaError(rc, load().sofa_last_error().decode())


def _stream(stream=None):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


class Index:
    """An SFA index over N series of length n (sofa_build_ex)."""

    def __init__(self, data: torch.Tensor, l: int = 16, alphabet: int = 256, *, sample_ratio: float = 0.1,
                 binning: str = "equi-depth", select: str = "variance", pool_coeffs: int = 0,
                 leaf_tiles: int = 0, precision: int = 0, user_sel=None, user_beta=None, stream=None):
        lib = load()
        if data.dtype != torch.float32 or data.dim() != 2:
            raise ValueError("data must be a 2-d float32 tensor")
        data = data.contiguous()
        o = BuildOpts()
        o.sample_ratio = sample_ratio
        o.binning = {"equi-depth": 0, "equi-width": 1}[binning]
        o.select = {"variance": 0, "first": 1}[select]
        o.pool_coeffs = pool_coeffs
        o.leaf_tiles = leaf_tiles
        o.precision = precision
        keep = []
        if user_sel is not None:
            us = torch.as_tensor(user_sel, dtype=torch.int32).contiguous()
            ub = torch.as_tensor(user_beta, dtype=torch.float32).contiguous()
            keep += [us, ub]
            o.user_sel = ctypes.cast(us.data_ptr(), ctypes.POINTER(ctypes.c_int32))
            o.user_nsel = us.numel()
            o.user_beta = ctypes.cast(ub.data_ptr(), ctypes.POINTER(ctypes.c_float))
        st = _stream(stream) if data.is_cuda else ctypes.c_void_p(0)
        h = lib.sofa_build_ex(_ptr(data), data.shape[0], data.shape[1], l, alphabet, ctypes.byref(o), st)
        if not h:
            raise SofaError(-1, lib.sofa_last_error().decode())
        self.h = ctypes.c_void_p(h)
        self.N, self.n, self.l, self.alphabet = data.shape[0], data.shape[1], l, alphabet

    def insert(self, data: torch.Tensor, stream=None):
        """sofa_insert: add the rows of data (N_add x n fp32, host or device);
        they get the row ids N, N+1, ... in order."""
        if data.dtype != torch.float32 or data.dim() != 2 or data.shape[1] != self.n:
            raise ValueError("data must be a 2-d float32 tensor with the index's series length")
        data = data.contiguous()
        st = _stream(stream) if data.is_cuda else ctypes.c_void_p(0)
        _check(load().sofa_insert(self.h, _ptr(data), data.shape[0], st))
        self.N += data.shape[0]

    def save(self, path: str):
        """sofa_save: every array of the index (and a trained proposal network) to one file."""
        _check(load().sofa_save(self.h, str(path).encode()))

    @classmethod
    def load(cls, path: str, stream=None) -> "Index":
        """sofa_load: an index recreated on the current device from a file of sofa_save."""
        lib = load()
        h = lib.sofa_load(str(path).encode(), _stream(stream))
        if not h:
            raise SofaError(-1, lib.sofa_last_error().decode())
        ix = cls.__new__(cls)
        ix.h = ctypes.c_void_p(h)
        inf = ix.info()
        ix.N, ix.n, ix.l, ix.alphabet = inf["N"], inf["n"], inf["l"], inf["alphabet"]
        return ix

    def close(self):
        if getattr(self, "h", None):
            load().sofa_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, q: torch.Tensor, k: int = 1, idx: torch.Tensor | None = None,
              dist: torch.Tensor | None = None, stream=None):
        """Exact k-NN of the rows of q; returns (idx int64 [Q,k], dist fp32 [Q,k])."""
        q = q.contiguous()
        Q = q.shape[0]
        dev = q.device
        if idx is None:
            idx = torch.empty((Q, k), dtype=torch.int64, device=dev)
        if dist is None:
            dist = torch.empty((Q, k), dtype=torch.float32, device=dev)
        _check(load().sofa_query(self.h, _ptr(q), Q, k, _ptr(idx), _ptr(dist), _stream(stream)))
        return idx, dist

    def query_window(self, q: torch.Tensor, k: int = 1, cap: int = MAX_WINDOW, stream=None):
        """sofa_query_window: per query, the rows within the tie window of its
        k-th distance in this index -- (ids int64 [Q,cap], d2 float64 [Q,cap],
        counts int32 [Q]), ascending by (distance, id), padded -1 / inf."""
        q = q.contiguous()
        Q = q.shape[0]
        dev = q.device
        ids = torch.empty((Q, cap), dtype=torch.int64, device=dev)
        d2 = torch.empty((Q, cap), dtype=torch.float64, device=dev)
        cnt = torch.empty((Q,), dtype=torch.int32, device=dev)
        _check(load().sofa_query_window(self.h, _ptr(q), Q, k, cap, _ptr(ids), _ptr(d2), _ptr(cnt), _stream(stream)))
        return ids, d2, cnt

    def set_tuning(self, group=0, cand_cap=0, seed_count=0, seed_window=0, bound_precision=0, pool_cap=0,
                   refine_filter=0, use_graph=0, cand_budget=0, dense=0, approximate=0, series_bound=0,
                   tile_checks=0):
        t = Tuning(group, cand_cap, seed_count, seed_window, bound_precision, pool_cap, refine_filter, use_graph,
                   cand_budget, dense, approximate, series_bound, tile_checks)
        _check(load().sofa_set_tuning(self.h, ctypes.byref(t)))

    def autotune(self, q: torch.Tensor, k: int = 1, cache_path: str | None = None, stream=None) -> dict:
        """Time candidate tunings on the sample queries q, apply the fastest."""
        q = q.contiguous()
        t = Tuning()
        _check(load().sofa_autotune(self.h, _ptr(q), q.shape[0], k,
                                    cache_path.encode() if cache_path else None, ctypes.byref(t), _stream(stream)))
        return {name: getattr(t, name) for name, _ in Tuning._fields_}

    def set_seed_mode(self, mode: int):
        _check(load().sofa_set_seed_mode(self.h, mode))

    def train_proposal(self, n_train=0, n_classes=0, epochs=0, batch=0, lr=0.0, seed=2, train_queries=None,
                       top_m=0, stream=None):
        o = TrainOpts(n_train, n_classes, epochs, batch, lr, seed,
                      train_queries.data_ptr() if train_queries is not None else None, top_m)
        _check(load().sofa_train_proposal(self.h, ctypes.byref(o), _stream(stream)))

    def status(self) -> int:
        return load().sofa_query_status(self.h)

    def stats(self, reset=False) -> dict:
        s = Stats()
        _check(load().sofa_stats(self.h, ctypes.byref(s), 1 if reset else 0))
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def set_profiling(self, on: bool = True):
        _check(load().sofa_set_profiling(self.h, 1 if on else 0))

    def profile(self, reset=False) -> dict:
        s = Profile()
        _check(load().sofa_profile(self.h, ctypes.byref(s), 1 if reset else 0))
        return {"ms": {PHASES[i]: s.ms[i] for i in range(8)},
                "launches": {PHASES[i]: s.launches[i] for i in range(8)},
                "scan_tile_loads": s.scan_tile_loads, "scan_tile_checks": s.scan_tile_checks}

    def info(self) -> dict:
        s = Info()
        _check(load().sofa_info(self.h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in Info._fields_}

    def summary(self):
        inf = self.info()
        sel = torch.empty(inf["nsel"], dtype=torch.int32)
        var = torch.empty(inf["nsel"], dtype=torch.float64)
        beta = torch.empty((self.l, self.alphabet + 1), dtype=torch.float32)
        _check(load().sofa_export_summary(self.h, _ptr(sel), _ptr(var), _ptr(beta)))
        return sel, var, beta

    def words(self) -> torch.Tensor:
        w = torch.empty((self.N, self.l), dtype=torch.uint8)
        _check(load().sofa_export_words(self.h, _ptr(w)))
        return w

    def perm(self) -> torch.Tensor:
        p = torch.empty(self.N, dtype=torch.int32)
        _check(load().sofa_export_perm(self.h, _ptr(p)))
        return p

    def lower_bounds(self, q: torch.Tensor, stream=None) -> torch.Tensor:
        q = q.contiguous()
        out = torch.empty((q.shape[0], self.N), dtype=torch.float32, device=q.device)
        _check(load().sofa_lower_bounds(self.h, _ptr(q), q.shape[0], _ptr(out), _stream(stream)))
        return out


def dense_sqdist(index: "Index", q: torch.Tensor, stream=None):
    """sofa_dense_sqdist: (Q x N approximate squared distances in sorted
    order, their error bound M)."""
    q = q.contiguous()
    out = torch.empty((q.shape[0], index.N), dtype=torch.float32, device=q.device)
    m = ctypes.c_float(0.0)
    _check(load().sofa_dense_sqdist(index.h, _ptr(q), q.shape[0], _ptr(out), ctypes.byref(m), _stream(stream)))
    return out, m.value


def value_bounds(index: "Index", q: torch.Tensor, stream=None):
    """sofa_value_bounds: (Q x N lower bounds of the tensor-core series bound
    in original row order, the rounding margin M')."""
    q = q.contiguous()
    out = torch.empty((q.shape[0], index.N), dtype=torch.float32, device=q.device)
    m = ctypes.c_float(0.0)
    _check(load().sofa_value_bounds(index.h, _ptr(q), q.shape[0], _ptr(out), ctypes.byref(m), _stream(stream)))
    return out, m.value


def lower_bounds_noalloc(index: "Index", q: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """sofa_lower_bounds_noalloc: the caller provides `out` (Q x N fp32, device);
    the library allocates nothing during the call."""
    q = q.contiguous()
    _check(load().sofa_lower_bounds_noalloc(index.h, _ptr(q), q.shape[0], _ptr(out), _stream(stream)))
    return out


def mlp_grad(params: torch.Tensor, x: torch.Tensor, y: torch.Tensor, din: int, hidden: int, classes: int,
             stream=None):
    """Loss and flat FP32 gradients of the proposal network on one batch."""
    params = params.contiguous()
    x = x.contiguous()
    y = y.to(torch.int32).contiguous()
    grads = torch.empty_like(params)
    loss = ctypes.c_float(0.0)
    _check(load().sofa_mlp_grad(din, hidden, classes, _ptr(params), _ptr(x), _ptr(y), x.shape[0], _ptr(grads),
                                ctypes.byref(loss), _stream(stream)))
    return loss.value, grads


def znorm(x: torch.Tensor, stream=None) -> torch.Tensor:
    x = x.contiguous()
    z = torch.empty_like(x)
    _check(load().sofa_znorm(_ptr(x), x.shape[0], x.shape[1], _ptr(z), _stream(stream)))
    return z


def query_multi(indexes, queries: torch.Tensor, q_offsets, q_len, q_k, out_offsets, total_out, stream=None):
    """Mixed-length / mixed-k queries over several indexes (sofa_query_multi)."""
    dev = queries.device
    arr = (ctypes.c_void_p * len(indexes))(*[ix.h.value for ix in indexes])
    qo = torch.as_tensor(q_offsets, dtype=torch.int64, device=dev).contiguous()
    ql = torch.as_tensor(q_len, dtype=torch.int32, device=dev).contiguous()
    qk = torch.as_tensor(q_k, dtype=torch.int32, device=dev).contiguous()
    oo = torch.as_tensor(out_offsets, dtype=torch.int64, device=dev).contiguous()
    idx = torch.full((total_out,), -1, dtype=torch.int64, device=dev)
    dist = torch.full((total_out,), float("inf"), dtype=torch.float32, device=dev)
    _check(load().sofa_query_multi(arr, len(indexes), _ptr(queries), _ptr(qo), _ptr(ql), _ptr(qk), qo.numel(),
                                   _ptr(idx), _ptr(dist), _ptr(oo), _stream(stream)))
    return idx, dist


def search(data: torch.Tensor, queries: torch.Tensor, k: int = 1, l: int = 16, alphabet: int = 256, **kw):
    """Build an index, answer the queries, free the index."""
    ix = Index(data, l, alphabet, **kw)
    try:
        return ix.query(queries, k)
    finally:
        ix.close()
