"""GB300 (sm_103a) FINGER greedy-search library: Python binding of libfinger.so.

Argument marshalling only: every step of the search, the graph build, the
FINGER tables and the ground truth runs in the library's CUDA kernels.  There
is no CPU fallback; if the extension cannot be built or loaded, importing the
binding's entry points raises.

Device buffers are torch CUDA tensors (torch supplies memory and streams);
host buffers are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["Index", "lib", "MODE_PLAIN", "MODE_FINGER", "MODE_FINGER_LP", "MODE_FINGER_MLP",
           "MODE_FINGER_F16", "MODE_FINGER_F8",
           "FingerError", "COUNTER_NAMES", "table_bytes"]

MODE_PLAIN, MODE_FINGER, MODE_FINGER_LP, MODE_FINGER_MLP, MODE_FINGER_F16 = 0, 1, 2, 3, 4
MODE_FINGER_F8 = 5
COUNTER_NAMES = ("expansions", "examined", "estimates", "skipped", "exact", "admitted", "upper",
                 "gathered")
STATUS = {0: "ok", 1: "invalid argument", 2: "i/o error", 3: "bad index file format",
          4: "out of memory", 5: "CUDA error", 6: "graph or tables not built",
          7: "kernel iteration or capacity limit reached", 8: "unsupported size"}

_lib = None


class FingerError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class GraphParams(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("candidates", ctypes.c_int), ("level_seed", ctypes.c_uint64),
                ("symmetric", ctypes.c_int), ("flat", ctypes.c_int),
                ("fp32_candidates", ctypes.c_int)]


class BuildParams(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("seed", ctypes.c_uint64), ("samples_per_node", ctypes.c_int),
                ("basis_host", ctypes.c_void_p), ("stats_host", ctypes.c_void_p),
                ("build_lp", ctypes.c_int), ("flags", ctypes.c_int)]

BUILD_NO_MATCHING, BUILD_NO_EPS, BUILD_HALF_CODES, BUILD_FP8_CODES = 1, 2, 4, 8


class TrainParams(ctypes.Structure):
    _fields_ = [("feat", ctypes.c_void_p), ("target", ctypes.c_void_p),
                ("n_train", ctypes.c_int64), ("n_val", ctypes.c_int64), ("epochs", ctypes.c_int),
                ("batch", ctypes.c_int), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int), ("deg0", ctypes.c_int),
                ("M", ctypes.c_int), ("maxlevel", ctypes.c_int), ("entry", ctypes.c_int),
                ("up_rows", ctypes.c_int64), ("r", ctypes.c_int), ("has_lp", ctypes.c_int),
                ("has_mlp", ctypes.c_int), ("device_bytes", ctypes.c_int64),
                ("has_half_codes", ctypes.c_int), ("has_fp8_codes", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("searches", ctypes.c_int64), ("counters", ctypes.c_int64 * 8),
                ("device_error", ctypes.c_int32), ("mu", ctypes.c_double),
                ("sigma", ctypes.c_double), ("mu_hat", ctypes.c_double),
                ("sigma_hat", ctypes.c_double), ("eps", ctypes.c_double),
                ("build_ms", ctypes.c_double), ("corr", ctypes.c_double),
                ("code_bytes", ctypes.c_int64)]


# name -> (restype, argtypes); every symbol include/finger.h declares
_P, _I, _I64, _U64, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
SIGNATURES = {
    "finger_index_create": (_I, [_I, _I64, _I, _P, _P]),
    "finger_index_set_graph": (_I, [_P, _I, _P, _P, _P, _I64, _I, _P, ctypes.c_int32,
                                    ctypes.c_int32]),
    "finger_build_graph": (_I, [_P, _P, _P]),
    "finger_get_graph": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "finger_get_info": (_I, [_P, _P]),
    "finger_index_save": (_I, [_P, ctypes.c_char_p]),
    "finger_index_load": (_I, [ctypes.c_char_p, _I, _P]),
    "finger_index_free": (None, [_P]),
    "finger_build_tables": (_I, [_P, _P, _P]),
    "finger_select_rank": (_I, [_P, _P, ctypes.c_double, _I, _I, _P, _P, _P]),
    "finger_get_tables": (_I, [_P, _P, _P, _P, _P, _P]),
    "finger_table_bytes": (_I64, [_I64, _I, _I, _I]),
    "finger_set_mode": (_I, [_P, _I, _I]),
    "finger_search": (_I, [_P, _P, _I64, _I, _I, _P, _P, _P]),
    "finger_search_host": (_I, [_P, _P, _I64, _I, _I, _P, _P, _P]),
    "finger_search_noalloc": (_I, [_P, _P, _I64, _I, _I, _P, _P, _P]),
    "finger_search_batch": (_I, [_P, _P, _I64, _P, _P, _I, _P, _P, _P, _P]),
    "finger_autotune": (_I, [_P, _P, _I64, _I, _I, _P, _P, _P, _P]),
    "finger_set_counters": (_I, [_P, _P]),
    "finger_set_limit": (_I, [_P, _I]),
    "finger_set_visited_slots": (_I, [_P, _I]),
    "finger_knn": (_I, [_P, _P, _I64, _I, _P, _P, _P]),
    "finger_sync": (_I, [_P]),
    "finger_get_stats": (_I, [_P, _P]),
    "finger_reset_stats": (_I, [_P]),
    "finger_status_str": (ctypes.c_char_p, [_I]),
    "finger_mlp_size": (_I64, [_I]),
    "finger_harvest": (_I, [_P, _P, _I64, _I, _I64, _P, _P, _P, _P, _P]),
    "finger_train_predictor": (_I, [_P, _P, _P, _P]),
    "finger_set_predictor": (_I, [_P, _P, _I64, _F]),
    "finger_get_predictor": (_I, [_P, _P, _P]),
    "finger_set_predictor_gate": (_I, [_P, _F]),
    "finger_get_tuned": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "finger_mlp_loss_grad": (_I, [_P, _I, _P, _P, _P, _I64, _P, _P, _P]),
    "finger_mlp_predict": (_I, [_P, _P, _I64, _P, _P]),
    "finger_merge_topk": (_I, [_P, _P, _I, _I64, _I, _P, _P, _P, _P]),
}


def lib(build: bool = True):
    """Load libfinger.so (building it first when stale).  Raises if it cannot."""
    global _lib
    if _lib is None:
        checked = os.environ.get("FINGER_CHECKED", "0") == "1"
        if build:
            path = _build.build(checked=checked)
        else:
            path = _build.LIB_CHECKED if checked else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libfinger.so is missing at {path}; build it with _build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise FingerError(st, what)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def merge_topk(ids, dists, id_offsets, stream=None):
    """K nearest over a partitioned database: the K smallest (distance, global
    id) keys of the parts' own lists.  ids, dists: CUDA tensors S x nq x K
    (part-major, local ids, -1 / +inf padded); id_offsets: the S first global
    ids.  Returns (ids, dists) as nq x K CUDA tensors."""
    import torch
    if ids.dim() != 3 or dists.shape != ids.shape:
        raise ValueError("ids and dists must both be S x nq x K")
    S, nq, K = ids.shape
    offs = np.ascontiguousarray(np.asarray(id_offsets, dtype=np.int64))
    if offs.shape != (S,):
        raise ValueError(f"id_offsets must hold {S} values")
    out_ids = torch.empty((nq, K), dtype=torch.int64, device=ids.device)
    out_d = torch.empty((nq, K), dtype=torch.float32, device=ids.device)
    with torch.cuda.device(ids.device):
        _check(lib().finger_merge_topk(_dev_ptr(ids, torch.int64, "ids"),
                                       _dev_ptr(dists, torch.float32, "dists"), S, nq, K,
                                       _np_ptr(offs), _dev_ptr(out_ids, torch.int64, "out_ids"),
                                       _dev_ptr(out_d, torch.float32, "out_dists"),
                                       _stream_ptr(stream)), "finger_merge_topk")
    return out_ids, out_d


def table_bytes(n: int, deg0: int, r: int, lp: bool = False) -> int:
    """Bytes of the per-edge FINGER tables, (r+2) * n * deg0 * 4 for FP32."""
    return int(lib().finger_table_bytes(n, deg0, r, int(lp)))


class Index:
    """A FINGER index on one CUDA device (vectors, HNSW-style graph, tables)."""

    def __init__(self, vectors: np.ndarray | None = None, device: int = 0, _handle=None):
        self._lib = lib()
        self.device = device
        if _handle is not None:
            self._h = _handle
            return
        x = np.ascontiguousarray(vectors, dtype=np.float32)
        if x.ndim != 2:
            raise ValueError("vectors must be n x m")
        h = ctypes.c_void_p()
        _check(self._lib.finger_index_create(device, x.shape[0], x.shape[1], _np_ptr(x),
                                             ctypes.byref(h)), "finger_index_create")
        self._h = h

    # ---------------------------------------------------------- lifecycle
    @classmethod
    def load(cls, path: str, device: int = 0) -> "Index":
        L = lib()
        h = ctypes.c_void_p()
        _check(L.finger_index_load(path.encode(), device, ctypes.byref(h)), "finger_index_load")
        return cls(device=device, _handle=h)

    def save(self, path: str):
        _check(self._lib.finger_index_save(self._h, path.encode()), "finger_index_save")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.finger_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = Info()
        _check(self._lib.finger_get_info(self._h, ctypes.byref(i)), "finger_get_info")
        return {k: getattr(i, k) for k, _ in Info._fields_}

    # -------------------------------------------------------------- graph
    def set_graph(self, adj0, level, up_off, up_adj, entry: int, maxlevel: int, M: int):
        adj0 = np.ascontiguousarray(adj0, dtype=np.int32)
        level = np.ascontiguousarray(level, dtype=np.int32)
        up_off = np.ascontiguousarray(up_off, dtype=np.int64)
        up_adj = np.ascontiguousarray(up_adj, dtype=np.int32).reshape(-1, M)
        _check(self._lib.finger_index_set_graph(
            self._h, adj0.shape[1], _np_ptr(adj0), _np_ptr(level), _np_ptr(up_off),
            up_adj.shape[0], M, _np_ptr(up_adj) if up_adj.size else None, entry, maxlevel),
            "finger_index_set_graph")

    def build_graph(self, M: int, candidates: int = 0, level_seed: int = 0,
                    symmetric: bool = False, flat: bool = False, fp32_candidates: bool = False,
                    stream=None):
        """finger_build_graph: HNSW on the device (insertion order by id, exact
        candidate search); symmetric=True draws candidates from all nodes;
        flat=True builds the single-layer graph (no hierarchy, entry node 0);
        fp32_candidates=True ranks layer-0 candidates with FP32 FFMA distances
        instead of the tensor cores."""
        p = GraphParams(M, candidates, level_seed, int(symmetric), int(flat), int(fp32_candidates))
        _check(self._lib.finger_build_graph(self._h, ctypes.byref(p), _stream_ptr(stream)),
               "finger_build_graph")

    def get_graph(self) -> dict:
        i = self.info()
        n, deg0, M, R = i["n"], i["deg0"], i["M"], i["up_rows"]
        adj0 = np.empty((n, deg0), np.int32)
        level = np.empty(n, np.int32)
        up_off = np.empty(n, np.int64)
        up_adj = np.empty((max(R, 1), max(M, 1)), np.int32)
        e = ctypes.c_int32()
        ml = ctypes.c_int32()
        _check(self._lib.finger_get_graph(self._h, _np_ptr(adj0), _np_ptr(level), _np_ptr(up_off),
                                          _np_ptr(up_adj), ctypes.byref(e), ctypes.byref(ml)),
               "finger_get_graph")
        return dict(adj0=adj0, level=level, up_off=up_off, up_adj=up_adj[:R], entry=e.value,
                    maxlevel=ml.value, M=M)

    # ------------------------------------------------------------- tables
    def build_tables(self, r: int, seed: int, samples_per_node: int = 1, basis=None, stats=None,
                     build_lp: bool = False, matching: bool = True, use_eps: bool = True,
                     half_codes: bool = False, fp8_codes: bool = False, stream=None):
        """finger_build_tables.  ``basis`` (r x m) replaces the SVD basis (e.g.
        a random Gaussian matrix: the RPLSH comparison of Sec. 4.3); ``matching``
        and ``use_eps`` False are the ablations of FINGER_BUILD_NO_MATCHING and
        FINGER_BUILD_NO_EPS; ``half_codes`` also stores the FP16 codes of
        MODE_FINGER_F16 (FINGER_BUILD_HALF_CODES), ``fp8_codes`` the FP8 codes
        of MODE_FINGER_F8 (FINGER_BUILD_FP8_CODES)."""
        keep = []
        bp = None
        sp = None
        if basis is not None:
            b = np.ascontiguousarray(basis, dtype=np.float32)
            keep.append(b)
            bp = _np_ptr(b)
        if stats is not None:
            s = np.ascontiguousarray(stats, dtype=np.float64)
            keep.append(s)
            sp = _np_ptr(s)
        flags = ((0 if matching else BUILD_NO_MATCHING) | (0 if use_eps else BUILD_NO_EPS) |
                 (BUILD_HALF_CODES if half_codes else 0) | (BUILD_FP8_CODES if fp8_codes else 0))
        p = BuildParams(r, seed, samples_per_node, bp, sp, int(build_lp), flags)
        _check(self._lib.finger_build_tables(self._h, ctypes.byref(p), _stream_ptr(stream)),
               "finger_build_tables")

    def select_rank(self, seed: int, threshold: float = 0.7, r_step: int = 8, r_max: int = 64,
                    samples_per_node: int = 1, build_lp: bool = False, half_codes: bool = False,
                    fp8_codes: bool = False, stream=None):
        """finger_select_rank: rank rule of Supplementary E, then the tables at
        that rank.  Returns (r, [correlation of each candidate tried])."""
        p = BuildParams(0, seed, samples_per_node, None, None, int(build_lp),
                        (BUILD_HALF_CODES if half_codes else 0) |
                        (BUILD_FP8_CODES if fp8_codes else 0))
        r_out = ctypes.c_int()
        trace = np.full(-(-r_max // r_step), np.nan)
        _check(self._lib.finger_select_rank(self._h, ctypes.byref(p), ctypes.c_double(threshold),
                                            r_step, r_max, ctypes.byref(r_out), _np_ptr(trace),
                                            _stream_ptr(stream)), "finger_select_rank")
        return r_out.value, [float(x) for x in trace if x == x]

    def get_tables(self) -> dict:
        i = self.info()
        n, m, r, deg0 = i["n"], i["m"], i["r"], i["deg0"]
        P = np.empty((r, m), np.float32)
        st = np.empty(5, np.float64)
        Pc = np.empty((n, r), np.float32)
        eu = np.empty((n, deg0, r), np.float32)
        es = np.empty((n, deg0, 2), np.float32)
        _check(self._lib.finger_get_tables(self._h, _np_ptr(P), _np_ptr(st), _np_ptr(Pc),
                                           _np_ptr(eu), _np_ptr(es)), "finger_get_tables")
        return dict(P=P, stats=st, node_proj=Pc, edge_u=eu, dres_norm=es[..., 0], b=es[..., 1])

    # ------------------------------------------------------------- search
    def set_mode(self, mode: int, warmup: int = -1):
        _check(self._lib.finger_set_mode(self._h, mode, warmup), "finger_set_mode")

    def set_limit(self, max_expansions: int):
        """Cap on expansions per query (0 = default n + 16)."""
        _check(self._lib.finger_set_limit(self._h, max_expansions), "finger_set_limit")

    def set_visited_slots(self, bits: int):
        """Visited-set slot width: 0 = 16-bit where the ids fit (default), 32 = always 32-bit."""
        _check(self._lib.finger_set_visited_slots(self._h, bits), "finger_set_visited_slots")

    def set_counters(self, counters):
        """Per-query counters (int32 CUDA tensor nq x 8) for later searches; None disables."""
        import torch
        p = None if counters is None else _dev_ptr(counters, torch.int32, "counters")
        _check(self._lib.finger_set_counters(self._h, p), "finger_set_counters")

    def search(self, queries, K: int, ef: int, out_ids=None, out_dists=None, stream=None):
        import torch
        nq = queries.shape[0]
        if out_ids is None:
            out_ids = torch.empty((nq, K), dtype=torch.int64, device=queries.device)
        if out_dists is None:
            out_dists = torch.empty((nq, K), dtype=torch.float32, device=queries.device)
        _check(self._lib.finger_search(self._h, _dev_ptr(queries, torch.float32, "queries"), nq, K,
                                       ef, _dev_ptr(out_ids, torch.int64, "out_ids"),
                                       _dev_ptr(out_dists, torch.float32, "out_dists"),
                                       _stream_ptr(stream)), "finger_search")
        return out_ids, out_dists

    def search_noalloc(self, queries, K: int, ef: int, out_ids, out_dists, stream=None):
        """finger_search_noalloc: same results as search(), scratch taken from the
        library's fixed device array, no allocation in the call (the caller passes
        preallocated output tensors)."""
        import torch
        nq = queries.shape[0]
        _check(self._lib.finger_search_noalloc(
            self._h, _dev_ptr(queries, torch.float32, "queries"), nq, K, ef,
            _dev_ptr(out_ids, torch.int64, "out_ids"),
            _dev_ptr(out_dists, torch.float32, "out_dists"), _stream_ptr(stream)),
            "finger_search_noalloc")
        return out_ids, out_dists

    def search_host(self, queries: np.ndarray, K: int, ef: int, out_ids=None, out_dists=None,
                    stream=None):
        q = np.ascontiguousarray(queries, dtype=np.float32)
        nq = q.shape[0]
        ids = out_ids if out_ids is not None else np.empty((nq, K), np.int64)
        d = out_dists if out_dists is not None else np.empty((nq, K), np.float32)
        _check(self._lib.finger_search_host(self._h, _np_ptr(q), nq, K, ef, _np_ptr(ids),
                                            _np_ptr(d), _stream_ptr(stream)),
               "finger_search_host")
        return ids, d

    def search_batch(self, queries, K, ef, max_ef: int | None = None, offsets=None,
                     total: int | None = None, stream=None):
        """Uneven batch: K, ef int32 CUDA tensors (per query).  Returns flat ids,
        dists and the int64 offsets of each query's results.  A caller that
        already has the exclusive prefix sum of K (``offsets``, int64 CUDA) and
        its total passes them to keep the call free of host synchronisation."""
        import torch
        nq = queries.shape[0]
        if offsets is None or total is None:
            Kc = K.to(torch.int64)
            off = torch.zeros(nq, dtype=torch.int64, device=queries.device)
            if nq > 1:
                off[1:] = torch.cumsum(Kc, 0)[:-1]
            total = int(Kc.sum().item()) if nq else 0
        else:
            off = offsets
        if max_ef is None:
            max_ef = int(ef.max().item())
        ids = torch.empty(max(total, 1), dtype=torch.int64, device=queries.device)
        d = torch.empty(max(total, 1), dtype=torch.float32, device=queries.device)
        _check(self._lib.finger_search_batch(
            self._h, _dev_ptr(queries, torch.float32, "queries"), nq,
            _dev_ptr(K, torch.int32, "K"), _dev_ptr(ef, torch.int32, "ef"), max_ef,
            _dev_ptr(off, torch.int64, "out_off"), _dev_ptr(ids, torch.int64, "out_ids"),
            _dev_ptr(d, torch.float32, "out_dists"), _stream_ptr(stream)), "finger_search_batch")
        return ids[:total], d[:total], off

    def autotune(self, queries, K: int, ef: int, stream=None) -> float:
        import torch
        nq = queries.shape[0]
        ids = torch.empty((nq, K), dtype=torch.int64, device=queries.device)
        d = torch.empty((nq, K), dtype=torch.float32, device=queries.device)
        best = ctypes.c_float()
        _check(self._lib.finger_autotune(self._h, _dev_ptr(queries, torch.float32, "queries"), nq,
                                         K, ef, _dev_ptr(ids, torch.int64, "ids"),
                                         _dev_ptr(d, torch.float32, "dists"), ctypes.byref(best),
                                         _stream_ptr(stream)), "finger_autotune")
        return best.value


    def tuned(self, ef: int) -> dict | None:
        """finger_get_tuned: the autotuner's pick for ef's bucket, or None."""
        w, h, o, rw = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_float()
        st = self._lib.finger_get_tuned(self._h, ef, ctypes.byref(w), ctypes.byref(h),
                                        ctypes.byref(o), ctypes.byref(rw), ctypes.byref(ms))
        if st == 6:      # FINGER_ERR_NOT_BUILT: not tuned
            return None
        _check(st, "finger_get_tuned")
        return {"warps_per_block": w.value, "hash_slots": h.value, "resident_warps": o.value,
                "rows_per_warp": rw.value,
                "best_ms": ms.value}
    def knn(self, queries, K: int, stream=None):
        """Exact K nearest neighbours by brute force on the GPU."""
        import torch
        nq = queries.shape[0]
        ids = torch.empty((nq, K), dtype=torch.int64, device=queries.device)
        d = torch.empty((nq, K), dtype=torch.float32, device=queries.device)
        _check(self._lib.finger_knn(self._h, _dev_ptr(queries, torch.float32, "queries"), nq, K,
                                    _dev_ptr(ids, torch.int64, "ids"),
                                    _dev_ptr(d, torch.float32, "dists"), _stream_ptr(stream)),
               "finger_knn")
        return ids, d

    # ------------------------------------------ learned predictor (extension)
    def mlp_size(self) -> int:
        return int(self._lib.finger_mlp_size(self.info()["r"]))

    def harvest(self, queries, ef: int, cap: int, stream=None):
        """Training triples from FINGER traversals: (features, targets, triples)
        as CUDA tensors trimmed to the number of records."""
        import torch
        nf = self.info()["r"] + 4
        feat = torch.empty((cap, nf), dtype=torch.float32, device=queries.device)
        tgt = torch.empty(cap, dtype=torch.float32, device=queries.device)
        trip = torch.empty((cap, 3), dtype=torch.int32, device=queries.device)
        cnt = ctypes.c_int64()
        _check(self._lib.finger_harvest(self._h, _dev_ptr(queries, torch.float32, "queries"),
                                        queries.shape[0], ef, cap, _dev_ptr(feat, torch.float32, "feat"),
                                        _dev_ptr(tgt, torch.float32, "target"),
                                        _dev_ptr(trip, torch.int32, "triples"), ctypes.byref(cnt),
                                        _stream_ptr(stream)), "finger_harvest")
        n = cnt.value
        return feat[:n], tgt[:n], trip[:n]

    def train_predictor(self, feat, target, n_val: int, epochs: int = 8, batch: int = 4096,
                        lr: float = 2e-3, seed: int = 5004, stream=None):
        import torch
        n = feat.shape[0]
        p = TrainParams(_dev_ptr(feat, torch.float32, "feat").value,
                        _dev_ptr(target, torch.float32, "target").value, n - n_val, n_val,
                        epochs, batch, lr, seed)
        losses = np.zeros(epochs, np.float32)
        _check(self._lib.finger_train_predictor(self._h, ctypes.byref(p), _np_ptr(losses),
                                                _stream_ptr(stream)), "finger_train_predictor")
        return losses

    def set_predictor(self, weights: np.ndarray, eps: float):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        _check(self._lib.finger_set_predictor(self._h, _np_ptr(w), w.size, eps),
               "finger_set_predictor")

    def set_predictor_gate(self, delta: float):
        """finger_set_predictor_gate: the learned predictor runs only where the
        matched estimate lies within delta * ub of ub (delta < 0: everywhere)."""
        _check(self._lib.finger_set_predictor_gate(self._h, float(delta)),
               "finger_set_predictor_gate")

    def get_predictor(self):
        w = np.empty(self.mlp_size(), np.float32)
        eps = ctypes.c_float()
        _check(self._lib.finger_get_predictor(self._h, _np_ptr(w), ctypes.byref(eps)),
               "finger_get_predictor")
        return w, eps.value

    def mlp_loss_grad(self, weights: np.ndarray, feat, target, stream=None):
        import torch
        w = np.ascontiguousarray(weights, dtype=np.float32)
        g = np.empty_like(w)
        loss = ctypes.c_double()
        _check(self._lib.finger_mlp_loss_grad(self._h, feat.shape[1], _np_ptr(w),
                                              _dev_ptr(feat, torch.float32, "feat"),
                                              _dev_ptr(target, torch.float32, "target"),
                                              feat.shape[0], _np_ptr(g), ctypes.byref(loss),
                                              _stream_ptr(stream)), "finger_mlp_loss_grad")
        return loss.value, g

    def mlp_predict(self, feat, stream=None):
        import torch
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        _check(self._lib.finger_mlp_predict(self._h, _dev_ptr(feat, torch.float32, "feat"),
                                            feat.shape[0], _dev_ptr(out, torch.float32, "out"),
                                            _stream_ptr(stream)), "finger_mlp_predict")
        return out

    # -------------------------------------------------------------- status
    def sync(self):
        _check(self._lib.finger_sync(self._h), "finger_sync")

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.finger_get_stats(self._h, ctypes.byref(s)), "finger_get_stats")
        out = {k: getattr(s, k) for k, _ in Stats._fields_ if k != "counters"}
        out["counters"] = dict(zip(COUNTER_NAMES, list(s.counters)))
        return out

    def reset_stats(self):
        _check(self._lib.finger_reset_stats(self._h), "finger_reset_stats")
