"""ctypes binding of libtw (include/tw.h): argument marshalling only.

Every computation runs inside libtw's CUDA kernels.  Arrays may be numpy
arrays (host memory) or CUDA torch tensors (device memory); libtw detects which
and copies accordingly.  Importing this module does not load the library;
:func:`lib` does, and it raises if ``libtw.so`` has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import graphgen

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtw.so")
MAX_N = 128
N_FEATURES = 12
N_PARAMS = 32 * 12 + 32 + 32 + 1

TW_OK, TW_ERR_INVALID, TW_ERR_CAPACITY, TW_ERR_TIMEOUT, TW_ERR_CUDA = 0, 1, 2, 3, 4


class TwError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} (status {status})")


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("fingerprints", ctypes.c_int), ("mem_cap_bytes", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("block_threads", ctypes.c_int), ("table_load_pct", ctypes.c_int),
                ("max_probes", ctypes.c_int), ("ub_shortcut", ctypes.c_int), ("graph_levels", ctypes.c_int),
                ("time_kernels", ctypes.c_int), ("clique_skip", ctypes.c_int), ("disjoint_paths", ctypes.c_int),
                ("autotune", ctypes.c_int), ("partition_table_mb", ctypes.c_int), ("mmw_prune", ctypes.c_int),
                ("spill_levels", ctypes.c_int), ("out_of_core", ctypes.c_int),
                ("fused_states", ctypes.c_int), ("batch_kernel", ctypes.c_int),
                ("host_cap_mb", ctypes.c_int), ("batch_arena_states", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("k", ctypes.c_int),
                ("level_size", ctypes.c_uint64 * (MAX_N + 1)),
                ("level_fp_sum", ctypes.c_uint64 * (MAX_N + 1)),
                ("level_fp_xor", ctypes.c_uint64 * (MAX_N + 1)),
                ("states_expanded", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("generated", ctypes.c_uint64), ("peak_frontier_bytes", ctypes.c_uint64),
                ("decide_runs", ctypes.c_uint64), ("level_retries", ctypes.c_uint64),
                ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_uint64),
                ("expand_launches", ctypes.c_uint64), ("expand_seconds", ctypes.c_double),
                ("expand_bytes", ctypes.c_double)]

    def as_dict(self) -> dict:
        L = self.levels
        return {"levels": L, "k": self.k, "level_size": list(self.level_size[:L]),
                "fp_sum": list(self.level_fp_sum[:L]), "fp_xor": list(self.level_fp_xor[:L]),
                "states_expanded": int(self.states_expanded), "candidates": int(self.candidates),
                "generated": int(self.generated), "peak_frontier_bytes": int(self.peak_frontier_bytes),
                "decide_runs": int(self.decide_runs), "level_retries": int(self.level_retries),
                "seconds": float(self.seconds), "kernel_launches": int(self.kernel_launches),
                "expand_launches": int(self.expand_launches), "expand_seconds": float(self.expand_seconds),
                "expand_bytes": float(self.expand_bytes)}


_lib = None
_vp = ctypes.c_void_p


def lib():
    """Loads libtw.so; raises if it is missing (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtw.so is not built ({LIB_PATH}); run python -m paper_1709_09990_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    L.tw_strerror.restype = ctypes.c_char_p
    L.tw_strerror.argtypes = [ctypes.c_int]
    L.tw_abi_version.restype = ctypes.c_int
    L.tw_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Config)]
    L.tw_destroy.argtypes = [_vp]
    L.tw_destroy.restype = None
    L.tw_decide.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.POINTER(Stats)]
    L.tw_decide_level.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Stats)]
    L.tw_decide_u32.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.POINTER(Stats)]
    L.tw_solve.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.POINTER(Stats)]
    L.tw_solve_batch.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.POINTER(Stats)]
    L.tw_decide_batch.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                  ctypes.POINTER(Stats)]
    L.tw_bounds.argtypes = [_vp, _vp, ctypes.c_int, _vp]
    L.tw_features_batch.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]
    L.tw_mlp_forward.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
    L.tw_mlp_grad.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]
    L.tw_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float]
    L.tw_mlp_train.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                               ctypes.c_float, _vp]
    _lib = L
    return L


def strerror(status: int) -> str:
    try:
        return lib().tw_strerror(status).decode()
    except RuntimeError:
        return f"status {status}"


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(rc: int, what: str) -> None:
    if rc != TW_OK:
        raise TwError(rc, what)


def rows_u64(adj) -> np.ndarray:
    """Python-int adjacency -> contiguous uint64 rows (numpy arrays pass through)."""
    if isinstance(adj, np.ndarray) or hasattr(adj, "data_ptr"):
        return adj
    return np.ascontiguousarray(graphgen.to_rows_u64(adj))


class Context:
    """One libtw context (one device, one stream)."""

    def __init__(self, device: int = 0, fingerprints: bool = False, mem_cap_bytes: int = 0,
                 stream: int = 0, block_threads: int = 0, table_load_pct: int = 0, max_probes: int = 0,
                 ub_shortcut: bool = False, time_kernels: bool = False, graph_levels: int = 0,
                 autotune: bool = False, clique_skip: bool = False, disjoint_paths: bool = False,
                 partition_table_mb: int = 0, mmw_prune: bool = False, spill_levels: bool = False,
                 out_of_core: bool = False, fused_states: int = 0, batch_kernel: int = 0,
                 host_cap_mb: int = 0, batch_arena_states: int = 0):
        cfg = Config()
        cfg.device = device
        cfg.fingerprints = int(fingerprints)
        cfg.mem_cap_bytes = mem_cap_bytes
        cfg.stream = stream or None
        cfg.block_threads = block_threads
        cfg.table_load_pct = table_load_pct
        cfg.max_probes = max_probes
        cfg.ub_shortcut = int(ub_shortcut)
        cfg.time_kernels = int(time_kernels)
        cfg.graph_levels = int(graph_levels)
        cfg.autotune = int(autotune)
        cfg.clique_skip = int(clique_skip)
        cfg.disjoint_paths = int(disjoint_paths)
        cfg.partition_table_mb = int(partition_table_mb)
        cfg.mmw_prune = int(mmw_prune)
        cfg.spill_levels = int(spill_levels)
        cfg.out_of_core = int(out_of_core)
        cfg.fused_states = int(fused_states)
        cfg.batch_kernel = int(batch_kernel)
        cfg.host_cap_mb = int(host_cap_mb)
        cfg.batch_arena_states = int(batch_arena_states)
        h = _vp()
        _check(lib().tw_create(ctypes.byref(h), ctypes.byref(cfg)), "tw_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().tw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- decide
    def decide(self, adj, n: Optional[int] = None, k: int = 0, want_order: bool = False,
               order_out=None, raise_on_error: bool = True):
        rows = rows_u64(adj)
        n = len(adj) if n is None else n
        yes = ctypes.c_int(-1)
        st = Stats()
        order = order_out if order_out is not None else (np.full(n, -1, np.int32) if want_order else None)
        rc = lib().tw_decide(self._h, _ptr(rows), n, k, ctypes.addressof(yes), _ptr(order), ctypes.byref(st))
        if raise_on_error:
            if rc != TW_OK:
                err = TwError(rc, "tw_decide")
                err.stats = st.as_dict()
                raise err
        return {"status": rc, "yes": bool(yes.value == 1), "order": order, "stats": st.as_dict()}

    def decide_level(self, adj, k: int, level: int, n: Optional[int] = None, keys_out=None,
                     count_only: bool = False):
        """The sets of level ``level`` of decide(k) as a (count, ceil(n/64))
        uint64 array (unordered).  keys_out (host array or device tensor of
        at least count * ceil(n/64) words) is used when given; otherwise a host
        array is sized from a first call that returns the count only.  With
        count_only no sets are copied (keys is None)."""
        rows = rows_u64(adj)
        n = len(adj) if n is None else n
        w = max(1, (n + 63) // 64)
        cnt = ctypes.c_uint64(0)
        st = Stats()
        if keys_out is None:
            rc = lib().tw_decide_level(self._h, _ptr(rows), n, k, level, None, 0, ctypes.byref(cnt),
                                       ctypes.byref(st))
            if rc not in (TW_OK, TW_ERR_CAPACITY) or (rc == TW_ERR_CAPACITY and cnt.value == 0):
                _check(rc, "tw_decide_level")
            if count_only:
                return {"keys": None, "count": int(cnt.value), "stats": st.as_dict()}
            keys_out = np.zeros((max(1, int(cnt.value)), w), np.uint64)
        cap = (keys_out.numel() if hasattr(keys_out, "numel") else keys_out.size) // w
        rc = lib().tw_decide_level(self._h, _ptr(rows), n, k, level, _ptr(keys_out), cap, ctypes.byref(cnt),
                                   ctypes.byref(st))
        _check(rc, "tw_decide_level")
        return {"keys": keys_out[: int(cnt.value)], "count": int(cnt.value), "stats": st.as_dict()}

    def decide_u32(self, adj_rows_u32: np.ndarray, n: int, k: int, want_order: bool = False):
        yes = ctypes.c_int(-1)
        st = Stats()
        order = np.full(n, -1, np.int32) if want_order else None
        rc = lib().tw_decide_u32(self._h, _ptr(adj_rows_u32), n, k, ctypes.addressof(yes), _ptr(order),
                                 ctypes.byref(st))
        _check(rc, "tw_decide_u32")
        return {"yes": bool(yes.value == 1), "order": order, "stats": st.as_dict()}

    # --------------------------------------------------------------- solve
    def solve(self, adj, n: Optional[int] = None, want_order: bool = True, want_td: bool = False,
              tw_out=None, order_out=None):
        rows = rows_u64(adj)
        n = len(adj) if n is None else n
        w = max(1, (n + 63) // 64)
        tw = tw_out if tw_out is not None else np.full(1, -1, np.int32)
        order = order_out if order_out is not None else (np.full(n, -1, np.int32) if want_order else None)
        parent = np.full(n, -2, np.int32) if want_td else None
        bags = np.zeros((n, w), np.uint64) if want_td else None
        st = Stats()
        rc = lib().tw_solve(self._h, _ptr(rows), n, _ptr(tw), _ptr(order), _ptr(parent), _ptr(bags),
                            ctypes.byref(st))
        _check(rc, "tw_solve")
        tw_val = int(tw[0]) if isinstance(tw, np.ndarray) else None
        return {"tw": tw_val, "order": order, "td_parent": parent, "td_bags": bags, "stats": st.as_dict()}

    def solve_batch(self, graphs: Sequence, k_hint: Optional[np.ndarray] = None, want_orders: bool = True):
        adj, ns, offs = graphgen.concat_rows_u64(graphs)
        G = len(graphs)
        tw = np.full(G, -1, np.int32)
        status = np.full(G, -1, np.int32)
        orders = np.full(int(ns.sum()), -1, np.int32) if want_orders else None
        hint = None if k_hint is None else np.ascontiguousarray(k_hint, dtype=np.float32)
        st = Stats()
        rc = lib().tw_solve_batch(self._h, _ptr(adj), _ptr(ns), _ptr(offs), G, _ptr(tw), _ptr(orders),
                                  _ptr(status), _ptr(hint), ctypes.byref(st))
        return {"status": rc, "tw": tw, "per_graph_status": status, "orders": orders, "n": ns,
                "stats": st.as_dict()}

    def decide_batch(self, graphs: Sequence, k, fingerprints: bool = True):
        """decide(k[g]) for every graph through the batched kernel: answers,
        per-graph level sizes (and fingerprints) of each run."""
        adj, ns, offs = graphgen.concat_rows_u64(graphs)
        G = len(graphs)
        kk = np.ascontiguousarray(k, dtype=np.int32)
        yes = np.full(G, -1, np.int32)
        status = np.full(G, -1, np.int32)
        L = MAX_N + 1
        ls = np.zeros((G, L), np.uint64)
        fs = np.zeros((G, L), np.uint64) if fingerprints else None
        fx = np.zeros((G, L), np.uint64) if fingerprints else None
        st = Stats()
        rc = lib().tw_decide_batch(self._h, _ptr(adj), _ptr(ns), _ptr(offs), G, _ptr(kk), _ptr(yes), _ptr(status),
                                   _ptr(ls), _ptr(fs), _ptr(fx), ctypes.byref(st))
        return {"status": rc, "yes": yes, "per_graph_status": status, "level_size": ls, "fp_sum": fs,
                "fp_xor": fx, "stats": st.as_dict()}

    # -------------------------------------------------------------- bounds
    def bounds(self, adj) -> np.ndarray:
        rows = rows_u64(adj)
        out = np.zeros(4, np.int32)
        _check(lib().tw_bounds(self._h, _ptr(rows), len(adj), _ptr(out)), "tw_bounds")
        return out

    def features(self, graphs: Sequence) -> np.ndarray:
        adj, ns, offs = graphgen.concat_rows_u64(graphs)
        out = np.zeros((len(graphs), N_FEATURES), np.float32)
        _check(lib().tw_features_batch(self._h, _ptr(adj), _ptr(ns), _ptr(offs), len(graphs), _ptr(out)),
               "tw_features_batch")
        return out

    # ------------------------------------------------------------- network
    def mlp_forward(self, params: np.ndarray, x: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(params, np.float32)
        xx = np.ascontiguousarray(x, np.float32)
        y = np.zeros(xx.shape[0], np.float32)
        _check(lib().tw_mlp_forward(self._h, _ptr(p), _ptr(xx), xx.shape[0], _ptr(y)), "tw_mlp_forward")
        return y

    def mlp_grad(self, params: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(params, np.float32)
        xx = np.ascontiguousarray(x, np.float32)
        yy = np.ascontiguousarray(y, np.float32)
        g = np.zeros(N_PARAMS, np.float32)
        _check(lib().tw_mlp_grad(self._h, _ptr(p), _ptr(xx), _ptr(yy), xx.shape[0], _ptr(g)), "tw_mlp_grad")
        return g

    def mlp_adam(self, params, grad, m, v, t: int, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().tw_mlp_adam(self._h, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), t, lr, beta1, beta2, eps),
               "tw_mlp_adam")

    def mlp_train(self, params: np.ndarray, x: np.ndarray, y: np.ndarray, minibatch: int, perm: np.ndarray,
                  lr: float = 1e-2) -> np.ndarray:
        p = params  # updated in place
        xx = np.ascontiguousarray(x, np.float32)
        yy = np.ascontiguousarray(y, np.float32)
        pm = np.ascontiguousarray(perm, np.int32)
        epochs = pm.shape[0]
        loss = np.zeros(epochs, np.float32)
        _check(lib().tw_mlp_train(self._h, _ptr(p), _ptr(xx), _ptr(yy), xx.shape[0], minibatch, epochs,
                                  _ptr(pm), lr, _ptr(loss)), "tw_mlp_train")
        return loss
