"""CPU oracle for the breadth-first treewidth DP (test infrastructure).

This package is the plain, slow reference that the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product package never does, and the two
share no code (the seeded input generators in
``paper_1709_09990_gb300.graphgen`` feed both sides but hold none of the
method's arithmetic).

Contents:
  * ``tw_oracle.cpp`` - the level-by-level test of van der Zanden &
    Bodlaender (arXiv 1709.09990, Section 3.1) over exact hash sets, with
    Q(S, v) computed from its Section 2 definition (paths from v whose inner
    vertices lie in S), brute force over all orderings, an independent subset
    DP, ordering and tree-decomposition checks.  Built with g++ by
    :func:`build`.
  * ``bounds.py`` - minimum-degree / minor-min-width lower bounds and
    min-degree / min-fill upper bounds (with their selection sequences), and
    the 12 graph features of the learned starting bound.
  * ``mlp.py`` - float64 forward/backward/Adam of the 12-32-1 network.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tw_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libtw_oracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (host code only, portable flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declares the C signatures on a loaded oracle library."""
    lib.orc_set_fingerprint.restype = ctypes.c_uint64
    lib.orc_set_fingerprint.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.orc_valid_graph.argtypes = [_u64p, ctypes.c_int]
    lib.orc_q_size.argtypes = [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
    lib.orc_q_set.argtypes = [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _u64p]
    lib.orc_decide.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, _i64p, _u64p, _u64p, _intp, _i64p, _i32p]
    lib.orc_solve.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, _i32p, _i64p]
    lib.orc_width_q.argtypes = [_u64p, ctypes.c_int, _i32p]
    lib.orc_width_elim.argtypes = [_u64p, ctypes.c_int, _i32p]
    lib.orc_brute_force_tw.argtypes = [_u64p, ctypes.c_int]
    lib.orc_subset_dp.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, _i64p, _u64p, _u64p, _intp]
    lib.orc_td_from_order.argtypes = [_u64p, ctypes.c_int, _i32p, _i32p, _u64p]
    lib.orc_verify_td.argtypes = [_u64p, ctypes.c_int, _i32p, _u64p]
    lib.orc_max_clique.argtypes = [_u64p, ctypes.c_int, _i32p]
    lib.orc_mmw_bound.argtypes = [_u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
    lib.orc_disjoint_paths.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_decide_opts.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _u64p, _u64p, _intp,
                                    _i64p, _i32p]
    if hasattr(lib, "orc_decide_prefix"):
        lib.orc_decide_prefix.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _u64p, _u64p,
                                          _i64p, ctypes.c_int]
    if hasattr(lib, "orc_level_keys"):
        lib.orc_level_keys.restype = ctypes.c_int64
        lib.orc_level_keys.argtypes = [_u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int64]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def rows(adj: Sequence[int]) -> np.ndarray:
    """Python-int adjacency -> contiguous n x ceil(n/64) uint64 rows."""
    n = len(adj)
    w = max(1, (n + 63) // 64)
    out = np.zeros((n, w), dtype=np.uint64)
    for i, r in enumerate(adj):
        for j in range(w):
            out[i, j] = (r >> (64 * j)) & 0xFFFFFFFFFFFFFFFF
    return np.ascontiguousarray(out)


def _key_words(s: int):
    return s & 0xFFFFFFFFFFFFFFFF, (s >> 64) & 0xFFFFFFFFFFFFFFFF


def fingerprint(s: int) -> int:
    w0, w1 = _key_words(s)
    return int(_load().orc_set_fingerprint(w0, w1))


def valid_graph(adj_rows: np.ndarray, n: int) -> bool:
    return bool(_load().orc_valid_graph(_ptr(adj_rows, _u64p), n))


def q_size(adj: Sequence[int], s: int, v: int) -> int:
    r = rows(adj)
    w0, w1 = _key_words(s)
    return int(_load().orc_q_size(_ptr(r, _u64p), len(adj), w0, w1, v))


def q_set(adj: Sequence[int], s: int, v: int) -> int:
    r = rows(adj)
    w0, w1 = _key_words(s)
    out = np.zeros(2, dtype=np.uint64)
    rc = _load().orc_q_set(_ptr(r, _u64p), len(adj), w0, w1, v, _ptr(out, _u64p))
    if rc != 0:
        raise ValueError("invalid graph or vertex")
    return int(out[0]) | (int(out[1]) << 64)


def decide(adj: Sequence[int], k: int, want_order: bool = False, count_canonical: bool = False) -> Dict:
    """Listing 1 at bound k.  Returns yes, levels, level_size, fp_sum, fp_xor,
    states_expanded, candidates, feasible and (optionally) order.  With
    count_canonical it also returns ``canonical``: the feasible pairs (S, v)
    whose v lies in the component of G[S u {v}] holding its lowest vertex."""
    if count_canonical:
        return decide_opts(adj, k, COUNT_CANONICAL, want_order)
    n = len(adj)
    r = rows(adj)
    ls = np.zeros(n + 1, dtype=np.int64)
    fs = np.zeros(n + 1, dtype=np.uint64)
    fx = np.zeros(n + 1, dtype=np.uint64)
    lv = ctypes.c_int(0)
    cnt = np.zeros(3, dtype=np.int64)
    order = np.full(n, -1, dtype=np.int32) if want_order else None
    yes = _load().orc_decide(_ptr(r, _u64p), n, k, _ptr(ls, _i64p), _ptr(fs, _u64p), _ptr(fx, _u64p),
                             ctypes.byref(lv), _ptr(cnt, _i64p),
                             _ptr(order, _i32p) if order is not None else None)
    if yes < 0:
        raise ValueError("invalid graph or k")
    return {"yes": bool(yes), "levels": lv.value, "level_size": ls[: lv.value].tolist(),
            "fp_sum": fs[: lv.value].tolist(), "fp_xor": fx[: lv.value].tolist(),
            "states_expanded": int(cnt[0]), "candidates": int(cnt[1]), "feasible": int(cnt[2]),
            "order": order.tolist() if (order is not None and yes) else None}


def decide_prefix(adj: Sequence[int], k: int, max_level: int, count_canonical: bool = True) -> Dict:
    """The first levels 0 .. max_level of the Section 3.1 test at bound k (for
    runs too large to finish here): level_size, fp_sum, fp_xor and the
    counters of the levels expanded so far (canonical pairs included when
    count_canonical)."""
    n = len(adj)
    r = rows(adj)
    ls = np.zeros(n + 1, dtype=np.int64)
    fs = np.zeros(n + 1, dtype=np.uint64)
    fx = np.zeros(n + 1, dtype=np.uint64)
    cnt = np.zeros(4, dtype=np.int64)
    lv = _load().orc_decide_prefix(_ptr(r, _u64p), n, k, max_level, _ptr(ls, _i64p), _ptr(fs, _u64p),
                                   _ptr(fx, _u64p), _ptr(cnt, _i64p), int(count_canonical))
    if lv < 0:
        raise ValueError("invalid graph, k or max_level")
    out = {"levels": lv, "level_size": ls[:lv].tolist(), "fp_sum": fs[:lv].tolist(), "fp_xor": fx[:lv].tolist(),
           "states_expanded": int(cnt[0]), "candidates": int(cnt[1]), "feasible": int(cnt[2])}
    if count_canonical:
        out["canonical"] = int(cnt[3])
    return out


def level_keys(adj: Sequence[int], k: int, level: int) -> np.ndarray:
    """The sets of level ``level`` of the test at bound k, as a
    (|L_level|, ceil(n/64)) uint64 array sorted by rows (word 0 first)."""
    n = len(adj)
    r = rows(adj)
    w = r.shape[1]
    lib = _load()
    count = lib.orc_level_keys(_ptr(r, _u64p), n, k, level, None, 0)
    if count < 0:
        raise ValueError("invalid graph, k or level")
    out = np.zeros((max(1, count), w), dtype=np.uint64)
    got = lib.orc_level_keys(_ptr(r, _u64p), n, k, level, _ptr(out, _u64p), count)
    assert got == count
    return sort_keys(out[:count])


def sort_keys(keys: np.ndarray) -> np.ndarray:
    """Rows of a (count, W) uint64 key array in increasing order (last word
    most significant)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    if keys.ndim == 1:
        keys = keys.reshape(len(keys), 1)
    if len(keys) == 0:
        return keys
    idx = np.lexsort(tuple(keys[:, j] for j in range(keys.shape[1])))
    return keys[idx]


CLIQUE_SKIP, DISJOINT_PATHS, MMW_PRUNE, COUNT_CANONICAL = 1, 2, 4, 8


def mmw_bound(adj: Sequence[int], s: int = 0) -> int:
    """Minor-min-width bound (second-smallest degree per step) of the graph
    left after eliminating the set s."""
    r = rows(adj)
    w0, w1 = _key_words(s)
    return int(_load().orc_mmw_bound(_ptr(r, _u64p), len(adj), w0, w1))


def decide_opts(adj: Sequence[int], k: int, opts: int, want_order: bool = False) -> Dict:
    """decide(k) with the optional reductions of Sections 3.1 and 3.3 (opts:
    CLIQUE_SKIP, DISJOINT_PATHS, MMW_PRUNE; COUNT_CANONICAL adds the
    ``canonical`` counter).  Same fields as :func:`decide`."""
    n = len(adj)
    r = rows(adj)
    ls = np.zeros(n + 1, dtype=np.int64)
    fs = np.zeros(n + 1, dtype=np.uint64)
    fx = np.zeros(n + 1, dtype=np.uint64)
    lv = ctypes.c_int(0)
    cnt = np.zeros(4, dtype=np.int64)
    order = np.full(n, -1, dtype=np.int32) if want_order else None
    yes = _load().orc_decide_opts(_ptr(r, _u64p), n, k, opts, _ptr(ls, _i64p), _ptr(fs, _u64p), _ptr(fx, _u64p),
                                  ctypes.byref(lv), _ptr(cnt, _i64p),
                                  _ptr(order, _i32p) if order is not None else None)
    if yes < 0:
        raise ValueError("invalid graph or k")
    return {"yes": bool(yes), "levels": lv.value, "level_size": ls[: lv.value].tolist(),
            "fp_sum": fs[: lv.value].tolist(), "fp_xor": fx[: lv.value].tolist(),
            "states_expanded": int(cnt[0]), "candidates": int(cnt[1]), "feasible": int(cnt[2]),
            "order": order.tolist() if (order is not None and yes) else None,
            **({"canonical": int(cnt[3])} if opts & COUNT_CANONICAL else {})}


def max_clique(adj: Sequence[int]) -> List[int]:
    r = rows(adj)
    out = np.zeros(len(adj), dtype=np.int32)
    m = _load().orc_max_clique(_ptr(r, _u64p), len(adj), _ptr(out, _i32p))
    return out[:m].tolist()


def disjoint_paths(adj: Sequence[int], u: int, v: int, limit: int) -> int:
    r = rows(adj)
    return int(_load().orc_disjoint_paths(_ptr(r, _u64p), len(adj), u, v, limit))


def solve(adj: Sequence[int], k_start: int = 0, want_order: bool = True) -> Dict:
    """Iterative deepening from k_start: tw, order, and counters summed over k."""
    n = len(adj)
    r = rows(adj)
    order = np.full(n, -1, dtype=np.int32) if want_order else None
    cnt = np.zeros(4, dtype=np.int64)
    tw = _load().orc_solve(_ptr(r, _u64p), n, k_start, _ptr(order, _i32p) if order is not None else None,
                           _ptr(cnt, _i64p))
    if tw < 0:
        raise ValueError("invalid graph")
    return {"tw": tw, "order": order.tolist() if order is not None else None,
            "states_expanded": int(cnt[0]), "candidates": int(cnt[1]), "feasible": int(cnt[2]),
            "k_tried": int(cnt[3])}


def width_q(adj: Sequence[int], order: Sequence[int]) -> int:
    r = rows(adj)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    return int(_load().orc_width_q(_ptr(r, _u64p), len(adj), _ptr(o, _i32p)))


def width_elim(adj: Sequence[int], order: Sequence[int]) -> int:
    r = rows(adj)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    return int(_load().orc_width_elim(_ptr(r, _u64p), len(adj), _ptr(o, _i32p)))


def brute_force_tw(adj: Sequence[int]) -> int:
    r = rows(adj)
    tw = _load().orc_brute_force_tw(_ptr(r, _u64p), len(adj))
    if tw < 0:
        raise ValueError("brute force needs n <= 10")
    return int(tw)


def subset_dp(adj: Sequence[int], k: int) -> Dict:
    n = len(adj)
    r = rows(adj)
    ls = np.zeros(n + 1, dtype=np.int64)
    fs = np.zeros(n + 1, dtype=np.uint64)
    fx = np.zeros(n + 1, dtype=np.uint64)
    lv = ctypes.c_int(0)
    yes = _load().orc_subset_dp(_ptr(r, _u64p), n, k, _ptr(ls, _i64p), _ptr(fs, _u64p), _ptr(fx, _u64p),
                                ctypes.byref(lv))
    if yes < 0:
        raise ValueError("subset DP needs n <= 22")
    return {"yes": bool(yes), "levels": lv.value, "level_size": ls[: lv.value].tolist(),
            "fp_sum": fs[: lv.value].tolist(), "fp_xor": fx[: lv.value].tolist()}


def td_from_order(adj: Sequence[int], order: Sequence[int]):
    n = len(adj)
    r = rows(adj)
    w = r.shape[1]
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    parent = np.zeros(n, dtype=np.int32)
    bags = np.zeros((n, w), dtype=np.uint64)
    width = _load().orc_td_from_order(_ptr(r, _u64p), n, _ptr(o, _i32p), _ptr(parent, _i32p),
                                      _ptr(bags, _u64p))
    return int(width), parent, bags


def verify_td(adj: Sequence[int], parent: np.ndarray, bags: np.ndarray) -> int:
    """Width of a valid tree decomposition, or -1."""
    r = rows(adj)
    p = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    b = np.ascontiguousarray(np.asarray(bags, dtype=np.uint64).reshape(len(adj), -1))
    return int(_load().orc_verify_td(_ptr(r, _u64p), len(adj), _ptr(p, _i32p), _ptr(b, _u64p)))


def verify_td_rows(adj_rows: np.ndarray, n: int, parent: np.ndarray, bags: np.ndarray) -> int:
    p = np.ascontiguousarray(np.asarray(parent, dtype=np.int32))
    b = np.ascontiguousarray(np.asarray(bags, dtype=np.uint64))
    r = np.ascontiguousarray(adj_rows, dtype=np.uint64)
    return int(_load().orc_verify_td(_ptr(r, _u64p), n, _ptr(p, _i32p), _ptr(b, _u64p)))
