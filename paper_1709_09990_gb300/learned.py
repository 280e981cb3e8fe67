"""Learned starting bound for the k sweep.

The paper's solver sweeps k upward and the first yes is the treewidth
(arXiv 1709.09990, Section 3.1).  Here a 12-32-1 ReLU network, trained on
exact treewidths produced by libtw itself, proposes the starting k; libtw then
runs decide at the proposal and one below and walks up or down until a yes at
tw and a no at tw-1 (or tw equal to the lower bound) certify the answer, so
every answer stays exact.  Features, training (forward, backward, Adam) and
inference all run in libtw's kernels; this module only draws the seeded
initial weights and epoch orders and marshals arrays.

Target: y = tw / n.  Proposal: k = round(n * yhat + offset), clamped by libtw
to [lower bound, n - 1]; a negative offset biases proposals downward, where a
wrong guess costs a cheap "no" run instead of an expensive "yes" run above tw.
"""
from __future__ import annotations

import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import graphgen as gg
from . import native

N_PARAMS = native.N_PARAMS


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = gg.Rng(seed)
    p = np.zeros(N_PARAMS, np.float32)
    b1 = 1.0 / math.sqrt(12.0)
    b2 = 1.0 / math.sqrt(32.0)
    for i in range(32 * 12):
        p[i] = (2.0 * rng.uniform() - 1.0) * b1
    for i in range(32):
        p[32 * 12 + 32 + i] = (2.0 * rng.uniform() - 1.0) * b2
    return p


def epoch_orders(count: int, epochs: int, seed: int) -> np.ndarray:
    """epochs x count sample orders (seeded Fisher-Yates shuffles)."""
    rng = gg.Rng(seed)
    out = np.empty((epochs, count), np.int32)
    base = np.arange(count, dtype=np.int32)
    for e in range(epochs):
        perm = base.copy()
        for i in range(count - 1, 0, -1):
            j = int(math.floor(rng.uniform() * (i + 1)))
            perm[i], perm[j] = perm[j], perm[i]
        out[e] = perm
    return out


def label(ctx: native.Context, graphs: Sequence) -> Dict:
    """Features (device) and exact treewidths (batched device solve)."""
    t0 = time.perf_counter()
    feats = ctx.features(graphs)
    res = ctx.solve_batch(graphs, want_orders=False)
    return {"x": feats, "tw": res["tw"], "status": res["per_graph_status"],
            "n": np.array([len(g) for g in graphs], np.int32), "seconds": time.perf_counter() - t0,
            "stats": res["stats"]}


def train(ctx: native.Context, x: np.ndarray, tw: np.ndarray, n: np.ndarray, epochs: int = 60,
          minibatch: int = 256, lr: float = 3e-3, seed: int = 7) -> Dict:
    """Minibatch Adam on the device; returns parameters and the loss curve."""
    y = (tw.astype(np.float64) / n.astype(np.float64)).astype(np.float32)
    params = init_params(seed)
    perm = epoch_orders(len(y), epochs, seed + 1)
    loss = ctx.mlp_train(params, x, y, minibatch, perm, lr=lr)
    return {"params": params, "loss": loss}


def propose(ctx: native.Context, params: np.ndarray, x: np.ndarray, n: np.ndarray,
            offset: float = 0.0) -> np.ndarray:
    """Proposed starting bound per graph (float, rounded inside libtw)."""
    yhat = ctx.mlp_forward(params, x)
    return (yhat.astype(np.float64) * n + offset).astype(np.float32)


def choose_offset(pred_k: np.ndarray, tw: np.ndarray, lb: np.ndarray,
                  candidates=(-2.0, -1.5, -1.0, -0.5, 0.0, 0.5)) -> float:
    """Offset minimising the expected number of decide runs on labelled data:
    a proposal k0 >= tw costs k0 - tw + 1 yes runs down to tw plus one no run
    at tw - 1 unless tw is the lower bound; k0 < tw costs tw - k0 + 1 runs (no
    runs up to tw - 1, then the yes).  k0 is clamped to the lower bound.  Runs
    above tw are the expensive ones, so they carry a small extra penalty."""
    best, best_cost = 0.0, None
    for off in candidates:
        k0 = np.maximum(np.rint(pred_k + off), lb)
        cost = np.where(k0 >= tw, (k0 - tw + 1) + (tw > lb), tw - k0 + 1)
        c = float(cost.mean()) + 0.25 * float((k0 > tw).mean())
        if best_cost is None or c < best_cost:
            best, best_cost = off, c
    return best
