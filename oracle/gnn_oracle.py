"""CPU oracle of the learned warm start (test infrastructure only).

This is the plain FP64 definition of the warm-start network that the GPU
library trains and runs (include/lorads.h, lorads_gnn_*).  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it;
the product path never imports it.

The paper has no such network: its solver starts every run from a random
factor (Sec. 2, App. A.1 draws the new columns at random).  The network
predicts a starting factor R0 for the Burer-Monteiro form X = R R^T of the
SDP (Eq. (1.1)) from the structure of C alone, and is trained on the factors
R* that the plain solver returns.  Its definition (all readings of this
module, since the paper fixes none of it):

* Graph: the off-diagonal pattern of C with signed weights w_ij = C_ij;
  deg_i = #{j != i : C_ij stored}, s_i = sum_j |w_ij|.
* Node features (F = 16): [1, log(1 + deg_i) / 4, sum_j w_ij / s_i,
  C_ii / s_i, 12 standard normals] (ratios taken as 0 when s_i = 0); the
  normals are the counter-based SplitMix64 / Box-Muller draws of
  ``gaussian_columns(n, 12, seed, FEATURE_STREAM)``.
* Three message-passing layers, hidden width H = 32:
      m_i = sum_j (w_ij / s_i) h_j          (0 when s_i = 0)
      h_i <- relu(W_s h_i + W_n m_i + b).
* Output: o_i = W_o h_i + b_o in R^r_out, r_hat_i = o_i / ||o_i||
  (unit rows: feasible for the MaxCut constraints X_ii = 1).
* Loss: mean over the edges {i < j} of (r_hat_i . r_hat_j - X*_ij)^2 with
  X*_ij = r*_i . r*_j from the solver's factor.  It depends on R_hat only
  through its Gram matrix, so it is invariant to rotations of the output
  space (R* is defined only up to R* Q).
* Parameters as one flat vector, in this order: for each layer l = 1..3,
  W_s (H x F_in, row-major), W_n (H x F_in), b (H); then W_o (r_out x H), b_o.
"""
from __future__ import annotations

import math

import numpy as np

from .lorads_oracle import gaussian_columns

__all__ = ["FEATURES", "HIDDEN", "LAYERS", "FEATURE_STREAM", "param_count", "param_shapes",
           "init_params", "flatten", "unflatten", "Graph", "node_features", "aggregate",
           "aggregate_transpose", "forward", "edge_targets", "edge_loss", "backward", "loss_and_grad"]

FEATURES = 16
N_STRUCT = 4
HIDDEN = 32
LAYERS = 3
FEATURE_STREAM = 0x474E4E                 # stream of the random node features


def param_shapes(r_out: int):
    shapes = []
    f_in = FEATURES
    for _ in range(LAYERS):
        shapes += [(HIDDEN, f_in), (HIDDEN, f_in), (HIDDEN,)]
        f_in = HIDDEN
    shapes += [(r_out, HIDDEN), (r_out,)]
    return shapes


def param_count(r_out: int) -> int:
    return int(sum(np.prod(s) for s in param_shapes(r_out)))


def unflatten(theta: np.ndarray, r_out: int):
    out, at = [], 0
    for s in param_shapes(r_out):
        k = int(np.prod(s))
        out.append(np.asarray(theta[at:at + k], dtype=np.float64).reshape(s))
        at += k
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def init_params(r_out: int, seed: int) -> np.ndarray:
    """Glorot-style uniform weights, zero biases (numpy generator; a starting point only)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in param_shapes(r_out):
        if len(s) == 2:
            lim = math.sqrt(6.0 / (s[0] + s[1]))
            parts.append(rng.uniform(-lim, lim, s))
        else:
            parts.append(np.zeros(s))
    return flatten(parts)


class Graph:
    """Off-diagonal pattern of C (CSR) with w_ij = C_ij, plus deg, s and diag."""

    def __init__(self, inst):
        n = int(inst.n)
        rp = np.asarray(inst.rowptr, dtype=np.int64)
        ci = np.asarray(inst.colind, dtype=np.int64)
        cv = np.asarray(inst.val, dtype=np.float64)
        self.n = n
        rows = np.repeat(np.arange(n), np.diff(rp))
        off = ci != rows
        self.diag = np.zeros(n)
        np.add.at(self.diag, rows[~off], cv[~off])
        self.rows = rows[off]
        self.cols = ci[off]
        self.w = cv[off]
        self.deg = np.bincount(self.rows, minlength=n).astype(np.float64)
        self.s = np.zeros(n)
        np.add.at(self.s, self.rows, np.abs(self.w))
        self.wsum = np.zeros(n)
        np.add.at(self.wsum, self.rows, self.w)
        self.inv_s = np.where(self.s > 0, 1.0 / np.where(self.s > 0, self.s, 1.0), 0.0)
        upper = self.rows < self.cols
        self.n_edges = int(np.count_nonzero(upper))


def node_features(g: Graph, seed: int) -> np.ndarray:
    x = np.zeros((g.n, FEATURES))
    x[:, 0] = 1.0
    x[:, 1] = np.log1p(g.deg) / 4.0
    x[:, 2] = g.wsum * g.inv_s
    x[:, 3] = g.diag * g.inv_s
    x[:, N_STRUCT:] = gaussian_columns(g.n, FEATURES - N_STRUCT, seed, FEATURE_STREAM)
    return x


def aggregate(g: Graph, h: np.ndarray) -> np.ndarray:
    """m_i = sum_j (w_ij / s_i) h_j, by an explicit loop over the stored entries."""
    m = np.zeros_like(h)
    np.add.at(m, g.rows, g.w[:, None] * h[g.cols])
    return m * g.inv_s[:, None]


def aggregate_transpose(g: Graph, v: np.ndarray) -> np.ndarray:
    """The adjoint of ``aggregate``: out_j = sum_i (w_ij / s_i) v_i."""
    out = np.zeros_like(v)
    np.add.at(out, g.cols, (g.w * g.inv_s[g.rows])[:, None] * v[g.rows])
    return out


def forward(g: Graph, x: np.ndarray, theta: np.ndarray, r_out: int):
    """Returns (r_hat, cache)."""
    parts = unflatten(theta, r_out)
    hs, ms, us = [x], [], []
    h = x
    for l in range(LAYERS):
        Ws, Wn, b = parts[3 * l: 3 * l + 3]
        m = aggregate(g, h)
        u = h @ Ws.T + m @ Wn.T + b
        h = np.maximum(u, 0.0)
        ms.append(m)
        us.append(u)
        hs.append(h)
    Wo, bo = parts[3 * LAYERS:]
    o = h @ Wo.T + bo
    nrm = np.linalg.norm(o, axis=1)
    r_hat = o / nrm[:, None]
    return r_hat, dict(hs=hs, ms=ms, us=us, o=o, nrm=nrm, r_hat=r_hat, parts=parts)


def edge_targets(g: Graph, R_star: np.ndarray) -> np.ndarray:
    """X*_ij = r*_i . r*_j on every stored off-diagonal entry (CSR order of the off pattern)."""
    return np.einsum("ec,ec->e", R_star[g.rows], R_star[g.cols])


def edge_loss(g: Graph, r_hat: np.ndarray, target: np.ndarray):
    """Mean over edges i < j of (r_hat_i . r_hat_j - X*_ij)^2 and its gradient in r_hat."""
    dots = np.einsum("ec,ec->e", r_hat[g.rows], r_hat[g.cols])
    diff = dots - target
    upper = g.rows < g.cols
    ne = max(g.n_edges, 1)
    loss = float(np.sum(diff[upper] ** 2)) / ne
    # each edge appears as (i, j) and (j, i): d/dr_i of (r_i.r_j - t)^2 = 2 diff r_j
    d = np.zeros_like(r_hat)
    np.add.at(d, g.rows, (2.0 / ne) * diff[:, None] * r_hat[g.cols])
    return loss, d


def backward(g: Graph, cache: dict, d_rhat: np.ndarray, r_out: int) -> np.ndarray:
    """Gradient of the loss in the flat parameter vector (reverse-mode, by hand)."""
    parts = cache["parts"]
    r_hat, nrm = cache["r_hat"], cache["nrm"]
    # r_hat = o / ||o||:  do = (d - r_hat (r_hat . d)) / ||o||
    do = (d_rhat - r_hat * np.sum(r_hat * d_rhat, axis=1, keepdims=True)) / nrm[:, None]
    h = cache["hs"][-1]
    Wo = parts[3 * LAYERS]
    grads = [None] * len(parts)
    grads[3 * LAYERS] = do.T @ h
    grads[3 * LAYERS + 1] = do.sum(axis=0)
    dh = do @ Wo
    for l in reversed(range(LAYERS)):
        Ws, Wn, _ = parts[3 * l: 3 * l + 3]
        u, m, h_in = cache["us"][l], cache["ms"][l], cache["hs"][l]
        du = dh * (u > 0)
        grads[3 * l] = du.T @ h_in
        grads[3 * l + 1] = du.T @ m
        grads[3 * l + 2] = du.sum(axis=0)
        dh = du @ Ws + aggregate_transpose(g, du @ Wn)
    return flatten(grads)


def loss_and_grad(g: Graph, x: np.ndarray, theta: np.ndarray, r_out: int, target: np.ndarray):
    r_hat, cache = forward(g, x, theta, r_out)
    loss, d = edge_loss(g, r_hat, target)
    return loss, backward(g, cache, d, r_out), r_hat
