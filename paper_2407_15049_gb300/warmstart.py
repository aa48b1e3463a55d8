"""Learned warm start around the lorads_gnn_* entry points.

Host-side plumbing only: device copies of a graph, the parameter
initialisation, and the epoch loop over training graphs.  The forward pass,
the loss, the backward pass and the Adam step all run in the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

from . import _native as N

FEATURES, HIDDEN, LAYERS = 16, 32, 3


def param_shapes(r_out: int):
    shapes, f_in = [], FEATURES
    for _ in range(LAYERS):
        shapes += [(HIDDEN, f_in), (HIDDEN, f_in), (HIDDEN,)]
        f_in = HIDDEN
    return shapes + [(r_out, HIDDEN), (r_out,)]


def init_params(r_out: int, seed: int) -> np.ndarray:
    """Glorot-uniform matrices and zero biases, in the library's parameter order."""
    rng = np.random.default_rng(seed)
    out = []
    for s in param_shapes(r_out):
        if len(s) == 2:
            lim = math.sqrt(6.0 / (s[0] + s[1]))
            out.append(rng.uniform(-lim, lim, s).ravel())
        else:
            out.append(np.zeros(s[0]))
    return np.concatenate(out).astype(np.float32)


def device_graph(inst, device: str = "cuda") -> dict:
    """Device CSR of C (int64 rowptr, int32 colind, float64 val) and its edge count."""
    import torch
    rp = np.asarray(inst.rowptr, dtype=np.int64)
    ci = np.asarray(inst.colind, dtype=np.int32)
    rows = np.repeat(np.arange(inst.n), np.diff(rp))
    n_edges = int(np.count_nonzero(rows < ci))
    return dict(n=int(inst.n), n_edges=max(n_edges, 1),
                rowptr=torch.as_tensor(rp, device=device),
                colind=torch.as_tensor(ci, device=device),
                val=torch.as_tensor(np.asarray(inst.val, dtype=np.float64), device=device))


def edge_targets(graph: dict, R, r: int):
    """X*_ij = r_i . r_j for every stored entry of C, from a factor R (n x ld, device FP64)."""
    import torch
    t = torch.empty(graph["colind"].numel(), dtype=torch.float32, device=R.device)
    N.lorads_gnn_edge_targets(graph, R, r, R.shape[1], t, torch.cuda.current_stream().cuda_stream)
    return t


class WarmStart:
    """The warm-start network on the GPU (r_out outputs, bf16 or float activations)."""

    def __init__(self, r_out: int = 24, act: str = "bf16", seed: int = 0, theta: np.ndarray | None = None,
                 stream: int | None = None):
        self.r_out = int(r_out)
        self.act = N.LORADS_BF16 if act == "bf16" else N.LORADS_FP32
        th = init_params(r_out, seed) if theta is None else np.asarray(theta, dtype=np.float32)
        self.net = N.lorads_gnn_create(r_out, th, self.act, stream)

    def close(self):
        N.lorads_gnn_destroy(self.net)
        self.net = None

    def __del__(self):
        if getattr(self, "net", None):
            self.close()

    @property
    def params(self) -> np.ndarray:
        return N.lorads_gnn_get_params(self.net, self.r_out)

    @params.setter
    def params(self, theta: np.ndarray):
        N.lorads_gnn_set_params(self.net, theta)

    def predict(self, graph: dict, feature_seed: int = 0, ld: int | None = None):
        """R0 (n x ld, device FP64, unit rows in columns 0..r_out-1)."""
        import torch
        ld = ld or N.padded_ld(self.r_out)
        R = torch.empty((graph["n"], ld), dtype=torch.float64, device=graph["rowptr"].device)
        N.lorads_gnn_predict(self.net, graph, feature_seed, R, ld)
        return R

    def train_step(self, graph: dict, targets, lr: float, feature_seed: int = 0, grad_out=None,
                   want_loss: bool = True):
        return N.lorads_gnn_train_step(self.net, graph, feature_seed, targets, lr, grad_out, want_loss)

    def fit(self, samples, epochs: int, lr: float, seed: int = 0, feature_seed: int = 0):
        """samples: list of (graph, targets).  One Adam step per graph, graphs shuffled
        each epoch; returns the mean loss of every epoch."""
        rng = np.random.default_rng(seed)
        hist = []
        for _ in range(epochs):
            order = rng.permutation(len(samples))
            tot = 0.0
            for k in order:
                g, t = samples[k]
                tot += self.train_step(g, t, lr, feature_seed)
            hist.append(tot / len(samples))
        return hist


def train_on_solved(instances, r: int, epochs: int = 40, lr: float = 3e-3, prec: int = N.LORADS_MIXED,
                    seed: int = 0, time_limit: float = 60.0):
    """Solves the training instances with the batched solver (one launch, rank r) and
    fits a network to the factors it returns.  Returns (network, info dict)."""
    import time
    import torch
    t0 = time.perf_counter()
    b = N.lorads_batch_create(instances, N.default_params(prec=prec, time_limit=time_limit),
                              r0=[r] * len(instances))
    try:
        res, stats = N.lorads_batch_solve(b, len(instances))
        samples = []
        for i, inst in enumerate(instances):
            if res[i]["status"] != 0:
                continue
            R, _ = N.lorads_batch_get_solution(b, i, inst.n, inst.m)
            dg = device_graph(inst)
            Rd = torch.zeros((inst.n, N.padded_ld(R.shape[1])), dtype=torch.float64, device=dg["rowptr"].device)
            Rd[:, :R.shape[1]] = torch.as_tensor(R, device=Rd.device)
            samples.append((dg, edge_targets(dg, Rd, R.shape[1])))
    finally:
        N.lorads_batch_destroy(b)
    t1 = time.perf_counter()
    net = WarmStart(r, act="bf16", seed=seed, stream=torch.cuda.current_stream().cuda_stream)
    hist = []
    for ep in range(epochs):
        hist += net.fit(samples, epochs=1, lr=lr if ep < 0.7 * epochs else lr / 3, seed=seed + ep)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"graphs": len(instances), "solved": len(samples), "solve_s": t1 - t0, "train_s": t2 - t1,
                 "epochs": epochs, "loss_first": hist[0] if hist else None, "loss_last": hist[-1] if hist else None,
                 "batch_stats": stats}
