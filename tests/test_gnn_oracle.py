"""Pins of the warm-start network oracle (oracle/gnn_oracle.py) to facts fixed by
its definition and by calculus, independent of the way the oracle computes them."""
import numpy as np
import pytest

import workloads as W
from oracle import gnn_oracle as G
from oracle import lorads_oracle as O

R_OUT = 6


def _graph(n=14, seed=0, weights="pm1"):
    inst = W.maxcut_instance(n, W.er_graph(n, 3 * n, seed, weights))
    return inst, G.Graph(inst)


def test_aggregate_equals_dense_row_normalised_product():
    inst, g = _graph(20, 1)
    C = O.Problem(inst).C.toarray()
    A = C - np.diag(np.diag(C))
    s = np.abs(A).sum(axis=1)
    An = A / np.where(s > 0, s, 1.0)[:, None]
    h = np.random.default_rng(0).standard_normal((20, 5))
    assert np.allclose(G.aggregate(g, h), An @ h, rtol=1e-13, atol=1e-13)


def test_aggregate_transpose_is_the_adjoint():
    _, g = _graph(25, 2)
    rng = np.random.default_rng(1)
    h, v = rng.standard_normal((25, 7)), rng.standard_normal((25, 7))
    assert np.sum(G.aggregate(g, h) * v) == pytest.approx(np.sum(h * G.aggregate_transpose(g, v)), rel=1e-12)


def test_features_of_a_maxcut_instance():
    """For C = -L/4 the diagonal feature is the negated signed balance, and the
    degree feature counts neighbours."""
    inst, g = _graph(30, 3)
    x = G.node_features(g, seed=5)
    assert np.all(x[:, 0] == 1.0)
    i, j, _ = inst.meta["edges"]
    deg = np.bincount(np.concatenate([i, j]), minlength=30)
    assert np.allclose(x[:, 1], np.log1p(deg) / 4.0)
    has = deg > 0
    assert np.allclose(x[has, 3], -x[has, 2])
    assert np.all(np.abs(x[:, 2]) <= 1.0 + 1e-12)
    assert np.array_equal(x[:, 4:], O.gaussian_columns(30, 12, 5, G.FEATURE_STREAM))


def test_rows_are_unit_and_isolated_nodes_are_handled():
    inst = W.maxcut_instance(9, (np.array([0, 1]), np.array([1, 2]), np.array([1.0, -1.0])))
    g = G.Graph(inst)
    theta = G.init_params(R_OUT, 3)
    r_hat, _ = G.forward(g, G.node_features(g, 1), theta, R_OUT)
    assert np.allclose(np.linalg.norm(r_hat, axis=1), 1.0)
    assert g.n_edges == 2 and np.all(g.inv_s[3:] == 0.0)


def test_constant_network_closed_form_loss():
    """All weights zero, biases set: every node gets the same output row, every
    edge dot is 1, and the loss is the mean of (1 - X*_ij)^2."""
    _, g = _graph(16, 4)
    parts = G.unflatten(np.zeros(G.param_count(R_OUT)), R_OUT)
    parts[2][:] = 0.5                       # b of layer 1 -> h = relu(0.5) at layer 1
    parts[-1][:] = np.arange(1, R_OUT + 1)  # b_o
    theta = G.flatten(parts)
    r_hat, _ = G.forward(g, G.node_features(g, 2), theta, R_OUT)
    assert np.allclose(r_hat, r_hat[0])
    t = np.random.default_rng(3).uniform(-1, 1, len(g.rows))       # one value per stored entry
    loss, _ = G.edge_loss(g, r_hat, t)
    upper = g.rows < g.cols
    assert loss == pytest.approx(np.mean((1.0 - t[upper]) ** 2), rel=1e-12)


def test_loss_is_zero_at_own_gram_and_rotation_invariant():
    _, g = _graph(18, 5)
    theta = G.init_params(R_OUT, 7)
    x = G.node_features(g, 9)
    r_hat, _ = G.forward(g, x, theta, R_OUT)
    t_own = G.edge_targets(g, r_hat)
    assert G.edge_loss(g, r_hat, t_own)[0] == pytest.approx(0.0, abs=1e-28)
    R_star = np.random.default_rng(2).standard_normal((18, 4))
    R_star /= np.linalg.norm(R_star, axis=1, keepdims=True)
    t = G.edge_targets(g, R_star)
    loss = G.edge_loss(g, r_hat, t)[0]
    Q, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((R_OUT, R_OUT)))
    parts = G.unflatten(theta, R_OUT)
    parts[-2] = Q @ parts[-2]
    parts[-1] = Q @ parts[-1]
    r_rot, _ = G.forward(g, x, G.flatten(parts), R_OUT)
    assert np.allclose(r_rot, r_hat @ Q.T)
    assert G.edge_loss(g, r_rot, t)[0] == pytest.approx(loss, rel=1e-12)


def test_permutation_equivariance():
    inst, g = _graph(15, 6)
    theta = G.init_params(R_OUT, 8)
    x = G.node_features(g, 3)
    r_hat, _ = G.forward(g, x, theta, R_OUT)
    perm = np.random.default_rng(5).permutation(15)
    inv = np.argsort(perm)
    i, j, w = inst.meta["edges"]
    inst2 = W.maxcut_instance(15, (inv[i], inv[j], w))      # node k of inst is node inv[k] of inst2
    g2 = G.Graph(inst2)
    r2, _ = G.forward(g2, x[perm], theta, R_OUT)
    assert np.allclose(r2, r_hat[perm], atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_central_differences(seed):
    _, g = _graph(12, 10 + seed)
    theta = G.init_params(R_OUT, seed) + 0.05           # nonzero biases: active relus both ways
    x = G.node_features(g, seed)
    R_star = np.random.default_rng(seed).standard_normal((12, 3))
    R_star /= np.linalg.norm(R_star, axis=1, keepdims=True)
    t = G.edge_targets(g, R_star)
    loss, grad, _ = G.loss_and_grad(g, x, theta, R_OUT, t)
    rng = np.random.default_rng(100 + seed)
    # every parameter group, several entries each
    idx, at = [], 0
    for s in G.param_shapes(R_OUT):
        k = int(np.prod(s))
        idx += list(at + rng.choice(k, size=min(k, 6), replace=False))
        at += k
    eps = 1e-6
    for q in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[q] += eps
        tm[q] -= eps
        lp = G.loss_and_grad(g, x, tp, R_OUT, t)[0]
        lm = G.loss_and_grad(g, x, tm, R_OUT, t)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad[q]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (q, fd, grad[q])
