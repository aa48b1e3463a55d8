"""Warm-start network on the GPU against its FP64 CPU oracle (oracle/gnn_oracle.py),
then what training buys: a better starting factor than the random one."""
import numpy as np
import pytest

import workloads as W
from oracle import gnn_oracle as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402
from paper_2407_15049_gb300 import warmstart as WS  # noqa: E402

R_OUT = 12


@pytest.fixture(scope="module", autouse=True)
def _built():
    L.build()


def _setup(n=300, seed=1, r_star=5):
    inst = W.maxcut_instance(n, W.er_graph(n, 3 * n, seed, "pm1"))
    g = G.Graph(inst)
    dg = WS.device_graph(inst)
    R_star = np.random.default_rng(seed).standard_normal((n, r_star))
    R_star /= np.linalg.norm(R_star, axis=1, keepdims=True)
    return inst, g, dg, R_star


def _group_errs(got, want, r_out):
    out, at = [], 0
    for s in G.param_shapes(r_out):
        k = int(np.prod(s))
        a, b = got[at:at + k], want[at:at + k]
        out.append(float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-30))
        at += k
    return out


def test_edge_targets_match_oracle():
    inst, g, dg, R_star = _setup()
    Rd = torch.zeros((inst.n, 8), dtype=torch.float64, device="cuda")
    Rd[:, :5] = torch.as_tensor(R_star, device="cuda")
    t = WS.edge_targets(dg, Rd, 5).cpu().numpy().astype(np.float64)
    rp = inst.rowptr
    rows = np.repeat(np.arange(inst.n), np.diff(rp))
    off = inst.colind != rows
    assert np.allclose(t[off], G.edge_targets(g, R_star), atol=1e-6)
    assert np.all(t[~off] == 0.0)


def _group_cosines(got, want, r_out):
    out, at = [], 0
    for s in G.param_shapes(r_out):
        k = int(np.prod(s))
        a, b = got[at:at + k], want[at:at + k]
        out.append(float(a @ b) / max(float(np.linalg.norm(a) * np.linalg.norm(b)), 1e-300))
        at += k
    return out


@pytest.mark.parametrize("act,tol_r,tol_g", [("fp32", 2e-5, 2e-4), ("bf16", 4e-2, 0.1)])
def test_forward_loss_and_gradient_match_oracle(act, tol_r, tol_g):
    inst, g, dg, R_star = _setup()
    theta = G.init_params(R_OUT, 3).astype(np.float32)
    theta[np.arange(theta.size) % 7 == 0] += 0.05          # nonzero biases
    th64 = theta.astype(np.float64)
    x = G.node_features(g, 11)
    t_host = G.edge_targets(g, R_star)
    r_ref, _ = G.forward(g, x, th64, R_OUT)
    loss_ref, grad_ref, _ = G.loss_and_grad(g, x, th64, R_OUT, t_host)
    net = WS.WarmStart(R_OUT, act=act, theta=theta)
    try:
        R = net.predict(dg, feature_seed=11)
        r_gpu = R[:, :R_OUT].cpu().numpy()
        assert np.max(np.abs(r_gpu - r_ref)) <= tol_r
        assert np.allclose(np.linalg.norm(r_gpu, axis=1), 1.0, atol=1e-5)
        Rd = torch.zeros((inst.n, 8), dtype=torch.float64, device="cuda")
        Rd[:, :5] = torch.as_tensor(R_star, device="cuda")
        targets = WS.edge_targets(dg, Rd, 5)
        grad = torch.zeros(theta.size, dtype=torch.float32, device="cuda")
        loss = net.train_step(dg, targets, 0.0, feature_seed=11, grad_out=grad)
        assert np.array_equal(net.params, theta)                 # lr = 0: no update
        assert loss == pytest.approx(loss_ref, rel=tol_g)
        gg = grad.cpu().numpy().astype(np.float64)
        if act == "fp32":
            errs = _group_errs(gg, grad_ref, R_OUT)
            assert max(errs) <= tol_g, errs
        else:
            # bf16 activations (unit roundoff 2^-8) perturb every stored value; the
            # gradient must still point the same way, group by group
            rel = np.linalg.norm(gg - grad_ref) / np.linalg.norm(grad_ref)
            cos = _group_cosines(gg, grad_ref, R_OUT)
            assert rel <= tol_g and min(cos) >= 0.98, (rel, cos)
    finally:
        net.close()


def test_training_step_is_adam_on_the_gradient():
    inst, g, dg, R_star = _setup(200, 4)
    theta = G.init_params(R_OUT, 5).astype(np.float32)
    net = WS.WarmStart(R_OUT, act="fp32", theta=theta)
    try:
        Rd = torch.zeros((inst.n, 8), dtype=torch.float64, device="cuda")
        Rd[:, :5] = torch.as_tensor(R_star, device="cuda")
        targets = WS.edge_targets(dg, Rd, 5)
        grad = torch.zeros(theta.size, dtype=torch.float32, device="cuda")
        net.train_step(dg, targets, 1e-3, feature_seed=2, grad_out=grad)
        gr = grad.cpu().numpy().astype(np.float64)
        # first Adam step: theta - lr * g / (|g| + eps)  (bias corrections cancel)
        want = theta - 1e-3 * gr / (np.abs(gr) + 1e-8)
        assert np.allclose(net.params, want, rtol=1e-5, atol=1e-7)
    finally:
        net.close()


def _solve_factor(inst, r, seed):
    ctx = L.lorads_create(inst, L.default_params())
    try:
        res = L.lorads_solve(ctx, W.initial_factor(inst, r, seed))
        R, _ = L.lorads_get_solution(ctx, inst.n, inst.m)
    finally:
        L.lorads_destroy(ctx)
    assert res["status_name"] == "LORADS_OK"
    return R, res


def test_trained_network_starts_closer_to_the_optimum():
    """Trained on solver factors of small random graphs, the network's R0 has a
    smaller objective gap on held-out graphs than the random unit-row start."""
    r = R_OUT
    train, held = [], []
    for k in range(24):
        n = 150 + 25 * k
        inst = W.maxcut_instance(n, W.er_graph(n, 2 * n, 100 + k, "pm1"))
        R, _ = _solve_factor(inst, r, k)
        dg = WS.device_graph(inst)
        Rd = torch.zeros((n, L.padded_ld(r)), dtype=torch.float64, device="cuda")
        Rd[:, :R.shape[1]] = torch.as_tensor(R, device="cuda")
        train.append((dg, WS.edge_targets(dg, Rd, R.shape[1])))
    net = WS.WarmStart(r, act="bf16", seed=0)
    try:
        hist = net.fit(train, epochs=60, lr=3e-3, seed=1)
        assert hist[-1] < 0.7 * hist[0], hist[::10]
        gains, iters = [], []
        for k in range(3):
            n = 900 + 100 * k
            inst = W.maxcut_instance(n, W.er_graph(n, 2 * n, 900 + k, "pm1"))
            R_opt, res = _solve_factor(inst, r, 50 + k)
            opt = res["primal_obj"]
            P = inst
            dg = WS.device_graph(inst)
            R0 = net.predict(dg)[:, :r].cpu().numpy()
            Rr = W.initial_factor(inst, r, 7 + k)
            from oracle import lorads_oracle as O
            Pb = O.Problem(P)
            gap_net = O.objective(Pb, R0) - opt
            gap_rand = O.objective(Pb, Rr) - opt
            gains.append(gap_rand / gap_net)
            assert gap_net < gap_rand, (gap_net, gap_rand)
            # started from the network's factor, the solve reaches the same optimum
            # (both at rel. KKT 1e-5 with err2); the iteration counts are reported
            ctx = L.lorads_create(inst, L.default_params(compute_err2=1))
            try:
                res_w = L.lorads_solve(ctx, R0)
                res_c = L.lorads_solve(ctx, Rr)
            finally:
                L.lorads_destroy(ctx)
            for rr in (res_w, res_c):
                assert rr["status_name"] == "LORADS_OK", rr
                assert max(rr["err1"], abs(rr["err3"]), rr["err2"]) <= 1e-5
                assert rr["primal_obj"] == pytest.approx(opt, rel=1e-4)
            iters.append((res_w["inner_iters"], res_c["inner_iters"]))
    finally:
        net.close()
    print("objective-gap ratio random / network:", gains, "iterations network / random start:", iters)
