"""Pins of the ADMM-stage oracle (Sec. 2.2) against the definitions.

* The operator frakA_V against the dense n r x n r matrix of Eq. (2.4),
  assembled from the dense A_k (brute-force definition).
* The solution of the block system is a stationary point of L_rho: central
  finite differences of L_rho itself (not of the system's formula) vanish,
  for the U step and for the V step.
* Conjugate gradients (Algorithm 2) reach the dense solution.
* Every block step lowers L_rho (each block problem is a convex quadratic and
  CG from the current iterate only lowers it).
* The two-stage solver reaches closed-form MaxCut SDP values, the ALM-only
  optimum, and the matrix-completion optimum 2 ||M||_*.
"""
from pathlib import Path

import numpy as np
import pytest

import workloads as W
from oracle import admm_oracle as A
from oracle import lorads_oracle as O


def _instances():
    return {
        "maxcut_er": W.maxcut_instance(12, W.er_graph(12, 25, 3, "pm1")),
        "mc": W.mc_instance(5, 6, 2, 18, seed=4),
    }


INST = _instances()


def _dense_operator(P, V, rho):
    """rho (sum_k vec(A_k V) vec(A_k V)^T + I), vec = row-major flattening."""
    nr = V.size
    M = rho * np.eye(nr)
    for k in range(P.m):
        v = (P.A_dense(k) @ V).reshape(-1)
        M += rho * np.outer(v, v)
    return M


@pytest.mark.parametrize("name", list(INST))
def test_operator_matches_dense_system(name):
    P = O.Problem(INST[name])
    rng = np.random.default_rng(1)
    V = rng.standard_normal((P.n, 3))
    X = rng.standard_normal((P.n, 3))
    rho = 1.7
    want = (_dense_operator(P, V, rho) @ X.reshape(-1)).reshape(X.shape)
    np.testing.assert_allclose(A.system_operator(P, V, X, rho), want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name", list(INST))
def test_split_lagrangian_reduces_to_the_alm_lagrangian(name):
    """With U = V the penalty term vanishes and Eq. (1.3) is Eq. (1.2)."""
    P = O.Problem(INST[name])
    rng = np.random.default_rng(4)
    R = rng.standard_normal((P.n, 3))
    y = rng.standard_normal(P.m)
    assert A.split_lagrangian(P, R, R, y, 1.3) == pytest.approx(O.lagrangian(P, R, y, 1.3), rel=1e-13)
    U = R + 0.1 * rng.standard_normal(R.shape)
    d = A.split_lagrangian(P, U, R, y, 1.3) - A.split_lagrangian(P, U, R, y, 0.0)
    z = O.constraint_map(P, U, R) - P.b
    assert d == pytest.approx(0.65 * (float(z @ z) + float(np.sum((U - R) ** 2))), rel=1e-12)


def _fd_grad(f, X, h=1e-6):
    G = np.zeros_like(X)
    for idx in np.ndindex(*X.shape):
        E = np.zeros_like(X)
        E[idx] = h
        G[idx] = (f(X + E) - f(X - E)) / (2 * h)
    return G


@pytest.mark.parametrize("name", list(INST))
def test_block_solutions_are_stationary_points_of_the_lagrangian(name):
    P = O.Problem(INST[name])
    rng = np.random.default_rng(2)
    U = rng.standard_normal((P.n, 2))
    V = rng.standard_normal((P.n, 2))
    y = rng.standard_normal(P.m)
    rho = 2.5
    # U step: dense solve of Eq. (2.3) with V fixed
    Us = np.linalg.solve(_dense_operator(P, V, rho), A.system_rhs(P, V, y, rho).reshape(-1)).reshape(U.shape)
    g = _fd_grad(lambda X: A.split_lagrangian(P, X, V, y, rho), Us)
    scale = 1 + np.abs(_fd_grad(lambda X: A.split_lagrangian(P, X, V, y, rho), U)).max()
    assert np.abs(g).max() <= 1e-6 * scale
    # V step: the same system with U and V exchanged
    Vs = np.linalg.solve(_dense_operator(P, Us, rho), A.system_rhs(P, Us, y, rho).reshape(-1)).reshape(V.shape)
    g = _fd_grad(lambda X: A.split_lagrangian(P, Us, X, y, rho), Vs)
    assert np.abs(g).max() <= 1e-6 * scale


@pytest.mark.parametrize("name", list(INST))
def test_cg_reaches_the_dense_solution(name):
    P = O.Problem(INST[name])
    rng = np.random.default_rng(3)
    V = rng.standard_normal((P.n, 3))
    y = rng.standard_normal(P.m)
    rho = 0.8
    rhs = A.system_rhs(P, V, y, rho)
    want = np.linalg.solve(_dense_operator(P, V, rho), rhs.reshape(-1)).reshape(V.shape)
    X, steps = A.cg(P, V, np.zeros_like(V), rhs, rho, cg_rel=1e-13, cg_max=4 * V.size)
    assert 0 < steps <= 4 * V.size
    np.testing.assert_allclose(X, want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("name", list(INST))
def test_cg_terminates_within_the_distinct_eigenvalue_count(name):
    """frakA_V = rho I + rho sum_k v_k v_k^T has at most m + 1 distinct
    eigenvalues, so exact-arithmetic CG (Algorithm 2) ends within m + 1 steps;
    in FP64 it is at the dense solution to ~1e-8 after them (a wrong alpha or
    beta does not)."""
    P = O.Problem(INST[name])
    rng = np.random.default_rng(8)
    V = rng.standard_normal((P.n, 3))
    y = rng.standard_normal(P.m)
    rho = 1.1
    rhs = A.system_rhs(P, V, y, rho)
    assert P.m + 1 < V.size                        # fewer steps than unknowns
    want = np.linalg.solve(_dense_operator(P, V, rho), rhs.reshape(-1)).reshape(V.shape)
    X, steps = A.cg(P, V, np.zeros_like(V), rhs, rho, cg_rel=0.0, cg_max=P.m + 1)
    assert np.abs(X - want).max() <= 1e-8 * np.abs(want).max()


def test_block_steps_lower_the_lagrangian():
    P = O.Problem(INST["maxcut_er"])
    R = W.initial_factor(INST["maxcut_er"], 4, 5)
    U, V = R.copy(), R.copy()
    y = np.zeros(P.m)
    rho = 3.0
    prm = A.AdmmParams()
    for _ in range(15):
        L0 = A.split_lagrangian(P, U, V, y, rho)
        U, _ = A.cg(P, V, U, A.system_rhs(P, V, y, rho), rho, prm.cg_rel, prm.cg_max)
        L1 = A.split_lagrangian(P, U, V, y, rho)
        V, _ = A.cg(P, U, V, A.system_rhs(P, U, y, rho), rho, prm.cg_rel, prm.cg_max)
        L2 = A.split_lagrangian(P, U, V, y, rho)
        assert L1 <= L0 + 1e-12 * abs(L0) and L2 <= L1 + 1e-12 * abs(L1)
        y = y - rho * (O.constraint_map(P, U, V) - P.b)


def _closed_forms():
    path = Path(__file__).resolve().parent / "golden" / "maxcut_sdp_values.txt"
    rows = []
    for line in path.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            fam, size, value = line.split()[:3]
            rows.append((fam, int(size), float(value)))
    return [r for r in rows if r[1] in (7, 10, 5, 4)]


@pytest.mark.parametrize("fam,size,value", _closed_forms())
def test_two_stage_reaches_closed_form_values(fam, size, value):
    if fam == "complete":
        n, edges, r = size, W.complete_graph(size), W.rank_log2(size)
    elif fam == "odd_cycle":
        n, edges, r = size, W.cycle_graph(size), 3
    else:
        n, edges, r = size * size, W.bipartite_torus_graph(size), W.rank_log2(size * size)
    inst = W.maxcut_instance(n, edges)
    P = O.Problem(inst)
    res = A.solve_two_stage(P, W.initial_factor(inst, r, 1), admm=A.AdmmParams(switch_err1=1e-1))
    assert res["status"] == "ok" and res["stage"] == "admm" and res["admm_iters"] > 0
    assert -res["primal_obj"] == pytest.approx(value, rel=1e-5)


def test_two_stage_is_certified_against_the_alm_optimum():
    """At rel. KKT 1e-5 the two stages may stop at different near-optimal
    points (the stop test bounds err1 and err3, not sigma_min): each result's
    dual bound b^T y + n sigma_min(C - A*(y)) must lie below the other's
    objective (weak duality, trace X = n), and both pass err2 <= 1e-5."""
    n = 60
    inst = W.maxcut_instance(n, W.er_graph(n, 200, 11, "pm1"))
    P = O.Problem(inst)
    R0 = W.initial_factor(inst, 10, 2)
    ref = O.solve(P, R0, O.Params())
    assert ref["status"] == "ok"
    for switch in (1e-2, 1e-3):
        res = A.solve_two_stage(P, R0, admm=A.AdmmParams(switch_err1=switch))
        assert res["status"] == "ok" and res["stage"] == "admm"
        e = O.errors(P, res["R"], res["y"], with_err2=True)
        assert e["err1"] <= 1e-5 and abs(e["err3"]) <= 1e-5 and e["err2"] <= 1e-5
        slack = 1e-4                                # primal infeasibility of the iterates (err1 <= 1e-5)
        lower_admm = float(P.b @ res["y"]) + n * min(0.0, O.sigma_min(P, res["y"]))
        lower_ref = float(P.b @ ref["y"]) + n * min(0.0, O.sigma_min(P, ref["y"]))
        assert lower_admm <= ref["primal_obj"] + slack
        assert lower_ref <= res["primal_obj"] + slack
        assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=1e-4)


def test_two_stage_matrix_completion_recovers_nuclear_norm():
    n1 = n2 = 20
    inst = W.mc_instance(n1, n2, 2, 300, seed=5)
    P = O.Problem(inst)
    R0 = W.initial_factor(inst, W.rank_log2(inst.m), 3)
    res = A.solve_two_stage(P, R0, O.Params(max_outer=300), A.AdmmParams(switch_err1=1e-2))
    assert res["status"] == "ok"
    M = inst.meta["U"] @ inst.meta["V"].T
    assert res["primal_obj"] == pytest.approx(2 * np.linalg.svd(M, compute_uv=False).sum(), rel=1e-3)
