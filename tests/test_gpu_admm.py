"""GPU parity of the splitting (ADMM) stage of Sec. 2.2 against the FP64 oracle
(oracle/admm_oracle.py).

* Operator: frakA_V(X) = rho A*(A(X V^T)) V + rho X (Eq. (2.3)) on instances
  with diagonal, off-diagonal and mixed constraints, ranks spanning one to
  several four-element units per lane, ragged row counts; 1e-12 in FP64 and
  1e-5 in FP32 (normwise).
* CG: Algorithm 2 on frakA_V(X) = frakb_V from the same start takes the same
  number of steps and reaches the same iterate (FP64); in FP32 the solution
  meets the same residual test when checked with the FP64 operator.
* Stage: 1 and 5 ADMM iterations from the same (R, y, rho) give the oracle's
  R = (U + V)/2 and y (FP64 1e-9, mixed 1e-5) and the same CG step counts.
* Two stages: lorads_solve with the ALM -> ADMM switch reaches rel. KKT 1e-5
  at the oracle's two-stage objective.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O
from oracle import admm_oracle as A
from tests._util import mixed_instance, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402

PREC = {"fp64": L.LORADS_FP64, "mixed": L.LORADS_MIXED, "df64": L.LORADS_DF64, "fp32": L.LORADS_FP32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    L.build()


def _instance(name):
    if name == "maxcut_er_1000":
        return W.maxcut_instance(1000, W.er_graph(1000, 4000, 0, "unit"))
    if name == "maxcut_pm1_2000":
        return W.maxcut_instance(2000, W.er_graph(2000, 4000, 3, "pm1"))
    if name == "mc_60x80":
        return W.mc_instance(60, 80, 3, 2500, seed=2)
    return mixed_instance(613, seed=4)


def _dev(a, dtype, ld):
    t = torch.zeros((a.shape[0], ld), dtype=dtype, device="cuda")
    t[:, :a.shape[1]] = torch.as_tensor(a, dtype=dtype, device="cuda")
    return t


@pytest.mark.parametrize("r", [1, 5, 12, 20, 33])
@pytest.mark.parametrize("name", ["maxcut_er_1000", "mc_60x80", "mixed_613"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_operator_matches_oracle(name, r, prec):
    inst = _instance(name)
    P = O.Problem(inst)
    rng = np.random.default_rng(r)
    V = rng.standard_normal((inst.n, r))
    X = rng.standard_normal((inst.n, r))
    rho = 3.7
    want = A.system_operator(P, V, X, rho)
    ld = L.padded_ld(r)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Vd, Xd = _dev(V, dt, ld), _dev(X, dt, ld)
    out = torch.full_like(Vd, float("nan"))
    ctx = L.lorads_create(inst)
    try:
        L.lorads_admm_operator(ctx, Vd, Xd, out, rho, r=r)
        torch.cuda.synchronize()
    finally:
        L.lorads_destroy(ctx)
    got = out.double().cpu().numpy()
    assert rel_err(got[:, :r], want) <= (1e-12 if prec == "fp64" else 1e-5)
    assert np.all(got[:, r:] == 0.0)


@pytest.mark.parametrize("cg_rel", [1e-2, 1e-8])
@pytest.mark.parametrize("name", ["maxcut_er_1000", "mc_60x80", "mixed_613"])
def test_cg_matches_oracle(name, cg_rel):
    inst = _instance(name)
    P = O.Problem(inst)
    rng = np.random.default_rng(7)
    r = 6
    V = rng.standard_normal((inst.n, r))
    X0 = rng.standard_normal((inst.n, r))
    y = rng.standard_normal(inst.m)
    rho = 2.5
    X_ref, k_ref = A.cg(P, V, X0, A.system_rhs(P, V, y, rho), rho, cg_rel, 50)
    ld = L.padded_ld(r)
    Vd, Xd = _dev(V, torch.float64, ld), _dev(X0, torch.float64, ld)
    ctx = L.lorads_create(inst)
    try:
        k = L.lorads_admm_cg(ctx, Vd, Xd, torch.as_tensor(y, device="cuda"), rho, cg_rel=cg_rel, cg_max=50, r=r)
    finally:
        L.lorads_destroy(ctx)
    assert k == k_ref
    # Algorithm 2 stops at a relative residual: the iterate it returns responds to
    # rounding differences (another reduction order) through the Krylov polynomial;
    # the bound is 10x the oracle's own response to a 1e-15 change of its right side
    rhs = A.system_rhs(P, V, y, rho)
    sens = max(rel_err(A.cg(P, V, X0, rhs * f, rho, cg_rel, 50)[0], X_ref) for f in (1 + 1e-15, 1 - 1e-15))
    assert rel_err(Xd.cpu().numpy()[:, :r], X_ref) <= max(1e-10, 10 * sens)


@pytest.mark.parametrize("name", ["maxcut_er_1000", "mc_60x80"])
def test_cg_fp32_meets_the_residual_test(name):
    inst = _instance(name)
    P = O.Problem(inst)
    rng = np.random.default_rng(8)
    r = 6
    V = rng.standard_normal((inst.n, r))
    X0 = rng.standard_normal((inst.n, r))
    y = rng.standard_normal(inst.m)
    rho = 2.5
    rhs = A.system_rhs(P, V, y, rho)
    r0 = np.linalg.norm(rhs - A.system_operator(P, V, X0, rho))
    ld = L.padded_ld(r)
    Vd, Xd = _dev(V, torch.float32, ld), _dev(X0, torch.float32, ld)
    ctx = L.lorads_create(inst)
    try:
        k = L.lorads_admm_cg(ctx, Vd, Xd, torch.as_tensor(y, device="cuda"), rho, cg_rel=1e-2, cg_max=50, r=r)
    finally:
        L.lorads_destroy(ctx)
    X = Xd.double().cpu().numpy()[:, :r]
    assert 1 <= k < 50
    assert np.linalg.norm(rhs - A.system_operator(P, V, X, rho)) <= 1.1e-2 * r0


def _alm_start(name, switch):
    """(R, y, rho) where the oracle's ALM stage hands over at err1, |err3| <= switch."""
    inst = _instance(name)
    P = O.Problem(inst)
    r = 10 if inst.kind == "maxcut" else 12
    R0 = W.initial_factor(inst, r, 1 if inst.kind == "maxcut" else 4)
    first = O.solve(P, R0, O.Params(tol=switch))
    return inst, P, first


@pytest.mark.parametrize("k", [1, 5])
@pytest.mark.parametrize("name", ["maxcut_er_1000", "maxcut_pm1_2000", "mc_60x80"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stage_trajectory_matches_oracle(name, k, prec):
    inst, P, first = _alm_start(name, 1e-2)
    ref = A.admm_stage(P, first["R"], first["y"], first["rho"], A.AdmmParams(max_iter=k, tol=1e-300))
    ctx = L.lorads_create(inst, L.default_params(prec=PREC[prec], admm_max_iter=k, tol=1e-300))
    try:
        res = L.lorads_admm_stage(ctx, first["R"], first["y"], first["rho"])
        R, y = L.lorads_get_solution(ctx, inst.n, inst.m)
    finally:
        L.lorads_destroy(ctx)
    assert res["admm_iters"] == ref["iters"] == k
    if prec == "fp64":
        assert res["cg_steps"] == ref["cg_steps"]
        tol = 1e-9
    else:
        tol = 1e-5
    assert rel_err(R, ref["R"]) <= tol
    assert rel_err(y, ref["y"]) <= tol
    assert res["err1"] == pytest.approx(ref["err1"], rel=10 * tol)
    assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=tol)


@pytest.mark.parametrize("switch", [1e-2, 1e-3])
@pytest.mark.parametrize("case", [("maxcut_er_1000", 10), ("maxcut_er_1000", 30), ("maxcut_pm1_2000", 30),
                                  ("mc_60x80", 12)], ids=lambda c: f"{c[0]}-r{c[1]}")
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_stage_solve_matches_oracle(case, switch, prec):
    """The GPU two-stage solve against the oracle's (solve_two_stage) from the same R0.

    FP64 on the unit-weight graph at r = 10 and on the completion instance follows the
    oracle's trajectory: the same ALM iterations, ADMM iterations and objective to
    1e-7.  Elsewhere rounding differences of the reduction orders move the ALM stage's
    hand-over by a few iterations and the stage stops at another point of the KKT-1e-5
    set: the objectives then agree to 2e-5 (for scale: the oracle's own two-stage
    objective lies 1.4e-5 above its ALM-only one on the +-1 graph at r = 30, switch 1e-2)."""
    name, r = case
    inst = _instance(name)
    P = O.Problem(inst)
    R0 = W.initial_factor(inst, r, 1 if inst.kind == "maxcut" else 4)
    ref = A.solve_two_stage(P, R0, O.Params(), A.AdmmParams(switch_err1=switch))
    ctx = L.lorads_create(inst, L.default_params(prec=PREC[prec], admm_switch=switch))
    try:
        res = L.lorads_solve(ctx, R0)
    finally:
        L.lorads_destroy(ctx)
    assert ref["status"] == "ok" and res["status_name"] == "LORADS_OK", res
    assert res["err1"] <= 1e-5 and abs(res["err3"]) <= 1e-5
    if prec == "fp64" and case in (("maxcut_er_1000", 10), ("mc_60x80", 12)):
        assert res["inner_iters"] == ref["alm_inner"]
        assert res["admm_iters"] == ref["admm_iters"]
        assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=1e-7)
    else:
        assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=2e-5)


@pytest.mark.parametrize("mem", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_stage_with_short_memory(mem, prec):
    """With T = 1 or 2 stored pairs the stage takes its arrays from the solver state
    (history, gradient, C D and the direction; for the mixed form at T = 2 the history
    holds U and V exactly) or, mixed at T = 1, allocates its own: the result is the
    oracle's two-stage solve with the same memory."""
    inst = _instance("maxcut_er_1000")
    P = O.Problem(inst)
    R0 = W.initial_factor(inst, 10, 1)
    ref = A.solve_two_stage(P, R0, O.Params(lbfgs_mem=mem), A.AdmmParams(switch_err1=1e-3))
    ctx = L.lorads_create(inst, L.default_params(prec=PREC[prec], admm_switch=1e-3, lbfgs_mem=mem))
    try:
        res = L.lorads_solve(ctx, R0)
    finally:
        L.lorads_destroy(ctx)
    assert ref["status"] == "ok" and res["status_name"] == "LORADS_OK", res
    assert res["admm_iters"] >= 1
    assert res["err1"] <= 1e-5 and abs(res["err3"]) <= 1e-5
    if prec == "fp64":
        assert res["inner_iters"] == ref["alm_inner"]
        assert res["admm_iters"] == ref["admm_iters"]
        assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=1e-7)
    else:
        assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=2e-5)


def test_stage_rejects_bad_rho():
    inst = _instance("maxcut_er_1000")
    ctx = L.lorads_create(inst)
    try:
        with pytest.raises(L.LoradsError):
            L.lorads_admm_stage(ctx, W.initial_factor(inst, 4, 1), None, -1.0)
    finally:
        L.lorads_destroy(ctx)
