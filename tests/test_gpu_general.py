"""GPU parity on general constraints (the class of Sec. 4.5): constraints with
several entries, several constraints on one entry, and a dense C.

Instances: the Lovasz theta SDP (tr X = 1 over all n diagonal entries, X_ij = 0 on
the edges, C = -J), and MaxCut SDPs with added constraints summing several
off-diagonal entries plus X_00 + X_11 = 2 over entries the row constraints
already fix.

* Kernels: the constraint map, (C - A*(v)) R and the line-search coefficients
  against the FP64 oracle (1e-12 FP64, 1e-5 FP32).
* Trajectory: 1, 5 and 30 L-BFGS steps equal the oracle's (FP64).
* Convergence: theta(C_5) = sqrt 5, theta(C_7), theta(Petersen) = 4 in FP64 and
  the mixed form, and the oracle's objective on the MaxCut instance.
* ADMM stage (Sec. 2.2) on this form: Algorithm 2's CG, 1 and 5 ADMM iterations
  from the same (R, y, rho) and two-stage solves against the oracle; the
  theta closed forms through the two stages.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O
from oracle import admm_oracle as A
from tests._util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402

PREC = {"fp64": L.LORADS_FP64, "mixed": L.LORADS_MIXED, "df64": L.LORADS_DF64, "fp32": L.LORADS_FP32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    L.build()


def _instance(name):
    if name == "theta_petersen":
        return W.theta_instance(10, W.petersen_graph())
    if name == "theta_c7":
        return W.theta_instance(7, W.cycle_graph(7))
    if name == "theta_er60":
        return W.theta_instance(60, W.er_graph(60, 200, 4, "unit"))
    return W.maxcut_with_sums(300, W.er_graph(300, 900, 2, "pm1"), 4, 12, 3)


def _dev(a, dtype, ld):
    t = torch.zeros((a.shape[0], ld), dtype=dtype, device="cuda")
    t[:, :a.shape[1]] = torch.as_tensor(a, dtype=dtype, device="cuda")
    return t


def _start(inst, r, seed):
    """Seeded Gaussian start: ||R0||_F = 1 for theta (tr X = 1), unit rows otherwise (X_ii = 1)."""
    R0 = np.random.default_rng(seed).standard_normal((inst.n, r))
    if inst.kind == "theta":
        return R0 / np.linalg.norm(R0)
    return R0 / np.linalg.norm(R0, axis=1, keepdims=True)


NAMES = ["theta_petersen", "theta_er60", "maxcut_sums_300"]


@pytest.mark.parametrize("r", [1, 6, 17])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kernels_match_oracle(name, r, prec):
    inst = _instance(name)
    P = O.Problem(inst)
    rng = np.random.default_rng(r + 1)
    U, V, D = (rng.standard_normal((inst.n, r)) for _ in range(3))
    v = rng.standard_normal(inst.m)
    y = rng.standard_normal(inst.m)
    rho = 1.7
    ld = L.padded_ld(r)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    ctx = L.lorads_create(inst)
    try:
        out = torch.zeros(inst.m, dtype=torch.float64, device="cuda")
        L.lorads_constraint_eval(ctx, _dev(U, dt, ld), _dev(V, dt, ld), out, r=r)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), O.constraint_map(P, U, V)) <= tol
        sp = torch.zeros((inst.n, ld), dtype=dt, device="cuda")
        L.lorads_spmm(ctx, _dev(U, dt, ld), torch.as_tensor(v, device="cuda"), sp, r=r)
        torch.cuda.synchronize()
        assert rel_err(sp.double().cpu().numpy()[:, :r], O.spmm(P, U, v)) <= tol
        a, _ = L.lorads_linesearch_coeffs(ctx, _dev(U, dt, ld), _dev(D, dt, ld), torch.as_tensor(y, device="cuda"),
                                          rho, r=r)
    finally:
        L.lorads_destroy(ctx)
    a_ref, parts = O.linesearch_coeffs(P, U, D, y, rho)
    # cancellation-aware scale of each coefficient: the magnitudes of its terms
    q1, q2, q0 = parts["q1"], parts["q2"], parts["q0"]
    w = np.abs(y) + rho * np.abs(q0)
    Cabs = abs(P.C)
    scale = np.array([0.5 * rho * float(q2 @ q2), rho * float(np.abs(q1) @ np.abs(q2)),
                      float(np.sum((Cabs @ np.abs(D)) * np.abs(D))) + float(w @ np.abs(q2)) + 0.5 * rho * float(q1 @ q1),
                      2 * float(np.sum((Cabs @ np.abs(U)) * np.abs(D))) + float(w @ np.abs(q1))])
    assert np.all(np.abs(a - a_ref) <= tol * scale), (a, a_ref)


@pytest.mark.parametrize("k", [1, 5, 30])
@pytest.mark.parametrize("name", ["theta_er60", "maxcut_sums_300"])
def test_trajectory_matches_oracle(name, k):
    inst = _instance(name)
    R0 = _start(inst, 6, 2)
    caps = dict(max_outer=1, max_inner=k, tol=1e-300)
    ref = O.solve(O.Problem(inst), R0, O.Params(**caps))
    ctx = L.lorads_create(inst, L.default_params(prec=L.LORADS_FP64, **caps))
    try:
        res = L.lorads_solve(ctx, R0)
        R, y = L.lorads_get_solution(ctx, inst.n, inst.m)
    finally:
        L.lorads_destroy(ctx)
    assert res["inner_iters"] == ref["inner"]
    assert np.max(np.abs(R - ref["R"])) <= 1e-9 * np.abs(ref["R"]).max() * max(1, k / 10)
    assert np.max(np.abs(y - ref["y"])) <= 1e-8 * (1 + np.abs(ref["y"]).max())


@pytest.mark.parametrize("name", ["C5", "C7", "petersen"])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "df64"])
def test_theta_closed_forms(name, prec):
    if name == "petersen":
        inst, value = W.theta_instance(10, W.petersen_graph()), 4.0
    else:
        n = int(name[1:])
        c = math.cos(math.pi / n)
        inst, value = W.theta_instance(n, W.cycle_graph(n)), n * c / (1 + c)
    R0 = _start(inst, 3, 1)
    ctx = L.lorads_create(inst, L.default_params(prec=PREC[prec], compute_err2=1))
    try:
        res = L.lorads_solve(ctx, R0)
    finally:
        L.lorads_destroy(ctx)
    assert res["status_name"] == "LORADS_OK", res
    assert -res["primal_obj"] == pytest.approx(value, rel=1e-5)
    assert res["err1"] <= 1e-5 and abs(res["err3"]) <= 1e-5
    # err2 is checked at the end, not in the stop test (Sec. 4.2): on the cycles the
    # multiplier is dual feasible to 1e-5; on Petersen the rank-3 stationary point's is not
    # (the oracle from the same start: err2 = 1.2e-3 at r = 3, 3.0e-5 at r = 6)
    if name != "petersen":
        assert res["err2"] <= 1e-5


@pytest.mark.parametrize("switch", [0.0, 1e-3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_maxcut_with_sums_converges_to_oracle_objective(prec, switch):
    """FP64 with power-of-two row groups (kernel_variant 10, whose row sums happen to
    keep to the oracle's trajectory here) ends at the oracle's objective to 1e-6.
    With the default packed groups the row norms are summed in another order, the
    trajectory departs at rounding level and ends at another point of the KKT-1e-5
    set: the ALM solve still lands within 2e-5; the two-stage solve within 1e-4 (the
    oracle's own two-stage objective moves by up to 4.4e-5 over three starts at
    switch 1e-3, its ADMM stage stopping short of the ALM optimum)."""
    inst = _instance("maxcut_sums_300")
    R0 = _start(inst, 20, 1)
    P = O.Problem(inst)
    ref = (O.solve(P, R0, O.Params()) if switch == 0.0
           else A.solve_two_stage(P, R0, O.Params(), A.AdmmParams(switch_err1=switch)))
    assert ref["status"] == "ok"
    forms = [(10, 1e-6), (None, 2e-5 if switch == 0.0 else 1e-4)] if prec == "fp64" else [(None, 2e-5)]
    for kv, tol in forms:
        kw = {} if kv is None else {"kernel_variant": kv}
        ctx = L.lorads_create(inst, L.default_params(prec=PREC[prec], admm_switch=switch, **kw))
        try:
            res = L.lorads_solve(ctx, R0)
            R, _ = L.lorads_get_solution(ctx, inst.n, inst.m)
        finally:
            L.lorads_destroy(ctx)
        assert res["status_name"] == "LORADS_OK", res
        assert res["primal_obj"] == pytest.approx(ref["primal_obj"], rel=tol), kv
        z = O.constraint_map(P, R, R) - inst.b
        assert np.linalg.norm(z) / (1 + np.abs(inst.b).max()) <= 1.0001e-5


@pytest.mark.parametrize("cg_rel", [1e-2, 1e-5])
@pytest.mark.parametrize("name", ["theta_er60", "maxcut_sums_300"])
def test_cg_matches_oracle(name, cg_rel):
    inst = _instance(name)
    P = O.Problem(inst)
    rng = np.random.default_rng(3)
    r = 5
    V = rng.standard_normal((inst.n, r))
    X0 = rng.standard_normal((inst.n, r))
    y = rng.standard_normal(inst.m)
    rho = 2.0
    X_ref, k_ref = A.cg(P, V, X0, A.system_rhs(P, V, y, rho), rho, cg_rel, 50)
    ld = L.padded_ld(r)
    Vd, Xd = _dev(V, torch.float64, ld), _dev(X0, torch.float64, ld)
    ctx = L.lorads_create(inst)
    try:
        k = L.lorads_admm_cg(ctx, Vd, Xd, torch.as_tensor(y, device="cuda"), rho, cg_rel=cg_rel, cg_max=50, r=r)
    finally:
        L.lorads_destroy(ctx)
    assert k == k_ref
    assert rel_err(Xd.cpu().numpy()[:, :r], X_ref) <= _cg_sensitivity(P, V, X0, y, rho, cg_rel, X_ref)


def _cg_sensitivity(P, V, X0, y, rho, cg_rel, X_ref):
    """Bound on the CG iterate's agreement: 10x the change of the oracle's own iterate
    when its right side moves by 1e-15 relative (Algorithm 2 stops at a relative
    residual, and the Krylov polynomial it stops at amplifies such changes: 2e-7 on
    the theta instance, 2e-6 on the MaxCut one), and at least 1e-10."""
    rhs = A.system_rhs(P, V, y, rho)
    worst = 0.0
    for f in (1 + 1e-15, 1 - 1e-15):
        Xp, _ = A.cg(P, V, X0, rhs * f, rho, cg_rel, 50)
        worst = max(worst, rel_err(Xp, X_ref))
    return max(1e-10, 10 * worst)


@pytest.mark.parametrize("k", [1, 5])
@pytest.mark.parametrize("name", ["theta_er60", "maxcut_sums_300"])
def test_admm_stage_trajectory_matches_oracle(name, k):
    inst = _instance(name)
    P = O.Problem(inst)
    first = O.solve(P, _start(inst, 6, 2), O.Params(tol=1e-2))
    ref = A.admm_stage(P, first["R"], first["y"], first["rho"], A.AdmmParams(max_iter=k, tol=1e-300))
    ctx = L.lorads_create(inst, L.default_params(prec=L.LORADS_FP64, admm_max_iter=k, tol=1e-300))
    try:
        res = L.lorads_admm_stage(ctx, first["R"], first["y"], first["rho"])
        R, y = L.lorads_get_solution(ctx, inst.n, inst.m)
    finally:
        L.lorads_destroy(ctx)
    assert res["admm_iters"] == k and res["cg_steps"] == ref["cg_steps"]
    assert rel_err(R, ref["R"]) <= 1e-9
    assert rel_err(y, ref["y"]) <= 1e-9


@pytest.mark.parametrize("name", ["C5", "petersen"])
def test_theta_closed_forms_two_stage(name):
    if name == "petersen":
        inst, value = W.theta_instance(10, W.petersen_graph()), 4.0
    else:
        inst, value = W.theta_instance(5, W.cycle_graph(5)), math.sqrt(5)
    ctx = L.lorads_create(inst, L.default_params(prec=L.LORADS_MIXED, admm_switch=1e-2))
    try:
        res = L.lorads_solve(ctx, _start(inst, 3, 1))
    finally:
        L.lorads_destroy(ctx)
    assert res["status_name"] == "LORADS_OK", res
    # the ADMM stage stops as soon as err1 and |err3| <= 1e-5: on these tiny instances
    # that leaves the value within 3e-5 of the closed form (the oracle's two stages from
    # the same start: 1.4e-5 on C_5, 1.5e-5 on Petersen)
    assert -res["primal_obj"] == pytest.approx(value, rel=3e-5)
