"""GPU parity of the standalone hot-path entry points against the FP64 oracle.

Sizes span many blocks with ragged tails; FP64 must match to 1e-12 (normwise),
FP32 and BF16-storage to 1e-5 against the oracle evaluated on the same rounded
inputs.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O
from tests._util import mixed_instance, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}


def _instances():
    return {
        "maxcut_er_3001": W.maxcut_instance(3001, W.er_graph(3001, 6002, 7, "pm1")),
        "mc_700x900": W.mc_instance(700, 900, 3, 30000, seed=8),
        "mixed_1031": mixed_instance(1031, seed=9),
    }


@pytest.fixture(scope="module")
def problems():
    L.build()
    out = {}
    for name, inst in _instances().items():
        ctx = L.lorads_create(inst)
        out[name] = (inst, O.Problem(inst), ctx)
    yield out
    for _, _, ctx in out.values():
        L.lorads_destroy(ctx)


def _factor(n, r, seed, prec):
    """Random n x r factor, rounded to the storage precision, and its padded device copy."""
    R = np.random.default_rng(seed).standard_normal((n, r))
    t = torch.zeros((n, L.padded_ld(r)), dtype=DT[prec], device="cuda")
    t[:, :r] = torch.as_tensor(R, device="cuda").to(DT[prec])
    R_rounded = t[:, :r].double().cpu().numpy()
    return t, R_rounded


RANKS = [1, 3, 10, 20, 24, 28, 32]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", ["maxcut_er_3001", "mc_700x900", "mixed_1031"])
@pytest.mark.parametrize("r", RANKS)
def test_spmm_parity(problems, name, prec, r):
    inst, P, ctx = problems[name]
    R, Rr = _factor(inst.n, r, 10 + r, prec)
    odt = torch.float64 if prec == "fp64" else torch.float32
    for use_v in (False, True):
        v = np.random.default_rng(r).standard_normal(inst.m) if use_v else None
        out = torch.full((inst.n, R.shape[1]), float("nan"), dtype=odt, device="cuda")
        L.lorads_spmm(ctx, R, torch.as_tensor(v, device="cuda") if use_v else None, out, r=r)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        want = O.spmm(P, Rr, v)
        assert rel_err(got[:, :r], want) <= TOL[prec], (use_v, rel_err(got[:, :r], want))
        assert np.all(got[:, r:] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", ["maxcut_er_3001", "mc_700x900", "mixed_1031"])
@pytest.mark.parametrize("r", [1, 10, 24, 28])
def test_constraint_eval_parity(problems, name, prec, r):
    inst, P, ctx = problems[name]
    U, Ur = _factor(inst.n, r, 30 + r, prec)
    V, Vr = _factor(inst.n, r, 40 + r, prec)
    out = torch.full((inst.m,), float("nan"), dtype=torch.float64, device="cuda")
    for (A, Ar, B, Br) in [(U, Ur, V, Vr), (U, Ur, U, Ur)]:
        L.lorads_constraint_eval(ctx, A, B, out, r=r)
        torch.cuda.synchronize()
        want = O.constraint_map(P, Ar, Br)
        assert rel_err(out.cpu().numpy(), want) <= TOL[prec]


def _coef_scales(P, R, D, y, rho):
    """Scale of each a_i: the sum of the magnitudes of its terms (cancellation-aware)."""
    a, parts = O.linesearch_coeffs(P, R, D, y, rho)
    q0, q1, q2 = parts["q0"], parts["q1"], parts["q2"]
    w = np.abs(y) + rho * np.abs(q0)
    CRabs = np.abs(P.C) @ np.abs(R)
    CDabs = np.abs(P.C) @ np.abs(D)
    s1 = 0.5 * rho * float(q2 @ q2)
    s2 = rho * float(np.abs(q1) @ np.abs(q2))
    s3 = float(np.sum(CDabs * np.abs(D))) + float(w @ np.abs(q2)) + 0.5 * rho * float(q1 @ q1)
    s4 = 2 * float(np.sum(CRabs * np.abs(D))) + float(w @ np.abs(q1))
    return a, np.array([s1, s2, s3, s4])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", ["maxcut_er_3001", "mc_700x900", "mixed_1031"])
@pytest.mark.parametrize("r", [3, 10, 24])
def test_linesearch_coeffs_parity(problems, name, prec, r):
    inst, P, ctx = problems[name]
    R, Rr = _factor(inst.n, r, 50 + r, prec)
    D, Dr = _factor(inst.n, r, 60 + r, prec)
    Dr_small = Dr
    y = np.random.default_rng(r).standard_normal(inst.m)
    rho = 3.5
    a_gpu, tau_gpu = L.lorads_linesearch_coeffs(ctx, R, D, torch.as_tensor(y, device="cuda"), rho, r=r)
    a_ref, scale = _coef_scales(P, Rr, Dr_small, y, rho)
    tol = TOL[prec]
    assert np.all(np.abs(a_gpu - a_ref) <= tol * scale), (a_gpu, a_ref, scale)
    if prec == "fp64":
        tau_ref = O.quartic_step(a_ref)
        assert tau_gpu == pytest.approx(tau_ref, rel=1e-9, abs=1e-300)
    # the GPU root is a root of the GPU's own cubic
    tau_own = O.quartic_step(a_gpu)
    assert tau_gpu == pytest.approx(tau_own, rel=1e-9, abs=1e-300)


def test_linesearch_step_on_descent_direction(problems):
    """Along -grad the step is positive and lowers the Lagrangian (FP64)."""
    inst, P, ctx = problems["maxcut_er_3001"]
    r = 10
    R = W.initial_factor(inst, r, 3)
    y = np.zeros(inst.m)
    rho = 2.0
    G = O.gradient(P, R, y, rho)
    ld = L.padded_ld(r)
    Rt = torch.zeros((inst.n, ld), dtype=torch.float64, device="cuda")
    Dt = torch.zeros_like(Rt)
    Rt[:, :r] = torch.as_tensor(R, device="cuda")
    Dt[:, :r] = torch.as_tensor(-G, device="cuda")
    a, tau = L.lorads_linesearch_coeffs(ctx, Rt, Dt, torch.as_tensor(y, device="cuda"), rho, r=r)
    assert tau > 0
    assert O.lagrangian(P, R - tau * G, y, rho) < O.lagrangian(P, R, y, rho)


def test_empty_rows_and_tiny_problem():
    """n = 1 and rows without any stored entry."""
    inst = mixed_instance(37, seed=3, empty_every=5)
    P = O.Problem(inst)
    ctx = L.lorads_create(inst)
    try:
        R, Rr = _factor(inst.n, 5, 1, "fp64")
        out = torch.zeros_like(R)
        L.lorads_spmm(ctx, R, None, out, r=5)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy()[:, :5], O.spmm(P, Rr, None)) <= 1e-12
    finally:
        L.lorads_destroy(ctx)
    one = W.SDPInstance(n=1, rowptr=np.array([0, 1]), colind=np.array([0], np.int32), val=np.array([2.0]), m=1,
                        con=np.array([0], np.int32), row=np.array([0], np.int32), col=np.array([0], np.int32),
                        aval=np.array([1.0]), b=np.array([1.0]))
    ctx = L.lorads_create(one)
    try:
        R = torch.tensor([[1.5, 0, 0, 0]], dtype=torch.float64, device="cuda")
        out = torch.zeros_like(R)
        L.lorads_spmm(ctx, R, torch.tensor([0.5], dtype=torch.float64, device="cuda"), out, r=1)
        torch.cuda.synchronize()
        assert out[0, 0].item() == pytest.approx((2.0 - 0.5) * 1.5, rel=1e-15)
    finally:
        L.lorads_destroy(ctx)


def test_rejects_bad_layout(problems):
    inst, P, ctx = problems["maxcut_er_3001"]
    R = torch.zeros((inst.n, 6), dtype=torch.float64, device="cuda")     # ld not a multiple of 4
    with pytest.raises(L.LoradsError):
        L.lorads_spmm(ctx, R, None, torch.zeros_like(R))
    R = torch.zeros((inst.n, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LoradsError):
        L.lorads_spmm(ctx, R, None, R)                                    # aliasing
