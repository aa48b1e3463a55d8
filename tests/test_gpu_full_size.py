"""GPU parity at the benchmark's full size: the MaxCut SDP of an Erdos-Renyi
graph with n = 1e7 vertices (average degree 4, w in {-1,+1}) at r = 24.

The FP64 oracle cannot run the solve at this size, so the entry points are
checked where the oracle can follow them: the SpMM (C - A*(v)) R on a seeded
sample of rows (each output row needs only its own CSR row), the constraint
map diag(R R^T) on every row, the line-search coefficients a1..a4 in full
(one oracle pass of a few sparse products), and the solver's own first
L-BFGS iteration and multiplier step (a handful of oracle passes).  Tolerances as for the small
cases: 1e-12 normwise in FP64, 1e-5 in FP32 against the oracle on the same
rounded inputs; a1..a4 relative to the sum of the magnitudes of their terms.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O
from tests._util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402

N = 10_000_000
R_COLS = 24
TOL = {"fp64": 1e-12, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


@pytest.fixture(scope="module")
def full():
    L.build()
    inst = W.maxcut_instance(N, W.er_graph(N, 2 * N, 0, "pm1"))
    ctx = L.lorads_create(inst)
    yield inst, O.Problem(inst), ctx
    L.lorads_destroy(ctx)


def _factor(n, r, seed, prec):
    R = np.random.default_rng(seed).standard_normal((n, r))
    t = torch.zeros((n, L.padded_ld(r)), dtype=DT[prec], device="cuda")
    t[:, :r] = torch.as_tensor(R, device="cuda").to(DT[prec])
    return t, t[:, :r].double().cpu().numpy()


def sampled_spmm_rows(P, R, v, rows):
    """Rows `rows` of (C - A*(v)) R, each from its own CSR row (oracle maps)."""
    out = P.C[rows] @ R
    if v is not None:
        out = out - O.adjoint(P, v)[rows] @ R
    return out


def sample_rows(n, count, seed):
    """Seeded sample: the first and last rows plus `count` distinct random rows."""
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=count, replace=False)]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_spmm_on_sampled_rows(full, prec):
    inst, P, ctx = full
    R, Rr = _factor(N, R_COLS, 101, prec)
    odt = torch.float64 if prec == "fp64" else torch.float32
    rows = sample_rows(N, 4096, 7)
    for use_v in (False, True):
        v = np.random.default_rng(3).standard_normal(inst.m) if use_v else None
        out = torch.full(R.shape, float("nan"), dtype=odt, device="cuda")
        L.lorads_spmm(ctx, R, torch.as_tensor(v, device="cuda") if use_v else None, out, r=R_COLS)
        torch.cuda.synchronize()
        idx = torch.as_tensor(rows, device="cuda")
        got = out[idx].double().cpu().numpy()
        want = sampled_spmm_rows(P, Rr, v, rows)
        assert rel_err(got[:, :R_COLS], want) <= TOL[prec], (use_v, rel_err(got[:, :R_COLS], want))
        assert np.all(got[:, R_COLS:] == 0.0)
        assert not torch.isnan(out).any().item()
        del out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_constraint_map(full, prec):
    inst, P, ctx = full
    R, Rr = _factor(N, R_COLS, 102, prec)
    out = torch.full((inst.m,), float("nan"), dtype=torch.float64, device="cuda")
    L.lorads_constraint_eval(ctx, R, R, out, r=R_COLS)
    torch.cuda.synchronize()
    want = np.einsum("ij,ij->i", Rr, Rr)          # diag(R R^T): MaxCut's A(R R^T)
    assert rel_err(out.cpu().numpy(), want) <= TOL[prec]


def coef_scales(P, R, D, y, rho):
    """a1..a4 of the oracle and the sum of the magnitudes of each one's terms."""
    a, parts = O.linesearch_coeffs(P, R, D, y, rho)
    q0, q1, q2 = parts["q0"], parts["q1"], parts["q2"]
    w = np.abs(y) + rho * np.abs(q0)
    Cabs = abs(P.C)
    s1 = 0.5 * rho * float(q2 @ q2)
    s2 = rho * float(np.abs(q1) @ np.abs(q2))
    s3 = float(np.sum((Cabs @ np.abs(D)) * np.abs(D))) + float(w @ np.abs(q2)) + 0.5 * rho * float(q1 @ q1)
    s4 = 2 * float(np.sum((Cabs @ np.abs(R)) * np.abs(D))) + float(w @ np.abs(q1))
    return a, np.array([s1, s2, s3, s4])


@pytest.fixture(scope="module")
def linesearch_case(full):
    """R, D with FP32-representable entries (so that both storage forms hold the
    same values), y, rho and the oracle's a1..a4 with their term scales: one
    oracle pass serves both precisions."""
    inst, P, _ = full
    R = np.random.default_rng(103).standard_normal((N, R_COLS)).astype(np.float32).astype(np.float64)
    D = np.random.default_rng(104).standard_normal((N, R_COLS)).astype(np.float32).astype(np.float64)
    y = np.random.default_rng(5).standard_normal(inst.m)
    rho = 3.5
    a_ref, scale = coef_scales(P, R, D, y, rho)
    return R, D, y, rho, a_ref, scale


def _device(X, prec):
    t = torch.zeros((X.shape[0], L.padded_ld(X.shape[1])), dtype=DT[prec], device="cuda")
    t[:, :X.shape[1]] = torch.as_tensor(X, device="cuda").to(DT[prec])
    return t


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_linesearch_coeffs(full, linesearch_case, prec):
    inst, P, ctx = full
    R, D, y, rho, a_ref, scale = linesearch_case
    a_gpu, tau_gpu = L.lorads_linesearch_coeffs(ctx, _device(R, prec), _device(D, prec),
                                                torch.as_tensor(y, device="cuda"), rho, r=R_COLS)
    assert np.all(np.abs(a_gpu - a_ref) <= TOL[prec] * scale), (a_gpu, a_ref, scale)
    assert tau_gpu == pytest.approx(O.quartic_step(a_gpu), rel=1e-9, abs=1e-300)


FIRST_STEP_CAPS = dict(max_outer=1, max_inner=1, tol=1e-300)


@pytest.fixture(scope="module")
def first_step_ref(full):
    """The oracle's first L-BFGS iteration and multiplier step from the seeded start."""
    inst, P, _ = full
    R0 = W.initial_factor(inst, R_COLS, 1)
    return R0, O.solve(P, R0, O.Params(**FIRST_STEP_CAPS))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_first_iteration_matches_oracle(full, first_step_ref, prec):
    """The solver itself (captured iteration graph, default kernel forms), capped
    at one L-BFGS iteration and one multiplier step from the seeded start: R and
    y equal the FP64 oracle's to 1e-9 / 1e-8 (FP64) or 1e-5 (mixed), normwise."""
    inst, P, _ = full
    R0, ref = first_step_ref
    caps = FIRST_STEP_CAPS
    code = {"fp64": L.LORADS_FP64, "mixed": L.LORADS_MIXED}[prec]
    ctx = L.lorads_create(inst, L.default_params(prec=code, **caps))
    try:
        res = L.lorads_solve(ctx, R0)
        R, y = L.lorads_get_solution(ctx, inst.n, inst.m)
    finally:
        L.lorads_destroy(ctx)
    assert res["inner_iters"] == ref["inner"] == 1
    tol_r, tol_y = (1e-9, 1e-8) if prec == "fp64" else (1e-5, 1e-5)
    assert rel_err(R, ref["R"]) <= tol_r, rel_err(R, ref["R"])
    assert np.max(np.abs(y - ref["y"])) <= tol_y * (1 + np.abs(ref["y"]).max())
