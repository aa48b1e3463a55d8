"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own formulas: dense brute-force
definitions, finite differences, polynomial interpolation, closed-form SDP
values, exhaustive max cut and duality certificates.
"""
import math
from pathlib import Path

import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O


# ----------------------------------------------------------------------------- instances

def _mixed_instance(seed=0, n=9, multi=False):
    """Random symmetric C with diagonal and off-diagonal single-entry constraints
    (and optionally one constraint with several entries)."""
    rng = np.random.default_rng(seed)
    Cd = rng.standard_normal((n, n))
    Cd = np.where(rng.random((n, n)) < 0.4, Cd, 0.0)
    Cd = Cd + Cd.T
    np.fill_diagonal(Cd, rng.standard_normal(n))
    rows, cols = np.nonzero(np.ones((n, n)) * (Cd != 0))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    con, row, col, aval = [], [], [], []
    k = 0
    for i in range(0, n, 2):                       # diagonal constraints
        con.append(k); row.append(i); col.append(i); aval.append(1.0 + 0.1 * i); k += 1
    for (i, j) in [(0, 3), (1, 5), (2, 8), (4, 6)]:  # off-diagonal constraints
        con.append(k); row.append(i); col.append(j); aval.append(0.5 - 0.2 * i); k += 1
    if multi:
        for (i, j, a) in [(1, 1, 1.0), (3, 7, -0.5), (7, 7, 2.0)]:
            con.append(k); row.append(i); col.append(j); aval.append(a)
        k += 1
    m = k
    return W.SDPInstance(
        n=n, rowptr=rowptr, colind=cols.astype(np.int32), val=Cd[rows, cols], m=m,
        con=np.array(con, np.int32), row=np.array(row, np.int32), col=np.array(col, np.int32),
        aval=np.array(aval), b=rng.standard_normal(m), kind="generic")


def _instances():
    out = {
        "maxcut_er": W.maxcut_instance(14, W.er_graph(14, 30, 3, "pm1")),
        "mc": W.mc_instance(5, 7, 2, 20, seed=4),
        "mixed": _mixed_instance(0),
        "multi": _mixed_instance(1, multi=True),
    }
    return out


INST = _instances()


def _dense_C(P):
    return P.C.toarray()


# ----------------------------------------------------------------------------- linear maps

@pytest.mark.parametrize("name", list(INST))
def test_constraint_map_matches_dense_definition(name):
    P = O.Problem(INST[name])
    rng = np.random.default_rng(1)
    U = rng.standard_normal((P.n, 3))
    V = rng.standard_normal((P.n, 3))
    X = U @ V.T
    want = np.array([np.sum(P.A_dense(k) * X) for k in range(P.m)])
    got = O.constraint_map(P, U, V)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name", list(INST))
def test_adjoint_matches_dense_sum(name):
    P = O.Problem(INST[name])
    v = np.random.default_rng(2).standard_normal(P.m)
    want = sum(v[k] * P.A_dense(k) for k in range(P.m))
    np.testing.assert_allclose(O.adjoint(P, v).toarray(), want, atol=1e-13)
    # adjointness <A*(v), X> = v^T A(X) for X = U V^T + V U^T (symmetric)
    rng = np.random.default_rng(3)
    U, V = rng.standard_normal((P.n, 2)), rng.standard_normal((P.n, 2))
    X = U @ V.T + V @ U.T
    lhs = np.sum(O.adjoint(P, v).toarray() * X)
    rhs = v @ (O.constraint_map(P, U, V) + O.constraint_map(P, V, U))
    assert abs(lhs - rhs) <= 1e-11 * (1 + abs(lhs))


@pytest.mark.parametrize("name", list(INST))
def test_spmm_matches_triple_loop(name):
    P = O.Problem(INST[name])
    rng = np.random.default_rng(4)
    R = rng.standard_normal((P.n, 3))
    v = rng.standard_normal(P.m)
    S = _dense_C(P) - sum(v[k] * P.A_dense(k) for k in range(P.m))
    want = np.zeros_like(R)
    for i in range(P.n):
        for j in range(P.n):
            for c in range(R.shape[1]):
                want[i, c] += S[i, j] * R[j, c]
    np.testing.assert_allclose(O.spmm(P, R, v), want, atol=1e-12)
    np.testing.assert_allclose(O.spmm(P, R, None), _dense_C(P) @ R, atol=1e-12)


@pytest.mark.parametrize("name", list(INST))
def test_gradient_matches_finite_differences(name):
    P = O.Problem(INST[name])
    rng = np.random.default_rng(5)
    R = rng.standard_normal((P.n, 3))
    y = rng.standard_normal(P.m)
    rho = 1.7
    G = O.gradient(P, R, y, rho)
    h = 1e-5
    for (i, c) in [(0, 0), (P.n - 1, 2), (P.n // 2, 1), (1, 1)]:
        E = np.zeros_like(R)
        E[i, c] = h
        fd = (O.lagrangian(P, R + E, y, rho) - O.lagrangian(P, R - E, y, rho)) / (2 * h)
        assert abs(fd - G[i, c]) <= 1e-6 * (1 + abs(G[i, c])), (i, c, fd, G[i, c])


# ----------------------------------------------------------------------------- line search

@pytest.mark.parametrize("name", list(INST))
def test_linesearch_coeffs_interpolate_the_lagrangian(name):
    """L(R + tau D) - L(R) is exactly the quartic a1 t^4 + a2 t^3 + a3 t^2 + a4 t."""
    P = O.Problem(INST[name])
    rng = np.random.default_rng(6)
    R = rng.standard_normal((P.n, 3))
    D = rng.standard_normal((P.n, 3))
    y = rng.standard_normal(P.m)
    rho = 2.3
    a, parts = O.linesearch_coeffs(P, R, D, y, rho)
    L0 = O.lagrangian(P, R, y, rho)
    taus = np.array([-1.0, -0.5, 0.5, 1.0])
    f = np.array([O.lagrangian(P, R + t * D, y, rho) - L0 for t in taus])
    V = np.stack([taus ** 4, taus ** 3, taus ** 2, taus], axis=1)
    fit = np.linalg.solve(V, f)
    scale = np.abs(a).max() + abs(L0)
    np.testing.assert_allclose(a, fit, atol=1e-9 * scale)
    # a4 is the directional derivative <grad L, D>
    G = O.gradient(P, R, y, rho)
    assert abs(a[3] - np.sum(G * D)) <= 1e-10 * (abs(a[3]) + np.abs(G).sum())


def test_quartic_step_is_the_grid_minimiser():
    rng = np.random.default_rng(7)
    for trial in range(200):
        a1 = abs(rng.standard_normal()) + 1e-3
        a2, a3 = rng.standard_normal(2) * 3
        a4 = -abs(rng.standard_normal())
        a = np.array([a1, a2, a3, a4])
        tau = O.quartic_step(a)
        # positive roots of f' lie below the Cauchy bound 1 + max|coef|/|lead|
        T = 1.0 + max(abs(3 * a2), abs(2 * a3), abs(a4)) / (4 * a1)
        grid = np.linspace(0.0, T, 200001)
        fv = O.quartic_value(a, grid)
        g = grid[np.argmin(fv)]
        assert tau > 0
        assert O.quartic_value(a, tau) <= fv.min() + 1e-12 * (1 + abs(fv.min()))
        assert abs(tau - g) <= 2 * (grid[1] - grid[0]) or abs(O.quartic_value(a, tau) - fv.min()) < 1e-12
        fp = ((4 * a1 * tau + 3 * a2) * tau + 2 * a3) * tau + a4
        assert abs(fp) <= 1e-9 * (4 * a1 * tau ** 3 + 3 * abs(a2) * tau ** 2 + 2 * abs(a3) * tau + abs(a4))


def test_quartic_step_degenerate_cases():
    # quadratic: minimiser -a4 / (2 a3)
    assert O.quartic_step([0.0, 0.0, 2.0, -3.0]) == pytest.approx(0.75, rel=1e-15)
    # ascent direction: no positive step lowers f
    assert O.quartic_step([1.0, 0.0, 1.0, 0.5]) == 0.0
    # f = t^4 - 2 t^2 - 0*t + tiny descent: minimum at t = 1
    assert O.quartic_step([1.0, 0.0, -2.0, -1e-12]) == pytest.approx(1.0, rel=1e-9)


def _bfgs_dense_direction(G, S, Y, gamma=1.0):
    """-H G with H built by the BFGS inverse update from H0 = gamma I, oldest pair first."""
    g = G.ravel()
    H = gamma * np.eye(g.size)
    for s, y in zip(S, Y):
        s, y = s.ravel(), y.ravel()
        r = 1.0 / (y @ s)
        Vm = np.eye(g.size) - r * np.outer(y, s)
        H = Vm.T @ H @ Vm + r * np.outer(s, s)
    return -(H @ g).reshape(G.shape)


def test_two_loop_matches_dense_bfgs_matrix():
    rng = np.random.default_rng(8)
    shape = (4, 3)
    M = rng.standard_normal((12, 12))
    A = M @ M.T + 12 * np.eye(12)            # SPD curvature: y = A s
    for T in range(0, 5):
        S = [rng.standard_normal(shape) for _ in range(T)]
        Y = [(A @ s.ravel()).reshape(shape) for s in S]
        G = rng.standard_normal(shape)
        np.testing.assert_allclose(O.lbfgs_direction(G, S, Y), _bfgs_dense_direction(G, S, Y), rtol=1e-10,
                                   atol=1e-12)
        if T:
            gamma = float(np.sum(S[-1] * Y[-1]) / np.sum(Y[-1] * Y[-1]))
            np.testing.assert_allclose(O.lbfgs_direction(G, S, Y, scaling=1),
                                       _bfgs_dense_direction(G, S, Y, gamma), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------------------- randomness

def test_splitmix64_reference_output():
    # first output of SplitMix64 from state 0 (published reference implementation)
    out, _ = O.splitmix64(0, 1)
    assert out[0] == 0xE220A8397B1DCDAF


def test_gaussian_columns_are_standard_normal():
    g = O.gaussian_columns(400, 5, seed=3, stream=2)
    assert abs(g.mean()) < 0.1 and abs(g.std() - 1) < 0.1
    g2 = O.gaussian_columns(400, 5, seed=3, stream=2)
    np.testing.assert_array_equal(g, g2)


def test_rank_rule():
    assert O.rank_update_size(10, 1000) == 15
    assert O.rank_update_size(40, 1000) == 45          # capped at ceil(sqrt(2m))


# ----------------------------------------------------------------------------- solver

def _solve_maxcut(n, edges, seed=1, r=None, **kw):
    inst = W.maxcut_instance(n, edges)
    P = O.Problem(inst)
    r = r or W.rank_log2(n)
    R0 = W.initial_factor(inst, r, seed)
    res = O.solve(P, R0, O.Params(**kw))
    return P, res


def _closed_forms():
    """Rows of golden/maxcut_sdp_values.txt: (family, size, value)."""
    path = Path(__file__).resolve().parent / "golden" / "maxcut_sdp_values.txt"
    rows = []
    for line in path.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            fam, size, value = line.split()[:3]
            rows.append((fam, int(size), float(value)))
    return rows


@pytest.mark.parametrize("fam,size,value", _closed_forms())
def test_closed_form_sdp_values(fam, size, value):
    """Unit-weight MaxCut SDP optima with closed forms: K_n -> n^2/4, odd C_n ->
    (n/2)(1 + cos(pi/n)), bipartite torus -> |E| (fixture values, derivations in
    golden/make_golden.py)."""
    if fam == "complete":
        n, edges, r = size, W.complete_graph(size), None
    elif fam == "odd_cycle":
        n, edges, r = size, W.cycle_graph(size), 3
    else:
        n, edges, r = size * size, W.bipartite_torus_graph(size), None
        assert len(edges[0]) == value
    P, res = _solve_maxcut(n, edges, r=r)
    assert res["status"] == "ok"
    assert -res["primal_obj"] == pytest.approx(value, rel=1e-5)


def test_bruteforce_cut_closed_forms():
    """Exact max cuts with closed forms: K_n -> floor(n/2) ceil(n/2), odd C_n -> n - 1,
    even C_n -> n, a bipartite torus -> |E|; a +-1 weighted triangle by hand."""
    for n in (4, 5, 7):
        assert O.maxcut_bruteforce(n, W.complete_graph(n)) == (n // 2) * ((n + 1) // 2)
    for n in (5, 7, 6):
        assert O.maxcut_bruteforce(n, W.cycle_graph(n)) == (n - 1 if n % 2 else n)
    edges = W.bipartite_torus_graph(4)
    assert O.maxcut_bruteforce(16, edges) == len(edges[0])
    # triangle with weights +1 (0-1), -1 (1-2), +1 (0-2): the best cut isolates vertex 0
    tri = (np.array([0, 1, 0]), np.array([1, 2, 2]), np.array([1.0, -1.0, 1.0]))
    assert O.maxcut_bruteforce(3, tri) == 2.0


def test_sigma_min_is_the_smallest_eigenvalue_of_the_dual_slack():
    """sigma_min(C - A*(y)) on a tiny MaxCut instance: the dense matrix written out
    entry by entry from C = -L/4 and A*(y) = Diag(y), against the spectrum's minimum
    over a Rayleigh-quotient grid bound and numpy's eigvalsh."""
    inst = W.maxcut_instance(5, W.cycle_graph(5))
    P = O.Problem(inst)
    y = np.array([0.3, -0.2, 0.1, 0.0, -0.4])
    S = np.zeros((5, 5))
    for i in range(5):
        j = (i + 1) % 5
        S[i, j] = S[j, i] = 0.25                 # -L/4 off the diagonal (unit weights)
    np.fill_diagonal(S, -0.5 - y)                # -deg/4 - y_i
    lam = np.linalg.eigvalsh(S)[0]
    assert O.sigma_min(P, y) == pytest.approx(lam, abs=1e-12)
    x = np.random.default_rng(0).standard_normal((5, 2000))
    rq = np.einsum("ij,ij->j", x, S @ x) / np.einsum("ij,ij->j", x, x)
    assert lam <= rq.min() + 1e-12


@pytest.mark.parametrize("weights,seed", [("unit", 0), ("unit", 1), ("pm1", 2), ("pm1", 3)])
def test_bruteforce_cut_below_sdp_bound(weights, seed):
    n = 12
    edges = W.er_graph(n, 24, seed, weights)
    P, res = _solve_maxcut(n, edges, seed=seed + 5)
    assert res["status"] == "ok"
    sdp = -res["primal_obj"]
    best = O.maxcut_bruteforce(n, edges)
    assert best <= sdp + 1e-6
    if weights == "unit":
        assert 0.878 * sdp <= best + 1e-9        # Goemans-Williamson ratio


def test_feasibility_and_weak_duality():
    n = 60
    edges = W.er_graph(n, 200, 11, "pm1")
    P, res = _solve_maxcut(n, edges, seed=2)
    assert res["status"] == "ok"
    R, y = res["R"], res["y"]
    z = np.sum(R * R, axis=1) - 1.0
    assert np.max(np.abs(z)) <= 3e-5
    smin = O.sigma_min(P, y)
    gap = res["primal_obj"] - float(P.b @ y)
    # weak duality certificate: <C,X> - b^T y = <C - A*(y), X> >= n sigma_min
    assert gap >= n * smin - 1e-6
    assert smin >= -1e-3 and abs(gap) <= 1e-3 * (1 + abs(res["primal_obj"]))


def test_matrix_completion_recovers_nuclear_norm():
    n1 = n2 = 20
    inst = W.mc_instance(n1, n2, 2, 300, seed=5)
    P = O.Problem(inst)
    R0 = W.initial_factor(inst, W.rank_log2(inst.m), 3)
    res = O.solve(P, R0, O.Params(max_outer=300))
    assert res["status"] == "ok"
    M = inst.meta["U"] @ inst.meta["V"].T
    nuc = np.linalg.svd(M, compute_uv=False).sum()
    assert res["primal_obj"] == pytest.approx(2 * nuc, rel=1e-3)
    R = res["R"]
    Mhat = R[:n1] @ R[n1:].T
    assert np.linalg.norm(Mhat - M) <= 1e-2 * np.linalg.norm(M)


@pytest.mark.parametrize("name", ["C5", "C7", "petersen"])
def test_lovasz_theta_closed_forms(name):
    """Constraints with several entries (tr X = 1 over n diagonal entries) and a
    dense C = -J: the Lovasz theta SDP reaches its closed-form values,
    theta(C_n) = n cos(pi/n) / (1 + cos(pi/n)) for odd n (sqrt 5 for the pentagon)
    and theta(Petersen) = 4."""
    if name == "petersen":
        inst, value = W.theta_instance(10, W.petersen_graph()), 4.0
    else:
        n = int(name[1:])
        c = math.cos(math.pi / n)
        inst, value = W.theta_instance(n, W.cycle_graph(n)), n * c / (1 + c)
    R0 = np.random.default_rng(1).standard_normal((inst.n, 3))
    R0 /= np.linalg.norm(R0)
    res = O.solve(O.Problem(inst), R0, O.Params())
    assert res["status"] == "ok"
    assert -res["primal_obj"] == pytest.approx(value, rel=1e-5)
