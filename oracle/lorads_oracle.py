"""Plain FP64 CPU oracle of the LoRADS Burer-Monteiro / ALM stage.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or run this module;
the GPU library never calls it and shares no code with it.

Everything here is written to be checked against the paper by eye: dense or
``scipy.sparse`` definitions, literal loops over the L-BFGS memory, numpy's
polynomial root finder, no fusion and no reordering of the algorithm's steps.

Sign convention.  The body of the paper writes the Lagrangian as
<C,RR^T> + <A(RR^T)-b, lam> + rho/2 ||A(RR^T)-b||^2 with the ascent step
lam += rho (A(RR^T)-b) (Eq. (1.2), Sec. 2.1), while the line-search appendix
and the error formulas (Sec. 4.2) use lam^T (b - A(X)) and C - A*(lam).  Only
the latter pair is consistent, so this module uses the standard dual variable
y (= -lam of the body):

    L_rho(R, y) = <C, RR^T> - y^T (A(RR^T) - b) + rho/2 ||A(RR^T) - b||^2
    grad_R L    = 2 (C - A*(y_tilde)) R,     y_tilde = y - rho (A(RR^T) - b)
    y          <- y_tilde                    (multiplier step of Sec. 2.1)

Constraint convention.  A constraint is a list of triplets (i <= j, a);
<A_k, X> = sum a * X_ij * (1 if i == j else 2), i.e. A_k is the symmetric
matrix with a at (i,j) and (j,i).

Parity pins: tests/test_oracle.py (closed forms, brute force, finite
differences, polynomial interpolation, duality certificates).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field, asdict

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem", "Params", "constraint_map", "adjoint", "spmm", "objective",
    "lagrangian", "gradient", "linesearch_coeffs", "quartic_step",
    "lbfgs_direction", "errors", "sigma_min", "solve", "maxcut_bruteforce",
    "rank_update_size", "splitmix64", "gaussian_columns",
]


# ----------------------------------------------------------------------------- problem

class Problem:
    """Primal SDP of Eq. (1.1): min <C,X> s.t. A(X) = b, X psd (host, FP64)."""

    def __init__(self, inst):
        self.n = int(inst.n)
        self.m = int(inst.m)
        self.C = sp.csr_matrix(
            (np.asarray(inst.val, dtype=np.float64),
             np.asarray(inst.colind, dtype=np.int64),
             np.asarray(inst.rowptr, dtype=np.int64)),
            shape=(self.n, self.n))
        self.con = np.asarray(inst.con, dtype=np.int64)
        self.row = np.asarray(inst.row, dtype=np.int64)
        self.col = np.asarray(inst.col, dtype=np.int64)
        self.aval = np.asarray(inst.aval, dtype=np.float64)
        self.b = np.asarray(inst.b, dtype=np.float64)
        self.is_diag = self.row == self.col

    def A_dense(self, k: int) -> np.ndarray:
        """A_k as a dense symmetric matrix (brute-force definition, small n only)."""
        M = np.zeros((self.n, self.n))
        sel = self.con == k
        for i, j, a in zip(self.row[sel], self.col[sel], self.aval[sel]):
            M[i, j] += a
            if i != j:
                M[j, i] += a
        return M


# ----------------------------------------------------------------------------- linear maps

def constraint_map(P: Problem, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """A(U V^T)_k = <A_k, U V^T>  (Sec. 1.2 notation; the map behind Sec. 3.4's
    compressed outer product, evaluated only on the nonzero positions of A)."""
    uv = np.einsum("kr,kr->k", U[P.row], V[P.col])          # (U V^T)_{ij}
    vu = np.einsum("kr,kr->k", U[P.col], V[P.row])          # (U V^T)_{ji}
    term = np.where(P.is_diag, P.aval * uv, P.aval * (uv + vu))
    return np.bincount(P.con, weights=term, minlength=P.m)


def adjoint(P: Problem, v: np.ndarray) -> sp.csr_matrix:
    """A*(v) = sum_k v_k A_k (Sec. 1.2), as a sparse symmetric matrix."""
    w = v[P.con] * P.aval
    off = ~P.is_diag
    rows = np.concatenate([P.row, P.col[off]])
    cols = np.concatenate([P.col, P.row[off]])
    vals = np.concatenate([w, w[off]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(P.n, P.n))


def spmm(P: Problem, R: np.ndarray, v: np.ndarray | None) -> np.ndarray:
    """(C - A*(v)) R: the sparse-times-tall-skinny product of the gradient
    (Sec. 2 gradient formula; Eq. (3.1) with the multiplier folded in)."""
    if v is None:
        return P.C @ R
    return (P.C - adjoint(P, v)) @ R


def objective(P: Problem, R: np.ndarray) -> float:
    """<C, R R^T>."""
    return float(np.sum((P.C @ R) * R))


def lagrangian(P: Problem, R: np.ndarray, y: np.ndarray, rho: float) -> float:
    """L_rho(R, y) of Eq. (1.2) in the dual-variable sign (module docstring)."""
    z = constraint_map(P, R, R) - P.b
    return objective(P, R) - float(y @ z) + 0.5 * rho * float(z @ z)


def gradient(P: Problem, R: np.ndarray, y: np.ndarray, rho: float) -> np.ndarray:
    """grad_R L = 2CR - 2A*(y)R + 2 rho A*(A(RR^T) - b) R  (Sec. 2, sign of y)."""
    z = constraint_map(P, R, R) - P.b
    y_tilde = y - rho * z
    return 2.0 * spmm(P, R, y_tilde)


# ----------------------------------------------------------------------------- line search

def linesearch_coeffs(P: Problem, R, D, y, rho):
    """Coefficients a1..a4 of the exact line search (App. A.2), lam := y.

    f(tau) = L(R + tau D) - L(R) = a1 tau^4 + a2 tau^3 + a3 tau^2 + a4 tau with
      p1 = <C, RD^T + DR^T>, p2 = <C, DD^T>, q0 = b - A(RR^T),
      q1 = A(RD^T + DR^T),   q2 = A(DD^T),
      a1 = rho/2 ||q2||^2,  a2 = rho q1^T q2,
      a3 = p2 - (y + rho q0)^T q2 + rho/2 ||q1||^2,
      a4 = p1 - (y + rho q0)^T q1.
    Returns (a, parts) with a = [a1, a2, a3, a4].
    """
    CR = P.C @ R
    CD = P.C @ D
    p1 = float(np.sum(CR * D) + np.sum(CD * R))
    p2 = float(np.sum(CD * D))
    q0 = P.b - constraint_map(P, R, R)
    q1 = constraint_map(P, R, D) + constraint_map(P, D, R)
    q2 = constraint_map(P, D, D)
    w = y + rho * q0
    a1 = 0.5 * rho * float(q2 @ q2)
    a2 = rho * float(q1 @ q2)
    a3 = p2 - float(w @ q2) + 0.5 * rho * float(q1 @ q1)
    a4 = p1 - float(w @ q1)
    parts = dict(p1=p1, p2=p2, q0=q0, q1=q1, q2=q2)
    return np.array([a1, a2, a3, a4]), parts


def quartic_value(a, tau):
    return ((a[0] * tau + a[1]) * tau + a[2]) * tau * tau + a[3] * tau


def quartic_step(a) -> float:
    """Step of the exact line search: a real root of 4a1 t^3 + 3a2 t^2 + 2a3 t + a4 = 0
    (App. A.2).  Among the positive real roots the one with the lowest quartic
    value is taken (the smaller on a tie).  Returns 0.0 when no positive root
    lowers the quartic (not a descent direction)."""
    a1, a2, a3, a4 = (float(x) for x in a)
    coeffs = [4.0 * a1, 3.0 * a2, 2.0 * a3, a4]
    # strip leading zeros (degenerate quartic)
    while coeffs and coeffs[0] == 0.0:
        coeffs = coeffs[1:]
    if len(coeffs) <= 1:
        return 0.0
    roots = np.roots(coeffs)
    scale = max(1.0, float(np.max(np.abs(roots)))) if len(roots) else 1.0
    real = [float(t.real) for t in roots if abs(t.imag) <= 1e-9 * scale]

    def fp(t):
        return ((4.0 * a1 * t + 3.0 * a2) * t + 2.0 * a3) * t + a4

    def fpp(t):
        return (12.0 * a1 * t + 6.0 * a2) * t + 2.0 * a3

    polished = []
    for t in real:
        for _ in range(3):                       # Newton polish in FP64
            d = fpp(t)
            if d == 0.0:
                break
            t_new = t - fp(t) / d
            if not math.isfinite(t_new):
                break
            t = t_new
        polished.append(t)
    best, best_f = 0.0, 0.0
    for t in sorted(polished):
        if t <= 0.0:
            continue
        f = quartic_value((a1, a2, a3, a4), t)
        if f < best_f:
            best, best_f = t, f
    return best


# ----------------------------------------------------------------------------- L-BFGS

def lbfgs_direction(G: np.ndarray, S: list, Y: list, scaling: int = 0) -> np.ndarray:
    """Search direction of Algorithm 1 (two-loop recursion).

    ``S`` and ``Y`` hold the stored pairs oldest first; beta_t = 1/<y^t, s^t>.
    The initial matrix is I as printed (scaling = 0) or gamma I with
    gamma = <s,y>/<y,y> of the newest pair (scaling = 1, the usual L-BFGS choice).
    """
    D = -G.copy()
    T = len(S)
    alpha = [0.0] * T
    beta = [1.0 / float(np.sum(Y[t] * S[t])) for t in range(T)]
    for t in range(T - 1, -1, -1):                  # newest to oldest
        alpha[t] = beta[t] * float(np.sum(S[t] * D))
        D = D - alpha[t] * Y[t]
    if scaling and T:
        D = D * (float(np.sum(S[-1] * Y[-1])) / float(np.sum(Y[-1] * Y[-1])))
    for t in range(T):                              # oldest to newest
        D = D + (alpha[t] - beta[t] * float(np.sum(Y[t] * D))) * S[t]
    return D


# ----------------------------------------------------------------------------- errors

def sigma_min(P: Problem, y: np.ndarray, dense_limit: int = 3000) -> float:
    """Smallest eigenvalue of the dual slack C - A*(y) (Sec. 4.2, err2)."""
    S = (P.C - adjoint(P, y)).tocsr()
    if P.n <= dense_limit:
        return float(np.linalg.eigvalsh(S.toarray())[0])
    from scipy.sparse.linalg import eigsh
    vals = eigsh(S, k=1, which="SA", tol=1e-10, maxiter=20000,
                 v0=np.ones(P.n), return_eigenvectors=False)
    return float(vals[0])


def errors(P: Problem, R: np.ndarray, y: np.ndarray, with_err2: bool = False):
    """Error measures of Sec. 4.2 with the readings used by the solver:
    err1 normalised by 1 + ||b||_inf, err3 signed, err2 by 1 + ||vec C||_1."""
    z = constraint_map(P, R, R) - P.b
    obj = objective(P, R)
    dual = float(P.b @ y)
    out = dict(
        err1=float(np.linalg.norm(z)) / (1.0 + float(np.max(np.abs(P.b)))),
        err1_l1=float(np.linalg.norm(z)) / (1.0 + float(np.sum(np.abs(P.b)))),
        err3=(obj - dual) / (1.0 + abs(obj) + abs(dual)),
        primal_obj=obj, dual_obj=dual,
    )
    if with_err2:
        smin = sigma_min(P, y)
        out["sigma_min"] = smin
        out["err2"] = abs(min(0.0, smin)) / (1.0 + float(np.abs(P.C.data).sum()))
    return out


# ----------------------------------------------------------------------------- randomness

_MASK = (1 << 64) - 1


def splitmix64(state: int, count: int):
    """SplitMix64 (Steele, Lea, Flood 2014), the published 64-bit mixing generator.
    Returns (outputs, new_state)."""
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return out, state


def gaussian_columns(n: int, k: int, seed: int, stream: int) -> np.ndarray:
    """n x k standard normals for new rank columns: entry (i, c) uses the two
    SplitMix64 outputs at counter 2*(i*k + c) of the sequence seeded by
    seed ^ (stream * golden), turned into a normal by Box-Muller
    (u1 in (0,1], u2 in [0,1): sqrt(-2 ln u1) cos(2 pi u2))."""
    base = (seed ^ ((stream * 0x9E3779B97F4A7C15) & _MASK)) & _MASK
    out = np.empty((n, k))
    for i in range(n):
        for c in range(k):
            ctr = 2 * (i * k + c)
            (x1, x2), _ = splitmix64((base + ctr * 0x9E3779B97F4A7C15) & _MASK, 2)
            u1 = ((x1 >> 11) + 1) * (1.0 / 9007199254740992.0)
            u2 = (x2 >> 11) * (1.0 / 9007199254740992.0)
            out[i, c] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
    return out


def rank_update_size(r: int, m: int) -> int:
    """r_new = min(ceil(1.5 r), ceil(sqrt(2m)))  (App. A.1)."""
    return int(min(math.ceil(1.5 * r), math.ceil(math.sqrt(2.0 * m))))


# ----------------------------------------------------------------------------- solver

@dataclass
class Params:
    """Solver constants.  The paper leaves all but ``tol`` and the rank rule
    unspecified (it defers them to the CPU LoRADS paper); the values below are
    the readings the GPU library uses too."""
    tol: float = 1e-5                 # epsilon of Sec. 4.2
    lbfgs_mem: int = 4                # T of Algorithm 1
    max_inner: int = 500              # K of Algorithm 1 (per outer step)
    max_outer: int = 200
    rho0: float = 0.0                 # <= 0: 1 / mean |C_ij| over stored entries
    rho_growth: float = 2.0
    rho_max: float = 1e12
    infeas_decrease: float = 0.25     # rho grows unless err1 shrank by this factor
    inner_rel: float = 1.0            # inner stop: ||G||_F <= inner_rel * max(||A(RR^T)-b||, tol (1+||b||_inf))
    rank_update_threshold: int = 3    # outer steps in a row that hit max_inner
    lbfgs_scaling: int = 1            # 0: initial matrix I (Algorithm 1); 1: gamma I
    rho_policy: int = 2               # 1: rho grows only after a converged inner loop;
                                      # 2: also after a capped loop that raised err1
    inner_scale: int = 2              # 1: inner stop against rho ||z|| instead of ||z||;
                                      # 2: as 1, capped by inner_progress * ||G|| at the loop start
    inner_progress: float = 0.1
    seed: int = 0
    time_limit: float = 1e4           # seconds (Sec. 4.2)
    stop_rule: int = 0                # 0: err1 and |err3| <= tol; 1: err1 <= tol alone (the
                                      # primal-feasibility stop that precedes re-opt, Sec. 4.1)


def auto_rho(P: Problem) -> float:
    d = np.abs(P.C.data)
    d = d[d > 0]
    return 1.0 / float(d.mean()) if len(d) else 1.0


def solve(P: Problem, R0: np.ndarray, params: Params | None = None,
          y0: np.ndarray | None = None, rho: float | None = None,
          record: list | None = None):
    """ALM on the Burer-Monteiro factorisation (Sec. 2.1) with the L-BFGS inner
    solver of Algorithm 1, the exact line search of App. A.2 and the rank rule
    of App. A.1.  Returns a dict with R, y, rho, errors and counters."""
    prm = params or Params()
    t0 = time.perf_counter()
    R = np.array(R0, dtype=np.float64, copy=True)
    y = np.zeros(P.m) if y0 is None else np.array(y0, dtype=np.float64, copy=True)
    rho = prm.rho0 if (rho is None and prm.rho0 > 0) else (rho or auto_rho(P))
    bnorm_inf = float(np.max(np.abs(P.b))) if P.m else 0.0

    z = constraint_map(P, R, R) - P.b
    err1 = float(np.linalg.norm(z)) / (1.0 + bnorm_inf)
    total_inner = 0
    hit_cap_streak = 0
    status = "maxiter"
    outer = 0
    for outer in range(prm.max_outer):
        # ---- inner: argmin_R L_rho(R, y) by Algorithm 1
        S: list = []
        Yh: list = []
        G = gradient(P, R, y, rho)
        g0 = float(np.linalg.norm(G))
        k = 0                                   # directions computed
        while k < prm.max_inner:
            # stop once the gradient is small next to the current infeasibility
            zc = float(np.linalg.norm(constraint_map(P, R, R) - P.b))
            if prm.inner_scale == 0:
                thr = prm.inner_rel * max(zc, prm.tol * (1.0 + bnorm_inf))
            elif prm.inner_scale == 1:
                thr = prm.inner_rel * max(rho * zc, prm.tol * (1.0 + bnorm_inf))
            else:
                thr = max(prm.tol * (1.0 + bnorm_inf), min(prm.inner_rel * rho * zc, prm.inner_progress * g0))
            if float(np.linalg.norm(G)) <= thr:
                break
            D = lbfgs_direction(G, S, Yh, prm.lbfgs_scaling)
            k += 1
            a, _ = linesearch_coeffs(P, R, D, y, rho)
            tau = quartic_step(a)
            if tau <= 0.0:
                if S:                           # no descent along -H G: drop the memory,
                    S.clear()                   # the next direction is -G
                    Yh.clear()
                    continue
                break
            R_new = R + tau * D
            G_new = gradient(P, R_new, y, rho)
            s = tau * D
            yv = G_new - G
            ys = float(np.sum(yv * s))
            if ys > 1e-16 * float(np.linalg.norm(yv)) * float(np.linalg.norm(s)):
                S.append(s)
                Yh.append(yv)
                if len(S) > prm.lbfgs_mem:
                    S.pop(0)
                    Yh.pop(0)
            else:
                S.clear()
                Yh.clear()
            R, G = R_new, G_new
        total_inner += k
        # ---- multiplier step (Sec. 2.1) and error check (Sec. 4.2)
        z = constraint_map(P, R, R) - P.b
        y = y - rho * z
        err1_new = float(np.linalg.norm(z)) / (1.0 + bnorm_inf)
        e = errors(P, R, y)
        if record is not None:
            record.append(dict(outer=outer, inner=k, rho=rho, err1=err1_new,
                               err3=e["err3"], obj=e["primal_obj"], r=R.shape[1]))
        if err1_new <= prm.tol and (prm.stop_rule == 1 or abs(e["err3"]) <= prm.tol):
            status = "ok"
            err1 = err1_new
            break
        grow = err1_new > prm.infeas_decrease * err1
        if prm.rho_policy == 1:
            grow = grow and k < prm.max_inner
        elif prm.rho_policy == 2:
            grow = grow and (k < prm.max_inner or err1_new > err1)
        if grow:
            rho = min(rho * prm.rho_growth, prm.rho_max)
        err1 = err1_new
        if outer == prm.max_outer - 1:
            break                               # out of outer steps: no rank update after the last one
        # ---- dynamic rank (App. A.1)
        hit_cap_streak = hit_cap_streak + 1 if k >= prm.max_inner else 0
        if hit_cap_streak >= prm.rank_update_threshold:
            r_new = rank_update_size(R.shape[1], P.m)
            if r_new > R.shape[1]:
                scale = 1e-3 * float(np.linalg.norm(R)) / math.sqrt(R.size)
                extra = scale * gaussian_columns(P.n, r_new - R.shape[1], prm.seed, outer)
                R = np.hstack([R, extra])
            hit_cap_streak = 0
        if time.perf_counter() - t0 > prm.time_limit:
            status = "timeout"
            break
    e = errors(P, R, y)
    return dict(R=R, y=y, rho=rho, status=status, outer=outer + 1,
                inner=total_inner, seconds=time.perf_counter() - t0, **e)


# ----------------------------------------------------------------------------- brute force

def maxcut_bruteforce(n: int, edges) -> float:
    """Exact max cut value by enumerating all 2^(n-1) cuts (n <= ~20)."""
    i, j, w = (np.asarray(x) for x in edges)
    best = -np.inf
    for mask in range(1 << (n - 1)):
        side = (mask >> np.arange(n)) & 1
        val = float(np.sum(w[side[i] != side[j]]))
        best = max(best, val)
    return best
