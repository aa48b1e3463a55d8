"""Plain FP64 CPU oracle of the splitting (ADMM) stage of LoRADS, Sec. 2.2.

TEST INFRASTRUCTURE.  Only the tests may import or run this module; the GPU
library never calls it and shares no code with it.  It reuses the linear maps
of ``lorads_oracle`` (A(UV^T), A*(v), C R) and that module's sign convention:
the dual variable is y = -lambda of the paper's body.

The stage.  Once the ALM stage (Sec. 2.1; ``lorads_oracle.solve``) has brought
the primal infeasibility below a switch threshold, LoRADS splits X = U V^T and
works on the Lagrangian of Eq. (1.3), here in the sign of y:

    L_rho(U, V, y) = <C, U V^T> - y^T (A(U V^T) - b) + rho/2 ||A(U V^T) - b||^2
                     + rho/2 ||U - V||_F^2

with the three ADMM steps of Eq. (2.2):

    U <- argmin_U L_rho(U, V, y),   V <- argmin_V L_rho(U, V, y),
    y <- y - rho (A(U V^T) - b).

Each argmin is the positive definite linear system of Eq. (2.3).  For the U
step (V fixed):

    frakA_V(U) = rho A*(A(U V^T)) V + rho U
    frakb_V    = -C V + A*(y) V + rho A*(b) V + rho V

This is what setting the U-gradient of L_rho to zero gives.  The vectorised
form printed as Eq. (2.4) drops the factor rho of the sum and flips the sign
of the rho A*(b) V term; read it as
(rho sum_k vec(A_k V) vec(A_k V)^T + rho I) vec(U) = vec(frakb_V), which agrees
with Eq. (2.3).  C and every A_k are symmetric, so A(U V^T) = A(V U^T) and the V step is the
same system with U and V exchanged.  Both are solved by the conjugate
gradients of Algorithm 2, started from the current iterate.

Readings where the paper is silent (all are parameters of ``AdmmParams``):
  * CG stop: ||r_k||_F <= cg_rel * ||r_0||_F, at most cg_max steps (the
    tolerance epsilon and cap K of Algorithm 2 are not given);
  * switch: the ALM stage runs with its own stopping test (err1 and |err3|,
    Sec. 4.2) at the looser tolerance switch_err1; the ADMM stage then starts
    from U = V = R and the ALM stage's y;
  * rho: the ALM stage's last rho, held fixed through the ADMM stage (no
    schedule is given for it);
  * stop: the errors of Sec. 4.2 at R = (U + V)/2, whose X = R R^T is positive
    semidefinite; err1 and |err3| <= tol, as in the ALM stage.

Parity pins: tests/test_admm_oracle.py -- the operator against the dense
n r x n r matrix of Eq. (2.4) assembled from the A_k, the system's solution
against a dense solve and a zero finite-difference gradient of L_rho, CG
against the dense solve, monotone decrease of L_rho over the block steps,
closed-form MaxCut SDP values and the ALM-only optimum.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import lorads_oracle as O

__all__ = ["AdmmParams", "split_lagrangian", "system_operator", "system_rhs", "cg", "admm_stage",
           "solve_two_stage"]


@dataclass
class AdmmParams:
    """Constants of the ADMM stage (readings, module docstring)."""
    tol: float = 1e-5
    switch_err1: float = 1e-3
    cg_rel: float = 1e-2
    cg_max: int = 50
    max_iter: int = 20000
    time_limit: float = 1e4


def split_lagrangian(P: O.Problem, U: np.ndarray, V: np.ndarray, y: np.ndarray, rho: float) -> float:
    """L_rho(U, V, y) of Eq. (1.3), sign of y."""
    z = O.constraint_map(P, U, V) - P.b
    return (float(np.sum((P.C @ V) * U)) - float(y @ z) + 0.5 * rho * float(z @ z)
            + 0.5 * rho * float(np.sum((U - V) ** 2)))


def system_operator(P: O.Problem, V: np.ndarray, X: np.ndarray, rho: float) -> np.ndarray:
    """frakA_V(X) = rho A*(A(X V^T)) V + rho X  (left side of Eq. (2.3))."""
    return rho * (O.adjoint(P, O.constraint_map(P, X, V)) @ V) + rho * X


def system_rhs(P: O.Problem, V: np.ndarray, y: np.ndarray, rho: float) -> np.ndarray:
    """frakb_V = -C V + A*(y) V + rho A*(b) V + rho V  (right side of Eq. (2.3))."""
    return -(P.C @ V) + O.adjoint(P, y) @ V + rho * (O.adjoint(P, P.b) @ V) + rho * V


def cg(P: O.Problem, V: np.ndarray, X0: np.ndarray, rhs: np.ndarray, rho: float,
       cg_rel: float, cg_max: int):
    """Conjugate gradients of Algorithm 2 on frakA_V(X) = rhs from X0.

    Stops when ||r||_F <= cg_rel * ||r_0||_F or after cg_max steps.  Returns
    (X, steps)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    r = rhs - system_operator(P, V, X, rho)
    eps = cg_rel * float(np.linalg.norm(r))
    if float(np.linalg.norm(r)) <= eps or float(np.linalg.norm(r)) == 0.0:
        return X, 0
    p = r.copy()
    rr = float(np.sum(r * r))
    for k in range(cg_max):
        Q = system_operator(P, V, p, rho)
        alpha = rr / float(np.sum(p * Q))
        X = X + alpha * p
        r = r - alpha * Q
        rr_new = float(np.sum(r * r))
        if math.sqrt(rr_new) <= eps:
            return X, k + 1
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return X, cg_max


def admm_stage(P: O.Problem, R: np.ndarray, y: np.ndarray, rho: float, params: AdmmParams | None = None,
               record: list | None = None):
    """The ADMM stage of Eq. (2.2) from U = V = R.  Returns a dict with the
    averaged factor R = (U + V)/2, U, V, y, the errors of Sec. 4.2 at R and the
    iteration and CG-step counts."""
    prm = params or AdmmParams()
    t0 = time.perf_counter()
    U = np.array(R, dtype=np.float64, copy=True)
    V = U.copy()
    y = np.array(y, dtype=np.float64, copy=True)
    cg_steps = 0
    status = "maxiter"
    it = 0
    e = O.errors(P, U, y)
    for it in range(1, prm.max_iter + 1):
        U, k1 = cg(P, V, U, system_rhs(P, V, y, rho), rho, prm.cg_rel, prm.cg_max)
        V, k2 = cg(P, U, V, system_rhs(P, U, y, rho), rho, prm.cg_rel, prm.cg_max)
        cg_steps += k1 + k2
        y = y - rho * (O.constraint_map(P, U, V) - P.b)
        Rm = 0.5 * (U + V)
        e = O.errors(P, Rm, y)
        if record is not None:
            record.append(dict(it=it, cg=(k1, k2), err1=e["err1"], err3=e["err3"], obj=e["primal_obj"],
                               split=float(np.linalg.norm(U - V))))
        if e["err1"] <= prm.tol and abs(e["err3"]) <= prm.tol:
            status = "ok"
            break
        if time.perf_counter() - t0 > prm.time_limit:
            status = "timeout"
            break
    return dict(R=0.5 * (U + V), U=U, V=V, y=y, rho=rho, status=status, iters=it, cg_steps=cg_steps,
                seconds=time.perf_counter() - t0, **e)


def solve_two_stage(P: O.Problem, R0: np.ndarray, alm: O.Params | None = None,
                    admm: AdmmParams | None = None, record: list | None = None):
    """LoRADS's two stages: the ALM stage of Sec. 2.1 until err1 <= switch_err1
    (or its own convergence), then the ADMM stage of Sec. 2.2."""
    aprm = admm or AdmmParams()
    base = alm or O.Params()
    first = O.solve(P, R0, O.Params(**{**base.__dict__, "tol": max(aprm.switch_err1, base.tol)}))
    if first["err1"] <= aprm.tol and abs(first["err3"]) <= aprm.tol:
        return dict(first, stage="alm", alm_inner=first["inner"], admm_iters=0, cg_steps=0)
    second = admm_stage(P, first["R"], first["y"], first["rho"], aprm, record)
    return dict(second, stage="admm", alm_inner=first["inner"], alm_outer=first["outer"],
                admm_iters=second["iters"])
