"""Plain FP64 CPU oracle of the re-optimisation (re-opt) of cuLoRADS, Sec. 4.1.

TEST INFRASTRUCTURE.  Only the tests may import or run this module; the GPU
library never calls it and shares no code with it.  It drives the ALM solve
of ``lorads_oracle`` (sign convention y = -lambda, as there).

The procedure.  The solve first stops on primal feasibility alone (err1 with
1 + ||b||_inf at most tol: the reoptLevel-0 rule of Sec. 4.2).  If the final
criteria of the chosen level do not hold -- level 1: err1 with 1 + ||b||_1
and the primal-dual gap err3; level 2: also the dual infeasibility err2
(Sec. 4.2) -- the objective matrix is scaled down by the re-opt factor (0.1
in the paper), the scaled problem is solved again from the previous output,
and the errors are evaluated anew on the original problem; this repeats
until the criteria hold or the re-opt budget is spent.

Readings where the paper is silent:
  * warm start: R unchanged, the multiplier scaled with C (the scaled
    problem's dual is s y), so that y = y_s / s on the original problem;
    rho carries over unchanged;
  * the factor compounds: after k rounds C is scaled by factor^k;
  * the gap criterion compares |err3| (the same absolute value the main stop
    test uses);
  * at most max_reopt rounds (default 5).

Parity pins: tests/test_reopt_oracle.py -- the scaled problem's optimum and
multiplier against s times the original's (the exact scaling of an SDP), the
closed-form value of an odd cycle reached by a level-1 re-opt that the
primal-only stop leaves with err3 above tol, err2 below tol after level 2, and
no round when the criteria already hold.
"""
from __future__ import annotations

import copy
from dataclasses import asdict

from . import lorads_oracle as O

__all__ = ["scaled_problem", "criteria_met", "solve_reopt"]


def scaled_problem(P: O.Problem, s: float) -> O.Problem:
    """The same SDP with objective matrix s C."""
    Ps = copy.copy(P)
    Ps.C = P.C * s
    return Ps


def criteria_met(e: dict, level: int, tol: float) -> bool:
    """Final criteria of re-opt level 1 (err1 with 1 + ||b||_1, |err3|) or 2 (also err2), Sec. 4.2."""
    ok = e["err1_l1"] <= tol and abs(e["err3"]) <= tol
    if level >= 2:
        ok = ok and e["err2"] <= tol
    return ok


def solve_reopt(P: O.Problem, R0, level: int = 1, factor: float = 0.1, max_reopt: int = 5,
                params: O.Params | None = None):
    """ALM solve with the primal-feasibility stop, then re-opt rounds until the
    criteria of ``level`` hold.  Returns the original problem's R, y, errors,
    the number of rounds, the final scale and the total L-BFGS iterations."""
    prm = params or O.Params()
    base = O.Params(**{**asdict(prm), "stop_rule": 1})
    res = O.solve(P, R0, base)
    R, y_s, rho = res["R"], res["y"], res["rho"]
    scale, rounds, inner = 1.0, 0, res["inner"]
    while True:
        y = y_s / scale
        e = O.errors(P, R, y, with_err2=level >= 2)
        if level == 0 or criteria_met(e, level, prm.tol) or rounds >= max_reopt:
            break
        scale *= factor
        rounds += 1
        res = O.solve(scaled_problem(P, scale), R, base, y0=y * scale, rho=rho)
        R, y_s, rho = res["R"], res["y"], res["rho"]
        inner += res["inner"]
    met = res["status"] == "ok" if level == 0 else criteria_met(e, level, prm.tol)
    return dict(R=R, y=y, rho=rho, rounds=rounds, scale=scale, inner=inner,
                status="ok" if met else "maxiter", **e)
