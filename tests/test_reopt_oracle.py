"""Pins of the re-opt oracle (Sec. 4.1) against what the mathematics fixes.

* Scaling the objective matrix by s scales the SDP's optimal value and its
  dual optimum by s: independent tight solves of P and of s P agree after
  dividing by s (the mapping re-opt relies on).
* The primal-feasibility stop leaves the odd cycle C_7 with err3 above tol;
  level-1 re-opt restores it and reaches the closed-form value
  (n/2)(1 + cos(pi/n)); level 2 also meets err2.
* No round is taken when the criteria already hold.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O
from oracle import reopt_oracle as RO


@pytest.mark.parametrize("name", ["complete_10", "odd_cycle_7"])
def test_scaled_problem_scales_value_and_multiplier(name):
    inst = (W.maxcut_instance(10, W.complete_graph(10)) if name == "complete_10"
            else W.maxcut_instance(7, W.cycle_graph(7)))
    P = O.Problem(inst)
    R0 = W.initial_factor(inst, 4, 1)
    s = 0.1
    a = O.solve(P, R0, O.Params(tol=1e-9))
    b = O.solve(RO.scaled_problem(P, s), R0, O.Params(tol=1e-9))
    assert a["status"] == b["status"] == "ok"
    assert b["primal_obj"] / s == pytest.approx(a["primal_obj"], rel=1e-7)
    assert np.max(np.abs(b["y"] / s - a["y"])) <= 1e-6 * (1 + np.abs(a["y"]).max())
    # the scaled copy leaves the original problem untouched
    assert np.array_equal(P.C.toarray(), O.Problem(inst).C.toarray())


def _cycle():
    inst = W.maxcut_instance(7, W.cycle_graph(7))
    return O.Problem(inst), W.initial_factor(inst, 3, 1), 3.5 * (1 + math.cos(math.pi / 7))


def test_primal_stop_leaves_the_gap_open_on_the_odd_cycle():
    P, R0, _ = _cycle()
    res = RO.solve_reopt(P, R0, level=0)
    assert res["status"] == "ok" and res["rounds"] == 0
    assert res["err1"] <= 1e-5 and abs(res["err3"]) > 1e-5


@pytest.mark.parametrize("level", [1, 2])
def test_reopt_meets_the_level_criteria_and_the_closed_form(level):
    P, R0, value = _cycle()
    res = RO.solve_reopt(P, R0, level=level)
    assert res["status"] == "ok" and res["rounds"] >= 1 and res["scale"] < 1
    assert RO.criteria_met(res, level, 1e-5)
    if level == 2:
        assert res["err2"] <= 1e-5
    assert -res["primal_obj"] == pytest.approx(value, rel=1e-6)


def test_no_round_when_the_criteria_hold():
    inst = W.maxcut_instance(60, W.er_graph(60, 200, 11, "pm1"))
    res = RO.solve_reopt(O.Problem(inst), W.initial_factor(inst, 6, 1), level=2)
    assert res["status"] == "ok" and res["rounds"] == 0 and res["scale"] == 1.0
