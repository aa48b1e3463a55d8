"""Failure statuses of the solve, reached without any GPU fault (error handling
of the ABI: every call returns a status; Sec. 4.2 fixes the time limit).

* A host time limit shorter than one polling batch ends lorads_solve with
  LORADS_ERR_TIMEOUT; the context stays usable and the next solve converges.
* The batched solve's per-instance limit (device clock, checked after each
  outer step) marks those instances LORADS_ERR_TIMEOUT; the launch completes.
* A non-finite starting factor or multiplier reaches the iteration's
  finiteness checks and ends the solve with LORADS_ERR_NUMERIC.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    L.build()


def _er(n=2000, seed=3):
    return W.maxcut_instance(n, W.er_graph(n, 2 * n, seed, "pm1"))


def test_host_time_limit_returns_timeout_and_context_recovers():
    inst = _er()
    R0 = W.initial_factor(inst, 11, 1)
    ctx = L.lorads_create(inst, L.default_params(time_limit=1e-6))
    try:
        res = L.lorads_solve(ctx, R0)
        assert res["status_name"] == "LORADS_ERR_TIMEOUT", res
        assert 0 < res["inner_iters"] < 500
    finally:
        L.lorads_destroy(ctx)
    ctx = L.lorads_create(inst, L.default_params())
    try:
        assert L.lorads_solve(ctx, R0)["status_name"] == "LORADS_OK"
    finally:
        L.lorads_destroy(ctx)


def test_batch_instance_time_limit_returns_timeout():
    insts = [_er(600, 1), _er(900, 2)]
    R0 = [W.initial_factor(t, 10, 5 + i) for i, t in enumerate(insts)]
    b = L.lorads_batch_create(insts, L.default_params(time_limit=1e-9), R0=R0)
    try:
        res, stats = L.lorads_batch_solve(b, len(insts))
    finally:
        L.lorads_batch_destroy(b)
    assert [r["status_name"] for r in res] == ["LORADS_ERR_TIMEOUT"] * 2, res
    assert stats["solved"] == 0
    assert all(r["outer_iters"] == 1 for r in res)


@pytest.mark.parametrize("where", ["R0_nan", "R0_inf", "y0_nan"])
def test_non_finite_start_returns_numeric(where):
    inst = _er(500, 4)
    R0 = W.initial_factor(inst, 9, 2)
    y0 = None
    if where == "R0_nan":
        R0[17, 3] = np.nan
    elif where == "R0_inf":
        R0[250, 0] = np.inf
    else:
        y0 = np.zeros(inst.m)
        y0[42] = np.nan
    ctx = L.lorads_create(inst, L.default_params())
    try:
        res = L.lorads_solve(ctx, R0, y0=y0)
    finally:
        L.lorads_destroy(ctx)
    assert res["status_name"] == "LORADS_ERR_NUMERIC", res
