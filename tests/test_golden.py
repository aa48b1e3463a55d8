"""The oracle against the exact fixture ``golden/lagrangian_exact.txt``.

The fixture's values come from symbolic expansion of the definitions (the
augmented Lagrangian of Sec. 2 in the dual-variable sign, its derivative, the
quartic of the exact line search of App. A.2 and the constraint map), written
by ``golden/make_golden.py`` with sympy: a dropped term, a wrong sign of y or
rho, a missing factor 2 of an off-diagonal constraint or of the gradient fails
here independently of the oracle's own formulas.
"""
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import lorads_oracle as O

FIXTURE = Path(__file__).resolve().parent / "golden" / "lagrangian_exact.txt"


def _num(tok: str) -> float:
    return float(Fraction(tok))


def _matrix(text: str) -> np.ndarray:
    return np.array([[_num(t) for t in row.split()] for row in text.split(";")])


def _cases():
    cases, cur = [], None
    for line in FIXTURE.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "instance":
            cur = {"name": rest}
            cases.append(cur)
        else:
            cur[key] = rest
    return cases


CASES = _cases()


def _instance(c):
    n, m = int(c["n"]), int(c["m"])
    C = _matrix(c["C"])
    b = np.array([_num(t) for t in c["b"].split()])
    if "edges" in c:
        e = np.array([[int(t) for t in row.split()] for row in c["edges"].split(";")])
        inst = W.maxcut_instance(n, (e[:, 0], e[:, 1], e[:, 2].astype(float)))
        # the workload generator's C = -L/4 is the fixture's
        Cw = sp.csr_matrix((inst.val, inst.colind, inst.rowptr), shape=(n, n)).toarray()
        np.testing.assert_array_equal(Cw, C)
        np.testing.assert_array_equal(inst.b, b)
        return inst
    trip = np.array([[_num(t) for t in row.split()] for row in c["triplets"].split(";")])
    Cs = sp.csr_matrix(C)
    Cs.sort_indices()
    return W.SDPInstance(
        n=n, rowptr=Cs.indptr.astype(np.int64), colind=Cs.indices.astype(np.int32), val=Cs.data.astype(np.float64),
        m=m, con=trip[:, 0].astype(np.int32), row=trip[:, 1].astype(np.int32), col=trip[:, 2].astype(np.int32),
        aval=trip[:, 3].astype(np.float64), b=b, kind="generic")


def test_fixture_has_the_four_instances():
    assert [c["name"] for c in CASES] == ["maxcut_triangle", "mc_2x2", "generic_4", "multi_entry_4"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_oracle_matches_exact_definitions(case):
    P = O.Problem(_instance(case))
    R, D = _matrix(case["R"]), _matrix(case["D"])
    y = np.array([_num(t) for t in case["y"].split()])
    rho = _num(case["rho"])
    z = np.array([_num(t) for t in case["z"].split()])
    np.testing.assert_allclose(O.constraint_map(P, R, R), z, rtol=0, atol=1e-13)
    L = _num(case["L"])
    assert O.lagrangian(P, R, y, rho) == pytest.approx(L, rel=1e-14, abs=1e-13)
    G = _matrix(case["G"])
    np.testing.assert_allclose(O.gradient(P, R, y, rho), G, rtol=1e-14, atol=1e-13)
    a_exact = np.array([_num(t) for t in case["a"].split()])
    a, _ = O.linesearch_coeffs(P, R, D, y, rho)
    np.testing.assert_allclose(a, a_exact, rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_error_measures_match_exact_values(case):
    """errors() against Sec. 4.2's measures evaluated exactly (sympy): <C,X> and
    b^T y as fractions, err1 in both normalisations, the signed err3, and err2
    from the smallest root of the exact characteristic polynomial of C - A*(y).
    A wrong denominator, a sign of err3 or of y in the dual slack, or a dropped
    off-diagonal half of A*(y) fails one of them."""
    P = O.Problem(_instance(case))
    R = _matrix(case["R"])
    y = np.array([_num(t) for t in case["y"].split()])
    e = O.errors(P, R, y, with_err2=True)
    assert e["primal_obj"] == pytest.approx(_num(case["obj"]), rel=1e-14, abs=1e-14)
    assert e["dual_obj"] == pytest.approx(_num(case["by"]), rel=1e-14, abs=1e-14)
    assert e["err1"] == pytest.approx(float(case["err1"]), rel=1e-14)
    assert e["err1_l1"] == pytest.approx(float(case["err1_l1"]), rel=1e-14)
    assert e["err3"] == pytest.approx(_num(case["err3"]), rel=1e-14, abs=1e-15)
    assert e["sigma_min"] == pytest.approx(float(case["smin"]), rel=1e-12, abs=1e-13)
    assert e["err2"] == pytest.approx(float(case["err2"]), rel=1e-12, abs=1e-13)
