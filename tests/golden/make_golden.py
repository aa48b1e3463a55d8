"""Writes the exact fixtures ``lagrangian_exact.txt`` and ``maxcut_sdp_values.txt``
of this folder.

For four tiny SDPs with integer factors, the fixture holds, as exact
fractions obtained by symbolic expansion of the definitions (sympy; neither
the CUDA library nor the oracle is used):

* L_rho(R, y) = <C, R R^T> - y^T (A(R R^T) - b) + rho/2 ||A(R R^T) - b||^2, the
  augmented Lagrangian of Sec. 2 (Eq. (1.2)) written with the dual variable
  y = -lambda, and its gradient dL/dR (entry by entry, symbolic derivative);
* the coefficients of L_rho(R + tau D, y) - L_rho(R, y)
  = a1 tau^4 + a2 tau^3 + a3 tau^2 + a4 tau  (exact line search, App. A.2);
* the constraint values A(R R^T) (Sec. 2 notation: <A_k, X> with the
  single-entry convention <A_k, X> = a X_ii, or 2 a X_ij for i != j);
* the error measures of Sec. 4.2 at (R, y) with the readings the solver uses:
  <C, X>, b^T y, err1 = ||A(X) - b||_2 / (1 + ||b||_inf) (and its 1 + ||b||_1
  form), the signed err3 = (<C,X> - b^T y) / (1 + |<C,X>| + |b^T y|), and
  err2 = |min(0, sigma_min(C - A*(y)))| / (1 + ||vec C||_1), sigma_min taken as
  the smallest real root of the exact characteristic polynomial of the rational
  matrix C - A*(y), to 30 digits.

Instances: the MaxCut SDP of Sec. 4.3 on a triangle with weights +1, -1, +1
(C = -L/4, X_ii = 1); a 2 x 2 matrix-completion SDP of Sec. 4.4 (C = I of
order 4, two sampled entries, X_{i,2+j} + X_{2+j,i} = 2 M_ij); a generic
instance with a mixed-sign C, one diagonal and two off-diagonal constraints;
and one whose constraints have several entries each (general SDPs, Sec. 4.5).

``maxcut_sdp_values.txt`` holds closed-form optimal values of the MaxCut SDP
(max <L/4, X>, diag X = 1, X PSD) of Sec. 4.3 for unit weights: n^2/4 on the
complete graph K_n (X = (n I - J)/(n - 1) attains the bound <L/4, X> <= n^2/4);
(n/2)(1 + cos(pi/n)) on an odd cycle C_n (vectors at consecutive angles
pi (n-1)/n, the classical value of the cycle's relaxation); |E| on a bipartite
graph (each edge term (1 - X_ij)/2 is at most 1 and the cut of the bipartition
attains it).

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

from pathlib import Path

import sympy as S

HERE = Path(__file__).resolve().parent


def _frac(x) -> str:
    x = S.nsimplify(x)
    return f"{x.p}/{x.q}" if x.q != 1 else f"{x.p}"


def _cases():
    half = S.Rational(1, 2)
    cases = []
    # MaxCut triangle: edges (i, j, w); C = -L/4, L_ii = sum_k w_ik, L_ij = -w_ij
    edges = [(0, 1, 1), (1, 2, -1), (0, 2, 1)]
    n = 3
    C = S.zeros(n, n)
    for i, j, w in edges:
        C[i, j] += S.Rational(w, 4)
        C[j, i] += S.Rational(w, 4)
        C[i, i] -= S.Rational(w, 4)
        C[j, j] -= S.Rational(w, 4)
    cases.append(dict(
        name="maxcut_triangle", n=n, C=C, edges=edges,
        triplets=[(k, k, k, 1) for k in range(n)], b=[1, 1, 1],
        R=[[1, 0], [0, 2], [1, -1]], D=[[2, 1], [-1, 0], [0, 3]],
        y=[half, -1, S.Rational(3, 4)], rho=S.Rational(3, 2)))
    # matrix completion 2 x 2, rows of U are 0, 1 and rows of V are 2, 3; samples
    # (i, j) -> constraint u_i . v_j = M_ij, i.e. triplet (k, i, 2 + j, a = 1), b = 2 M_ij
    cases.append(dict(
        name="mc_2x2", n=4, C=S.eye(4), edges=None,
        triplets=[(0, 0, 2, 1), (1, 1, 3, 1)], b=[2 * 3, 2 * (-2)],
        R=[[1, 1], [0, -1], [2, 0], [1, 1]], D=[[0, 1], [1, 1], [-1, 0], [2, -1]],
        y=[-1, S.Rational(1, 3)], rho=2))
    # generic: mixed-sign symmetric C, one diagonal and two off-diagonal constraints
    Cg = S.Matrix([[2, -1, 0, half], [-1, 0, 3, 0], [0, 3, -1, 1], [half, 0, 1, 0]])
    cases.append(dict(
        name="generic_4", n=4, C=Cg, edges=None,
        triplets=[(0, 1, 1, S.Rational(3, 2)), (1, 0, 2, 1), (2, 2, 3, -half)], b=[1, -1, 2],
        R=[[1, 0], [1, 1], [0, -2], [3, 1]], D=[[1, -1], [0, 2], [1, 1], [-1, 0]],
        y=[2, -half, 1], rho=S.Rational(5, 4)))
    # a constraint with several entries (general SDPs, Sec. 4.5): k = 0 has three
    cases.append(dict(
        name="multi_entry_4", n=4, C=Cg, edges=None,
        triplets=[(0, 0, 0, 1), (0, 1, 3, -S.Rational(3, 2)), (0, 2, 2, 2), (1, 0, 1, half), (1, 3, 3, 1)],
        b=[3, -2], R=[[1, -1], [2, 0], [0, 1], [1, 1]], D=[[0, 2], [1, -1], [1, 0], [-2, 1]],
        y=[-half, S.Rational(3, 2)], rho=S.Rational(2, 3)))
    return cases


def _constraint_map(case, X):
    out = [S.Integer(0)] * len(case["b"])
    for k, i, j, a in case["triplets"]:
        out[k] += a * X[i, j] if i == j else 2 * a * X[i, j]
    return out


def _lagrangian(case, R, y, rho):
    X = R * R.T
    z = [zk - bk for zk, bk in zip(_constraint_map(case, X), case["b"])]
    obj = sum(case["C"][i, j] * X[i, j] for i in range(case["n"]) for j in range(case["n"]))
    return obj - sum(yk * zk for yk, zk in zip(y, z)) + rho / 2 * sum(zk * zk for zk in z)


def _adjoint(case, y):
    """A*(y) = sum_k y_k A_k, A_k symmetric with a at (i, j) and (j, i)."""
    n = case["n"]
    M = S.zeros(n, n)
    for k, i, j, a in case["triplets"]:
        M[i, j] += y[k] * a
        if i != j:
            M[j, i] += y[k] * a
    return M


def _errors(case, R, y):
    X = R * R.T
    n = case["n"]
    z = [zk - bk for zk, bk in zip(_constraint_map(case, X), case["b"])]
    obj = sum(case["C"][i, j] * X[i, j] for i in range(n) for j in range(n))
    dual = sum(S.nsimplify(bk) * yk for bk, yk in zip(case["b"], y))
    bmax = max(abs(S.nsimplify(v)) for v in case["b"])
    b1 = sum(abs(S.nsimplify(v)) for v in case["b"])
    znorm = S.sqrt(sum(zk * zk for zk in z))
    slack = case["C"] - _adjoint(case, y)
    lam = S.Symbol("lam")
    roots = S.Poly(slack.charpoly(lam).as_expr(), lam).nroots(n=30)
    smin = min(S.re(v) for v in roots)
    c1 = sum(abs(case["C"][i, j]) for i in range(n) for j in range(n))
    return dict(obj=obj, by=dual, err1=(znorm / (1 + bmax)).evalf(30), err1_l1=(znorm / (1 + b1)).evalf(30),
                err3=(obj - dual) / (1 + abs(obj) + abs(dual)), smin=smin,
                err2=(abs(min(S.Integer(0), smin)) / (1 + c1)).evalf(30))


def _block(rows) -> str:
    return "; ".join(" ".join(_frac(v) for v in row) for row in rows)


def main() -> None:
    tau = S.Symbol("tau")
    lines = [
        "# Exact values from the definitions (written by tests/golden/make_golden.py with sympy).",
        "# L = <C,RR^T> - y^T(A(RR^T)-b) + rho/2||A(RR^T)-b||^2  (Sec. 2, Eq. (1.2), y = -lambda);",
        "# a1..a4: L(R + tau D) - L(R) = a1 tau^4 + a2 tau^3 + a3 tau^2 + a4 tau  (App. A.2);",
        "# G = dL/dR; z = A(RR^T).  Matrices: rows separated by ';'.",
        "# obj = <C,RR^T>, by = b^T y, err1/err1_l1/err3/err2 of Sec. 4.2, smin = sigma_min(C - A*(y)).",
    ]
    for case in _cases():
        n = case["n"]
        r = len(case["R"][0])
        R = S.Matrix(case["R"])
        D = S.Matrix(case["D"])
        y = [S.nsimplify(v) for v in case["y"]]
        rho = S.nsimplify(case["rho"])
        L0 = S.expand(_lagrangian(case, R, y, rho))
        poly = S.Poly(S.expand(_lagrangian(case, R + tau * D, y, rho) - L0), tau)
        coeffs = [poly.coeff_monomial(tau ** p) for p in (4, 3, 2, 1)]
        assert poly.coeff_monomial(1) == 0
        Rs = S.Matrix(n, r, lambda i, c: S.Symbol(f"r_{i}_{c}"))
        Ls = _lagrangian(case, Rs, y, rho)
        subs = {Rs[i, c]: R[i, c] for i in range(n) for c in range(r)}
        G = [[S.diff(Ls, Rs[i, c]).subs(subs) for c in range(r)] for i in range(n)]
        z = _constraint_map(case, R * R.T)
        Cd = [[case["C"][i, j] for j in range(n)] for i in range(n)]
        lines += ["", f"instance {case['name']}", f"n {n}", f"m {len(case['b'])}", f"C {_block(Cd)}",
                  "triplets " + "; ".join(f"{k} {i} {j} {_frac(a)}" for k, i, j, a in case["triplets"]),
                  "b " + " ".join(_frac(v) for v in case["b"])]
        if case["edges"] is not None:
            lines.append("edges " + "; ".join(f"{i} {j} {w}" for i, j, w in case["edges"]))
        lines += [f"R {_block(case['R'])}", f"D {_block(case['D'])}", "y " + " ".join(_frac(v) for v in y),
                  f"rho {_frac(rho)}", f"L {_frac(L0)}",
                  "a " + " ".join(_frac(c) for c in coeffs),
                  f"G {_block(G)}", "z " + " ".join(_frac(v) for v in z)]
        e = _errors(case, R, y)
        lines += [f"obj {_frac(e['obj'])}", f"by {_frac(e['by'])}", f"err1 {e['err1']}", f"err1_l1 {e['err1_l1']}",
                  f"err3 {_frac(e['err3'])}", f"smin {S.N(e['smin'], 30)}", f"err2 {e['err2']}"]
    (HERE / "lagrangian_exact.txt").write_text("\n".join(lines) + "\n")
    vals = ["# Closed-form MaxCut SDP values, unit weights (written by tests/golden/make_golden.py).",
            "# family size value expression"]
    for n in (4, 7, 10):
        vals.append(f"complete {n} {S.Rational(n * n, 4).evalf(17)} n^2/4")
    for n in (5, 7, 9):
        v = S.Rational(n, 2) * (1 + S.cos(S.pi / n))
        vals.append(f"odd_cycle {n} {v.evalf(17)} (n/2)(1+cos(pi/n))")
    for side in (4, 6):
        vals.append(f"bipartite_torus {side} {2 * side * side} |E|=2*side^2")
    (HERE / "maxcut_sdp_values.txt").write_text("\n".join(vals) + "\n")


if __name__ == "__main__":
    main()
