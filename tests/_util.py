"""Test-side input builders and error measures (no method arithmetic)."""
import numpy as np

import workloads as W


def rel_err(got, want) -> float:
    """Normwise relative error ||got - want||_inf / max(||want||_inf, tiny)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(float(np.max(np.abs(want))) if want.size else 0.0, 1e-300)
    return float(np.max(np.abs(got - want))) / scale if want.size else 0.0


def mixed_instance(n: int, seed: int, density: float = 3.0, empty_every: int = 17,
                   diag_frac: float = 0.6, n_off: int | None = None) -> W.SDPInstance:
    """Random sparse symmetric C (some rows completely empty, no stored diagonal there)
    with diagonal constraints on a subset of rows and off-diagonal single-entry
    constraints on random distinct pairs."""
    rng = np.random.default_rng(seed)
    m_edges = int(density * n)
    i = rng.integers(0, n, m_edges)
    j = rng.integers(0, n, m_edges)
    keep = (i != j) & (i % empty_every != 0) & (j % empty_every != 0)
    lo, hi = np.minimum(i[keep], j[keep]), np.maximum(i[keep], j[keep])
    keys = np.unique(lo * n + hi)
    lo, hi = keys // n, keys % n
    w = rng.standard_normal(len(lo))
    diag_rows = np.array([r for r in range(n) if r % empty_every != 0 and r % 3 != 1])
    rows = np.concatenate([lo, hi, diag_rows])
    cols = np.concatenate([hi, lo, diag_rows])
    vals = np.concatenate([w, w, rng.standard_normal(len(diag_rows))])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    # constraints
    dsel = rng.random(n) < diag_frac
    drows = np.nonzero(dsel)[0]
    n_off = n_off if n_off is not None else n
    a = rng.integers(0, n, 3 * n_off)
    c = rng.integers(0, n, 3 * n_off)
    ok = a != c
    plo, phi = np.minimum(a[ok], c[ok]), np.maximum(a[ok], c[ok])
    pk = np.unique(plo * n + phi)[:n_off]
    plo, phi = pk // n, pk % n
    m = len(drows) + len(plo)
    perm = rng.permutation(m)                       # constraint ids in random order
    row = np.concatenate([drows, plo]).astype(np.int32)
    col = np.concatenate([drows, phi]).astype(np.int32)
    aval = rng.uniform(0.5, 1.5, m) * np.where(rng.random(m) < 0.5, -1.0, 1.0)
    return W.SDPInstance(n=n, rowptr=rowptr, colind=cols.astype(np.int32), val=vals, m=m,
                         con=perm.astype(np.int32), row=row, col=col, aval=aval,
                         b=rng.standard_normal(m), kind="generic")
