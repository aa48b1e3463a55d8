"""Seeded synthetic SDP instances shared by the oracle and the CUDA path.

This module only *generates inputs*: graphs, sampled matrix entries and the
primal SDP data (C, A, b) in the exchange format of the C-ABI, plus seeded
starting factors.  It holds none of the solver's arithmetic (no gradient, no
line search, no multiplier update), so that the oracle and the GPU library can
both consume it without sharing any part of the method.

Exchange format (the primal SDP of Eq. (1.1): min <C,X> s.t. <A_k,X> = b_k, X psd):

* ``rowptr`` int64 (n+1), ``colind`` int32, ``val`` float64: C as a full
  symmetric CSR matrix with sorted column indices in every row.
* constraint triplets ``con, row, col`` int32 and ``aval`` float64 with
  ``row <= col``; constraint k is  <A_k, X> = sum a * X_ij * (1 if i == j else 2).
* ``b`` float64 (m).

Workloads (Sec. 4.3 MaxCut SDP and Sec. 4.4 matrix-completion SDP):

* MaxCut: C = -L/4 with L the weighted graph Laplacian, constraints X_ii = 1
  (one diagonal triplet per row, b = 1).  The reported SDP value is -<C,X>.
* Matrix completion: X has order n1 + n2, C = I, constraint k <-> (i, j) in
  Omega is  X_{i,n1+j} + X_{n1+j,i} = 2 M_ij  (one off-diagonal triplet).
* General constraints (the class of Sec. 4.5, constraints with several
  entries): the Lovasz theta SDP of a graph, max <J, X> s.t. tr X = 1 and
  X_ij = 0 on the edges (C = -J, one constraint of n diagonal triplets), and
  MaxCut instances with added constraints over several entries.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SDPInstance", "er_graph", "torus_graph", "complete_graph", "cycle_graph",
    "bipartite_torus_graph", "maxcut_instance", "mc_instance", "initial_factor",
    "rank_log2", "config_instance", "theta_instance", "maxcut_with_sums",
]


@dataclass
class SDPInstance:
    """Primal SDP data in the C-ABI exchange format (all arrays host, contiguous)."""

    n: int
    rowptr: np.ndarray          # int64 (n+1)
    colind: np.ndarray          # int32 (nnz)
    val: np.ndarray             # float64 (nnz)
    m: int
    con: np.ndarray             # int32 (nnz_a)
    row: np.ndarray             # int32 (nnz_a), row <= col
    col: np.ndarray             # int32 (nnz_a)
    aval: np.ndarray            # float64 (nnz_a)
    b: np.ndarray               # float64 (m)
    kind: str = "generic"
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _sym_csr(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray, diag: np.ndarray):
    """Full symmetric CSR from upper off-diagonal entries (i<j, w) and a dense diagonal.

    Every diagonal slot is stored (also when its value is 0) so that the row
    structure does not depend on the weights.
    """
    import scipy.sparse as sp
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    rows = np.concatenate([i, j, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([j, i, np.arange(n, dtype=np.int64)])
    # the diagonal is added with a tiny offset and removed again so that explicit
    # zeros on the diagonal survive the duplicate summation
    vals = np.concatenate([np.asarray(w, np.float64), np.asarray(w, np.float64),
                           np.asarray(diag, np.float64) + 1.0])
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M.sum_duplicates()
    M.sort_indices()
    rowptr = M.indptr.astype(np.int64)
    colind = M.indices.astype(np.int32)
    val = M.data.astype(np.float64)
    # undo the +1 on the diagonal slots
    rr = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    dmask = rr == colind
    val[dmask] -= 1.0
    # restore exact diagonal values (the +1/-1 round trip may round)
    val[dmask] = np.asarray(diag, np.float64)[rr[dmask]]
    return rowptr, colind, np.ascontiguousarray(val)


# ----------------------------------------------------------------------------- graphs

def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent difference)."""
    a = np.sort(a)
    if len(a) == 0:
        return a
    keep = np.empty(len(a), dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _weights(rng, count: int, weights: str) -> np.ndarray:
    if weights == "unit":
        return np.ones(count, dtype=np.float64)
    if weights == "pm1":
        return rng.integers(0, 2, size=count).astype(np.float64) * 2.0 - 1.0
    raise ValueError(f"unknown weights {weights!r}")


def er_graph(n: int, n_edges: int, seed: int, weights: str = "unit"):
    """Erdos-Renyi G(n, M): ``n_edges`` distinct undirected edges drawn uniformly.

    Returns (i, j, w) with i < j, sorted by (i, j).
    """
    if n_edges > n * (n - 1) // 2:
        raise ValueError("too many edges")
    rng = np.random.default_rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while len(keys) < n_edges:
        draw = int((n_edges - len(keys)) * 1.02) + 64
        a = rng.integers(0, n, size=draw, dtype=np.int64)
        c = rng.integers(0, n, size=draw, dtype=np.int64)
        ok = a != c
        lo = np.minimum(a[ok], c[ok])
        hi = np.maximum(a[ok], c[ok])
        keys = _sorted_unique(np.concatenate([keys, lo * n + hi]))
    if len(keys) > n_edges:
        # drop a uniformly random subset of the surplus distinct pairs
        drop = rng.choice(len(keys), size=len(keys) - n_edges, replace=False)
        keys = np.delete(keys, drop)
    i = (keys // n).astype(np.int64)
    j = (keys % n).astype(np.int64)
    return i, j, _weights(rng, len(i), weights)


def torus_graph(side: int, seed: int, weights: str = "pm1"):
    """2D toroidal grid side x side (4-regular with wraparound)."""
    rng = np.random.default_rng(seed)
    idx = np.arange(side * side, dtype=np.int64).reshape(side, side)
    right = np.roll(idx, -1, axis=1)
    down = np.roll(idx, -1, axis=0)
    a = np.concatenate([idx.ravel(), idx.ravel()])
    c = np.concatenate([right.ravel(), down.ravel()])
    lo = np.minimum(a, c)
    hi = np.maximum(a, c)
    keys = _sorted_unique(lo * (side * side) + hi)
    n = side * side
    i = keys // n
    j = keys % n
    return i, j, _weights(rng, len(i), weights)


def bipartite_torus_graph(side: int):
    """Even torus with unit weights (bipartite when side is even)."""
    i, j, _ = torus_graph(side, seed=0, weights="unit")
    return i, j, np.ones(len(i))


def complete_graph(n: int):
    i, j = np.triu_indices(n, k=1)
    return i.astype(np.int64), j.astype(np.int64), np.ones(len(i))


def cycle_graph(n: int):
    i = np.arange(n, dtype=np.int64)
    j = (i + 1) % n
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    order = np.lexsort((hi, lo))
    return lo[order], hi[order], np.ones(n)


# ----------------------------------------------------------------------------- instances

def _sorted_distinct_upper(i: np.ndarray, j: np.ndarray) -> bool:
    """True when every pair has i < j and the pairs are strictly increasing in (i, j)."""
    if len(i) == 0:
        return True
    if not np.all(i < j):
        return False
    di = np.diff(i)
    return bool(np.all((di > 0) | ((di == 0) & (np.diff(j) > 0))))


def _sym_csr_upper_sorted(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray, diag: np.ndarray):
    """The CSR of ``_sym_csr`` built by counting, for distinct pairs i < j sorted by
    (i, j): row r holds the pairs whose larger end is r (columns ascending), then the
    diagonal, then the pairs whose smaller end is r.  Linear memory, no sparse-matrix
    conversion (graphs of 1e8 vertices and more)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    cnt_up = np.bincount(i, minlength=n).astype(np.int64)
    cnt_lo = np.bincount(j, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_lo + cnt_up + 1, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    rows = np.arange(n, dtype=np.int64)
    dpos = rowptr[:-1] + cnt_lo
    colind[dpos] = rows.astype(np.int32)
    val[dpos] = np.asarray(diag, dtype=np.float64)
    del dpos
    # upper entries: the pairs in their given order, k - (first pair of row i) after the diagonal
    first_up = np.zeros(n, dtype=np.int64)
    np.cumsum(cnt_up[:-1], out=first_up[1:])
    pos = rowptr[:-1][i] + cnt_lo[i] + 1 + (np.arange(len(i), dtype=np.int64) - first_up[i])
    colind[pos] = j.astype(np.int32)
    val[pos] = w
    del pos, first_up
    # lower entries: the pairs ordered by (j, i) (distinct keys: any sort gives this order)
    perm = np.argsort(j * n + i)
    js = j[perm]
    first_lo = np.zeros(n, dtype=np.int64)
    np.cumsum(cnt_lo[:-1], out=first_lo[1:])
    pos = rowptr[:-1][js] + (np.arange(len(js), dtype=np.int64) - first_lo[js])
    colind[pos] = i[perm].astype(np.int32)
    val[pos] = w[perm]
    return rowptr, colind, val


def maxcut_instance(n: int, edges) -> SDPInstance:
    """MaxCut SDP of Sec. 4.3 written as a minimisation: C = -L(G,w)/4, X_ii = 1."""
    i, j, w = edges
    w = np.asarray(w, dtype=np.float64)
    # weighted degrees, each accumulated in the order of the pairs (i ends, then j ends)
    deg = np.bincount(np.concatenate([np.asarray(i, np.int64), np.asarray(j, np.int64)]),
                      weights=np.concatenate([w, w]), minlength=n)
    # L_ij = -w_ij, L_ii = sum_k w_ik  ->  C = -L/4
    if _sorted_distinct_upper(np.asarray(i), np.asarray(j)):
        rowptr, colind, val = _sym_csr_upper_sorted(n, i, j, w / 4.0, -deg / 4.0)
    else:
        rowptr, colind, val = _sym_csr(n, i, j, w / 4.0, -deg / 4.0)
    k = np.arange(n, dtype=np.int32)
    return SDPInstance(
        n=n, rowptr=rowptr, colind=colind, val=val, m=n,
        con=k.copy(), row=k.copy(), col=k.copy(), aval=np.ones(n),
        b=np.ones(n), kind="maxcut",
        meta={"edges": (np.asarray(i), np.asarray(j), np.asarray(w, dtype=np.float64))},
    )


def mc_instance(n1: int, n2: int, rank: int, n_samples: int, seed: int) -> SDPInstance:
    """Matrix-completion SDP of Sec. 4.4 with M = U V^T, U, V iid N(0,1) of rank ``rank``.

    Omega is drawn uniformly without replacement.  X = [[W1, Y^T-block], ...] has
    order n1 + n2; constraint k <-> (i, j): X_{i, n1+j} + X_{n1+j, i} = 2 M_ij.
    """
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n1, rank))
    V = rng.standard_normal((n2, rank))
    total = n1 * n2
    if n_samples > total:
        raise ValueError("too many samples")
    if n_samples > total // 2:
        flat = rng.choice(total, size=n_samples, replace=False)
    else:
        flat = np.empty(0, dtype=np.int64)
        while len(flat) < n_samples:
            draw = rng.integers(0, total, size=int((n_samples - len(flat)) * 1.1) + 16)
            flat = _sorted_unique(np.concatenate([flat, draw]))
        flat = rng.permutation(flat)[:n_samples]
    flat = np.sort(flat)
    si = (flat // n2).astype(np.int64)
    sj = (flat % n2).astype(np.int64)
    mvals = np.einsum("kr,kr->k", U[si], V[sj])
    n = n1 + n2
    rowptr, colind, val = _sym_csr(n, np.empty(0, np.int64), np.empty(0, np.int64),
                                   np.empty(0), np.ones(n))
    m = n_samples
    return SDPInstance(
        n=n, rowptr=rowptr, colind=colind, val=val, m=m,
        con=np.arange(m, dtype=np.int32), row=si.astype(np.int32),
        col=(n1 + sj).astype(np.int32), aval=np.ones(m), b=2.0 * mvals,
        kind="mc", meta={"n1": n1, "n2": n2, "U": U, "V": V},
    )


def theta_instance(n: int, edges) -> SDPInstance:
    """Lovasz theta SDP of a graph: min <-J, X> s.t. tr X = 1 (constraint 0: n
    diagonal triplets, b = 1) and X_ij = 0 for every edge (one triplet (i, j, 1/2),
    b = 0).  C = -J is stored in full (n^2 entries).  The value is theta(G)."""
    i, j, _ = (np.asarray(x) for x in edges)
    lo, hi = np.minimum(i, j).astype(np.int64), np.maximum(i, j).astype(np.int64)
    keys = np.unique(lo * n + hi)
    lo, hi = keys // n, keys % n
    rowptr = np.arange(n + 1, dtype=np.int64) * n
    colind = np.tile(np.arange(n, dtype=np.int32), n)
    val = -np.ones(n * n)
    m = 1 + len(lo)
    con = np.concatenate([np.zeros(n, dtype=np.int32), np.arange(1, m, dtype=np.int32)])
    row = np.concatenate([np.arange(n), lo]).astype(np.int32)
    col = np.concatenate([np.arange(n), hi]).astype(np.int32)
    aval = np.concatenate([np.ones(n), 0.5 * np.ones(len(lo))])
    b = np.concatenate([[1.0], np.zeros(len(lo))])
    return SDPInstance(n=n, rowptr=rowptr, colind=colind, val=val, m=m, con=con, row=row, col=col, aval=aval, b=b,
                       kind="theta")


def petersen_graph():
    """The Petersen graph (10 vertices, 15 edges, unit weights): theta = 4."""
    outer = [(k, (k + 1) % 5) for k in range(5)]
    spokes = [(k, k + 5) for k in range(5)]
    inner = [(5 + k, 5 + (k + 2) % 5) for k in range(5)]
    e = np.array(outer + spokes + inner)
    return e[:, 0], e[:, 1], np.ones(len(e))


def maxcut_with_sums(n: int, edges, groups: int, size: int, seed: int) -> SDPInstance:
    """A MaxCut SDP (X_ii = 1) with `groups` added constraints over several entries
    each: sum of X_ij over `size` random off-diagonal pairs = 0, and one constraint
    X_00 + X_11 = 2 on two entries the diagonal constraints already fix.  X = I is
    feasible for all of them."""
    base = maxcut_instance(n, edges)
    rng = np.random.default_rng(seed)
    con, row, col, aval, b = [base.con], [base.row], [base.col], [base.aval], [base.b]
    k = base.m
    for _ in range(groups):
        a = rng.integers(0, n, 3 * size)
        c = rng.integers(0, n, 3 * size)
        ok = a != c
        lo, hi = np.minimum(a[ok], c[ok]), np.maximum(a[ok], c[ok])
        keys = np.unique(lo.astype(np.int64) * n + hi)[:size]
        con.append(np.full(len(keys), k, dtype=np.int32))
        row.append((keys // n).astype(np.int32))
        col.append((keys % n).astype(np.int32))
        aval.append(rng.uniform(0.5, 1.5, len(keys)))
        b.append([0.0])
        k += 1
    con.append(np.array([k, k], dtype=np.int32))
    row.append(np.array([0, 1], dtype=np.int32))
    col.append(np.array([0, 1], dtype=np.int32))
    aval.append(np.ones(2))
    b.append([2.0])
    k += 1
    return SDPInstance(n=n, rowptr=base.rowptr, colind=base.colind, val=base.val, m=k,
                       con=np.concatenate(con), row=np.concatenate(row), col=np.concatenate(col),
                       aval=np.concatenate(aval), b=np.concatenate(b).astype(np.float64), kind="generic")


def rank_log2(k: int) -> int:
    """ceil(log2 k): the logarithmic starting rank of App. A.1."""
    return max(1, int(math.ceil(math.log2(max(k, 2)))))


def initial_factor(inst: SDPInstance, r: int, seed: int) -> np.ndarray:
    """Seeded starting factor R0 (n x r), rows iid N(0, I_r).

    Rows of MaxCut instances are scaled to unit norm (feasible for X_ii = 1).
    Matrix-completion factors are scaled so that ||R0||_F^2 = ||b||_1 / 2.
    """
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((inst.n, r))
    if inst.kind == "maxcut":
        R /= np.linalg.norm(R, axis=1, keepdims=True)
    elif inst.kind == "mc":
        target = 0.5 * float(np.abs(inst.b).sum())
        R *= math.sqrt(max(target, 1.0) / float((R * R).sum()))
    return np.ascontiguousarray(R)


def serving_batch(count: int = 512, seed: int = 0, n_range=(200, 20000), side_range=(100, 5000)):
    """Uneven instances for batched solving: about 3/4 MaxCut SDPs on ER graphs
    (n log-uniform in n_range, average degree uniform in {3..20}, weights in
    {-1,+1}) and 1/4 matrix-completion SDPs (M side x side, side uniform in
    side_range, rank uniform in {2..5}, |Omega| = ceil(5 side ln side)).
    Instance k is generated from seed * 1_000_003 + k.  Returns a list."""
    rng = np.random.default_rng(seed)
    kinds = rng.random(count) < 0.75
    out = []
    for k in range(count):
        s = seed * 1_000_003 + k
        if kinds[k]:
            n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
            deg = int(rng.integers(3, 21))
            out.append(maxcut_instance(n, er_graph(n, max(1, deg * n // 2), s, "pm1")))
        else:
            side = int(rng.integers(side_range[0], side_range[1] + 1))
            rank = int(rng.integers(2, 6))
            n_samples = min(side * side, int(math.ceil(5 * side * math.log(side))))
            out.append(mc_instance(side, side, rank, n_samples, s))
    return out


def config_instance(name: str, seed: int = 0):
    """The named synthetic workloads (shapes and distributions of the paper's workloads).

    Returns (instance, r0).
    """
    if name == "maxcut_er_1e3":          # ER n=1000, avg degree 8, unit weights
        n = 1000
        inst = maxcut_instance(n, er_graph(n, 4 * n, seed, "unit"))
        return inst, rank_log2(n)
    if name == "maxcut_torus_1e6":       # 1000x1000 torus, weights in {-1,+1}
        side = 1000
        inst = maxcut_instance(side * side, torus_graph(side, seed, "pm1"))
        return inst, rank_log2(side * side)
    if name == "mc_5e4_rank3":           # 50000 x 50000, rank 3, |Omega| = ceil(5 n ln n)
        n = 50000
        k = int(math.ceil(5 * n * math.log(n)))
        inst = mc_instance(n, n, 3, k, seed)
        return inst, rank_log2(inst.m)
    if name == "maxcut_er_1e7":          # ER n=1e7, avg degree 4, weights in {-1,+1}
        n = 10_000_000
        inst = maxcut_instance(n, er_graph(n, 2 * n, seed, "pm1"))
        return inst, 24
    raise KeyError(name)
