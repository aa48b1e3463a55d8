"""Row partition of the SpMM (C - A*(v)) R across ranks: the exchange plan.

The hot path shards naturally by rows: rank q owns a contiguous block of rows
of C, R and every n x r iterate.  One SpMM needs, besides the rank's own rows
of R (or D), the *halo* rows: rows j owned by other ranks with C_ij stored for
some own row i.  Because C is symmetric, the rows rank q must send to rank p
are exactly its own rows that have a stored column in p's block, so every rank
builds both its receive and its send lists from its own rows, with no request
round.  The per-iteration exchange is then one neighbour send/receive of those
rows per SpMM (D changes every L-BFGS iteration), and the scalar reductions
(the line-search sums, the L-BFGS Gram entries, err1 / err3) are one small
all-reduce of a few dozen doubles.

This module holds index bookkeeping and the exchange only: no arithmetic of
the method.  It is not wired into the single-GPU library (each box of this
build has one GPU); its plan and exchange are tested with gloo ranks on the
CPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def row_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, nearly equal row blocks [lo, hi) for ranks 0..world-1."""
    bounds = [(n * q) // world for q in range(world + 1)]
    return [(bounds[q], bounds[q + 1]) for q in range(world)]


def owner_of(rows: np.ndarray, ranges: list[tuple[int, int]]) -> np.ndarray:
    """Rank owning each global row."""
    starts = np.array([lo for lo, _ in ranges])
    return np.searchsorted(starts, rows, side="right") - 1


@dataclass
class HaloPlan:
    """What one rank holds, receives and sends for one SpMM over C."""
    rank: int
    world: int
    lo: int
    hi: int
    # own rows of C with columns renumbered: own rows 0..n_own-1, then halo rows in
    # receive order (owner rank, then global row)
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    recv: dict = field(default_factory=dict)      # owner rank -> global rows received from it (sorted)
    send: dict = field(default_factory=dict)      # peer rank -> own global rows sent to it (sorted)

    @property
    def n_own(self) -> int:
        return self.hi - self.lo

    @property
    def n_halo(self) -> int:
        return int(sum(len(v) for v in self.recv.values()))

    @property
    def halo_rows(self) -> np.ndarray:
        """Global rows of the halo, in the order `exchange` returns them."""
        if not self.recv:
            return np.zeros(0, dtype=np.int64)
        return np.concatenate([np.asarray(self.recv[q], dtype=np.int64) for q in sorted(self.recv)])

    def local_index(self, rows) -> np.ndarray:
        """Position of each global row in [own rows; halo rows] (the row order of the
        local column numbering), or -1 for a row the rank neither owns nor receives."""
        rows = np.asarray(rows, dtype=np.int64)
        out = np.full(rows.shape, -1, dtype=np.int64)
        own = (rows >= self.lo) & (rows < self.hi)
        out[own] = rows[own] - self.lo
        halo = self.halo_rows
        if halo.size:
            order = np.argsort(halo, kind="stable")
            pos = np.searchsorted(halo[order], rows[~own])
            pos = np.minimum(pos, halo.size - 1)
            hit = halo[order][pos] == rows[~own]
            sub = np.full(pos.shape, -1, dtype=np.int64)
            sub[hit] = self.n_own + order[pos[hit]]
            out[~own] = sub
        return out


def build_plan(rowptr: np.ndarray, colind: np.ndarray, val: np.ndarray, n: int, world: int,
               rank: int) -> HaloPlan:
    """Plan of `rank` from the rows of the symmetric CSR matrix C it owns."""
    ranges = row_ranges(n, world)
    lo, hi = ranges[rank]
    s0, s1 = int(rowptr[lo]), int(rowptr[hi])
    cols = np.asarray(colind[s0:s1], dtype=np.int64)
    own = (cols >= lo) & (cols < hi)
    remote = np.unique(cols[~own])
    owners = owner_of(remote, ranges)
    recv = {int(q): remote[owners == q] for q in np.unique(owners)}
    # halo numbering: by owner rank, then by global row (np.unique sorts both)
    new_col = np.where(own, cols - lo, 0)
    if remote.size:
        pos = np.searchsorted(remote, cols[~own])
        new_col[~own] = (hi - lo) + pos
    # symmetric C: own row i goes to rank p iff row i has a stored column in p's block
    send = {}
    col_owner = owner_of(cols, ranges)
    row_of_entry = np.repeat(np.arange(lo, hi), np.diff(np.asarray(rowptr[lo:hi + 1], dtype=np.int64)))
    for p in np.unique(col_owner[col_owner != rank]):
        send[int(p)] = np.unique(row_of_entry[col_owner == p])
    return HaloPlan(rank=rank, world=world, lo=lo, hi=hi,
                    rowptr=np.asarray(rowptr[lo:hi + 1], dtype=np.int64) - s0, col=new_col,
                    val=np.asarray(val[s0:s1]), recv=recv, send=send)


def sdp_pattern_plan(n: int, rowptr, colind, val, con_row, con_col, world: int, rank: int):
    """Plan of `rank` for an SDP with constraints of one triplet each (constraint k on
    entry (con_row[k], con_col[k]), row <= col): the halo plan of the pattern of
    S~ = C - A*(y~) (C's stored entries and both triangles of every constraint entry),
    so that both rows of every constraint touching an own row are on the rank, and
    the constraint bookkeeping.  Returns (plan, touch, canonical): `touch` lists the
    constraints with a row on this rank (each is evaluated here, from the same two
    rows as on the other rank, so replicated multipliers stay identical) and
    `canonical` marks those this rank counts in global sums (the owner of the
    constraint's lower row), so every constraint is counted once."""
    import scipy.sparse as sp
    con_row = np.asarray(con_row, dtype=np.int64)
    con_col = np.asarray(con_col, dtype=np.int64)
    C = sp.csr_matrix((np.abs(np.asarray(val, dtype=np.float64)) + 1.0, np.asarray(colind), np.asarray(rowptr)),
                      shape=(n, n))
    A = sp.csr_matrix((np.ones(len(con_row)), (con_row, con_col)), shape=(n, n))
    pat = (C + A + A.T).tocsr()
    pat.sort_indices()
    plan = build_plan(pat.indptr, pat.indices, pat.data, n, world, rank)
    lo, hi = plan.lo, plan.hi
    touch = np.nonzero(((con_row >= lo) & (con_row < hi)) | ((con_col >= lo) & (con_col < hi)))[0]
    canonical = owner_of(con_row[touch], row_ranges(n, world)) == rank
    return plan, touch, canonical


def exchange(plan: HaloPlan, X_own, dist) -> "object":
    """Halo rows of X (a torch tensor holding this rank's rows, n_own x ld) in the
    plan's halo order, by one send/receive per neighbouring rank (torch.distributed
    point-to-point; any backend).  Returns an n_halo x ld tensor."""
    import torch
    ld = X_own.shape[1]
    ops = []
    out = {}
    for p, rows in sorted(plan.recv.items()):
        buf = torch.empty((len(rows), ld), dtype=X_own.dtype, device=X_own.device)
        out[p] = buf
        ops.append(dist.P2POp(dist.irecv, buf, p))
    sends = []
    for p, rows in sorted(plan.send.items()):
        payload = X_own[torch.as_tensor(rows - plan.lo, device=X_own.device)].contiguous()
        sends.append(payload)
        ops.append(dist.P2POp(dist.isend, payload, p))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if not out:
        return torch.empty((0, ld), dtype=X_own.dtype, device=X_own.device)
    return torch.cat([out[p] for p in sorted(out)], dim=0)
