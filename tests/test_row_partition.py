"""The row-partitioned SpMM's exchange plan (paper_2407_15049_gb300/partition.py)
on CPU ranks (gloo, world sizes 2 and 3).

Each rank owns a contiguous row block of C and R, receives its halo rows of R
from their owners through the plan's send/receive lists, multiplies its own
rows of C by [own rows; halo rows] and must obtain exactly its rows of the FP64
oracle's C R; the all-reduce of the per-rank partial <C R, R> must equal the
oracle's objective.  Unmeasured on hardware (the library runs on one GPU);
this covers the host-side logic of the multi-GPU design.
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instance(name):
    import workloads as W
    if name == "er":
        return W.maxcut_instance(3001, W.er_graph(3001, 6000, 5, "pm1"))
    return W.maxcut_instance(900, W.torus_graph(30, 2, "pm1"))


def _rank_main(rank: int, world: int, port: int, name: str, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import scipy.sparse as sp
        import workloads as W
        from oracle import lorads_oracle as O
        from paper_2407_15049_gb300 import partition as PT
        inst = _instance(name)
        R = W.initial_factor(inst, 7, 3)
        plan = PT.build_plan(inst.rowptr, inst.colind, inst.val, inst.n, world, rank)
        R_own = torch.as_tensor(R[plan.lo:plan.hi].copy())
        halo = PT.exchange(plan, R_own, dist)
        # received rows are the owners' rows, in the plan's order
        want_rows = np.concatenate([plan.recv[q] for q in sorted(plan.recv)]) if plan.recv else np.zeros(0, int)
        assert np.array_equal(halo.numpy(), R[want_rows])
        X = np.vstack([R_own.numpy(), halo.numpy()])
        C_loc = sp.csr_matrix((plan.val, plan.col, plan.rowptr), shape=(plan.n_own, X.shape[0]))
        CR = C_loc @ X
        want = O.spmm(O.Problem(inst), R, None)[plan.lo:plan.hi]
        err = float(np.max(np.abs(CR - want))) / float(np.max(np.abs(want)))
        part = torch.tensor([float(np.sum(CR * R_own.numpy()))], dtype=torch.float64)
        dist.all_reduce(part)
        obj = O.objective(O.Problem(inst), R)
        out[rank] = (err, float(part[0]), obj, plan.n_halo, {int(k): len(v) for k, v in plan.send.items()},
                     {int(k): len(v) for k, v in plan.recv.items()})
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", ["er", "torus"])
def test_row_partitioned_spmm_matches_oracle(name, world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        err, total, obj, n_halo, send, recv = res[r]
        assert err <= 1e-14
        assert total == pytest.approx(obj, rel=1e-12)
        assert n_halo > 0
        # what rank r receives from q is what q sends to r (symmetric pattern, no request round)
        for q, cnt in recv.items():
            assert res[q][4][r] == cnt


def test_plan_of_a_single_rank_has_no_halo():
    from paper_2407_15049_gb300 import partition as PT
    inst = _instance("torus")
    plan = PT.build_plan(inst.rowptr, inst.colind, inst.val, inst.n, 1, 0)
    assert plan.n_halo == 0 and plan.send == {} and plan.n_own == inst.n
    assert np.array_equal(plan.col, inst.colind)


def _partitioned_inner_loop(rank: int, world: int, port: int, k: int, out):
    """Algorithm 1 on row-partitioned ranks for the MaxCut SDP (constraint i on row i):
    k L-BFGS iterations of the first ALM outer step, then its multiplier step, with
    the oracle's inner-loop control (stop test, gamma-scaled two-loop, exact line
    search of App. A.2, pair acceptance).  Per iteration the ranks exchange the halo
    rows of D for C D, and every global sum is an all-reduce of per-rank partial
    sums; the seven line-search sums travel in one all-reduce."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import scipy.sparse as sp
        import workloads as W
        from oracle import lorads_oracle as O
        from paper_2407_15049_gb300 import partition as PT
        inst = _instance("er")
        r = 7
        R0 = W.initial_factor(inst, r, 3)
        plan = PT.build_plan(inst.rowptr, inst.colind, inst.val, inst.n, world, rank)
        C_loc = sp.csr_matrix((plan.val, plan.col, plan.rowptr), shape=(plan.n_own, plan.n_own + plan.n_halo))

        def allsum(*vals):
            t = torch.tensor([float(v) for v in vals], dtype=torch.float64)
            dist.all_reduce(t)
            return t.tolist()

        def cmul(X_own):                           # own rows of C X
            halo = PT.exchange(plan, torch.as_tensor(X_own), dist).numpy()
            return C_loc @ np.vstack([X_own, halo])

        def dot(a, b):
            return allsum(np.sum(a * b))[0]

        nz = np.abs(plan.val[plan.val != 0])
        s_abs, cnt = allsum(nz.sum(), nz.size)
        rho = cnt / s_abs                           # 1 / mean |C_ij| over the stored entries
        R = R0[plan.lo:plan.hi].copy()
        y = np.zeros(plan.n_own)
        b = np.ones(plan.n_own)
        tol_e = 1e-300 * 2.0                        # tol (1 + ||b||_inf), b = 1

        def grad(Rx, CRx):
            z = np.sum(Rx * Rx, axis=1) - b
            return 2.0 * (CRx - (y - rho * z)[:, None] * Rx)

        CR = cmul(R)
        G = grad(R, CR)
        g0 = math.sqrt(dot(G, G))
        S, Yh, it = [], [], 0
        while it < k:
            zc = math.sqrt(dot(*(2 * [np.sum(R * R, axis=1) - b])))
            thr = max(tol_e, min(1.0 * rho * zc, 0.1 * g0))
            if math.sqrt(dot(G, G)) <= thr:
                break
            # two-loop recursion, gamma I initial matrix (the oracle's default)
            D = -G.copy()
            T = len(S)
            alpha = [0.0] * T
            beta = [1.0 / dot(Yh[t], S[t]) for t in range(T)]
            for t in range(T - 1, -1, -1):
                alpha[t] = beta[t] * dot(S[t], D)
                D = D - alpha[t] * Yh[t]
            if T:
                D = D * (dot(S[-1], Yh[-1]) / dot(Yh[-1], Yh[-1]))
            for t in range(T):
                D = D + (alpha[t] - beta[t] * dot(Yh[t], D)) * S[t]
            it += 1
            CD = cmul(D)
            q0 = b - np.sum(R * R, axis=1)
            q1 = 2.0 * np.sum(R * D, axis=1)
            q2 = np.sum(D * D, axis=1)
            w = y + rho * q0
            p1, p2, s22, s12, sw2, s11, sw1 = allsum(
                np.sum(CR * D) + np.sum(CD * R), np.sum(CD * D), q2 @ q2, q1 @ q2, w @ q2, q1 @ q1, w @ q1)
            a = np.array([0.5 * rho * s22, rho * s12, p2 - sw2 + 0.5 * rho * s11, p1 - sw1])
            tau = O.quartic_step(a)
            if tau <= 0.0:
                if S:
                    S.clear()
                    Yh.clear()
                    continue
                break
            R_new = R + tau * D
            CR_new = CR + tau * CD
            G_new = grad(R_new, CR_new)
            s, yv = tau * D, G_new - G
            ys, yy, ss = allsum(np.sum(yv * s), np.sum(yv * yv), np.sum(s * s))
            if ys > 1e-16 * math.sqrt(yy) * math.sqrt(ss):
                S.append(s)
                Yh.append(yv)
                if len(S) > 4:
                    S.pop(0)
                    Yh.pop(0)
            else:
                S.clear()
                Yh.clear()
            R, G, CR = R_new, G_new, CR_new
        y = y - rho * (np.sum(R * R, axis=1) - b)      # multiplier step of the outer loop
        out[rank] = (plan.lo, plan.hi, R, y, it, rho)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("k", [1, 5])
def test_row_partitioned_inner_loop_follows_the_oracle(world, k):
    """After k row-partitioned L-BFGS iterations and the multiplier step, every rank's
    rows of R and y equal the FP64 oracle's single-process iterate (O.solve with one
    outer step of k inner iterations) up to the summation order of the global sums."""
    import workloads as W
    from oracle import lorads_oracle as O
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_partitioned_inner_loop, args=(r, world, port, k, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        res = dict(out)
    inst = _instance("er")
    P = O.Problem(inst)
    ref = O.solve(P, W.initial_factor(inst, 7, 3), O.Params(max_outer=1, max_inner=k, tol=1e-300))
    assert ref["inner"] == k
    R = np.vstack([res[q][2] for q in range(world)])
    y = np.concatenate([res[q][3] for q in range(world)])
    assert all(res[q][4] == k for q in range(world))
    assert res[0][5] == pytest.approx(O.auto_rho(P), rel=1e-14)
    assert np.max(np.abs(R - ref["R"])) <= 1e-10 * np.max(np.abs(ref["R"]))
    assert np.max(np.abs(y - ref["y"])) <= 1e-10 * np.max(np.abs(ref["y"]))


def _partitioned_triplet_loop(rank: int, world: int, port: int, k: int, out):
    """The partitioned inner loop for constraints of one triplet each, on the
    matrix-completion SDP (constraint k couples row i of U with row n1 + j of V,
    often on another rank).  The halo plan is built on the pattern of
    S~ = C - A*(y~), so both ends of every constraint that touches an own row are on
    the rank.  A constraint whose rows lie on two ranks is evaluated on both, from
    the same two rows: the replicated multipliers stay identical.  Global sums
    count each constraint once, on the owner of its lower row."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import scipy.sparse as sp
        import workloads as W
        from oracle import lorads_oracle as O
        from paper_2407_15049_gb300 import partition as PT
        inst = _mc_instance()
        n = inst.n
        R0 = W.initial_factor(inst, 5, 4)
        C = sp.csr_matrix((inst.val, inst.colind, inst.rowptr), shape=(n, n))
        plan, touch, canon = PT.sdp_pattern_plan(n, inst.rowptr, inst.colind, inst.val, inst.row, inst.col,
                                                 world, rank)
        lo, hi, n_own = plan.lo, plan.hi, plan.n_own
        halo_rows = plan.halo_rows
        loc = plan.local_index(np.arange(n))
        row, col, av = inst.row.astype(np.int64), inst.col.astype(np.int64), inst.aval
        ui, vj, ak, bk = loc[row[touch]], loc[col[touch]], av[touch], inst.b[touch]
        assert np.all(ui >= 0) and np.all(vj >= 0)
        diag = row[touch] == col[touch]
        own_i, own_j = (row[touch] >= lo) & (row[touch] < hi), (col[touch] >= lo) & (col[touch] < hi)
        Cl = C[lo:hi].tocoo()
        C_loc = sp.csr_matrix((Cl.data, (Cl.row, loc[Cl.col])), shape=(n_own, n_own + plan.n_halo))

        def allsum(*vals):
            t = torch.tensor([float(v) for v in vals], dtype=torch.float64)
            dist.all_reduce(t)
            return t.tolist()

        def full(X_own):
            return np.vstack([X_own, PT.exchange(plan, torch.as_tensor(X_own), dist).numpy()])

        def amap(Xu, Xv):                          # A(U V^T) on the touching constraints
            uv = np.sum(Xu[ui] * Xv[vj], axis=1)
            vu = np.sum(Xu[vj] * Xv[ui], axis=1)
            return np.where(diag, ak * uv, ak * (uv + vu))

        def astar(v, Xf):                          # own rows of A*(v) X
            res = np.zeros((n_own, Xf.shape[1]))
            w = v * ak
            np.add.at(res, ui[own_i], (w[own_i])[:, None] * Xf[vj[own_i]])
            off = own_j & ~diag
            np.add.at(res, vj[off], (w[off])[:, None] * Xf[ui[off]])
            return res

        def dot(a, b):
            return allsum(np.sum(a * b))[0]

        cabs = np.abs(Cl.data[Cl.data != 0])
        s_abs, cnt = allsum(cabs.sum(), cabs.size)
        rho = cnt / s_abs
        bmax = torch.tensor([float(np.max(np.abs(bk))) if bk.size else 0.0], dtype=torch.float64)
        dist.all_reduce(bmax, op=dist.ReduceOp.MAX)
        tol_e = 1e-300 * (1.0 + float(bmax[0]))
        R = R0[lo:hi].copy()
        y = np.zeros(len(touch))

        def grad(Rf):
            y_t = y - rho * (amap(Rf, Rf) - bk)
            return 2.0 * (C_loc @ Rf - astar(y_t, Rf))

        Rf = full(R)
        G = grad(Rf)
        g0 = math.sqrt(dot(G, G))
        S, Yh, it = [], [], 0
        while it < k:
            zc = math.sqrt(allsum(np.sum(((amap(Rf, Rf) - bk) ** 2)[canon]))[0])
            if math.sqrt(dot(G, G)) <= max(tol_e, min(rho * zc, 0.1 * g0)):
                break
            D = -G.copy()
            T = len(S)
            alpha = [0.0] * T
            beta = [1.0 / dot(Yh[t], S[t]) for t in range(T)]
            for t in range(T - 1, -1, -1):
                alpha[t] = beta[t] * dot(S[t], D)
                D = D - alpha[t] * Yh[t]
            if T:
                D = D * (dot(S[-1], Yh[-1]) / dot(Yh[-1], Yh[-1]))
            for t in range(T):
                D = D + (alpha[t] - beta[t] * dot(Yh[t], D)) * S[t]
            it += 1
            Df = full(D)
            CR, CD = C_loc @ Rf, C_loc @ Df
            q0 = bk - amap(Rf, Rf)
            q1 = amap(Rf, Df) + amap(Df, Rf)
            q2 = amap(Df, Df)
            w = y + rho * q0
            c = canon
            p1, p2, s22, s12, sw2, s11, sw1 = allsum(
                np.sum(CR * D) + np.sum(CD * R), np.sum(CD * D), q2[c] @ q2[c], q1[c] @ q2[c], w[c] @ q2[c],
                q1[c] @ q1[c], w[c] @ q1[c])
            a = np.array([0.5 * rho * s22, rho * s12, p2 - sw2 + 0.5 * rho * s11, p1 - sw1])
            tau = O.quartic_step(a)
            if tau <= 0.0:
                if S:
                    S.clear()
                    Yh.clear()
                    continue
                break
            R_new = R + tau * D
            Rf_new = full(R_new)
            G_new = grad(Rf_new)
            s, yv = tau * D, G_new - G
            ys, yy, ss = allsum(np.sum(yv * s), np.sum(yv * yv), np.sum(s * s))
            if ys > 1e-16 * math.sqrt(yy) * math.sqrt(ss):
                S.append(s)
                Yh.append(yv)
                if len(S) > 4:
                    S.pop(0)
                    Yh.pop(0)
            else:
                S.clear()
                Yh.clear()
            R, Rf, G = R_new, Rf_new, G_new
        y = y - rho * (amap(Rf, Rf) - bk)
        out[rank] = (lo, hi, R, touch[canon], y[canon], it, len(halo_rows))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _mc_instance():
    import workloads as W
    return W.mc_instance(40, 50, 3, 600, seed=3)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("k", [1, 5])
def test_row_partitioned_matrix_completion_follows_the_oracle(world, k):
    """Matrix completion on the row partition: every rank's rows of R and the
    multipliers of the constraints it owns equal the FP64 oracle's iterate after k
    L-BFGS iterations and the multiplier step, and the constraints couple ranks
    (the halo is not empty)."""
    import workloads as W
    from oracle import lorads_oracle as O
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_partitioned_triplet_loop, args=(r, world, port, k, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        res = dict(out)
    inst = _mc_instance()
    ref = O.solve(O.Problem(inst), W.initial_factor(inst, 5, 4), O.Params(max_outer=1, max_inner=k, tol=1e-300))
    assert ref["inner"] == k
    R = np.vstack([res[q][2] for q in range(world)])
    owned = np.concatenate([res[q][3] for q in range(world)])
    y = np.concatenate([res[q][4] for q in range(world)])
    assert np.array_equal(np.sort(owned), np.arange(inst.m))          # every constraint owned once
    assert all(res[q][5] == k for q in range(world)) and all(res[q][6] > 0 for q in range(world))
    assert np.max(np.abs(R - ref["R"])) <= 1e-10 * np.max(np.abs(ref["R"]))
    assert np.max(np.abs(y - ref["y"][owned])) <= 1e-10 * np.max(np.abs(ref["y"]))


def test_local_index_follows_the_halo_order():
    """local_index maps own rows to 0..n_own-1 and halo rows to n_own + their position
    in the exchange order (owner rank, then row), and every other row to -1; the
    local column numbering of the plan's CSR uses the same map."""
    from paper_2407_15049_gb300 import partition as PT
    inst = _instance("er")
    for world in (2, 3):
        for rank in range(world):
            plan = PT.build_plan(inst.rowptr, inst.colind, inst.val, inst.n, world, rank)
            loc = plan.local_index(np.arange(inst.n))
            assert np.array_equal(loc[plan.lo:plan.hi], np.arange(plan.n_own))
            assert np.array_equal(loc[plan.halo_rows], plan.n_own + np.arange(plan.n_halo))
            others = np.setdiff1d(np.setdiff1d(np.arange(inst.n), np.arange(plan.lo, plan.hi)), plan.halo_rows)
            assert np.all(loc[others] == -1)
            s0, s1 = inst.rowptr[plan.lo], inst.rowptr[plan.hi]
            assert np.array_equal(plan.col, loc[inst.colind[s0:s1]])


def test_sdp_pattern_plan_counts_every_constraint_once():
    """On every rank, the constraints it evaluates are exactly those with a row it
    owns, both rows of each are own or halo rows, and over the ranks each
    constraint is counted (canonical) exactly once."""
    from paper_2407_15049_gb300 import partition as PT
    inst = _mc_instance()
    for world in (1, 2, 3):
        counted = np.zeros(inst.m, dtype=int)
        for rank in range(world):
            plan, touch, canon = PT.sdp_pattern_plan(inst.n, inst.rowptr, inst.colind, inst.val, inst.row,
                                                     inst.col, world, rank)
            row, col = inst.row.astype(np.int64), inst.col.astype(np.int64)
            mine = ((row >= plan.lo) & (row < plan.hi)) | ((col >= plan.lo) & (col < plan.hi))
            assert np.array_equal(touch, np.nonzero(mine)[0])
            assert np.all(plan.local_index(row[touch]) >= 0) and np.all(plan.local_index(col[touch]) >= 0)
            counted[touch[canon]] += 1
        assert np.all(counted == 1)
