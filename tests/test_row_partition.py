"""The row-partitioned SpMM's exchange plan (paper_2407_15049_gb300/partition.py)
on CPU ranks (gloo, world sizes 2 and 3).

Each rank owns a contiguous row block of C and R, receives its halo rows of R
from their owners through the plan's send/receive lists, multiplies its own
rows of C by [own rows; halo rows] and must obtain exactly its rows of the FP64
oracle's C R; the all-reduce of the per-rank partial <C R, R> must equal the
oracle's objective.  Unmeasured on hardware (the library runs on one GPU);
this covers the host-side logic of the multi-GPU design.
"""
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
