"""lorads_linesearch_coeffs_noalloc: the context-free line-search entry point for
callers that cannot allocate device memory (a framework's caching allocator
owns it, or a latency-critical loop cannot take cudaMalloc's synchronisation).
Its scratch is a fixed device array inside the
library, so the test checks it against the context entry point and against
the FP64 oracle's coefficients of App. A.2 on two calls in a row (the second
sees the first call's leftovers in that array), on small instances and on one
of 300,000 rows, where both reduction grids hit the 1024-block cap and every
block's grid-stride loop covers several row tiles.

This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import lorads_oracle as O
from tests._util import mixed_instance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2407_15049_gb300 as L  # noqa: E402


def _scales(P, R, D, y, rho):
    """Magnitude of the terms of each a_i (cancellation-aware tolerance scale)."""
    a, parts = O.linesearch_coeffs(P, R, D, y, rho)
    q0, q1, q2 = parts["q0"], parts["q1"], parts["q2"]
    w = np.abs(y) + rho * np.abs(q0)
    CRabs = np.abs(P.C) @ np.abs(R)
    CDabs = np.abs(P.C) @ np.abs(D)
    return np.array([0.5 * rho * float(q2 @ q2), rho * float(np.abs(q1) @ np.abs(q2)),
                     float(np.sum(CDabs * np.abs(D))) + float(w @ np.abs(q2)) + 0.5 * rho * float(q1 @ q1),
                     2 * float(np.sum(CRabs * np.abs(D))) + float(w @ np.abs(q1))])


def _instance(name):
    if name == "mixed_1031":
        return mixed_instance(1031, seed=9)
    if name == "maxcut_er_2001":
        return W.maxcut_instance(2001, W.er_graph(2001, 4002, 3, "pm1"))
    # 300,000 rows at ld = 12: 64 rows per 256-thread block, 4,688 row tiles > 1024 blocks
    return W.maxcut_instance(300_000, W.er_graph(300_000, 600_000, 7, "pm1"))


@pytest.mark.parametrize("name", ["mixed_1031", "maxcut_er_2001", "maxcut_er_300000"])
def test_noalloc_matches_context_entry_point(name):
    L.build()
    lib = L.load()
    inst = _instance(name)
    P = O.Problem(inst)
    r = 10
    ld = L.padded_ld(r)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    rowptr = dev(inst.rowptr, torch.int64)
    colind = dev(inst.colind, torch.int32)
    val = dev(inst.val, torch.float64)
    con = dev(inst.con, torch.int32)
    row = dev(inst.row, torch.int32)
    col = dev(inst.col, torch.int32)
    aval = dev(inst.aval, torch.float64)
    b = dev(inst.b, torch.float64)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    ctx = L.lorads_create(inst)
    try:
        rng = np.random.default_rng(5)
        for call in range(2):
            Rh = rng.standard_normal((inst.n, r))
            Dh = rng.standard_normal((inst.n, r))
            yh = rng.standard_normal(inst.m)
            rho = 2.5 + call
            R = torch.zeros((inst.n, ld), dtype=torch.float64, device="cuda")
            D = torch.zeros_like(R)
            R[:, :r] = dev(Rh, torch.float64)
            D[:, :r] = dev(Dh, torch.float64)
            y = dev(yh, torch.float64)
            a_ref, tau_ref = L.lorads_linesearch_coeffs(ctx, R, D, y, rho, r=r)
            st = lib.lorads_linesearch_coeffs_noalloc(
                inst.n, rowptr.data_ptr(), colind.data_ptr(), val.data_ptr(), inst.m, con.data_ptr(),
                row.data_ptr(), col.data_ptr(), aval.data_ptr(), b.data_ptr(), R.data_ptr(), D.data_ptr(),
                r, ld, y.data_ptr(), C.c_double(rho), out.data_ptr(),
                C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == 0, lib.lorads_noalloc_error().decode()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = _scales(P, Rh, Dh, yh, rho)
            assert np.all(np.abs(got[:4] - a_ref) <= 1e-12 * scale), (call, got[:4], a_ref)
            assert got[4] == pytest.approx(tau_ref, rel=1e-9, abs=1e-300)
            a_orc, _ = O.linesearch_coeffs(P, Rh, Dh, yh, rho)
            assert np.all(np.abs(got[:4] - a_orc) <= 1e-12 * scale), (call, got[:4], a_orc)
            assert got[4] == pytest.approx(O.quartic_step(a_orc), rel=1e-9, abs=1e-300)
    finally:
        L.lorads_destroy(ctx)


def test_noalloc_rejects_bad_sizes():
    lib = L.load()
    null = None
    st = lib.lorads_linesearch_coeffs_noalloc(0, null, null, null, 1, null, null, null, null, null, null, null,
                                              1, 4, null, C.c_double(1.0), null, null)
    assert st == 1 and b"n and m" in lib.lorads_noalloc_error()
    st = lib.lorads_linesearch_coeffs_noalloc(10, null, null, null, 10, null, null, null, null, null, null, null,
                                              4, 1024, null, C.c_double(1.0), null, null)
    assert st == 1 and b"512" in lib.lorads_noalloc_error()
