"""CPU tests of the C-ABI library: it builds, loads, exports every declared
symbol, and rejects invalid inputs on the host (before any device call)."""
import re
from pathlib import Path

import numpy as np
import pytest

import workloads as W
import paper_2407_15049_gb300 as L
from paper_2407_15049_gb300 import _native as N

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    L.build()
    return N.load()


def _declared_functions():
    text = (ROOT / "include" / "lorads.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lorads_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = _declared_functions()
    for want in ["lorads_create", "lorads_spmm", "lorads_constraint_eval", "lorads_linesearch_coeffs",
                 "lorads_solve", "lorads_destroy"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_declared_functions()) == set(N.SIGNATURES), "binding and header disagree"


def test_default_params(lib):
    p = N.default_params()
    assert p.tol == 1e-5 and p.lbfgs_mem == 4 and p.max_inner == 500 and p.rho_growth == 2.0
    assert p.lbfgs_scaling == 1 and p.rho_policy == 2 and p.inner_scale == 2 and p.rank_update_threshold == 3
    assert p.inner_progress == 0.1
    assert p.inner_rel == 1.0 and p.infeas_decrease == 0.25 and p.time_limit == 1e4


def _maxcut(n=12, seed=0):
    return W.maxcut_instance(n, W.er_graph(n, 20, seed, "pm1"))


def _expect(status_name, inst, **kw):
    with pytest.raises(N.LoradsError) as ei:
        N.lorads_create(inst, **kw)
    assert N.STATUS_NAMES[ei.value.status] == status_name, str(ei.value)
    return str(ei.value)


def test_rejects_asymmetric_C(lib):
    inst = _maxcut()
    inst.val = inst.val.copy()
    s = inst.rowptr[3]
    if inst.colind[s] == 3:
        s += 1
    inst.val[s] += 0.5
    _expect("LORADS_ERR_NOT_SYMMETRIC", inst)


def test_asymmetry_reports_the_lowest_row_on_a_large_C(lib):
    """C large enough for the threaded symmetry check: with two broken entries in
    different row ranges, the message names the lowest row that sees a mismatch
    (a broken (i, j) is seen from row i and from row j), as a sequential scan would."""
    n = 1_200_000
    inst = W.maxcut_instance(n, W.er_graph(n, 2 * n, 9, "pm1"))
    assert inst.nnz >= 1 << 22
    inst.val = inst.val.copy()
    seen = []
    for row in (1_000_003, 400_001):
        s = inst.rowptr[row]
        if inst.colind[s] == row:
            s += 1
        inst.val[s] += 0.5
        seen += [row, int(inst.colind[s])]
    msg = _expect("LORADS_ERR_NOT_SYMMETRIC", inst)
    assert f"at ({min(seen)}," in msg, msg


def test_rejects_out_of_range_index(lib):
    inst = _maxcut()
    inst.colind = inst.colind.copy()
    inst.colind[-1] = inst.n
    _expect("LORADS_ERR_INVALID_ARG", inst)


def test_rejects_unsorted_row(lib):
    inst = _maxcut()
    inst.colind = inst.colind.copy()
    r = next(i for i in range(inst.n) if inst.rowptr[i + 1] - inst.rowptr[i] >= 2)
    s = inst.rowptr[r]
    inst.colind[s], inst.colind[s + 1] = inst.colind[s + 1], inst.colind[s]
    _expect("LORADS_ERR_INVALID_ARG", inst)


def test_rejects_nan(lib):
    inst = _maxcut()
    inst.b = inst.b.copy()
    inst.b[2] = np.nan
    _expect("LORADS_ERR_INVALID_ARG", inst)
    inst = _maxcut()
    inst.val = inst.val.copy()
    inst.val[0] = np.inf
    _expect("LORADS_ERR_INVALID_ARG", inst)


def test_rejects_lower_triangle_triplet(lib):
    inst = W.mc_instance(4, 5, 2, 6, seed=1)
    inst.row, inst.col = inst.col.copy(), inst.row.copy()
    _expect("LORADS_ERR_INVALID_ARG", inst)


def test_rejects_constraint_without_triplet(lib):
    inst = _maxcut()
    inst.con = inst.con.copy()
    inst.con[1] = 0                    # constraint 0 gets two triplets, constraint 1 none
    msg = _expect("LORADS_ERR_INVALID_ARG", inst)
    assert "no triplet" in msg


def test_rejects_an_entry_listed_twice_in_one_constraint(lib):
    inst = W.theta_instance(5, W.cycle_graph(5))
    inst.row = inst.row.copy()
    inst.col = inst.col.copy()
    inst.row[1], inst.col[1] = inst.row[0], inst.col[0]     # tr X lists X_00 twice
    msg = _expect("LORADS_ERR_INVALID_ARG", inst)
    assert "twice" in msg


def test_batch_rejects_the_general_form(lib):
    """Several constraints on one entry are the general form: lorads_solve takes it,
    the batched solve does not (host check, before any device call)."""
    inst = W.mc_instance(4, 5, 2, 6, seed=1)
    inst.row = inst.row.copy()
    inst.col = inst.col.copy()
    inst.row[1], inst.col[1] = inst.row[0], inst.col[0]
    with pytest.raises(N.LoradsError) as ei:
        N.lorads_batch_create([inst])
    assert N.STATUS_NAMES[ei.value.status] == "LORADS_ERR_UNSUPPORTED"
    assert "general form" in str(ei.value)


def test_rejects_empty_problem(lib):
    inst = _maxcut()
    inst.m = 0
    inst.con = inst.con[:0]
    inst.row = inst.row[:0]
    inst.col = inst.col[:0]
    inst.aval = inst.aval[:0]
    inst.b = inst.b[:0]
    _expect("LORADS_ERR_INVALID_ARG", inst)


def test_rejects_bad_lbfgs_memory(lib):
    _expect("LORADS_ERR_INVALID_ARG", _maxcut(), params=N.default_params(lbfgs_mem=9))


@pytest.mark.parametrize("field,value,word", [
    ("tol", float("nan"), "tol"), ("tol", 0.0, "tol"), ("time_limit", 0.0, "time_limit"),
    ("max_inner", 0, "max_inner"), ("max_outer", 0, "max_outer"),
    ("rank_update_threshold", 0, "rank_update_threshold"), ("rho0", float("inf"), "rho0"),
    ("rho_growth", 0.5, "rho_growth"), ("rho_max", float("nan"), "rho_max"),
    ("infeas_decrease", -0.1, "infeas_decrease"), ("inner_rel", 0.0, "inner_rel"),
    ("inner_progress", float("inf"), "inner_progress"), ("lanczos_steps", 0, "lanczos_steps"),
    ("lbfgs_scaling", 2, "lbfgs_scaling"), ("rho_policy", 3, "rho_policy"), ("inner_scale", -1, "inner_scale"),
    ("cg_rel", 1.0, "cg_rel"), ("reopt_factor", 1.0, "reopt_factor"),
])
def test_rejects_solver_constants_out_of_range(lib, field, value, word):
    """Each solver constant outside its documented range is refused by lorads_create
    and by lorads_batch_create, with a message that names it; the defaults and the
    values the tests and the bench use pass."""
    msg = _expect("LORADS_ERR_INVALID_ARG", _maxcut(), params=N.default_params(**{field: value}))
    assert word in msg, msg
    msg = _expect_batch("LORADS_ERR_INVALID_ARG", [_maxcut()], params=N.default_params(**{field: value}))
    assert word in msg, msg


def _expect_batch(status_name, insts, **kw):
    with pytest.raises(N.LoradsError) as ei:
        N.lorads_batch_create(insts, **kw)
    assert N.STATUS_NAMES[ei.value.status] == status_name, str(ei.value)
    return str(ei.value)


def test_batch_rejects_a_bad_instance_and_names_it(lib):
    good = _maxcut()
    bad = _maxcut(seed=1)
    bad.colind = bad.colind.copy()
    bad.colind[-1] = bad.n
    msg = _expect_batch("LORADS_ERR_INVALID_ARG", [good, good, bad])
    assert "instance 2" in msg
    asym = _maxcut(seed=2)
    asym.val = asym.val.copy()
    asym.val[asym.rowptr[5] + 1] += 1.0
    msg = _expect_batch("LORADS_ERR_NOT_SYMMETRIC", [asym, good])
    assert "instance 0" in msg


def test_batch_rejects_bad_precision_and_rank(lib):
    good = _maxcut()
    _expect_batch("LORADS_ERR_INVALID_ARG", [good], params=N.default_params(prec=N.LORADS_DF64))
    _expect_batch("LORADS_ERR_INVALID_ARG", [good], params=N.default_params(lbfgs_mem=0))
    msg = _expect_batch("LORADS_ERR_INVALID_ARG", [good, good], r0=[4, 200])
    assert "instance 1" in msg and "r0" in msg


def test_workload_generators_shapes():
    inst = W.maxcut_instance(50, W.er_graph(50, 100, 0, "pm1"))
    assert inst.rowptr[-1] == 2 * 100 + 50 and inst.m == 50
    i, j, w = W.torus_graph(10, 0)
    assert len(i) == 200 and set(np.unique(w)) <= {-1.0, 1.0}
    mc = W.mc_instance(30, 40, 3, 200, seed=2)
    assert mc.n == 70 and mc.m == 200 and np.all(mc.col >= 30)
    assert W.rank_log2(1000) == 10 and W.rank_log2(10**6) == 20 and W.rank_log2(10**7) == 24


@pytest.mark.parametrize("graph", ["er_pm1", "er_unit_isolated", "torus", "cycle", "complete", "uniform"])
def test_counting_csr_equals_the_sparse_conversion(graph):
    """The counting CSR build (sorted distinct pairs) gives the arrays of the general
    sparse-matrix conversion bit for bit: same row pointers, columns and values."""
    rng = np.random.default_rng(5)
    if graph == "er_pm1":
        n, e = 300, W.er_graph(300, 1200, 1, "pm1")
    elif graph == "er_unit_isolated":
        n, e = 500, W.er_graph(500, 120, 2, "unit")         # many rows without an edge
    elif graph == "torus":
        n, e = 144, W.torus_graph(12, 3)
    elif graph == "cycle":
        n, e = 9, W.cycle_graph(9)
    elif graph == "complete":
        n, e = 12, W.complete_graph(12)
    else:
        i, j, _ = W.er_graph(200, 900, 4, "unit")
        n, e = 200, (i, j, rng.uniform(-1, 1, len(i)))
    i, j, w = e
    assert W._sorted_distinct_upper(np.asarray(i), np.asarray(j))
    deg = np.bincount(np.concatenate([i, j]), weights=np.concatenate([w, w]), minlength=n)
    a = W._sym_csr(n, i, j, np.asarray(w) / 4.0, -deg / 4.0)
    b = W._sym_csr_upper_sorted(n, i, j, np.asarray(w) / 4.0, -deg / 4.0)
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and np.array_equal(x, y)
    inst = W.maxcut_instance(n, e)
    assert np.array_equal(inst.colind, a[1]) and np.array_equal(inst.val, a[2])


def test_unsorted_pairs_take_the_sparse_conversion():
    i, j, w = W.er_graph(100, 300, 7, "pm1")
    perm = np.random.default_rng(0).permutation(len(i))
    assert not W._sorted_distinct_upper(i[perm], j[perm])
    a = W.maxcut_instance(100, (i, j, w))
    b = W.maxcut_instance(100, (i[perm], j[perm], w[perm]))
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.colind, b.colind)
    assert np.allclose(a.val, b.val, rtol=0, atol=1e-15)


@pytest.mark.parametrize("overrides", [
    {}, dict(prec=N.LORADS_MIXED, compute_err2=1, admm_switch=3e-4, lbfgs_mem=2),
    dict(max_outer=10**6, max_inner=200, rank_update_threshold=10**6, verbose=2),
    dict(max_outer=1, max_inner=5, tol=1e-300), dict(time_limit=1e-9), dict(reopt_level=2, lanczos_steps=300),
    dict(lbfgs_scaling=0, rank_update_threshold=1), dict(infeas_decrease=0.0, rho_growth=1.0),
])
def test_accepts_the_solver_constants_in_use(lib, overrides):
    """The parameter sets of the bench, smoke() and the GPU tests pass the range checks:
    without a GPU the call gets as far as the first device call, with one it succeeds."""
    pairs = ((lambda p: N.lorads_create(_maxcut(), p), N.lorads_destroy),
             (lambda p: N.lorads_batch_create([_maxcut()], p), N.lorads_batch_destroy))
    for create, destroy in pairs:
        try:
            handle = create(N.default_params(**overrides))
        except N.LoradsError as e:
            assert N.STATUS_NAMES[e.status] in ("LORADS_ERR_CUDA", "LORADS_ERR_OOM"), str(e)
        else:
            destroy(handle)
