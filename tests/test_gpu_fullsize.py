"""Full-size C2 workload (m = 2^25, n = 2^24, FP32 values), checked on sampled outputs the
oracle computes one by one (Algorithms MvPA / MvPAt on unit vectors) and on properties that
hold at any size (IGen's optimum certifies at once)."""

import numpy as np
import pytest

import workloads as W
from oracle.generator import GenParams, angles, igen_matrix_free, make_factors, stage_first, stage_pairs
from oracle.operators import mvpa, mvpat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    inst = ctx.generate(W.C2)
    f = make_factors(GenParams.from_dict(W.C2))
    yield ctx, inst, f
    inst.free()
    ctx.close()


def _unit(size, k):
    import torch
    v = torch.zeros(size, dtype=torch.float32, device="cuda")
    v[k] = 1.0
    return v


def test_c2_vectors_and_scalars(c2):
    ctx, inst, f = c2
    m, n = inst.m, inst.n
    b_ref, e_ref = igen_matrix_free(f)
    b = np.zeros(m)
    xs = np.zeros(n)
    sg = np.zeros(n)
    pm = np.zeros(m, np.int64)
    import ctypes
    import paper_1503_03520_gb300 as l1
    st = l1.lib.l1ls_inst_export(inst._h, None, None, None, b.ctypes.data, xs.ctypes.data, sg.ctypes.data,
                                 pm.ctypes.data)
    assert st == 0
    assert np.array_equal(pm, f.perm)
    assert np.array_equal(xs, f.xstar)
    assert np.allclose(sg, f.sigma, rtol=4e-16, atol=0)
    assert np.abs(b - b_ref).max() <= 50 * W.C2["kappa"] * 2.2e-16 * np.abs(b_ref).max()
    f_star = np.abs(f.xstar).sum() + 0.5 * float(e_ref @ e_ref)
    assert inst.info["f_star"] == pytest.approx(f_star, rel=1e-12)
    assert 7.5 * n <= inst.nnz <= 8 * n          # "about 8 nonzeros per column"


def test_c2_sampled_columns_and_rows(c2):
    ctx, inst, f = c2
    m, n = inst.m, inst.n
    rng = np.random.default_rng(0)
    cols = [0, 1, n // 2, n - 1] + list(rng.integers(0, n, 4))
    for j in cols:
        y = inst.matvec(_unit(n, int(j))).double().cpu().numpy()
        e = np.zeros(n)
        e[j] = 1.0
        ref = mvpa(f, e).astype(np.float32).astype(np.float64)
        assert np.all(np.abs(y - ref) <= np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)), j
        assert 4 <= np.count_nonzero(ref) <= 8
    rows = [0, m - 1] + list(rng.integers(0, m, 4))
    for i in rows:
        x = inst.rmatvec(_unit(m, int(i))).double().cpu().numpy()
        e = np.zeros(m)
        e[i] = 1.0
        ref = mvpat(f, e).astype(np.float32).astype(np.float64)
        assert np.all(np.abs(x - ref) <= np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)), i


def test_c2_optimum_certifies_at_full_size(c2):
    ctx, inst, f = c2
    x, r = inst.solve_fista(x0=f.xstar.copy(), tau=1.0, tol=W.C2_TOL, max_iter=4)
    assert r["status"] == 0 and r["iters"] == 0
    x, r = inst.solve_pdncg(x0=f.xstar.copy(), tau=1.0, tol=W.C2_TOL, max_iter=4)
    assert r["status"] == 0 and r["iters"] == 0


def _abs_stage(v, first, c, s):
    """|T| v for one stage of rotations: (v_i, v_j) <- (|c| v_i + |s| v_j, |s| v_i + |c| v_j)."""
    i, j = stage_pairs(len(v), first)
    vi = v[i].copy()
    vj = v[j].copy()
    v[i] = abs(c) * vi + abs(s) * vj
    v[j] = abs(s) * vi + abs(c) * vj
    return v


def _abs_mvpa(f, x):
    """An entrywise majorant of |A| x for x >= 0: A = L Sigma R^T with every rotation replaced
    by its entrywise absolute value (|sum| <= sum of |terms| stage by stage)."""
    p = f.params
    c, s, ct, st = angles(p)
    y = np.array(x, dtype=np.float64, copy=True)
    for k in range(p.right_stages, 0, -1):
        _abs_stage(y, stage_first(k), c, s)
    yt = np.zeros(p.m)
    yt[:p.n] = f.sigma * y
    if p.left_stages > 0:
        yt = yt[f.perm]
        for k in range(1, p.left_stages + 1):
            _abs_stage(yt, stage_first(k), ct, st)
        yt = yt[f.perm]
    return yt


def _abs_mvpat(f, y):
    """The transpose of _abs_mvpa: a majorant of |A|^T y for y >= 0."""
    p = f.params
    c, s, ct, st = angles(p)
    xt = np.array(y, dtype=np.float64, copy=True)
    if p.left_stages > 0:
        tmp = np.empty(p.m)
        tmp[f.perm] = xt
        xt = tmp
        for k in range(p.left_stages, 0, -1):
            _abs_stage(xt, stage_first(k), ct, st)
        tmp = np.empty(p.m)
        tmp[f.perm] = xt
        xt = tmp
    x = f.sigma * xt[:p.n]
    for k in range(1, p.right_stages + 1):
        _abs_stage(x, stage_first(k), c, s)
    return x


def test_c2_one_fused_iteration_every_entry(c2):
    """The bench's kernels at full size (K1 / K2 on the C2 instance, the grids `bench.py` times):
    one FISTA iteration from x0 = x* + seeded noise, every entry of x1 against the oracle's
    x1 = S_tau(x0 + A^T (b - A x0)) by Algorithms MvPA / MvPAt in FP64.  The device works on the
    FP32-rounded A and b and gathers x0 rounded to FP32; with M >= |A| entrywise (the factors
    with every rotation made nonnegative, _abs_mvpa), the difference of the two is bounded per
    entry by eps ((kmax + 4) M^T M |x0| + (kmax + 4) M^T |r| + |g|) to first order, eps = 2^-24,
    plus the float-float iterate."""
    ctx, inst, f = c2
    n = inst.n
    eps = 2.0 ** -24
    kmax = 4 * W.C2["right_stages"] + 2
    rng = np.random.default_rng(21)
    x0 = f.xstar + 0.1 * rng.standard_normal(n)
    x1, r = inst.solve_fista(x0=x0.copy(), tau=1.0, tol=1e-12, max_iter=1)
    assert r["status"] == 5 and r["iters"] == 1
    b, _ = igen_matrix_free(f)
    res = b - mvpa(f, x0)
    g = mvpat(f, res)
    want = np.sign(x0 + g) * np.maximum(np.abs(x0 + g) - 1.0, 0.0)
    mm = _abs_mvpat(f, _abs_mvpa(f, np.abs(x0)))
    mr = _abs_mvpat(f, np.abs(res))
    tol = eps * ((kmax + 4) * mm + (kmax + 4) * mr + np.abs(g)) * 1.01 + 2.0 ** -45 * (np.abs(x0) + np.abs(g))
    err = np.abs(x1 - want)
    assert np.all(err <= tol), (int(np.argmax(err / tol)), float((err / tol).max()))
    # the bound is far below the size of an entry a mis-staged tile would corrupt
    assert np.median(tol[want != 0]) <= 1e-3 * np.median(np.abs(want[want != 0]))
