"""Full-size C2 workload (m = 2^25, n = 2^24, FP32 values), checked on sampled outputs the
oracle computes one by one (Algorithms MvPA / MvPAt on unit vectors) and on properties that
hold at any size (IGen's optimum certifies at once)."""

import numpy as np
import pytest

import workloads as W
from oracle.generator import GenParams, igen_matrix_free, make_factors
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
