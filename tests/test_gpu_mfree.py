"""Matrix-free products (Algorithms MvPA / MvPAt of Sec. 4 on the device: the stages of R,
Sigma, the permutation and the left rotations applied in FP32) against the oracle's assembled
A, and FISTA on matrix-free instances against the oracle's FISTA."""

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance
from oracle import solvers

pytestmark = pytest.mark.gpu

EPS32 = 6e-8


@pytest.fixture(scope="module")
def ctx():
    import paper_1503_03520_gb300 as l1
    c = l1.Context(0)
    yield c
    c.close()


def _factored_abs(ref, v, transpose):
    """The products of the absolute values of every factor, stage by stage, applied to |v|:
    the scale of the rounding errors of the factored product (it can exceed |A| |v|)."""
    from oracle.generator import angles, stage_first, stage_matrix
    p = ref.params
    c, s, _, _ = angles(p)
    n = ref.sigma.shape[0]
    T = [abs(stage_matrix(n, stage_first(k), c, s)) for k in range(1, p.right_stages + 1)]
    L = abs(ref.Lmat)
    if not transpose:
        z = np.abs(v)
        for Tk in reversed(T):
            z = Tk.T @ z
        zz = np.zeros(L.shape[1])
        zz[:n] = ref.sigma * z
        return L @ zz
    z = ref.sigma * (L.T @ np.abs(v))[:n]
    for Tk in T:
        z = Tk @ z
    return z


@pytest.mark.parametrize("shape", [(2048, 1024, 1, 1), (20002, 10001, 2, 1), (9000, 4500, 4, 1),
                                   (3001, 1000, 3, 0), (8, 3, 2, 0), (4098, 2049, 8, 1)])
def test_matrix_free_products_match_oracle(ctx, shape):
    import torch
    m, n, w, left = shape
    params = W.params(m=m, n=n, right_stages=w, left_stages=left, kappa=1e3, value_dtype="f32", seed=5)
    ref = oracle_instance(params)
    inst = ctx.generate(dict(params, matrix_free=1))
    try:
        assert inst.info["matrix_free"] == 1 and inst.nnz == ref.A.nnz
        xr = W.random_vector(n, 1).astype(np.float32).astype(np.float64)
        yr = W.random_vector(m, 2).astype(np.float32).astype(np.float64)
        ax = inst.matvec(torch.tensor(xr, dtype=torch.float32, device="cuda")).double().cpu().numpy()
        aty = inst.rmatvec(torch.tensor(yr, dtype=torch.float32, device="cuda")).double().cpu().numpy()
        k = 2 * w + 6
        assert np.all(np.abs(ax - ref.A @ xr) <= k * EPS32 * _factored_abs(ref, np.abs(xr), False) + 1e-30)
        assert np.all(np.abs(aty - ref.A.T @ yr) <= k * EPS32 * _factored_abs(ref, np.abs(yr), True) + 1e-30)
        # host buffers through the same entry points
        assert np.array_equal(inst.matvec(xr.astype(np.float32)).astype(np.float64), ax)
    finally:
        inst.free()


def test_matrix_free_instance_matches_the_stored_one(ctx):
    """The same parameters with and without the assembled matrix: same b, x*, f*, lambda_max;
    the FP32 products agree to FP32 rounding."""
    import torch
    params = W.params(m=50000, n=25000, right_stages=2, left_stages=1, kappa=1e4, value_dtype="f32", seed=7)
    a = ctx.generate(params)
    b = ctx.generate(dict(params, matrix_free=1))
    try:
        for k in ("f_star", "lam_max", "lipschitz", "s", "nnz"):
            assert a.info[k] == b.info[k]
        assert b.info["device_bytes"] < a.info["device_bytes"] / 3
        ea, eb = a.export(), b.export_vectors()
        assert np.array_equal(ea["b"], eb["b"]) and np.array_equal(ea["xstar"], eb["xstar"])
        x = torch.tensor(W.random_vector(25000, 3), dtype=torch.float32, device="cuda")
        ya, yb = a.matvec(x), b.matvec(x)
        scale = float(torch.abs(ya).max())
        assert float(torch.abs(ya - yb).max()) <= 1e-5 * scale
    finally:
        a.free()
        b.free()


@pytest.mark.parametrize("restart", [0, 1])
def test_fista_matrix_free_matches_oracle(ctx, restart):
    params = W.params(m=6000, n=3000, right_stages=2, left_stages=1, kappa=10.0 ** 2.2, seed=9, xstar_frac=0.02,
                      value_dtype="f32")
    ref = oracle_instance(params)
    inst = ctx.generate(dict(params, matrix_free=1))
    try:
        tau = 1.0 if not restart else 0.3 * ref.lam_max
        x, r = inst.solve_fista(tau=tau, tol=1e-6, max_iter=100000, restart=restart)
        o = solvers.fista(ref.A, ref.b, tau, 1.0, 1e-6, 100000, restart=bool(restart))
        assert o["status"] == 0
        assert r["status"] == 0 and r["rel_gap"] <= 1e-6
        assert abs(r["iters"] - o["iters"]) <= max(5, 0.05 * o["iters"]), (r["iters"], o["iters"])
        # the certificate of the returned x on the FP64 problem (FP32 products: 1e-5)
        assert solvers.certificate(ref.A, ref.b, tau, x)[3] <= 1e-5
    finally:
        inst.free()


def test_matrix_free_rejections(ctx):
    import paper_1503_03520_gb300 as l1
    for bad in (dict(m=256, n=512), dict(m=512, n=256, value_dtype="f64")):
        with pytest.raises(l1.L1LSError) as e:
            ctx.generate(W.params(matrix_free=1, **bad))
        assert e.value.status == 1
    inst = ctx.generate(W.params(m=512, n=256, value_dtype="f32", matrix_free=1))
    try:
        for call in (lambda: inst.solve_pdncg(tau=1.0), lambda: inst.export(), lambda: inst.export_t(),
                     lambda: inst.solve_fista(tau=1.0, accum=1)):
            with pytest.raises(l1.L1LSError) as e:
                call()
            assert e.value.status == 1
    finally:
        inst.free()
