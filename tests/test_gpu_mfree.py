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
        for call in (lambda: inst.export(), lambda: inst.export_t(), lambda: inst.solve_fista(tau=1.0, accum=1)):
            with pytest.raises(l1.L1LSError) as e:
                call()
            assert e.value.status == 1
    finally:
        inst.free()


# ---- pdNCG on matrix-free instances ---------------------------------------------------------
# Gradient and certificate by one FP64 sweep (A^T r = A^T b - R Sigma^2 R^T x), the PCG product
# by one FP32 sweep (A^T A = R Sigma^2 R^T), the line search's sums by one FP64 sweep.


@pytest.mark.parametrize("left,w", [(1, 2), (0, 2), (1, 5), (0, 8)])
def test_pdncg_matrix_free_certificate_at_x0(ctx, left, w):
    """max_iter = 0 returns the first certificate at x0: P and D against the oracle's at the same
    x0 on the FP64 A (A^T b, ||b||^2, ||Sigma R^T x||^2 and max |A^T r| all enter them).  Two
    tiles with a ragged second one (n = 3001)."""
    n = 3001
    params = W.params(m=2 * n + 2, n=n, right_stages=w, left_stages=left, kappa=1e3, seed=11, xstar_frac=0.02,
                      value_dtype="f32")
    ref = oracle_instance(params)
    inst = ctx.generate(dict(params, matrix_free=1))
    try:
        for seed, tau in ((4, 1.0), (5, 0.3 * ref.lam_max)):
            x0 = ref.xstar + 0.1 * W.random_vector(n, seed)
            x, r = inst.solve_pdncg(x0=x0.copy(), tau=tau, tol=1e-12, max_iter=0, allow=(4, 5))
            P, D, gap, rel = solvers.certificate(ref.A, ref.b, tau, x0)
            assert r["iters"] == 0 and np.array_equal(x, x0)
            assert r["f"] == pytest.approx(P, rel=1e-11)
            assert r["dual"] == pytest.approx(D, rel=1e-10, abs=1e-10 * abs(P))
    finally:
        inst.free()


@pytest.mark.parametrize("left", [1, 0])
def test_pdncg_matrix_free_matches_oracle(ctx, left):
    """pdNCG to 1e-6 on a matrix-free instance: the oracle re-certifies the returned x on the FP64
    A, f is compared with f*, and the oracle's pdNCG bounds the Newton count."""
    n = 3000
    params = W.params(m=2 * n, n=n, right_stages=2, left_stages=left, kappa=1e3, seed=9, xstar_frac=0.02,
                      value_dtype="f32")
    ref = oracle_instance(params)
    inst = ctx.generate(dict(params, matrix_free=1))
    try:
        x, r = inst.solve_pdncg(tau=1.0, tol=1e-6, max_iter=200)
        assert r["status"] == 0 and r["rel_gap"] <= 1e-6
        P, D, gap, rel = solvers.certificate(ref.A, ref.b, 1.0, x)
        assert rel <= 1.01e-6 and P == pytest.approx(r["f"], rel=1e-11)
        assert abs(P - ref.f_star) <= 2e-6 * ref.f_star
        o = solvers.pdncg(ref.A, ref.b, 1.0, 1e-6)
        assert o["status"] == 0
        assert r["iters"] <= 2 * o["iters"] + 3, (r["iters"], o["iters"])
    finally:
        inst.free()


def test_pdncg_matrix_free_sec89_shape(ctx):
    """Sec. 8.9's instance shape (A = Sigma G^T, L = I, sigma 0.1 / 100, x* entries -1e4 and 0.1)
    at n = 2^12: matrix-free pdNCG to 1e-6 against the stored FP32 instance (float-float
    gradient) and the oracle's x*."""
    params = W.sec89(12, "f32")
    ref = oracle_instance(params)
    a = ctx.generate(dict(params, matrix_free=1))
    b = ctx.generate(params)
    try:
        xa, ra = a.solve_pdncg(tau=1.0, tol=1e-6, max_iter=200)
        xb, rb = b.solve_pdncg(tau=1.0, tol=1e-6, max_iter=200, accum=1)
        assert ra["status"] == 0 and rb["status"] == 0
        assert solvers.certificate(ref.A, ref.b, 1.0, xa)[3] <= 1.01e-6
        assert np.linalg.norm(xa - ref.xstar) <= 1e-6 * np.linalg.norm(ref.xstar)
        assert abs(ra["iters"] - rb["iters"]) <= max(3, rb["iters"] // 4), (ra["iters"], rb["iters"])
    finally:
        a.free()
        b.free()


def test_pdncg_matrix_free_several_tiles_per_block(ctx):
    """C2 recipe at n = 2^22 (2048 tiles, more than one block's share on this grid): the
    certificate at x* is the one of the exact minimiser, and pdNCG to 1e-6 takes about the
    Newton steps of the stored FP32 instance."""
    params = W.c2_scaled(22)
    a = ctx.generate(dict(params, matrix_free=1))
    b = ctx.generate(params)
    try:
        xs = a.xstar()
        _, r0 = a.solve_pdncg(x0=xs.copy(), tau=1.0, tol=1e-12, max_iter=0, allow=(4, 5))
        assert abs(r0["f"] - a.info["f_star"]) <= 1e-12 * a.info["f_star"]
        assert r0["rel_gap"] <= 1e-10
        xa, ra = a.solve_pdncg(tau=1.0, tol=W.C2_TOL, max_iter=200)
        xb, rb = b.solve_pdncg(tau=1.0, tol=W.C2_TOL, max_iter=200, accum=1)
        assert ra["status"] == 0 and rb["status"] == 0
        assert abs(ra["f"] - a.info["f_star"]) <= 2 * W.C2_TOL * a.info["f_star"]
        assert abs(ra["iters"] - rb["iters"]) <= max(3, rb["iters"] // 4), (ra["iters"], rb["iters"])
    finally:
        a.free()
        b.free()
