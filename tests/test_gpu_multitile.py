"""Parity at the sizes where one warp traverses several tiles (C2 recipe at n = 2^19, 2^20).

The fused FISTA kernels and the plain products run on a grid capped at (SMs x resident
blocks); with 152 SMs, 4 blocks of 8 warps per SM and tiles of 32 row pairs (A x) or 32
columns (A^T y), a warp takes several tiles once m/2 or n exceeds about 155,000: at
n = 2^19 each warp sums about 3.4 tiles of each kind, at n = 2^20 about 6.7.  These tests
exercise the next-tile staging, the stage parity flip and the stage reuse element by element
against the oracle's assembled A (Eq. bd8), which the smaller parity tests do not reach.
"""

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance, stored_values
from oracle import solvers

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", params=[19, 20])
def case(request):
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    out = {}
    for dt in ("f32", "f64"):
        params = W.c2_scaled(request.param, value_dtype=dt)
        out[dt] = (params, ctx.generate(params))
    ref = oracle_instance(out["f32"][0])      # the FP64 matrix is the same for both stored types
    yield request.param, ref, out
    for _, inst in out.values():
        inst.free()
    ctx.close()


def test_products_several_tiles_per_warp(case):
    """A x and A^T y on random FP32 vectors within the entry-wise rounding bound of a sum of
    at most kmax FP32 products (plus the final rounding), as in the small-size product tests."""
    import torch
    log2n, ref, insts = case
    params, inst = insts["f32"]
    A = stored_values(ref.A, "f32")
    absA = abs(A)
    m, n = A.shape
    for seed in (0, 1):
        xd = torch.tensor(W.random_vector(n, 100 + seed), dtype=torch.float32, device="cuda")
        yd = torch.tensor(W.random_vector(m, 200 + seed), dtype=torch.float32, device="cuda")
        xr = xd.double().cpu().numpy()
        yr = yd.double().cpu().numpy()
        ax = inst.matvec(xd).double().cpu().numpy()
        aty = inst.rmatvec(yd).double().cpu().numpy()
        torch.cuda.synchronize()
        kmax = 4 * params["right_stages"] + 2
        ry = A @ xr
        rx = A.T @ yr
        bound_y = kmax * 6e-8 * (absA @ np.abs(xr)) + 6e-8 * np.abs(ry) + 1e-300
        bound_x = kmax * 6e-8 * (absA.T @ np.abs(yr)) + 6e-8 * np.abs(rx) + 1e-300
        assert np.all(np.abs(ax - ry) <= bound_y), np.argmax(np.abs(ax - ry) / bound_y)
        assert np.all(np.abs(aty - rx) <= bound_x), np.argmax(np.abs(aty - rx) / bound_x)


def _fista_rounding_bound(A, b, iters, eps, kmax):
    """2-norm bound on the distance between FISTA whose products round with unit roundoff eps
    and FISTA in exact arithmetic on the same A and b after `iters` iterations (L = 1).  With
    L >= ||A||^2 the map y -> S(y + A^T(b - A y)) is nonexpansive (I - A^T A has eigenvalues in
    [0, 1), the shrinkage is nonexpansive), so an iterate error E_k obeys
      E_k <= (1 + beta_k) E_{k-1} + beta_k E_{k-2} + delta_k,
    with delta_k = || c eps (|A|^T (|A| |y|~ + |b|) + |A^T r_k|) ||_2 covering the <= kmax-term
    sums of both products, A y formed by linearity ((1 + beta) |x_{k-1}| + beta |x_{k-2}| for
    |y|~) and the roundings of the residual and the results (c = 2 kmax + 4)."""
    absA = abs(A)
    c = 2 * kmax + 4
    n = A.shape[1]
    x_cur = np.zeros(n)
    x_old = np.zeros(n)
    t, beta = 1.0, 0.0
    E_cur = E_old = 0.0
    for _ in range(iters):
        y = x_cur + beta * (x_cur - x_old)
        yabs = (1 + beta) * np.abs(x_cur) + beta * np.abs(x_old)
        g = A.T @ (b - A @ y)
        delta = c * eps * np.linalg.norm(absA.T @ (absA @ yabs + np.abs(b)) + np.abs(g))
        E_new = (1 + beta) * E_cur + beta * E_old + delta
        x_new = solvers.soft_threshold(y + g, 1.0)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_new
        t = t_new
        x_old, x_cur = x_cur, x_new
        E_old, E_cur = E_cur, E_new
    return x_cur, E_cur


def test_fista_ten_iterations_fp64_values(case):
    """FP64 values: the fused K1 / K2 with their epilogues against the oracle's FISTA after 10
    iterations; the two differ only in the order of FP64 roundings, bounded by
    _fista_rounding_bound for both sides (twice the bound of one)."""
    log2n, ref, insts = case
    params, inst = insts["f64"]
    x, r = inst.solve_fista(tau=1.0, tol=1e-12, max_iter=10)
    assert r["status"] == 5 and r["iters"] == 10
    o = solvers.fista(ref.A, ref.b, 1.0, 1.0, 1e-12, 10)
    x_b, E = _fista_rounding_bound(ref.A, ref.b, 10, 2.0 ** -53, 4 * params["right_stages"] + 2)
    assert np.allclose(x_b, o["x"], rtol=1e-9, atol=1e-9)
    assert np.linalg.norm(x - o["x"]) <= 2 * E
    assert E <= 1e-8 * np.linalg.norm(o["x"])      # far below what a mis-staged tile would change
    assert r["f"] == pytest.approx(o["P"], rel=1e-12)


def test_fista_one_step_fp32_values(case):
    """FP32 values (the C2 path): one fused iteration (K1, K2 and the shrinkage epilogue) from
    x0 = x* + seeded noise, entry by entry against the oracle's step on the FP32-rounded A and b.
    The first iteration is the prox-gradient step x1 = S_tau(x0 + A^T (b - A x0)) (L = 1).  Its
    rounding: K1 gathers x0 rounded to FP32 and sums at most kmax FP32 products per row, the
    residual b - A x0 is rounded once, K2 sums at most kmax FP32 products per column; the
    shrinkage is 1-Lipschitz per entry.  So, to first order in eps = 2^-24,
      |dx1| <= eps ((kmax + 2) |A|^T |A| |x0| + (kmax + 2) |A|^T |r| + |A^T r|),
    plus the float-float iterate (about 2^-45 of |x0| + |A^T r|)."""
    log2n, ref, insts = case
    params, inst = insts["f32"]
    A = stored_values(ref.A, "f32")
    b = ref.b.astype(np.float32).astype(np.float64)
    absA = abs(A)
    kmax = 4 * params["right_stages"] + 2
    for seed in (3, 4):
        x0 = ref.xstar + 0.1 * W.random_vector(A.shape[1], seed)
        x, r = inst.solve_fista(x0=x0.copy(), tau=1.0, tol=1e-12, max_iter=1)
        assert r["status"] == 5 and r["iters"] == 1
        o = solvers.fista(A, b, 1.0, 1.0, 1e-12, 1, x0=x0)
        res = b - A @ x0
        g = A.T @ res
        bound = EPS32 * ((kmax + 2) * (absA.T @ (absA @ np.abs(x0))) + (kmax + 2) * (absA.T @ np.abs(res))
                         + np.abs(g)) * 1.01 + 2.0 ** -45 * (np.abs(x0) + np.abs(g)) + 1e-300
        err = np.abs(x - o["x"])
        assert np.all(err <= bound), (int(np.argmax(err / bound)), float((err / bound).max()))


def test_fista_iteration_count_fp32_values(case):
    """FISTA to the 1e-6 gap with FP32 values: the device's iteration count against the oracle's
    FP64 FISTA on the stored problem (the same certificate rule; they may part only where the
    rounding of a certificate crosses the threshold)."""
    log2n, ref, insts = case
    params, inst = insts["f32"]
    A = stored_values(ref.A, "f32")
    b = ref.b.astype(np.float32).astype(np.float64)
    tol = W.C2_TOL
    x, r = inst.solve_fista(tau=1.0, tol=tol, max_iter=20000)
    assert r["status"] == 0
    o = solvers.fista(A, b, 1.0, 1.0, tol, 20000)
    assert o["status"] == 0
    assert abs(r["iters"] - o["iters"]) <= max(3, 0.01 * o["iters"]), (r["iters"], o["iters"])
    assert r["f"] == pytest.approx(o["P"], rel=1e-9)


def test_fista_to_gap_several_tiles_per_warp(case):
    """FISTA to the 1e-6 gap on the FP32 instance: the oracle re-certifies the returned x on the
    stored problem, f is compared with the generator's f*, and the distance to x* obeys the
    strong-convexity bound of the FP64 problem, ||x - x*||^2 <= 2 (P(x) - f*) / sigma_min^2."""
    log2n, ref, insts = case
    params, inst = insts["f32"]
    tol = W.C2_TOL
    x, r = inst.solve_fista(tau=1.0, tol=tol, max_iter=20000)
    assert r["status"] == 0 and r["rel_gap"] <= tol
    A = stored_values(ref.A, "f32")
    b = ref.b.astype(np.float32).astype(np.float64)
    P, D, gap, rel = solvers.certificate(A, b, 1.0, x)
    assert rel <= 20 * tol
    f64 = solvers.objective(ref.A, ref.b, 1.0, x)
    assert abs(f64 - ref.f_star) <= 20 * tol * ref.f_star
    excess = max(f64 - ref.f_star, 0.0)
    smin = ref.sigma.min()
    assert float(np.sum((x - ref.xstar) ** 2)) <= 2.0 * excess / smin ** 2 + 1e-9 * float(ref.xstar @ ref.xstar)


def test_pdncg_to_gap_several_tiles_per_warp(case):
    """pdNCG on the FP32 instance (its products traverse several tiles per warp): the oracle
    re-certifies the returned x on the stored problem, and the oracle's pdNCG on that problem
    bounds the Newton count."""
    log2n, ref, insts = case
    params, inst = insts["f32"]
    tol = W.C2_TOL
    x, r = inst.solve_pdncg(tau=1.0, tol=tol, max_iter=200)
    assert r["status"] == 0 and r["rel_gap"] <= tol
    A = stored_values(ref.A, "f32")
    b = ref.b.astype(np.float32).astype(np.float64)
    P, D, gap, rel = solvers.certificate(A, b, 1.0, x)
    assert rel <= 20 * tol
    if log2n == 19:
        o = solvers.pdncg(A, b, 1.0, tol)
        assert o["status"] == 0
        assert r["iters"] <= 2 * o["iters"] + 3, (r["iters"], o["iters"])
