"""FISTA and pdNCG on the device against the oracle (Sec. 8.1; IGen's known optimum)."""

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance, stored_values
from oracle import solvers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1503_03520_gb300 as l1
    c = l1.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def c1(ctx):
    ref = oracle_instance(W.C1)
    inst = ctx.generate(W.C1)
    yield ref, inst
    inst.free()


def test_fista_c1_matches_oracle(c1):
    ref, inst = c1
    tol = W.C1_TOL
    x, r = inst.solve_fista(tau=1.0, tol=tol, max_iter=200000)
    assert r["status"] == 0 and r["rel_gap"] <= tol
    o = solvers.fista(ref.A, ref.b, 1.0, ref.lipschitz, tol, 200000)
    # same rule, same iteration count up to rounding-order effects at the threshold
    assert abs(r["iters"] - o["iters"]) <= max(3, 0.01 * o["iters"])
    # primal suboptimality by the oracle's objective against the known optimum
    f = solvers.objective(ref.A, ref.b, 1.0, x)
    assert f - ref.f_star <= 1.01 * tol * ref.f_star
    assert np.sum((x - ref.xstar) ** 2) <= 2.0 * 1.01 * tol * ref.f_star / ref.sigma.min() ** 2


def test_pdncg_c1_matches_oracle(c1):
    ref, inst = c1
    tol = W.C1_TOL
    x, r = inst.solve_pdncg(tau=1.0, tol=tol, max_iter=200)
    assert r["status"] == 0 and r["rel_gap"] <= tol
    o = solvers.pdncg(ref.A, ref.b, 1.0, tol)
    assert abs(r["iters"] - o["iters"]) <= 2
    assert r["iters"] <= 30
    f = solvers.objective(ref.A, ref.b, 1.0, x)
    assert f - ref.f_star <= 1.01 * tol * ref.f_star


@pytest.mark.parametrize("method", ["fista", "pdncg"])
@pytest.mark.parametrize("tau", [0.5, 2.0])
def test_tau_off_generator_matches_oracle_solution(ctx, method, tau):
    """tau != tau_gen: no closed form; compare with the oracle's own solve."""
    params = W.params(m=1024, n=512, right_stages=2, kappa=30.0, seed=4, xstar_frac=0.05)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        fn = inst.solve_fista if method == "fista" else inst.solve_pdncg
        x, r = fn(tau=tau, tol=1e-10, max_iter=500000 if method == "fista" else 200)
        assert r["status"] == 0
        o = (solvers.fista(ref.A, ref.b, tau, 1.0, 1e-10, 500000) if method == "fista"
             else solvers.pdncg(ref.A, ref.b, tau, 1e-10))
        fo = solvers.objective(ref.A, ref.b, tau, o["x"])
        fg = solvers.objective(ref.A, ref.b, tau, x)
        assert abs(fg - fo) <= 2e-10 * fo
    finally:
        inst.free()


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("method", ["fista", "pdncg"])
def test_reduced_precision_certificate_holds_on_the_stored_problem(ctx, dt, method):
    """FP32 / BF16 values define their own problem (A rounded once); the oracle re-checks the
    device's answer on that problem with its own certificate."""
    tol = 1e-6 if dt == "f32" else 1e-4
    params = W.params(m=16384, n=8192, right_stages=2, kappa=1e3, seed=6, xstar_frac=0.01, value_dtype=dt)
    ref = oracle_instance(params)
    A = stored_values(ref.A, dt)
    b = ref.b.astype(np.float32).astype(np.float64)
    inst = ctx.generate(params)
    try:
        fn = inst.solve_fista if method == "fista" else inst.solve_pdncg
        x, r = fn(tau=1.0, tol=tol, max_iter=200000 if method == "fista" else 200)
        assert r["status"] == 0 and r["rel_gap"] <= tol
        P, D, gap, rel = solvers.certificate(A, b, 1.0, x)
        assert rel <= 20 * tol
        # stated per result: relative error of f_tau against the FP64 optimum
        f64 = solvers.objective(ref.A, ref.b, 1.0, x)
        assert abs(f64 - ref.f_star) / ref.f_star <= 100 * tol
    finally:
        inst.free()


def test_warm_start_at_optimum_certifies_immediately(c1):
    ref, inst = c1
    x, r = inst.solve_fista(x0=ref.xstar.copy(), tau=1.0, tol=1e-10, max_iter=10)
    assert r["status"] == 0 and r["iters"] == 0
    x, r = inst.solve_pdncg(x0=ref.xstar.copy(), tau=1.0, tol=1e-10, max_iter=10)
    assert r["status"] == 0 and r["iters"] == 0


def test_iteration_limit_reports_noconv(c1):
    ref, inst = c1
    x, r = inst.solve_fista(tau=1.0, tol=1e-14, max_iter=10)
    assert r["status"] == 5 and r["iters"] == 10
    o = solvers.fista(ref.A, ref.b, 1.0, 1.0, 0.0, 10)
    assert np.allclose(x, o["x"], rtol=1e-12, atol=1e-12)


def test_device_buffers_in_place(c1):
    import torch
    ref, inst = c1
    x0 = torch.zeros(inst.n, dtype=torch.float64, device="cuda")
    xo = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    xr, r = inst.solve_fista(x0=x0, x_out=xo, tau=1.0, tol=1e-8, max_iter=100000)
    torch.cuda.synchronize()
    assert r["status"] == 0
    xh, rh = inst.solve_fista(tau=1.0, tol=1e-8, max_iter=100000)
    assert np.array_equal(xo.cpu().numpy(), xh)      # deterministic reductions
    assert rh["iters"] == r["iters"]


@pytest.mark.parametrize("tau", [0.3, 0.05])
def test_fista_restart_matches_oracle(ctx, tau):
    """FISTA with the gradient restart (an option; not in the paper) against the oracle's."""
    params = W.params(m=2000, n=1000, right_stages=2, kappa=300.0, seed=41, xstar_frac=0.02)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        x, r = inst.solve_fista(tau=tau, tol=1e-8, max_iter=200000, restart=1)
        assert r["status"] == 0 and r["rel_gap"] <= 1e-8
        o = solvers.fista(ref.A, ref.b, tau, 1.0, 1e-8, 200000, restart=True)
        assert o["status"] == 0
        assert abs(r["iters"] - o["iters"]) <= max(5, 0.15 * o["iters"])
        fo = solvers.objective(ref.A, ref.b, tau, o["x"])
        fg = solvers.objective(ref.A, ref.b, tau, x)
        assert abs(fg - fo) <= 2e-8 * fo
    finally:
        inst.free()


@pytest.mark.parametrize("restart,tau_exp,w,dt", [(0, 0.5, 2, "f32"), (1, 2.0, 2, "f32"), (1, 1.0, 8, "f32"),
                                                  (1, 1.0, 8, "bf16")])
def test_fista_compensated_products_reach_small_gaps_at_small_tau(ctx, restart, tau_exp, w, dt):
    """accum = 1 (float-float products) against the oracle's FP64 FISTA on the stored FP32
    problem, down to a tau (1e-2 of lambda_max) where FP32 sums of the products stall above
    the 1e-6 gap.  (Without the restart FISTA needs more than 1e5 iterations there.)  With
    w = 8 a tile of 32 row pairs holds about 18 entries per pair, more than one shared-memory
    stage: the staged float-float traversal then streams each tile in pieces."""
    params = W.params(m=2000, n=1000, right_stages=w, left_stages=1, kappa=10.0 ** 2.2, seed=41, xstar_frac=0.02,
                      value_dtype=dt)
    ref = oracle_instance(params)
    A = stored_values(ref.A, dt)
    b = ref.b.astype(np.float32).astype(np.float64)
    tau = 0.9 * ref.lam_max * 10.0 ** -tau_exp
    inst = ctx.generate(params)
    try:
        x, r = inst.solve_fista(tau=tau, tol=1e-6, max_iter=100000, restart=restart, accum=1)
        o = solvers.fista(A, b, tau, 1.0, 1e-6, 100000, restart=bool(restart))
        assert o["status"] == 0
        assert r["status"] == 0 and r["rel_gap"] <= 1e-6
        slack = max(3, 0.01 * o["iters"]) if not restart else max(5, 0.15 * o["iters"])
        assert abs(r["iters"] - o["iters"]) <= slack, (r["iters"], o["iters"])
        assert abs(r["f"] - o["P"]) <= 2e-6 * o["P"]
        assert solvers.certificate(A, b, tau, x)[3] <= 1e-5
    finally:
        inst.free()


def test_compensated_products_need_fp32_or_bf16_values(ctx):
    import paper_1503_03520_gb300 as l1
    inst = ctx.generate(W.params(m=512, n=256, value_dtype="f64"))
    try:
        with pytest.raises(l1.L1LSError) as e:
            inst.solve_fista(tau=1.0, accum=1)
        assert e.value.status == 1
    finally:
        inst.free()


@pytest.mark.parametrize("case,frac", [(dict(m=2000, n=1000, left_stages=0, value_dtype="f32", seed=43), 0.09),
                                       (dict(m=1000, n=2000, left_stages=1, value_dtype="f32", seed=46), 0.5),
                                       (dict(m=1500, n=3000, left_stages=0, value_dtype="bf16", seed=43), 0.09)],
                         ids=["plain", "igen2", "igen2_bf16"])
def test_fista_compensated_products_in_plain_storage(ctx, case, frac):
    """accum = 1 on instances without row pairs (no left stage, or IGen2) against the oracle.
    (IGen2's columns of N~ scaled by xi tau / |N_i^T e| make ||A||^2 large: FISTA is slow on
    them at small tau, so the IGen2 case takes tau = lambda_max / 2.)"""
    params = W.params(right_stages=2, kappa=10.0 ** 2.2, xstar_frac=0.02, **case)
    ref = oracle_instance(params)
    A = stored_values(ref.A, case["value_dtype"])
    b = ref.b.astype(np.float32).astype(np.float64)
    tau = frac * ref.lam_max
    inst = ctx.generate(params)
    try:
        assert inst.info["lipschitz"] == pytest.approx(ref.lipschitz, rel=1e-11)
        x, r = inst.solve_fista(tau=tau, tol=1e-6, max_iter=100000, restart=1, accum=1)
        o = solvers.fista(A, b, tau, inst.info["lipschitz"], 1e-6, 100000, restart=True)
        assert o["status"] == 0
        assert r["status"] == 0 and r["rel_gap"] <= 1e-6
        assert abs(r["iters"] - o["iters"]) <= max(5, 0.15 * o["iters"]), (r["iters"], o["iters"])
        assert abs(r["f"] - o["P"]) <= 2e-6 * o["P"]
    finally:
        inst.free()


@pytest.mark.parametrize("L0,tau_rel", [(1e-3, None), (0.3, 0.2), (4.0, 0.5)])
def test_fista_backtracking_matches_oracle(ctx, L0, tau_rel):
    """FISTA with backtracking on L (FP64 values and vectors) against the oracle's: the same
    increases of L (each a decision ||A d||^2 <= L ||d||^2 taken on both sides in FP64), the
    same final L, the iteration count within 2%, and the certified x."""
    params = W.params(m=4096, n=2048, right_stages=2, left_stages=1, kappa=100.0, value_dtype="f64", seed=21,
                      xstar_frac=0.05)
    ref = oracle_instance(params)
    tau = 1.0 if tau_rel is None else tau_rel * ref.lam_max
    inst = ctx.generate(params)
    try:
        x, r = inst.solve_fista_bt(L0, 2.0, tau=tau, tol=1e-8, max_iter=50000)
        o = solvers.fista_bt(ref.A, ref.b, tau, L0, 2.0, 1e-8, 50000)
        assert o["status"] == 0 and r["status"] == 0 and r["rel_gap"] <= 1e-8
        assert r["ls_trials"] == o["backtracks"] and r["L"] == o["L"], (r["ls_trials"], o["backtracks"], r["L"], o["L"])
        assert abs(r["iters"] - o["iters"]) <= max(2, 0.02 * o["iters"]), (r["iters"], o["iters"])
        assert r["products"] == 1 + 2 * r["iters"] + r["ls_trials"]
        assert o["products"] == 1 + 2 * o["iters"] + o["backtracks"]
        assert solvers.certificate(ref.A, ref.b, tau, x)[3] <= 2e-8
        if tau_rel is None:   # strong convexity: ||x - x*||^2 <= 2 gap / sigma_min^2
            assert float((x - ref.xstar) @ (x - ref.xstar)) <= 2.0 * r["gap"] * 100.0 ** 2
    finally:
        inst.free()


def test_fista_backtracking_fp32_values(ctx):
    """FP32 values (FP32 sums in the products): the C2 recipe at n = 2^16 from L0 = 1e-2 reaches
    the 1e-6 gap; L ends within [L0, 2 L_f] (L_f = sigma_max^2 = 1)."""
    params = W.c2_scaled(16)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        x, r = inst.solve_fista_bt(1e-2, 2.0, tau=1.0, tol=1e-6, max_iter=50000)
        assert r["status"] == 0 and r["rel_gap"] <= 1e-6
        assert 1e-2 < r["L"] <= 2.0 and r["ls_trials"] >= 6
        assert solvers.certificate(ref.A, ref.b, 1.0, x)[3] <= 1e-5
    finally:
        inst.free()


def test_fista_backtracking_rejections(ctx):
    import paper_1503_03520_gb300 as l1
    inst = ctx.generate(W.params(m=512, n=256, value_dtype="f32"))
    mf = ctx.generate(W.params(m=512, n=256, value_dtype="f32", matrix_free=1))
    try:
        for call in (lambda: inst.solve_fista_bt(0.0, 2.0), lambda: inst.solve_fista_bt(1.0, 1.0),
                     lambda: inst.solve_fista_bt(float("nan"), 2.0), lambda: mf.solve_fista_bt(1.0, 2.0)):
            with pytest.raises(l1.L1LSError) as e:
                call()
            assert e.value.status == 1
    finally:
        inst.free()
        mf.free()


def test_objective_target_matches_oracle(ctx):
    """f_target (the paper's rule for ending its comparison solvers, Sec. 8.3): FISTA and FISTA
    with backtracking stop at the same iteration as the oracle's; pdNCG stops below the target."""
    params = W.params(m=4096, n=2048, right_stages=2, left_stages=1, kappa=100.0, value_dtype="f64", seed=23,
                      xstar_frac=0.05)
    ref = oracle_instance(params)
    f0 = 0.5 * float(ref.b @ ref.b)             # the objective at x = 0
    target = ref.f_star + 1e-4 * (f0 - ref.f_star)
    inst = ctx.generate(params)
    try:
        runs = ((lambda: inst.solve_fista(tau=1.0, tol=0.0, max_iter=100000, f_target=target),
                 lambda: solvers.fista(ref.A, ref.b, 1.0, ref.lipschitz, 0.0, 100000, f_target=target)),
                (lambda: inst.solve_fista_bt(1e-2, 2.0, tau=1.0, tol=0.0, max_iter=100000, f_target=target),
                 lambda: solvers.fista_bt(ref.A, ref.b, 1.0, 1e-2, 2.0, 0.0, 100000, f_target=target)))
        for dev, orc in runs:
            x, r = dev()
            o = orc()
            assert r["status"] == 0 and o["status"] == 0 and o["iters"] >= 5
            assert r["iters"] == o["iters"] and r["f"] <= target, (r["iters"], o["iters"])
            assert solvers.objective(ref.A, ref.b, 1.0, x) <= target * (1.0 + 1e-12)
        x, r = inst.solve_pdncg(tau=1.0, tol=0.0, max_iter=200, f_target=target)
        assert r["status"] == 0 and r["f"] <= target
        assert solvers.objective(ref.A, ref.b, 1.0, x) <= target * (1.0 + 1e-12)
    finally:
        inst.free()


@pytest.mark.parametrize("factor", [1.0, 1.5])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tau_at_or_above_lambda_max_gives_zero(ctx, factor, dt):
    """The degenerate case of Eq. (prob1): for tau >= lambda_max = ||A^T b||_inf the minimiser is
    x = 0, and at x = 0 the dual point theta = b is feasible with D = P = ||b||^2 / 2, so every
    solver certifies the start without an iteration (lambda_max checked against the oracle)."""
    params = W.params(m=1024, n=512, right_stages=2, kappa=30.0, seed=4, xstar_frac=0.05, value_dtype=dt)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        assert inst.info["lam_max"] == pytest.approx(float(np.abs(ref.A.T @ ref.b).max()), rel=1e-12)
        # FP32 products: step just above the device's own lambda_max by their rounding
        tau = factor * inst.info["lam_max"] * (1.0 if dt == "f64" else 1.0 + 1e-5)
        for fn in (inst.solve_fista, inst.solve_pdncg):
            x, r = fn(tau=tau, tol=1e-12, max_iter=100)
            assert r["status"] == 0 and r["iters"] == 0 and not np.any(x)
        x, r = inst.solve_fista_bt(1e-2, 2.0, tau=tau, tol=1e-12, max_iter=100)
        assert r["status"] == 0 and not np.any(x)
    finally:
        inst.free()


@pytest.mark.parametrize("kappa", [1e4, 1e6])
def test_pdncg_compensated_gradient_at_large_kappa(ctx, kappa):
    """accum = 1: pdNCG's gradient products (r = b - A x, A^T r) in float-float, the PCG in FP32.
    The C3 recipe (16 per column, x* 2%) at n = 2^14 with FP32 values: at kappa = 1e6 the
    residual's entries reach 1 / sigma_min = 1e6 and FP32 sums of A^T r lose the gradient.  The
    oracle re-certifies the device's x on the stored problem, and its own pdNCG on that problem
    bounds the Newton count (the two part only through rounding in the line search)."""
    params = W.params(m=2 ** 15, n=2 ** 14, seed=0, kappa=kappa, xstar_frac=0.02, right_stages=4,
                      left_stages=1, value_dtype="f32")
    ref = oracle_instance(params)
    A = stored_values(ref.A, "f32")
    b = ref.b.astype(np.float32).astype(np.float64)
    inst = ctx.generate(params)
    try:
        x, r = inst.solve_pdncg(tau=1.0, tol=1e-6, max_iter=200, accum=1)
        assert r["status"] == 0 and r["rel_gap"] <= 1e-6
        P, D, gap, rel = solvers.certificate(A, b, 1.0, x)
        assert rel <= 2e-5
        o = solvers.pdncg(A, b, 1.0, 1e-6)
        assert o["status"] == 0
        assert r["iters"] <= 2 * o["iters"] + 3, (r["iters"], o["iters"])
    finally:
        inst.free()
