"""Pins of the oracle's objective, certificate, FISTA and pdNCG.

Closed forms (shrinkage for orthogonal A, Sec. 2), the generator's known optimum (IGen,
Sec. 3.1; unique because A has rank n), weak duality, and brute-force support
enumeration (Eq. bd9) for tiny n.
"""

import math

import numpy as np
import pytest

from oracle import solvers
from oracle.brute import brute_force
from oracle.generator import GenParams, generate


def _small(seed=0, kappa=20.0, tau=1.0, m=16, n=8, right=1, frac=0.25):
    return generate(GenParams(m=m, n=n, seed=seed, kappa=kappa, tau=tau, right_stages=right,
                              xstar_frac=frac))


def test_soft_threshold_definition():
    v = np.array([-3.0, -0.5, 0.0, 0.2, 2.5])
    assert np.array_equal(solvers.soft_threshold(v, 1.0), np.array([-2.0, -0.0, 0.0, 0.0, 1.5]))


@pytest.mark.parametrize("tau", [0.3, 1.0, 4.0])
def test_orthogonal_A_closed_form(tau):
    """A^T A = I: the minimiser is S_tau(A^T b); FISTA with L = 1 reaches it in one step."""
    inst = generate(GenParams(m=64, n=32, seed=1, kappa=1.0, right_stages=2, tau=1.0, xstar_frac=0.2))
    A, b = inst.A, inst.b
    x_cf = solvers.soft_threshold(A.T @ b, tau)
    r = solvers.fista(A, b, tau, 1.0, 1e-12, 10)
    assert r["iters"] == 1
    assert np.allclose(r["x"], x_cf, atol=1e-13)
    q = solvers.pdncg(A, b, tau, 1e-10)
    assert q["status"] == 0
    assert np.allclose(q["x"], x_cf, atol=1e-5)


def test_certificate_zero_at_generated_optimum_and_weak_duality():
    inst = generate(GenParams(m=256, n=128, seed=2, kappa=100.0, right_stages=2))
    A, b, tau = inst.A, inst.b, 1.0
    assert abs(solvers.certificate(A, b, tau, inst.xstar)[3]) < 1e-13
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = inst.xstar + rng.standard_normal(128)
        y = rng.standard_normal(128)
        r = b - A @ y
        D = solvers.dual_value(b, r, A.T @ r, tau)
        assert solvers.objective(A, b, tau, x) >= D
        assert D <= inst.f_star * (1 + 1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fista_and_pdncg_reach_the_generated_optimum(seed):
    inst = generate(GenParams(m=512, n=256, seed=seed, kappa=100.0, right_stages=2, xstar_frac=0.05))
    A, b = inst.A, inst.b
    smin = inst.sigma.min()
    for res in (solvers.fista(A, b, 1.0, inst.lipschitz, 1e-8, 100000), solvers.pdncg(A, b, 1.0, 1e-8)):
        assert res["status"] == 0
        assert res["rel_gap"] <= 1e-8
        # strong convexity: ||x - x*||^2 <= 2 gap / sigma_min^2
        err2 = float(np.sum((res["x"] - inst.xstar) ** 2))
        assert err2 <= 2.0 * res["gap"] / smin ** 2 + 1e-20
        assert res["P"] >= inst.f_star * (1 - 1e-14)


@pytest.mark.parametrize("tau_factor", [1.0, 0.4, 2.5])
@pytest.mark.parametrize("right", [1, 2])
def test_brute_force_agrees(tau_factor, right):
    inst = _small(seed=3, right=right, tau=1.0)
    A, b = inst.A, inst.b
    tau = tau_factor
    xb, fb = brute_force(A, b, tau)
    if tau_factor == 1.0:
        assert np.allclose(xb, inst.xstar, atol=1e-10)
    f = solvers.fista(A, b, tau, inst.lipschitz, 1e-12, 200000)
    q = solvers.pdncg(A, b, tau, 1e-12)
    for res in (f, q):
        assert res["status"] == 0
        assert np.allclose(res["x"], xb, atol=1e-4)
        assert math.isclose(res["P"], fb, rel_tol=1e-11)


def test_fista_warm_start_at_optimum_needs_no_iteration():
    inst = _small(seed=4)
    r = solvers.fista(inst.A, inst.b, 1.0, inst.lipschitz, 1e-12, 100, x0=inst.xstar)
    assert r["iters"] == 0


def test_fista_is_beck_teboulle_on_a_tiny_case():
    """Three iterations written out by hand from the FISTA recursion."""
    inst = _small(seed=5, kappa=5.0)
    A, b, L, tau = inst.A.toarray(), inst.b, inst.lipschitz, 0.6
    x_prev = np.zeros(8)
    y = x_prev.copy()
    t = 1.0
    for _ in range(3):
        x = solvers.soft_threshold(y - A.T @ (A @ y - b) / L, tau / L)
        t_new = (1 + math.sqrt(1 + 4 * t * t)) / 2
        y = x + ((t - 1) / t_new) * (x - x_prev)
        x_prev, t = x, t_new
    r = solvers.fista(inst.A, b, tau, L, 0.0, 3)
    assert r["iters"] == 3
    assert np.allclose(r["x"], x_prev, atol=1e-14)


def test_pdncg_newton_count_is_small_on_c1_shape():
    """The paper reports at most 30 pdNCG iterations on its Sec. 8.4 instances."""
    inst = generate(GenParams(m=2048, n=1024, seed=0, kappa=100.0, xstar_frac=0.05))
    r = solvers.pdncg(inst.A, inst.b, 1.0, 1e-8)
    assert r["status"] == 0 and r["iters"] <= 30


def test_planted_dual_scaling_error_is_caught(monkeypatch):
    """Dropping the scaling s of the dual point breaks weak duality at a random point."""
    inst = generate(GenParams(m=64, n=32, seed=1, kappa=10.0))
    A, b = inst.A, inst.b

    def bad_dual(b_, r, atr, tau):
        return float(b_ @ r) - 0.5 * float(r @ r)

    monkeypatch.setattr(solvers, "dual_value", bad_dual)
    y = np.zeros(32)
    r = b - A @ y
    assert solvers.dual_value(b, r, A.T @ r, 1.0) > inst.f_star


def test_fista_restart_recursion_written_out():
    """The gradient restart (O'Donoghue & Candes 2015) written out from its rule: after the
    prox step from y, if (y - x_new)^T (x_new - x) > 0 the momentum is dropped (t = 1)."""
    inst = _small(seed=6, kappa=100.0, m=24, n=12, right=2)
    A, b, L, tau = inst.A.toarray(), inst.b, inst.lipschitz, 0.3
    x, x_prev, t, beta, nres = np.zeros(12), np.zeros(12), 1.0, 0.0, 0
    for _ in range(1000):
        y = x + beta * (x - x_prev)
        xn = solvers.soft_threshold(y - A.T @ (A @ y - b) / L, tau / L)
        if (y - xn) @ (xn - x) > 0:
            t, beta, nres = 1.0, 0.0, nres + 1
        else:
            t_new = (1 + math.sqrt(1 + 4 * t * t)) / 2
            beta, t = (t - 1) / t_new, t_new
        x_prev, x = x, xn
    r = solvers.fista(inst.A, b, tau, L, 0.0, 1000, restart=True)
    assert nres >= 2 and r["restarts"] == nres
    assert np.allclose(r["x"], x, atol=1e-12)


@pytest.mark.parametrize("tau_factor", [1.0, 0.4])
def test_fista_restart_reaches_brute_force_optimum(tau_factor):
    inst = _small(seed=7, right=2, kappa=300.0)
    xb, fb = brute_force(inst.A, inst.b, tau_factor)
    r = solvers.fista(inst.A, inst.b, tau_factor, inst.lipschitz, 1e-12, 200000, restart=True)
    assert r["status"] == 0
    assert np.allclose(r["x"], xb, atol=1e-4)
    assert math.isclose(r["P"], fb, rel_tol=1e-11)


def test_fista_next_iterate_is_one_prox_step_past_the_certified_one():
    """x_next (the warm start of the next tau of a path) is the prox-gradient step from y_k:
    stopping one iteration later returns it as the certified iterate."""
    inst = generate(GenParams(m=256, n=128, seed=8, kappa=100.0, right_stages=2, xstar_frac=0.05))
    a = solvers.fista(inst.A, inst.b, 0.5, inst.lipschitz, 0.0, 17)
    c = solvers.fista(inst.A, inst.b, 0.5, inst.lipschitz, 0.0, 18)
    assert np.array_equal(a["x_next"], c["x"])


# ---- FISTA with backtracking on L (Beck & Teboulle, Sec. 4 of their paper) -------------------

def test_fista_bt_orthogonal_A_step_constant_in_closed_form():
    """A^T A = I: the sufficient-decrease test at y reads 1/2 ||d||^2 <= L/2 ||d||^2, so from
    L0 = 0.3 with eta = 2 the step constant ends at exactly 0.3 * 4 = 1.2 after two increases
    and never moves again; the iteration then reaches S_tau(A^T b)."""
    inst = generate(GenParams(m=64, n=32, seed=1, kappa=1.0, right_stages=2, tau=1.0, xstar_frac=0.2))
    A, b, tau = inst.A, inst.b, 0.5
    r = solvers.fista_bt(A, b, tau, 0.3, 2.0, 1e-12, 10000)
    assert r["status"] == 0
    assert r["L"] == 0.3 * 2.0 * 2.0 and r["backtracks"] == 2
    assert np.allclose(r["x"], solvers.soft_threshold(A.T @ b, tau), atol=1e-10)


def test_fista_bt_with_an_upper_bound_is_plain_fista():
    """L0 >= lambda_max(A^T A): no increase, and the iterates are FISTA's (pinned above)."""
    inst = _small(seed=5, kappa=5.0)
    for k in (1, 3, 7):
        r = solvers.fista_bt(inst.A, inst.b, 0.6, inst.lipschitz, 2.0, 0.0, k)
        f = solvers.fista(inst.A, inst.b, 0.6, inst.lipschitz, 0.0, k)
        assert r["backtracks"] == 0 and r["iters"] == k
        assert np.allclose(r["x"], f["x"], atol=1e-14)


def test_fista_bt_rate_bound_and_step_constant_bound():
    """Beck & Teboulle's Theorem 4.4: f(x_k) - f* <= 2 eta L_f ||x0 - x*||^2 / (k + 1)^2 for
    every k, and the step constant stays below eta L_f (L_f = sigma_max^2 = 1 here).  x* and f*
    are the generator's (tau = tau_gen)."""
    inst = generate(GenParams(m=256, n=128, seed=9, kappa=100.0, right_stages=2, xstar_frac=0.05))
    eta = 2.0
    r = solvers.fista_bt(inst.A, inst.b, 1.0, 1e-3, eta, 1e-10, 5000, trace=True)
    assert r["status"] == 0 and r["backtracks"] >= 9
    assert 1e-3 < r["L"] <= eta * 1.0
    bound = 2.0 * eta * 1.0 * float(inst.xstar @ inst.xstar)
    for k, (P, _) in enumerate(r["hist"], start=1):
        assert P - inst.f_star <= bound / (k + 1) ** 2 + 1e-9 * abs(inst.f_star)
    assert np.allclose(r["x"], inst.xstar, atol=1e-4)


@pytest.mark.parametrize("tau_factor", [1.0, 0.4, 2.5])
def test_fista_bt_reaches_brute_force_optimum(tau_factor):
    inst = _small(seed=3, right=2, tau=1.0)
    xb, fb = brute_force(inst.A, inst.b, tau_factor)
    r = solvers.fista_bt(inst.A, inst.b, tau_factor, 0.01, 2.0, 1e-12, 200000)
    assert r["status"] == 0
    assert np.allclose(r["x"], xb, atol=1e-4)
    assert math.isclose(r["P"], fb, rel_tol=1e-11)


def test_planted_factor_error_in_the_backtracking_test_is_caught(monkeypatch):
    """A test that drops the factor 1/2 of the model's quadratic term (||A d||^2 <= 2 L ||d||^2)
    accepts L = 0.6 on the orthogonal instance, and the closed form above catches it."""
    inst = generate(GenParams(m=64, n=32, seed=1, kappa=1.0, right_stages=2, tau=1.0, xstar_frac=0.2))
    monkeypatch.setattr(solvers, "sufficient_decrease", lambda Ad, d, L: float(Ad @ Ad) <= 2.0 * L * float(d @ d))
    with np.errstate(all="ignore"):   # the planted test lets the iteration diverge
        r = solvers.fista_bt(inst.A, inst.b, 0.5, 0.3, 2.0, 1e-12, 10000)
    assert r["L"] != 0.3 * 2.0 * 2.0


def test_objective_target_stops_at_the_first_iterate_below_it():
    """f_target (the paper's rule for ending its comparison solvers, Sec. 8.3): the returned
    iterate is the first certified one with P <= f_target, against a written-out trace."""
    inst = generate(GenParams(m=256, n=128, seed=9, kappa=100.0, right_stages=2, xstar_frac=0.05))
    A, b = inst.A, inst.b
    trace = [solvers.fista(A, b, 1.0, inst.lipschitz, 0.0, k)["P"] for k in range(0, 40)]
    target = inst.f_star + 1e-2 * (trace[0] - inst.f_star)
    first = next(k for k, P in enumerate(trace) if P <= target)
    assert first >= 3
    r = solvers.fista(A, b, 1.0, inst.lipschitz, 0.0, 100000, f_target=target)
    assert r["status"] == 0 and r["iters"] == first and r["P"] <= target
    q = solvers.fista_bt(A, b, 1.0, inst.lipschitz, 2.0, 0.0, 100000, f_target=target)
    assert q["status"] == 0 and q["P"] <= target and q["iters"] == first   # no increase of L: FISTA's iterates


def test_pseudo_huber_terms_against_high_precision():
    """Eq. (pseudoHuber) term by term, sqrt(mu^2 + x^2) - mu and its difference along a step,
    against 60-digit arithmetic: the oracle's cancellation-free forms keep a few ulps of
    relative error down to x ~ 1e-12 mu and up to x ~ 1e12 mu (the plain formula loses all
    digits at the small end)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    rng = np.random.default_rng(3)
    for mu in (1e-5, 1e-2, 1.0):
        x = np.concatenate([[0.0], mu * 10.0 ** rng.uniform(-12, 12, 64) * rng.choice([-1.0, 1.0], 64)])
        d = rng.standard_normal(x.size) * np.maximum(np.abs(x), mu)
        alpha = 0.37
        got = solvers.psi_terms(x, mu)
        got_diff = solvers.psi_diff_terms(x, d, alpha, mu)
        for i in range(x.size):
            ref = mpmath.sqrt(mpmath.mpf(mu) ** 2 + mpmath.mpf(x[i]) ** 2) - mu
            assert abs(got[i] - float(ref)) <= 4e-16 * float(ref) + 1e-300, (mu, x[i])
            xt = mpmath.mpf(x[i]) + mpmath.mpf(alpha * d[i])  # the oracle forms alpha*d in FP64 first
            ref_d = (mpmath.sqrt(mpmath.mpf(mu) ** 2 + xt ** 2) - mpmath.sqrt(mpmath.mpf(mu) ** 2 + mpmath.mpf(x[i]) ** 2))
            scale = abs(float(ref_d)) + 1e-300
            # x + alpha*d is rounded once in FP64 before the quotient: an error of about one ulp
            # of |x + alpha d| times the slope |xt| / sqrt(mu^2 + xt^2) <= 1
            tol = 8e-16 * scale + 2.3e-16 * abs(x[i] + alpha * d[i])
            assert abs(got_diff[i] - float(ref_d)) <= tol, (mu, x[i], d[i])


def test_pseudo_huber_slope_and_curvature():
    """The derivatives pdNCG builds on, checked by differences of the oracle's terms:
    psi' = x / sqrt(mu^2 + x^2) and psi'' = mu^2 / (mu^2 + x^2)^{3/2} (Eq. (pseudoHuber))."""
    mu, h = 0.5, 1e-4
    x = np.array([-3.0, -0.4, 0.0, 0.1, 2.0])
    w = np.sqrt(mu * mu + x * x)
    slope = (solvers.psi_terms(x + h, mu) - solvers.psi_terms(x - h, mu)) / (2 * h)
    assert np.allclose(slope, x / w, rtol=1e-7, atol=1e-10)
    curv = (solvers.psi_diff_terms(x, np.ones_like(x), h, mu)
            + solvers.psi_diff_terms(x, -np.ones_like(x), h, mu)) / (h * h)
    assert np.allclose(curv, mu * mu / w ** 3, rtol=1e-6)


@pytest.mark.parametrize("tau", [0.05, 1.4, 1.9, 2.5])
def test_brute_force_on_orthonormal_columns_is_shrinkage(tau):
    """A with orthonormal columns (a random Q of a QR factorisation, m = 9, n = 6): the unique
    minimiser of Eq. (prob1) is the soft threshold S_tau(A^T b), independent of the generator."""
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((9, 6)))
    b = rng.standard_normal(9) * 1.5
    xb, fb = brute_force(Q, b, tau)
    xs = solvers.soft_threshold(Q.T @ b, tau)
    assert np.allclose(xb, xs, atol=1e-12)
    assert math.isclose(fb, solvers.objective(Q, b, tau, xs), rel_tol=1e-12)


def test_pd_curvature_at_g_equal_x_over_w_is_the_hessian_of_bd4():
    """At g = x / w the primal-dual matrix diag(h) + A^T A equals the Hessian of the smoothed
    objective of Eq. (prob2), tau psi_mu'' + A^T A (the model bd4): psi_mu'' is taken here by
    symbolic differentiation of Eq. (pseudoHuber), independently of the oracle's formula."""
    sympy = pytest.importorskip("sympy")
    xs, ms = sympy.symbols("x mu", real=True)
    d2 = sympy.lambdify((xs, ms), sympy.diff(sympy.sqrt(ms ** 2 + xs ** 2) - ms, xs, 2), "mpmath")
    rng = np.random.default_rng(5)
    for mu in (1e-5, 1e-2, 1.0):
        x = mu * 10.0 ** rng.uniform(-3, 6, 40) * rng.choice([-1.0, 1.0], 40)
        w = np.sqrt(mu * mu + x * x)
        for tau in (0.3, 1.0):
            h, w2 = solvers.pd_curvature(x, x / w, mu, tau)
            assert np.array_equal(w2, w)
            ref = np.array([tau * float(d2(xi, mu)) for xi in x])
            # 1 - g x / w cancels when |x| >> mu: a few ulps of 1 relative to mu^2 / w^2
            tol = 1e-13 * ref + 8 * 2.3e-16 * tau / w
            assert np.all(np.abs(h - ref) <= tol), mu


def _pd_newton_step(A, b, x, g, mu, tau, dual_step=None):
    h, w = solvers.pd_curvature(x, g, mu, tau)
    grad = tau * x / w + A.T @ (A @ x - b)
    dx = np.linalg.solve(A.T @ A + np.diag(h), -grad)
    dg = (dual_step or solvers.pd_dual_step)(x, g, dx, mu)
    return dx, dg


def _pd_conditions(A, b, x, g, mu, tau):
    """The two conditions pdNCG's Newton step linearises: tau g + A^T (A x - b) = 0 and
    g_i sqrt(mu^2 + x_i^2) - x_i = 0 (complex arguments allowed)."""
    return tau * g + A.T @ (A @ x - b), g * np.sqrt(mu * mu + x * x) - x


def _check_pd_step_is_newton(A, b, x, g, mu, tau, dx, dg):
    # the first condition is linear in (x, g): a Newton step zeroes it exactly
    F1, _ = _pd_conditions(A, b, x + dx, g + dg, mu, tau)
    scale = tau + np.abs(A.T) @ (np.abs(A) @ (np.abs(x) + np.abs(dx)) + np.abs(b))
    ok1 = np.all(np.abs(F1) <= 1e-12 * scale)
    # the second: F2 + J2 (dx, dg) = 0, with J2 (dx, dg) the directional derivative taken by
    # the complex step (exact to rounding for an analytic function)
    hstep = 1e-30
    _, F2 = _pd_conditions(A, b, x, g, mu, tau)
    _, F2c = _pd_conditions(A, b, x + 1j * hstep * dx, g + 1j * hstep * dg, mu, tau)
    J2 = np.imag(F2c) / hstep
    w = np.sqrt(mu * mu + x * x)
    scale2 = np.abs(x) + w * (np.abs(g) + np.abs(dg)) + np.abs(dx)
    ok2 = np.all(np.abs(F2 + J2) <= 1e-12 * scale2)
    return ok1 and ok2


def test_pd_direction_and_dual_step_are_a_newton_step():
    """With dx from the oracle's primal-dual matrix (solved exactly) and dg from its dual step,
    (dx, dg) is Newton's step on the pair of conditions of pdNCG's primal-dual formulation at
    any (x, g), not only at g = x / w: the linear condition holds at (x + dx, g + dg) and the
    other's linearisation, taken by the complex step, vanishes."""
    rng = np.random.default_rng(9)
    for trial in range(6):
        A = rng.standard_normal((14, 9))
        b = rng.standard_normal(14)
        x = rng.standard_normal(9) * 10.0 ** rng.uniform(-3, 1, 9)
        g = rng.uniform(-1.0, 1.0, 9)
        for mu, tau in ((1e-2, 0.7), (1.0, 2.0)):
            dx, dg = _pd_newton_step(A, b, x, g, mu, tau)
            assert _check_pd_step_is_newton(A, b, x, g, mu, tau, dx, dg), (trial, mu)


def test_planted_sign_error_in_the_dual_step_is_caught():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((14, 9))
    b = rng.standard_normal(14)
    x = rng.standard_normal(9)
    g = rng.uniform(-1.0, 1.0, 9)
    wrong = lambda x, g, d, mu: (x - (1.0 - g * x / np.sqrt(mu * mu + x * x)) * d) / np.sqrt(mu * mu + x * x) - g
    dx, dg = _pd_newton_step(A, b, x, g, 0.1, 1.0, dual_step=wrong)
    assert not _check_pd_step_is_newton(A, b, x, g, 0.1, 1.0, dx, dg)


def test_residual_dual_equals_the_newton_update_after_an_exact_full_step():
    """The reading behind pdNCG's dual estimate: the first condition tau g + A^T(Ax - b) = 0 is
    linear, so Newton's g + dg after an exact full step is A^T r(x + dx) / tau, the dual the
    oracle recomputes from the residual at the accepted point."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((16, 10))
    b = rng.standard_normal(16)
    x = rng.standard_normal(10)
    g = rng.uniform(-1.0, 1.0, 10)
    for mu, tau in ((1e-3, 0.5), (0.3, 1.5)):
        dx, dg = _pd_newton_step(A, b, x, g, mu, tau)
        xn = x + dx
        assert np.allclose(g + dg, A.T @ (b - A @ xn) / tau, rtol=1e-10, atol=1e-10)
