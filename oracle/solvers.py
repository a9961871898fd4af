"""Objective, duality-gap certificate, FISTA and pdNCG (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Objective f_tau(x) = tau ||x||_1 + 1/2 ||A x - b||^2, Eq. (prob1).
* Certificate.  The paper stops its comparison solvers at pdNCG's objective and gives no
  gap; this project certifies with the Lagrange dual of Eq. (prob1),
  max_theta b^T theta - 1/2 ||theta||^2 s.t. ||A^T theta||_inf <= tau, at the feasible
  point theta = s r with r = b - A y and s = min(1, tau / ||A^T r||_inf).  By weak
  duality P(x) - D(theta) >= P(x) - P(x*) for any x and any such y; at the optimum with
  y = x = x* it is zero (Sec. 3.1: A^T e = tau g).  rel_gap = gap / max(P, tiny).
* FISTA (Sec. 8.1; Beck & Teboulle): x_k = S_{tau/L}(y_k - A^T(A y_k - b) / L),
  t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, y_{k+1} = x_k + ((t_k - 1)/t_{k+1})(x_k - x_{k-1}),
  y_1 = x_0, t_1 = 1, L >= lambda_max(A^T A) (fixed, not TFOCS' dynamic L).
  Iteration k evaluates A x_{k-1} (which certifies x_{k-1} through P(x_{k-1})) and
  A^T r at y_k (which supplies a dual point); x_{k-1} is returned as soon as
  P(x_{k-1}) - max_{j<=k} D(y_j) is within the tolerance.  A y_k is formed by linearity
  from A x_{k-1} and A x_{k-2}.
* FISTA with backtracking on L (Beck & Teboulle, Sec. 4 of their paper; the paper's TFOCS
  runs use a dynamic L): see fista_bt.
* pdNCG (Sec. 8.1 and 8.3): Newton-CG on f^mu_tau(x) = tau psi_mu(x) + 1/2||Ax - b||^2 with
  the pseudo-Huber psi_mu of Eq. (pseudoHuber), mu = 1e-5.  The Newton system of the model
  (bd4) is solved by PCG with the inverse diagonal of its matrix as preconditioner, stopped
  at relative residual 0.1; then a backtracking (halving) Armijo line search with at most
  50 trials, accepting the last trial when none passes.
  Readings (the paper defers the details of its primal-dual method to its reference):
  - primal-dual direction: Newton's method on the pair of conditions
    tau g + A^T(Ax - b) = 0 and g_i sqrt(mu^2 + x_i^2) = x_i, linearised in (x, g) and with
    dx eliminated for, gives [A^T A + tau diag((1 - g_i x_i / w_i) / w_i)] dx = -grad f^mu(x)
    (w_i = sqrt(mu^2 + x_i^2)); with g = x / w this is exactly the Newton system of (bd4).
    The dual estimate entering each Newton step is the first condition solved for g at the
    current x and projected onto [-1, 1]^n, g = clip(A^T r / tau) with r = b - A x.  The first
    condition is linear, so after a full step with dx solved exactly this is the Newton update
    g + dg, dg = (x + (1 - g x / w) dx) / w - g (pd_dual_step); after a damped or inexact step
    it keeps g consistent with the accepted x instead of with the undamped point.  (Measured
    on the C2 recipe, n = 2^18 / 2^20: 17 / 20 Newton steps and 123 / 150 PCG iterations,
    against 31 / 51 and 746 / 4715 with the full-step update, whose dual estimate kept the wrong
    sign on coordinates the line search had not moved across zero.  The purely primal system
    stalls on these instances: its curvature mu^2 / w^3 spans ~15 decades and steps shrink to
    ~1e-4.)
  - Armijo constant 1e-4; psi_mu evaluated as x^2 / (sqrt(mu^2 + x^2) + mu) and the line
    search through per-coordinate differences, the same quantities without cancellation.
  - PCG's relative residual is measured in the norm of the preconditioner,
    sqrt(res^T M^{-1} res) <= 0.1 sqrt(grad^T M^{-1} grad).  In the 2-norm the residual is
    dominated by the coordinates at zero (curvature ~ tau/mu) that the diagonal
    preconditioner resolves in one step, so PCG stopped before solving the support block.
  - mu-continuation: mu starts at mu_start (1, the scale of x*) and is divided by 10 after
    every full Newton step (alpha = 1) until it reaches the paper's mu; the smoothed minimiser
    then still carries an O(mu) bias in the l1 certificate (about 0.2 tau mu per zero of
    x*), so below mu a full step that fails to halve the gap divides mu by 10 again, down
    to mu_min.  With mu fixed at 1e-5 from x = 0 the iteration stalls on instances with
    n >= 2^16 (measured), because coordinates leave zero only by grad / (tau / mu) per step.
"""

import math

import numpy as np

TINY = 1e-300

STATUS_OK = 0
STATUS_NOCONV = 5      # the library's L1LS_ENOCONV
STATUS_NUMERIC = 6     # L1LS_ENUMERIC


def objective(A, b, tau, x):
    """f_tau(x), Eq. (prob1)."""
    r = A @ x - b
    return tau * np.abs(x).sum() + 0.5 * float(r @ r)


def dual_value(b, r, atr, tau):
    """Lagrange dual of Eq. (prob1), D(theta) = b^T theta - 1/2 ||theta||^2 over
    ||A^T theta||_inf <= tau, at theta = s r, s = min(1, tau/||A^T r||_inf).  The paper states
    no stopping test; this certificate is the reading used on both sides."""
    amax = float(np.abs(atr).max()) if len(atr) else 0.0
    s = 1.0 if amax <= tau else tau / amax
    return s * float(b @ r) - 0.5 * s * s * float(r @ r)


def certificate(A, b, tau, x):
    """(P, D, gap, rel_gap) at x with the dual point built from r = b - A x; zero gap exactly
    at the minimisers of Eq. (prob1), whose optimality condition is Eq. (bd7)."""
    r = b - A @ x
    atr = A.T @ r
    P = tau * np.abs(x).sum() + 0.5 * float(r @ r)
    D = dual_value(b, r, atr, tau)
    gap = P - D
    return P, D, gap, gap / max(abs(P), TINY)


def soft_threshold(v, t):
    """Shrinkage S_t(v) = sign(v) max(|v| - t, 0), the exact minimiser of the separable
    model (bd1) with H = L I (Sec. 2)."""
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def fista(A, b, tau, L, tol, max_iter, x0=None, restart=False, f_target=-math.inf):
    """FISTA with the certificate above.  Returns dict(x, x_next, iters, products, P, D, gap,
    rel_gap, status, restarts).  It also stops (status OK) at the first certified x_{k-1} with
    P(x_{k-1}) <= f_target: the paper ends its comparison solvers once their objective is
    below pdNCG's (Sec. 8.3).

    restart=True adds the gradient restart of O'Donoghue & Candes (2015, "Adaptive restart for
    accelerated gradient schemes"), not used by the paper: when (y_k - x_k)^T (x_k - x_{k-1}) > 0
    the momentum is dropped (t <- 1, so y_{k+1} = x_k)."""
    n = A.shape[1]
    x_cur = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)   # x_{k-1}
    x_old = x_cur.copy()                                                              # x_{k-2}
    Ax_old = A @ x_old
    products = 1
    t = 1.0
    beta = 0.0
    best_D = -math.inf
    k = 1
    restarts = 0
    while True:
        u = A @ x_cur                                   # A x_{k-1}
        P = tau * np.abs(x_cur).sum() + 0.5 * float((u - b) @ (u - b))
        y = x_cur + beta * (x_cur - x_old)              # y_k
        Ay = u + beta * (u - Ax_old)
        r = b - Ay
        g = A.T @ r                                     # -grad of the smooth part at y_k
        products += 2
        best_D = max(best_D, dual_value(b, r, g, tau))
        gap = P - best_D
        rel = gap / max(abs(P), TINY)
        x_new = soft_threshold(y + g / L, tau / L)
        if rel <= tol or P <= f_target or k - 1 >= max_iter:
            # x_next: the prox-gradient step from y_k, one past the certified iterate
            ok = rel <= tol or P <= f_target
            return dict(x=x_cur, x_next=x_new, iters=k - 1, products=products, P=P, D=best_D, gap=gap,
                        rel_gap=rel, status=STATUS_OK if ok else STATUS_NOCONV, restarts=restarts)
        if restart and float((y - x_new) @ (x_new - x_cur)) > 0.0:
            t = 1.0
            beta = 0.0
            restarts += 1
        else:
            t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            beta = (t - 1.0) / t_new
            t = t_new
        x_old, x_cur = x_cur, x_new
        Ax_old = u
        k += 1


def sufficient_decrease(Ad, d, L):
    """The backtracking test of FISTA with backtracking (Beck & Teboulle 2009) for the quadratic smooth part
    h(x) = 1/2 ||A x - b||^2: h(x) <= h(y) + grad h(y)^T d + L/2 ||d||^2 with d = x - y.  Since
    h(y + d) - h(y) - grad h(y)^T d = 1/2 ||A d||^2 exactly, the test is ||A d||^2 <= L ||d||^2;
    evaluated in this form it has no cancellation (the difference of the two objective values
    near the optimum is below their rounding)."""
    return float(Ad @ Ad) <= L * float(d @ d)


def fista_bt(A, b, tau, L0, eta, tol, max_iter, x0=None, max_trials=60, trace=False, f_target=-math.inf):
    """FISTA with backtracking on L (Beck & Teboulle 2009, "A fast iterative shrinkage-
    thresholding algorithm for linear inverse problems", Sec. 4): the step constant of
    iteration k is the smallest L = eta^i L_{k-1} (i >= 0) for which the prox-gradient point
    x = S_{tau/L}(y_k + g/L), g = A^T (b - A y_k), passes sufficient_decrease with
    d = x - y_k and A d = A x - A y_k.  L never decreases.  The momentum is FISTA's.
    Iteration k certifies its own output x_k by P(x_k) - max_{j<=k} D(theta(y_j)).  A y_k is
    formed by linearity from A x_{k-1} and A x_{k-2}.

    Returns dict(x, iters, products, P, D, gap, rel_gap, status, L, backtracks) and, with
    trace, hist = [(P(x_k), L_k)] per iteration.  f_target as for fista."""
    n = A.shape[1]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)   # x_{k-1}
    x_prev = x.copy()                                                             # x_{k-2}
    Ax = A @ x
    Ax_prev = Ax.copy()
    products = 1
    t = 1.0
    beta = 0.0
    L = float(L0)
    best_D = -math.inf
    backtracks = 0
    hist = []
    k = 1
    while True:
        y = x + beta * (x - x_prev)
        Ay = Ax + beta * (Ax - Ax_prev)
        r = b - Ay
        g = A.T @ r
        products += 1
        best_D = max(best_D, dual_value(b, r, g, tau))
        trials = 0
        while True:
            x_new = soft_threshold(y + g / L, tau / L)
            Ax_new = A @ x_new
            products += 1
            if sufficient_decrease(Ax_new - Ay, x_new - y, L):
                break
            trials += 1
            if trials > max_trials:
                return dict(x=x, iters=k - 1, products=products, P=math.nan, D=best_D, gap=math.nan,
                            rel_gap=math.nan, status=STATUS_NUMERIC, L=L, backtracks=backtracks, hist=hist)
            L *= eta
            backtracks += 1
        res_new = Ax_new - b
        P = tau * float(np.abs(x_new).sum()) + 0.5 * float(res_new @ res_new)
        gap = P - best_D
        rel = gap / max(abs(P), TINY)
        hist.append((P, L))
        if rel <= tol or P <= f_target or k >= max_iter:
            ok = rel <= tol or P <= f_target
            out = dict(x=x_new, iters=k, products=products, P=P, D=best_D, gap=gap, rel_gap=rel,
                       status=STATUS_OK if ok else STATUS_NOCONV, L=L, backtracks=backtracks)
            if trace:
                out["hist"] = hist
            return out
        t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_new
        t = t_new
        x_prev, x = x, x_new
        Ax_prev, Ax = Ax, Ax_new
        k += 1


def psi_terms(x, mu):
    """Per-coordinate sqrt(mu^2 + x^2) - mu of Eq. (pseudoHuber), cancellation-free."""
    return x * x / (np.sqrt(mu * mu + x * x) + mu)


def psi_diff_terms(x, d, alpha, mu):
    """Per-coordinate psi(x + alpha d) - psi(x) of Eq. (pseudoHuber), cancellation-free."""
    xt = x + alpha * d
    return (alpha * d) * (x + xt) / (np.sqrt(mu * mu + xt * xt) + np.sqrt(mu * mu + x * x))


def pd_curvature(x, gd, mu, tau):
    """Diagonal of the primal-dual Newton matrix, tau (1 - g_i x_i / w_i) / w_i with
    w_i = sqrt(mu^2 + x_i^2): the Newton system of the conditions tau g + A^T(Ax - b) = 0 and
    g_i w_i = x_i (pdNCG, Sec. 8.1) after eliminating dg.  Returns (h, w)."""
    w = np.sqrt(mu * mu + x * x)
    return tau * (1.0 - gd * x / w) / w, w


def pd_dual_step(x, gd, d, mu):
    """Newton step of the dual estimate g for the primal step d, from the linearised
    condition g_i w_i = x_i: dg = (x + (1 - g x / w) d) / w - g."""
    w = np.sqrt(mu * mu + x * x)
    return (x + (1.0 - gd * x / w) * d) / w - gd


def pdncg(A, b, tau, tol, max_newton=200, mu0=1e-5, mu_min=1e-14, pcg_rtol=0.1, pcg_max=1000,
          ls_max=50, armijo=1e-4, stall=0.5, x0=None, mu_start=1.0):
    """Primal-dual Newton-CG (pdNCG, Sec. 8.1) on f_tau^mu of Eq. (prob2) with the pseudo-Huber
    smoothing of Eq. (pseudoHuber), stopped by the certificate above.

    Returns dict(x, iters, products, cg_iters, ls_trials, P, D, gap, rel_gap, mu, status).
    """
    m, n = A.shape
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    mu = max(mu_start, mu0)
    colnorm2 = np.asarray(A.multiply(A).sum(axis=0)).ravel()       # diag(A^T A)
    products = 0
    cg_total = 0
    ls_total = 0
    it = 0
    prev_gap = math.inf
    prev_full = False
    while True:
        Ax = A @ x
        r = b - Ax
        atr = A.T @ r
        products += 2
        P = tau * np.abs(x).sum() + 0.5 * float(r @ r)
        D = dual_value(b, r, atr, tau)
        gap = P - D
        rel = gap / max(abs(P), TINY)
        if rel <= tol or it >= max_newton:
            return dict(x=x, iters=it, products=products, cg_iters=cg_total, ls_trials=ls_total,
                        P=P, D=D, gap=gap, rel_gap=rel, mu=mu,
                        status=STATUS_OK if rel <= tol else STATUS_NOCONV)
        if prev_full and mu > mu0:
            mu = max(mu * 0.1, mu0)
        elif prev_full and gap > stall * prev_gap:
            mu = max(mu * 0.1, mu_min)
        prev_gap = gap
        gd = np.clip(atr / tau, -1.0, 1.0)                          # dual estimate g at x
        hdiag, w = pd_curvature(x, gd, mu, tau)                     # primal-dual psi curvature
        grad = tau * x / w - atr                                    # grad f^mu
        minv = 1.0 / (hdiag + colnorm2)
        # PCG on (diag(hdiag) + A^T A) d = -grad from d = 0.
        d = np.zeros(n)
        res = -grad
        z = minv * res
        p = z.copy()
        rz = float(res @ z)
        rz0 = rz
        for _ in range(pcg_max):
            Ap = A @ p
            Hp = hdiag * p + A.T @ Ap
            products += 2
            cg_total += 1
            pHp = float(p @ Hp)
            if pHp <= 0.0:
                break
            alpha = rz / pHp
            d += alpha * p
            res -= alpha * Hp
            z = minv * res
            rz_new = float(res @ z)
            if math.sqrt(rz_new) <= pcg_rtol * math.sqrt(rz0):
                break
            p = z + (rz_new / rz) * p
            rz = rz_new
        # Backtracking Armijo line search on f^mu.
        Ad = A @ d
        products += 1
        slope = float(grad @ d)
        rAd = float(r @ Ad)
        AdAd = float(Ad @ Ad)
        step = 1.0
        for trial in range(ls_max):
            ls_total += 1
            df = tau * float(psi_diff_terms(x, d, step, mu).sum()) - step * rAd + 0.5 * step * step * AdAd
            if df <= armijo * step * slope or trial == ls_max - 1:
                break                                               # the last trial is accepted
            step *= 0.5
        x = x + step * d
        prev_full = step == 1.0
        it += 1
