"""Pins of the oracle's instance generator against what the paper fixes.

Sec. 4 (Givens layout, Eq. bd8, known SVD, cheap (A^T A)^{-1}), Sec. 4.2 (printed nonzero
counts), Procedure IGen / IGen2 (optimality by construction, Eqs. bd7 and bd10),
Procedure OsGen, Algorithms MvPA / MvPAt.
"""

import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import generator as gen
from oracle.generator import GenParams, generate
from oracle.operators import mvpa, mvpat
from oracle.solvers import certificate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_spy():
    rows = []
    with open(os.path.join(GOLDEN, "spy_counts_sec4_2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            stages, name, nnz_a, nnz_ata = line.split()
            rows.append((int(stages), name, int(nnz_a), int(nnz_ata)))
    return rows


def test_givens_layout_matches_sec4():
    c, s = math.cos(0.3), math.sin(0.3)
    G = gen.givens(5, 1, 3, c, s)
    assert G[1, 1] == c and G[3, 3] == c and G[1, 3] == -s and G[3, 1] == s
    assert np.allclose(G @ G.T, np.eye(5), atol=1e-15)
    # G rotates the plane (i, j) by theta: e_i -> (c, s) in that plane.
    v = G @ np.eye(5)[1]
    assert np.isclose(v[1], c) and np.isclose(v[3], s)


@pytest.mark.parametrize("first", [0, 1])
@pytest.mark.parametrize("size", [8, 9])
def test_stage_is_product_of_its_rotations(first, size):
    c, s = math.cos(2 * math.pi / 10), math.sin(2 * math.pi / 10)
    prod = np.eye(size)
    for i in range(first, size - 1, 2):
        prod = prod @ gen.givens(size, i, i + 1, c, s)
    assert np.array_equal(gen.stage_matrix(size, first, c, s).toarray(), prod)


def test_spy_counts_of_AtA_sec4_2():
    """nnz(A^T A) = 16, 38, 56, 62 for G, G2G, GG2G, G2GG2G at n = 8, m = 16 (Sec. 4.2)."""
    for stages, name, _nnz_a, nnz_ata in _golden_spy():
        inst = generate(GenParams(m=16, n=8, seed=3, kappa=10.0, right_stages=stages, left_stages=1,
                                  xstar_frac=0.25))
        A = inst.A.toarray()
        AtA = A.T @ A
        # exact zeros of R Sigma^2 R^T show up as rounding residue; drop it
        assert np.count_nonzero(np.abs(AtA) > 1e-12 * np.abs(AtA).max()) == nnz_ata, name
        pat = (gen._structure(inst.R) @ gen._structure(inst.R).T)
        assert pat.nnz == nnz_ata, name


def test_nnz_A_of_sec4_2_attainable():
    """28 nonzeros (Sec. 4.2, one stage each side) occurs for some permutation P."""
    seen = set()
    for seed in range(200):
        seen.add(generate(GenParams(m=16, n=8, seed=seed, right_stages=1, left_stages=1)).A.nnz)
    assert 28 in seen
    assert max(seen) == 32          # 2 left rows per 2 right entries per column


@pytest.mark.parametrize("n", [8, 16, 64])
def test_nnz_closed_forms(n):
    forms = {1: (2 * n, 2 * n), 2: (4 * n - 4, 6 * n - 10), 3: (6 * n - 8, 10 * n - 24),
             4: (8 * n - 16, 14 * n - 50)}
    c, s = math.cos(0.7), math.sin(0.7)
    for w, (nnz_r, nnz_rrt) in forms.items():
        R = gen._structure(gen.right_factor(n, w, c, s))
        assert R.nnz == nnz_r
        assert (R @ R.T).nnz == nnz_rrt


@pytest.mark.parametrize("right,left", [(1, 1), (2, 1), (4, 1), (3, 0)])
def test_known_svd_and_inverse(right, left):
    p = GenParams(m=24, n=12, seed=5, kappa=50.0, right_stages=right, left_stages=left)
    inst = generate(p)
    A = inst.A.toarray()
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(np.sort(sv), np.sort(inst.sigma), rtol=1e-12)
    R = inst.R.toarray()
    inv = R @ np.diag(1.0 / inst.sigma ** 2) @ R.T       # G (Sigma^T Sigma)^{-1} G^T
    assert np.allclose(inv, np.linalg.inv(A.T @ A), rtol=1e-9, atol=1e-9)


def test_sigma_exactly_logspaced():
    inst = generate(GenParams(m=64, n=32, seed=1, kappa=1e4))
    srt = np.sort(inst.sigma)[::-1]
    assert srt[0] == 1.0
    assert np.allclose(srt, 1e4 ** (-np.arange(32) / 31.0), rtol=1e-14)
    assert math.isclose(srt[-1], 1e-4, rel_tol=1e-14)
    assert inst.lipschitz == 1.0


def test_osgen_support_and_values():
    p = GenParams(m=2048, n=1024, seed=0, xstar_frac=0.05)
    inst = generate(p)
    assert len(inst.support) == 51
    nz = np.flatnonzero(inst.xstar)
    assert np.array_equal(nz, inst.support)
    mags = np.abs(inst.xstar[nz])
    assert mags.min() >= 1.0 and mags.max() <= 10.0
    assert 10 < (inst.xstar > 0).sum() < 41
    g = inst.g
    assert np.array_equal(g[nz], np.sign(inst.xstar[nz]))
    off = np.setdiff1d(np.arange(1024), nz)
    assert np.abs(g[off]).max() <= 1.0 and np.abs(g[off]).min() < 0.1


@pytest.mark.parametrize("kappa", [1e2, 1e4])
@pytest.mark.parametrize("right", [1, 2, 4])
def test_igen_optimality_by_construction(kappa, right):
    """A^T e = tau g (Eq. bd7), hence A^T(A x* - b) in -tau d||x*||_1 and the gap is 0."""
    p = GenParams(m=512, n=256, seed=2, kappa=kappa, right_stages=right, tau=0.7)
    inst = generate(p)
    A = inst.A
    atr = A.T @ inst.e
    assert np.abs(atr - p.tau * inst.g).max() <= 1e-11 * kappa
    P, D, gap, rel = certificate(A, inst.b, p.tau, inst.xstar)
    assert abs(rel) < 1e-13 * kappa
    assert math.isclose(P, inst.f_star, rel_tol=1e-14)


def test_e_equals_dense_solve():
    p = GenParams(m=64, n=32, seed=4, kappa=30.0, right_stages=2)
    inst = generate(p)
    A = inst.A.toarray()
    e_dense = p.tau * A @ np.linalg.solve(A.T @ A, inst.g)
    assert np.allclose(inst.e, e_dense, rtol=1e-10, atol=1e-10)
    assert np.allclose(inst.b, A @ inst.xstar + e_dense, rtol=1e-10, atol=1e-10)


def test_orthogonal_when_kappa_is_one():
    inst = generate(GenParams(m=64, n=32, seed=9, kappa=1.0, right_stages=3))
    A = inst.A.toarray()
    assert np.allclose(A.T @ A, np.eye(32), atol=1e-14)


@pytest.mark.parametrize("right,left,m,n", [(1, 1, 64, 32), (2, 1, 80, 40), (4, 1, 64, 64),
                                            (2, 0, 64, 32), (3, 1, 66, 34)])
def test_mvpa_mvpat_match_assembled_A(right, left, m, n):
    inst = generate(GenParams(m=m, n=n, seed=11, kappa=100.0, right_stages=right, left_stages=left))
    x = np.random.default_rng(0).standard_normal(n)
    y = np.random.default_rng(1).standard_normal(m)
    assert np.allclose(mvpa(inst, x), inst.A @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(mvpat(inst, y), inst.A.T @ y, rtol=1e-14, atol=1e-14)


def test_mvpa_matches_dense_bd8():
    """Eq. (bd8) written with dense Givens products, rotation by rotation."""
    m, n = 12, 6
    p = GenParams(m=m, n=n, seed=2, kappa=20.0, right_stages=2, left_stages=1)
    inst = generate(p)
    c, s, ct, st = gen.angles(p)
    T1 = np.eye(n)
    for i in range(0, n - 1, 2):
        T1 = T1 @ gen.givens(n, i, i + 1, c, s)
    T2 = np.eye(n)
    for i in range(1, n - 1, 2):
        T2 = T2 @ gen.givens(n, i, i + 1, c, s)
    G = T2 @ T1
    Gt = np.eye(m)
    for i in range(0, m - 1, 2):
        Gt = Gt @ gen.givens(m, i, i + 1, ct, st)
    P = np.zeros((m, m))
    P[np.arange(m), inst.perm] = 1.0
    Sig = np.zeros((m, n))
    Sig[np.arange(n), np.arange(n)] = inst.sigma
    A = (P @ Gt @ P) @ Sig @ G.T
    assert np.allclose(inst.A.toarray(), A, atol=1e-15)


def test_igen2_conditions():
    """m < n: B^T e = tau g_B and |N~^T e| <= tau (Eq. bd10); x* optimal, gap 0."""
    p = GenParams(m=64, n=128, seed=6, kappa=100.0, right_stages=2, xstar_frac=0.1, tau=0.5)
    inst = generate(p)
    B, N = inst.extra["B"], inst.extra["N"]
    assert np.abs(B.T @ inst.e - p.tau * inst.g[:64]).max() < 1e-11
    ne = N.T @ inst.e
    assert np.abs(ne).max() <= p.tau * (1 + 1e-12)
    # N~_i^T e = xi tau sign(N_i^T e), so its magnitude is |xi| tau
    assert np.allclose(np.abs(ne), p.tau * np.abs(inst.extra["xi"]), rtol=1e-12)
    assert np.all(inst.support < 64)
    P, D, gap, rel = certificate(inst.A, inst.b, p.tau, inst.xstar)
    assert abs(rel) < 1e-12
    assert N.getnnz(axis=0).min() == 8 and N.getnnz(axis=0).max() == 8


def test_structural_pattern_independent_of_values():
    """Changing only the angles leaves the structure unchanged."""
    a = generate(GenParams(m=64, n=32, seed=3, right_stages=2, theta=0.4))
    b = generate(GenParams(m=64, n=32, seed=3, right_stages=2, theta=1.3))
    assert np.array_equal(a.A.indptr, b.A.indptr) and np.array_equal(a.A.indices, b.A.indices)


def test_planted_sign_error_is_caught(monkeypatch):
    """A transposed rotation in the assembly breaks the MvPA pin and the optimality pin."""
    orig = gen.stage_matrix
    monkeypatch.setattr(gen, "stage_matrix", lambda size, first, c, s: orig(size, first, c, -s))
    inst = generate(GenParams(m=64, n=32, seed=1, kappa=10.0, right_stages=2))
    x = np.random.default_rng(0).standard_normal(32)
    assert not np.allclose(mvpa(inst, x), inst.A @ x, atol=1e-8)


def test_igen2_step_size_bounds_the_spectrum():
    """IGen2's FISTA step size: sigma_max^2 + ||N~||_1 ||N~||_inf >= ||A||_2^2, since
    ||[B N~]||^2 <= ||B||^2 + ||N~||^2 and ||N~||_2^2 <= ||N~||_1 ||N~||_inf."""
    for seed in (1, 2):
        inst = generate(GenParams(m=48, n=80, seed=seed, kappa=30.0, right_stages=2, xstar_frac=0.1,
                                  n_nnz_per_col=5))
        top = np.linalg.svd(inst.A.toarray(), compute_uv=False)[0]
        assert inst.lipschitz >= top ** 2 * (1 - 1e-12)
        assert inst.lipschitz <= 1.0 + 5.0 * 48


def test_sec89_instance_shape():
    """Sec. 8.9's instances: sigma_i = 0.1 for odd i and 100 for even i, so A^T A = G Sigma^2 G^T
    has exactly the eigenvalues 0.01 and 1e4, n/2 times each; half of the nonzeros of x* are
    -1e4 and the rest 0.1; x* is optimal at tau (Eq. bd7, zero gap)."""
    p = GenParams(m=128, n=64, seed=3, right_stages=2, left_stages=0, theta=2.0 * math.pi / 3.0, sigma_mode=1,
                  sigma_odd=0.1, sigma_even=100.0, xstar_mode=1, xstar_lo=0.1, xstar_hi=1e4, xstar_frac=1.0 / 8.0)
    inst = generate(p)
    assert np.array_equal(inst.sigma[0::2], np.full(32, 0.1)) and np.array_equal(inst.sigma[1::2], np.full(32, 100.0))
    ev = np.sort(np.linalg.eigvalsh((inst.A.T @ inst.A).toarray()))
    assert np.allclose(ev[:32], 0.01, rtol=1e-9) and np.allclose(ev[32:], 1e4, rtol=1e-12)
    S = inst.support
    assert len(S) == 8 and np.array_equal(inst.xstar[S[:4]], np.full(4, -1e4))
    assert np.array_equal(inst.xstar[S[4:]], np.full(4, 0.1))
    assert np.count_nonzero(inst.xstar) == 8
    assert inst.lipschitz == 1e4
    assert np.abs(inst.A.T @ inst.e - p.tau * inst.g).max() < 1e-7
    # b carries A x* with entries near 1e6, so the gap at x* is zero only to FP64 rounding
    assert abs(certificate(inst.A, inst.b, p.tau, inst.xstar)[3]) < 1e-7


def test_osgen3_unconstrained_solution_and_selection():
    """Procedure OsGen3 (Sec. 6): with every component kept, G^T x* = gamma (Sigma^T Sigma)^{-1} 1
    (the exact least-squares solution, G orthonormal); with s < n the kept components are the
    s1 smallest nonzero and s2 largest |x_i| of that solution."""
    from oracle.generator import osgen3
    full = GenParams(m=96, n=48, seed=5, kappa=30.0, right_stages=3, xstar_mode=2, gamma=100.0, xstar_frac=1.0)
    inst = generate(full)
    assert np.allclose(inst.R.T @ inst.xstar, 100.0 / inst.sigma ** 2, rtol=1e-12, atol=0)
    sparse = GenParams(m=96, n=48, seed=5, kappa=30.0, right_stages=3, xstar_mode=2, gamma=100.0, xstar_frac=0.25)
    xs, S = osgen3(sparse, inst.sigma)
    x = inst.xstar                                     # the unconstrained solution of the same G, Sigma
    order = np.argsort(np.abs(x), kind="stable")
    assert len(S) == 12
    assert set(S) == set(order[:6]) | set(order[-6:])
    assert np.array_equal(xs[S], x[S]) and np.count_nonzero(xs) == 12


def test_kappa_rho_against_an_eigendecomposition():
    """Eq. (bd12) through R and Sigma against the eigenvectors of the assembled A^T A."""
    from oracle.generator import kappa_rho
    p = GenParams(m=80, n=40, seed=6, kappa=100.0, right_stages=2, xstar_mode=2, gamma=100.0, xstar_frac=0.2)
    inst = generate(p)
    lam, V = np.linalg.eigh((inst.A.T @ inst.A).toarray())
    for rho in (1e-5, 1e-3, 0.01, 0.1, 0.5, 2.0):
        Vr = V[:, lam >= rho * (1 - 1e-9)]
        proj = np.linalg.norm(Vr @ (Vr.T @ inst.xstar))
        want = math.inf if proj == 0 else np.linalg.norm(inst.xstar) / proj
        got = kappa_rho(inst.sigma, inst.R, inst.xstar, rho)
        assert (math.isinf(want) and math.isinf(got)) or math.isclose(got, want, rel_tol=1e-9)
    assert kappa_rho(inst.sigma, inst.R, inst.xstar, inst.sigma.min() ** 2) == pytest.approx(1.0)
    assert math.isinf(kappa_rho(inst.sigma, inst.R, inst.xstar, 2.0))
    # the OsGen3 optimum is optimal at tau (Eq. bd7)
    assert abs(certificate(inst.A, inst.b, p.tau, inst.xstar)[3]) < 1e-10
