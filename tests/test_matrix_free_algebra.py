"""The algebra that matrix-free pdNCG rests on, checked on the oracle's generated instances
(CPU).  A = L Sigma R^T with L = P1 G~ P2 orthogonal (Eq. bd8), so:
  * A^T A = R Sigma^2 R^T, whatever the left factor (the Hessian's product needs no left stage);
  * ||b - A x||^2 = ||b||^2 - 2 (A^T b).x + ||Sigma R^T x||^2 and b.(b - A x) = ||b||^2 - (A^T b).x,
    so the gradient A^T r = A^T b - R Sigma^2 R^T x and the certificate need A^T b once;
  * r.(A d) = (A^T r).d and ||A d|| = ||Sigma R^T d||, the line search's two sums;
  * R has half-bandwidth w (w stages of neighbour rotations), so R Sigma^2 R^T has at most 2w
    (2w - 1 measured for w >= 2), and its product with the indicator of {i = q mod (2w + 1)}
    equals its diagonal on those i.
A wrong sign, a dropped factor of Sigma or a transposed R fails one of these."""

import numpy as np
import pytest

import workloads as W
from oracle.generator import GenParams, generate


def _inst(left, w, m=400, n=200, seed=3):
    p = W.params(m=m, n=n, right_stages=w, left_stages=left, kappa=1e3, seed=seed, xstar_frac=0.05)
    return generate(GenParams.from_dict(p))


@pytest.mark.parametrize("left,w", [(1, 2), (0, 2), (1, 5), (0, 8)])
def test_gram_matrix_is_r_sigma2_rt(left, w):
    ref = _inst(left, w)
    A = ref.A.toarray()
    R = ref.R.toarray()
    G = R @ np.diag(ref.sigma ** 2) @ R.T
    assert np.allclose(A.T @ A, G, rtol=0, atol=1e-12 * np.abs(G).max())
    # half-bandwidth w of R, 2w of the Gram matrix
    i, j = np.nonzero(np.abs(R) > 0)
    assert np.abs(i - j).max() <= w
    i, j = np.nonzero(np.abs(G) > 1e-14 * np.abs(G).max())
    assert np.abs(i - j).max() <= 2 * w


@pytest.mark.parametrize("left", [1, 0])
def test_residual_sums_from_atb_and_sigma_rt(left):
    ref = _inst(left, 2)
    A, b = ref.A, ref.b
    R = ref.R
    c = A.T @ b
    for seed in (1, 2):
        x = ref.xstar + W.random_vector(A.shape[1], seed)
        d = W.random_vector(A.shape[1], seed + 10)
        r = b - A @ x
        u = ref.sigma * (R.T @ x)
        assert float(r @ r) == pytest.approx(float(b @ b) - 2 * float(c @ x) + float(u @ u), rel=1e-12)
        assert float(b @ r) == pytest.approx(float(b @ b) - float(c @ x), rel=1e-12)
        atr = c - R @ (ref.sigma * u)
        assert np.allclose(atr, A.T @ r, rtol=0, atol=1e-11 * np.abs(A.T @ r).max())
        Ad = A @ d
        v = ref.sigma * (R.T @ d)
        assert float(r @ Ad) == pytest.approx(float(atr @ d), rel=1e-11)
        assert float(Ad @ Ad) == pytest.approx(float(v @ v), rel=1e-12)


@pytest.mark.parametrize("left,w", [(1, 2), (0, 3), (1, 8)])
def test_probing_recovers_the_diagonal(left, w):
    ref = _inst(left, w, m=300, n=150)
    A = ref.A.toarray()
    want = (A * A).sum(axis=0)
    R = ref.R
    n = A.shape[1]
    K = 2 * w + 1
    got = np.zeros(n)
    for q in range(K):
        v = (np.arange(n) % K == q).astype(float)
        mv = R @ (ref.sigma ** 2 * (R.T @ v))
        got[np.arange(n) % K == q] = mv[np.arange(n) % K == q]
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    # with fewer probes than the band needs its neighbours leak in
    K = 2 * w - 1
    bad = np.zeros(n)
    for q in range(K):
        v = (np.arange(n) % K == q).astype(float)
        mv = R @ (ref.sigma ** 2 * (R.T @ v))
        bad[np.arange(n) % K == q] = mv[np.arange(n) % K == q]
    assert not np.allclose(bad, want, rtol=1e-6, atol=0)
