"""Instance generator of the paper, written out with sparse matrices (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows, in the paper's order:

* Sec. 4, Eq. (bd8):     A = (P1 G~ P2) Sigma G^T with Sigma the m x n rectangular diagonal
                         of singular values and G, G~ compositions of Givens rotations
                         G(i, j, theta) whose (i,i), (i,j), (j,i), (j,j) entries are
                         c, -s, s, c.
* Sec. 4.1:              one stage of rotations on the planes (1,2), (3,4), ... (1-based),
                         P1 = P2 = P a random permutation.
* Sec. 4.2:              a second kind of stage G2 on the planes (2,3), (4,5), ...; the
                         right factor alternates G, G2 G, G G2 G, G2 G G2 G.
* Procedure OsGen (Sec. 6): a random support S with |S| = s and random nonzeros.
* Procedure IGen (Sec. 3.1): g in the subdifferential of ||x*||_1 (Eq. bd6),
                         e = tau A (A^T A)^{-1} g with (A^T A)^{-1} = G (Sigma^T Sigma)^{-1} G^T
                         (end of Sec. 4: a diagonal scaling between a product with G^T and one with G),
                         b = A x* + e.
* Procedure IGen2 (Sec. 3.2): for m < n, A = [B, N~] with B square (built as above with
                         n = m), e = tau B^{-T} g, N~_i = xi tau / |N_i^T e| N_i.

Readings of the paper where it is silent (each also listed in the design notes):

* kappa is kappa(A) = sigma_max / sigma_min (the configs say "kappa(A)"); the singular
  values are exactly log-spaced, sigma_i = kappa^(-rank_i / (n-1)) with rank_i a random
  permutation of 0..n-1, so sigma_max = 1 and lambda_max(A^T A) = 1.
* The right factor R with w stages is R = T_w ... T_2 T_1 with T_1 of kind G (planes
  (0,1), (2,3), ... 0-based), T_2 of kind G2 (planes (1,2), (3,4), ...), alternating.
  The left factor with one stage is L = P G~ P (Sec. 4.1); with zero stages L = I (the
  experiments of Sec. 8 use A = Sigma G^T).
* Permutation convention: (P v)_i = v_{perm[i]}, perm = stable argsort of random keys.
* x*: |x*_i| = lo + (hi - lo) U, independent random sign; g_i = U(-1,1) off the support.
* A structural entry is one reached by some product of structural nonzeros of the
  factors; it is kept even if its value cancels to 0.0.
* IGen2: N has ``n_nnz_per_col`` distinct random rows per column with values U(-1,1);
  the support of x* lies in the first m columns; a column with N_i^T e = 0 is kept
  unscaled.  The step size bound for N~ is ||N~||_1 ||N~||_inf.
"""

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import rng


@dataclass
class GenParams:
    m: int
    n: int
    seed: int = 0
    kappa: float = 1e2
    tau: float = 1.0
    xstar_frac: float = 0.05
    xstar_lo: float = 1.0
    xstar_hi: float = 10.0
    right_stages: int = 1
    left_stages: int = 1
    theta: float = 2.0 * math.pi / 10.0
    vartheta: float = float("nan")   # nan: same angle as theta
    g_offsupport: int = 0            # 0: U(-1,1) off the support, 1: zero
    n_nnz_per_col: int = 8           # IGen2: nonzeros per column of N
    # Sec. 8.9's huge-scale instances: sigma_i alternating (sigma_odd for odd i = 1, 3, ...,
    # sigma_even for even i), and x* with half of its nonzeros -xstar_hi, the rest +xstar_lo
    sigma_mode: int = 0              # 0: log-spaced by kappa; 1: alternating
    sigma_odd: float = 0.1
    sigma_even: float = 100.0
    xstar_mode: int = 0              # 0: +-U[lo, hi]; 1: first half of the support -hi, rest +lo;
                                     # 2: Procedure OsGen3 (Sec. 6) with gamma, s1 = s // 2
    gamma: float = 100.0             # OsGen3's gamma

    @classmethod
    def from_dict(cls, d):
        """Build from a parameter dict (the generator parameters of Sec. 3-6), ignoring keys
        that only the CUDA path reads."""
        names = set(cls.__dataclass_fields__)
        return cls(**{k: v for k, v in d.items() if k in names})


@dataclass
class Instance:
    params: GenParams
    A: sp.csr_matrix                  # m x n, sorted indices, structural entries kept
    b: np.ndarray
    xstar: np.ndarray
    g: np.ndarray                     # subgradient used by IGen / IGen2 (length n)
    e: np.ndarray                     # b - A x*
    sigma: np.ndarray                 # singular values in index order
    perm: np.ndarray                  # row permutation (None when L = I)
    support: np.ndarray               # sorted support of x*
    R: sp.csr_matrix                  # right factor (n x n, or m x m for IGen2)
    Lmat: sp.csr_matrix               # left factor (m x m)
    f_star: float                     # f_tau(x*) at tau = params.tau
    lam_max: float                    # ||A^T b||_inf
    lipschitz: float                  # L >= lambda_max(A^T A)
    extra: dict = field(default_factory=dict)


def support_size(p: GenParams) -> int:
    """Number s of nonzeros of x* (Procedure OsGen, Sec. 6, takes s as given):
    s = floor(frac * n + 0.5), clamped to [1, min(m, n)]."""
    s = int(math.floor(p.xstar_frac * p.n + 0.5))
    return max(1, min(s, p.m, p.n))


def angles(p: GenParams):
    """(c, s, c~, s~) of the right and left rotations (angles theta and vartheta of the Givens
    matrices of Sec. 4 and 4.1), by the host libm."""
    vt = p.theta if math.isnan(p.vartheta) else p.vartheta
    return math.cos(p.theta), math.sin(p.theta), math.cos(vt), math.sin(vt)


def givens(size, i, j, c, s):
    """The Givens matrix G(i, j, theta) of Sec. 4 as a dense array (0-based i < j)."""
    G = np.eye(size)
    G[i, i] = c
    G[i, j] = -s
    G[j, i] = s
    G[j, j] = c
    return G


def stage_pairs(size, first):
    """Planes of one stage (Sec. 4.1 for G, Sec. 4.2 for G2): (first, first+1),
    (first+2, first+3), ... inside [0, size)."""
    i = np.arange(first, size - 1, 2, dtype=np.int64)
    return i, i + 1


def stage_matrix(size, first, c, s):
    """Composition of the rotations of one stage (G of Sec. 4.1, G2 of Sec. 4.2).

    The rotations of a stage act on disjoint planes, so their product is the block
    diagonal matrix with a 2x2 block [[c, -s], [s, c]] on each plane and 1 on every
    coordinate left unpaired.
    """
    i, j = stage_pairs(size, first)
    diag = np.ones(size)
    diag[i] = c
    diag[j] = c
    rows = np.concatenate([np.arange(size), i, j])
    cols = np.concatenate([np.arange(size), j, i])
    vals = np.concatenate([diag, np.full(len(i), -s), np.full(len(i), s)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(size, size))


def stage_first(k):
    """Kind of the k-th stage (1-based, Sec. 4.2 alternates them): odd stages are G (first
    plane 0), even are G2."""
    return (k - 1) % 2


def right_factor(size, stages, c, s):
    """Right singular vectors of Eq. (bd8): R = T_w ... T_2 T_1 (T_1 applied first to a
    vector), the products of stages of Sec. 4.2."""
    R = sp.identity(size, format="csr")
    for k in range(1, stages + 1):
        R = stage_matrix(size, stage_first(k), c, s) @ R
    return R.tocsr()


def perm_matrix(perm):
    """The random permutation matrix P of Sec. 4.1, with (P v)_i = v_{perm[i]}."""
    size = len(perm)
    return sp.csr_matrix((np.ones(size), (np.arange(size), perm)), shape=(size, size))


def left_factor(size, stages, perm, ct, st):
    """Left singular vectors of Eq. (bd8): L = P (T~_l ... T~_1) P (Sec. 4.1), or the
    identity when there is no left stage (the A = Sigma G^T of Sec. 8)."""
    if stages == 0:
        return sp.identity(size, format="csr")
    Gt = right_factor(size, stages, ct, st)
    P = perm_matrix(perm)
    return (P @ Gt @ P).tocsr()


def _structure(M):
    """Same sparsity as M with every stored entry replaced by 1."""
    M = M.tocsr(copy=True)
    M.data = np.ones_like(M.data)
    return M


def _values_on_pattern(pattern, values):
    """CSR with the structure of ``pattern`` and the entries of ``values`` (0 where absent)."""
    pattern = pattern.tocsr()
    pattern.sort_indices()
    m, n = pattern.shape
    V = values.tocoo()
    vkeys = V.row.astype(np.int64) * n + V.col.astype(np.int64)
    order = np.argsort(vkeys, kind="stable")
    vkeys = vkeys[order]
    vdata = V.data[order]
    prow = np.repeat(np.arange(m, dtype=np.int64), np.diff(pattern.indptr))
    pkeys = prow * n + pattern.indices.astype(np.int64)
    pos = np.searchsorted(vkeys, pkeys)
    posc = np.minimum(pos, max(len(vkeys) - 1, 0))
    found = (pos < len(vkeys)) & (vkeys[posc] == pkeys) if len(vkeys) else np.zeros(len(pkeys), bool)
    if found.sum() != len(vkeys):
        raise AssertionError("a computed entry lies outside the structural pattern")
    data = np.where(found, vdata[posc] if len(vkeys) else 0.0, 0.0)
    out = sp.csr_matrix((data, pattern.indices.copy(), pattern.indptr.copy()), shape=(m, n))
    out.has_sorted_indices = True
    return out


def sigma_of(p: GenParams, count):
    """The singular values of the square factor: log-spaced by kappa, or (sigma_mode 1,
    Sec. 8.9) sigma_i = sigma_odd for odd i and sigma_even for even i (1-based i)."""
    if p.sigma_mode == 1:
        return np.where(np.arange(count) % 2 == 0, p.sigma_odd, p.sigma_even).astype(np.float64)
    return singular_values(p.seed, count, p.kappa)


def singular_values(seed, count, kappa):
    """Diagonal of Sigma (Sec. 4) with kappa(A) = sigma_max / sigma_min = kappa: the paper
    fixes the condition number, not the spacing; here sigma_i = kappa^(-rank_i/(count-1)),
    ranks from the argsort of random keys."""
    if count == 1:
        return np.ones(1)
    keys = rng.draws(seed, rng.TAG_SIGMA, count)
    order = np.argsort(keys, kind="stable")
    rank = np.empty(count, dtype=np.int64)
    rank[order] = np.arange(count)
    return np.exp(-(rank.astype(np.float64) / float(count - 1)) * math.log(kappa))


def row_permutation(seed, m):
    """The random row permutation of Sec. 4.1: perm = stable argsort of random keys;
    P[i, perm[i]] = 1."""
    return np.argsort(rng.draws(seed, rng.TAG_PERM, m), kind="stable").astype(np.int64)


def optimal_solution(p: GenParams, ncols_support):
    """Procedure OsGen (Sec. 6) with the configs' magnitudes +-U[lo, hi].

    The support is the s indices with the smallest keys among the first
    ``ncols_support`` columns.  Returns (x*, sorted support).
    """
    s = support_size(p)
    s = min(s, ncols_support)
    keys = rng.draws(p.seed, rng.TAG_SUPPORT, ncols_support)
    S = np.sort(np.argsort(keys, kind="stable")[:s])
    xstar = np.zeros(p.n)
    if p.xstar_mode == 1:
        # Sec. 8.9: half of the nonzeros (the first in index order) -xstar_hi, the rest +xstar_lo
        h = len(S) // 2
        xstar[S[:h]] = -p.xstar_hi
        xstar[S[h:]] = p.xstar_lo
        return xstar, S
    mag = p.xstar_lo + (p.xstar_hi - p.xstar_lo) * rng.unit_uniform(rng.draws(p.seed, rng.TAG_XVAL, p.n))
    neg = (rng.draws(p.seed, rng.TAG_XSIGN, p.n) >> np.uint64(63)) == np.uint64(1)
    xstar[S] = np.where(neg[S], -mag[S], mag[S])
    return xstar, S


def osgen3(p: GenParams, sigma):
    """Procedure OsGen3 (Sec. 6): x = argmin ||G^T x - gamma (Sigma^T Sigma)^{-1} 1||, which is
    G (gamma / sigma^2) because G is orthonormal (G = R, the stages applied to the vector one by
    one, T_1 first); keep the s1 = s // 2 smallest nonzero and the s2 = s - s1 largest |x_i| (ties
    by index), zero the rest.  IGen only (m >= n).  Returns (x*, sorted support)."""
    from .operators import rotate   # local import: operators imports this module
    c, sn, _, _ = angles(p)
    n = p.n
    x = p.gamma / (sigma * sigma)
    for k in range(1, p.right_stages + 1):
        rotate(x, stage_first(k), c, sn)
    s = min(support_size(p), n)
    s1 = s // 2
    s2 = s - s1
    order = np.argsort(np.abs(x), kind="stable")
    nz = order[np.abs(x[order]) > 0.0]
    keep = np.union1d(nz[:s1], nz[max(0, len(nz) - s2):] if s2 > 0 else np.array([], dtype=np.int64))
    xstar = np.zeros(n)
    xstar[keep] = x[keep]
    return xstar, np.sort(keep.astype(np.int64))


def kappa_rho(sigma, R, xstar, rho):
    """Eq. (bd12): ||x*|| / ||P_rho x*||, P_rho the projection on the eigenvectors of A^T A with
    eigenvalue >= rho; with A^T A = R Sigma^2 R^T that is the mass of R^T x* on sigma_i^2 >= rho."""
    proj = np.linalg.norm((R.T @ xstar)[sigma * sigma >= rho])
    return math.inf if proj == 0.0 else float(np.linalg.norm(xstar) / proj)


def subgradient(p: GenParams, xstar, count):
    """g in the subdifferential of ||x*||_1 on the first ``count`` coordinates (Eq. bd6)."""
    g = np.zeros(count)
    if p.g_offsupport == 0:
        g = 2.0 * rng.unit_uniform(rng.draws(p.seed, rng.TAG_GOFF, count)) - 1.0
    nz = xstar[:count] != 0
    g[nz] = np.sign(xstar[:count][nz])
    return g


def _square_part(p: GenParams, size, rows):
    """(A0, R, L, sigma, perm) for A0 = L Sigma R^T with ``rows`` >= ``size`` rows."""
    c, s, ct, st = angles(p)
    sigma = sigma_of(p, size)
    R = right_factor(size, p.right_stages, c, s)
    perm = row_permutation(p.seed, rows) if p.left_stages > 0 else None
    L = left_factor(rows, p.left_stages, perm, ct, st)
    Sig = sp.csr_matrix((sigma, (np.arange(size), np.arange(size))), shape=(rows, size))
    values = L @ Sig @ R.T
    pattern = _structure(L) @ _structure(Sig) @ _structure(R).T
    A0 = _values_on_pattern(pattern, values)
    return A0, R, L, sigma, perm


def generate(p: GenParams) -> Instance:
    """IGen (m >= n) or IGen2 (m < n) on the matrix of Eq. (bd8)."""
    if p.m >= p.n:
        return _generate_igen(p)
    return _generate_igen2(p)


def _generate_igen(p: GenParams) -> Instance:
    m, n, tau = p.m, p.n, p.tau
    A, R, L, sigma, perm = _square_part(p, n, m)
    xstar, S = osgen3(p, sigma) if p.xstar_mode == 2 else optimal_solution(p, n)
    g = subgradient(p, xstar, n)
    # IGen's e = tau A (A^T A)^{-1} g (Sec. 3.1) with (A^T A)^{-1} = G (Sigma^T Sigma)^{-1} G^T (end of Sec. 4).
    v = R.T @ g
    v = v / (sigma * sigma)
    v = R @ v
    e = tau * (A @ v)
    # IGen's b = A x* + e (Sec. 3.1).
    b = A @ xstar + e
    f_star = tau * np.abs(xstar).sum() + 0.5 * float(e @ e)
    lam_max = float(np.abs(A.T @ b).max())
    lipschitz = float(sigma.max() ** 2)
    return Instance(p, A, b, xstar, g, e, sigma, perm, S, R, L, f_star, lam_max, lipschitz)


def n_columns(p: GenParams, e):
    """IGen2 columns N_i (i = 0 .. n-m-1) and the scaled N~_i (Sec. 3.2).

    Column i takes the first ``n_nnz_per_col`` distinct rows among the candidates
    draw(NROW, i*4096 + t) mod m, t = 0, 1, ...; the value of the k-th accepted row is
    2 U(draw(NVAL, i*d + k)) - 1; xi_i = 2 U(draw(XI, i)) - 1.
    """
    m, n, d = p.m, p.n, p.n_nnz_per_col
    ncols = n - m
    if d > m:
        raise ValueError("n_nnz_per_col exceeds m")
    key_rows = rng.stream_key(p.seed, rng.TAG_NROW)
    rows_all, cols_all, vals_all = [], [], []
    vals_u = 2.0 * rng.unit_uniform(rng.draws(p.seed, rng.TAG_NVAL, ncols * d)) - 1.0
    xi = 2.0 * rng.unit_uniform(rng.draws(p.seed, rng.TAG_XI, ncols)) - 1.0
    for i in range(ncols):
        chosen = []
        t = 0
        while len(chosen) < d:
            if t >= 4096:
                raise RuntimeError("row sampling for a column of N did not finish")
            r = int(rng.splitmix_output(key_rows, np.array([i * 4096 + t], np.uint64))[0] % np.uint64(m))
            t += 1
            if r not in chosen:
                chosen.append(r)
        vals = vals_u[i * d:(i + 1) * d]
        order = np.argsort(chosen)
        rows = np.array(chosen)[order]
        v = vals[order]
        dot = float(v @ e[rows])
        if dot != 0.0:
            v = (xi[i] * p.tau / abs(dot)) * v
        rows_all.append(rows)
        cols_all.append(np.full(d, i))
        vals_all.append(v)
    if ncols == 0:
        return sp.csr_matrix((m, 0)), xi
    N = sp.csr_matrix((np.concatenate(vals_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                      shape=(m, ncols))
    N.sort_indices()
    return N, xi


def _generate_igen2(p: GenParams) -> Instance:
    m, n, tau = p.m, p.n, p.tau
    if p.xstar_mode == 2:
        raise ValueError("OsGen3 (xstar_mode 2) is defined for m >= n")
    B, R, L, sigma, perm = _square_part(p, m, m)
    xstar, S = optimal_solution(p, m)
    gB = subgradient(p, xstar, m)
    # IGen2's e = tau B^{-T} g with B^{-T} = L Sigma^{-1} R^T.
    v = R.T @ gB
    v = v / sigma
    e = tau * (L @ v)
    Ntil, xi = n_columns(p, e)
    A = sp.hstack([B, Ntil], format="csr")
    A.sort_indices()
    b = A @ xstar + e
    g = np.concatenate([gB, xi])
    f_star = tau * np.abs(xstar).sum() + 0.5 * float(e @ e)
    lam_max = float(np.abs(A.T @ b).max())
    absN = abs(Ntil)
    bound = (float(absN.sum(axis=0).max()) * float(absN.sum(axis=1).max())) if Ntil.shape[1] else 0.0
    lipschitz = float(sigma.max() ** 2) + bound
    return Instance(p, A, b, xstar, g, e, sigma, perm, S, R, L, f_star, lam_max, lipschitz,
                    extra={"B": B, "N": Ntil, "xi": xi})


@dataclass
class Factors:
    """The ingredients of Eq. (bd8) and of x*, without assembling A (m >= n only)."""
    params: GenParams
    sigma: np.ndarray
    perm: np.ndarray
    xstar: np.ndarray
    support: np.ndarray
    g: np.ndarray


def make_factors(p: GenParams) -> Factors:
    """The factors of Eq. (bd8) and the x*, g of Procedures OsGen / OsGen3 (Sec. 6) and IGen
    (Eq. bd6), without assembling A (m >= n)."""
    if p.m < p.n:
        raise ValueError("make_factors covers IGen (m >= n)")
    sigma = sigma_of(p, p.n)
    perm = row_permutation(p.seed, p.m) if p.left_stages > 0 else None
    xstar, S = osgen3(p, sigma) if p.xstar_mode == 2 else optimal_solution(p, p.n)
    g = subgradient(p, xstar, p.n)
    return Factors(p, sigma, perm, xstar, S, g)


def igen_matrix_free(f: Factors):
    """(b, e) of Procedure IGen through Algorithm MvPA, the route the paper proposes when A is
    not stored (Sec. 4): e = tau A G (Sigma^T Sigma)^{-1} G^T g, b = A x* + e."""
    from .operators import rotate, rotate_t   # local import: operators imports this module
    p = f.params
    c, s, _, _ = angles(p)
    v = np.array(f.g, dtype=np.float64, copy=True)
    for k in range(p.right_stages, 0, -1):      # G^T g
        rotate_t(v, stage_first(k), c, s)
    v = v / (f.sigma * f.sigma)
    for k in range(1, p.right_stages + 1):      # G (...)
        rotate(v, stage_first(k), c, s)
    from .operators import mvpa
    e = p.tau * mvpa(f, v)
    b = mvpa(f, f.xstar) + e
    return b, e
