"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds only input recipes (instance parameters and seeded random vectors); none of the
method's arithmetic.  Both the CUDA path and the oracle build their own instance from
the same parameters.

Workloads (all synthetic; the paper uses no dataset):

* ``c1``  m=2048, n=1024, seed 0, kappa(A)=1e2, x* 5% nonzeros +-U[1,10], tau=1, one right
          stage (G) and one left stage (P G~ P) as in Sec. 4.1; FP64 values.
* ``c2``  m=2^25, n=2^24, kappa(A)=1e4, x* 1% nonzeros, right stages G2 G plus one left
          stage (about 8 nonzeros per column); FP32 values, int32 indices.
* ``c3``  m=2^22, n=2^21, x* 2% nonzeros, right stages G2 G G2 G plus one left stage (about
          16 nonzeros per column); kappa in {1e2, 1e4, 1e6}; values FP64 / FP32 / BF16.
* ``c4``  256 instances, n log-uniform in [2^12, 2^18] rounded to even, m = 2n, about 8
          nonzeros per column, kappa log-uniform in [1e2, 1e5], x* 1% nonzeros, seed i,
          16 tau values 0.9 lambda_max 10^(-3 j / 15).
* ``c5``  Poisson arrivals; n log-uniform in [2^10, 2^23] (even), m in {n/2, 2n}, kappa
          log-uniform in [1e2, 1e6], x* density U[0.5%, 5%], tau = 10^U[-2,0] lambda_max.
* ``sec89`` the huge-scale instances of Sec. 8.9 at a size one GPU holds.
"""

import math

import numpy as np

TWO_PI = 2.0 * math.pi

BASE = dict(seed=0, kappa=1e2, tau=1.0, xstar_frac=0.05, xstar_lo=1.0, xstar_hi=10.0,
            right_stages=1, left_stages=1, theta=TWO_PI / 10.0, vartheta=float("nan"),
            g_offsupport=0, n_nnz_per_col=8, value_dtype="f64")


def params(**kw):
    """A full parameter dict: BASE overridden by ``kw``."""
    out = dict(BASE)
    out.update(kw)
    return out


C1 = params(m=2048, n=1024, seed=0, kappa=1e2, xstar_frac=0.05, right_stages=1, left_stages=1,
            value_dtype="f64")
C1_TOL = 1e-8

C2 = params(m=2 ** 25, n=2 ** 24, seed=0, kappa=1e4, xstar_frac=0.01, right_stages=2,
            left_stages=1, value_dtype="f32")
C2_TOL = 1e-6


def c2_scaled(log2n, **kw):
    """The C2 recipe at n = 2^log2n (m = 2n)."""
    n = 2 ** log2n
    return params(**{**C2, "m": 2 * n, "n": n, **kw})


def c3(kappa, value_dtype):
    return params(m=2 ** 22, n=2 ** 21, seed=0, kappa=kappa, xstar_frac=0.02, right_stages=4,
                  left_stages=1, value_dtype=value_dtype)


def c4_batch(count=256, seed=12345, log2n_lo=12, log2n_hi=18):
    """Instance parameters of the ragged batch and their tau paths."""
    r = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(2.0 ** r.uniform(log2n_lo, log2n_hi)))
        n += n % 2
        kappa = float(10.0 ** r.uniform(2.0, 5.0))
        out.append(params(m=2 * n, n=n, seed=i, kappa=kappa, xstar_frac=0.01, right_stages=2,
                          left_stages=1, value_dtype="f32"))
    return out


def c4_tau_path(lam_max, count=16):
    return [0.9 * lam_max * 10.0 ** (-3.0 * j / (count - 1)) for j in range(count)]


def c5_requests(count, rate, seed=777, log2n_lo=10, log2n_hi=23):
    """Serving requests: (arrival time s, gen params, tau factor, method)."""
    r = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += r.exponential(1.0 / rate)
        n = int(round(2.0 ** r.uniform(log2n_lo, log2n_hi)))
        n += n % 2
        m = n // 2 if r.uniform() < 0.5 else 2 * n
        m += m % 2
        kappa = float(10.0 ** r.uniform(2.0, 6.0))
        frac = float(r.uniform(0.005, 0.05))
        tau_factor = float(10.0 ** r.uniform(-2.0, 0.0))
        method = "fista" if kappa <= 1e3 else "pdncg"
        out.append(dict(t=t, params=params(m=m, n=n, seed=100000 + i, kappa=kappa, xstar_frac=frac,
                                           right_stages=2, left_stages=1, value_dtype="f32"),
                        tau_factor=tau_factor, method=method))
    return out


def sec89(log2n, value_dtype="f32", seed=0):
    """The huge-scale instances of Sec. 8.9 at n = 2^log2n: A = Sigma G^T (no left stage),
    m = 2n, sigma_i = 0.1 (odd i) / 100 (even i), theta = 2 pi / 3, s = n / 2^10 nonzeros of x*,
    half -1e4 and half 0.1; G = G2 G (two stages, as constructed in Sec. 4.2)."""
    n = 2 ** log2n
    return params(m=2 * n, n=n, seed=seed, right_stages=2, left_stages=0, theta=2.0 * math.pi / 3.0,
                  sigma_mode=1, sigma_odd=0.1, sigma_even=100.0, xstar_mode=1, xstar_lo=0.1, xstar_hi=1e4,
                  xstar_frac=2.0 ** -10, value_dtype=value_dtype)


def random_vector(size, seed):
    """Standard normal FP64 vector."""
    return np.random.default_rng(seed).standard_normal(size)
