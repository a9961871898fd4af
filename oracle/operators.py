"""Algorithms MvPA and MvPAt of Sec. 4: products with A = (P1 G~ P2) Sigma G^T without A.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The composition G = G_1 G_2 ... G_K lists the rotations of the last stage first, so for
R = T_w ... T_1 MvPA applies T_w^T first and T_1^T last (y_k = G_k^T y_{k-1}), then
Sigma and P2, then the left rotations G~_{K~}, ..., G~_1 (T~_1 first), then P1.  MvPAt
runs the same steps transposed in the opposite order.  Rotations inside one stage act on
disjoint planes, so each stage is applied as one vectorised update; every pair still
sees exactly the arithmetic of its own rotation.
"""

import numpy as np

from .generator import angles, stage_first, stage_pairs


def rotate(v, first, c, s):
    """v <- T v for one stage (the rotation step of Algorithms MvPA / MvPAt, Sec. 4):
    (v_i, v_j) <- (c v_i - s v_j, s v_i + c v_j)."""
    i, j = stage_pairs(len(v), first)
    vi = v[i].copy()
    vj = v[j].copy()
    v[i] = c * vi - s * vj
    v[j] = s * vi + c * vj
    return v


def rotate_t(v, first, c, s):
    """v <- T^T v for one stage (Algorithms MvPA / MvPAt, Sec. 4):
    (v_i, v_j) <- (c v_i + s v_j, -s v_i + c v_j)."""
    i, j = stage_pairs(len(v), first)
    vi = v[i].copy()
    vj = v[j].copy()
    v[i] = c * vi + s * vj
    v[j] = -s * vi + c * vj
    return v


def _square_dims(inst):
    """Works for an Instance or a Factors object (both carry params, sigma and perm)."""
    p = inst.params
    size = p.n if p.m >= p.n else p.m
    return size, p.m


def mvpa(inst, x):
    """y = A x for the Givens part of A (Algorithm MvPA)."""
    p = inst.params
    c, s, ct, st = angles(p)
    size, m = _square_dims(inst)
    y = np.array(x[:size], dtype=np.float64, copy=True)
    for k in range(p.right_stages, 0, -1):          # G_1^T, ..., G_K^T
        rotate_t(y, stage_first(k), c, s)
    yt = np.zeros(m)
    yt[:size] = inst.sigma * y                       # Sigma y_K
    if p.left_stages > 0:
        yt = yt[inst.perm]                           # P2
        for k in range(1, p.left_stages + 1):        # G~_{K~}, ..., G~_1
            rotate(yt, stage_first(k), ct, st)
        yt = yt[inst.perm]                           # P1
    return yt


def mvpat(inst, y):
    """x = A^T y for the Givens part of A (Algorithm MvPAt)."""
    p = inst.params
    c, s, ct, st = angles(p)
    size, m = _square_dims(inst)
    xt = np.array(y, dtype=np.float64, copy=True)
    if p.left_stages > 0:
        tmp = np.empty(m)
        tmp[inst.perm] = xt                          # P1^T
        xt = tmp
        for k in range(p.left_stages, 0, -1):        # G~_1^T, ..., G~_{K~}^T
            rotate_t(xt, stage_first(k), ct, st)
        tmp = np.empty(m)
        tmp[inst.perm] = xt                          # P2^T
        xt = tmp
    x = inst.sigma * xt[:size]                       # Sigma^T
    for k in range(1, p.right_stages + 1):           # G_K, ..., G_1
        rotate(x, stage_first(k), c, s)
    return x
