"""Helpers for the GPU parity tests (reference-side conversions written from their
definitions; nothing here calls the CUDA path)."""

import numpy as np
import scipy.sparse as sp

from oracle.generator import GenParams, generate


def oracle_instance(params):
    return generate(GenParams.from_dict(params))


def round_bf16(a):
    """Round FP64 values directly to bfloat16 (8 significant bits, round half to even)."""
    v = np.asarray(a, dtype=np.float64)
    out = np.zeros_like(v)
    nz = v != 0
    e = np.floor(np.log2(np.abs(v[nz])))
    q = np.exp2(e - 7)                  # spacing of bf16 numbers in the binade of v
    out[nz] = np.round(v[nz] / q) * q   # exact scaling; np.round rounds half to even
    return out


def stored_values(A, dtype):
    """The oracle's matrix with its values rounded once to the storage type."""
    B = A.copy().astype(np.float64)
    if dtype == "f32":
        B.data = B.data.astype(np.float32).astype(np.float64)
    elif dtype == "bf16":
        B.data = round_bf16(B.data)
    return B


def ulp(x, dtype):
    x = np.abs(np.asarray(x, dtype=np.float64))
    if dtype == "f64":
        return np.spacing(x)
    if dtype == "f32":
        return np.spacing(x.astype(np.float32)).astype(np.float64)
    # bf16: 8 significand bits
    e = np.floor(np.log2(np.maximum(x, 1e-300)))
    return 2.0 ** (e - 7)


def csr_from_export(ex, m, n):
    return sp.csr_matrix((ex["data"], ex["indices"], ex["indptr"]), shape=(m, n))
