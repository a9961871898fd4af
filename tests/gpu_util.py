"""Helpers for the GPU parity tests (reference-side conversions written from their
definitions; nothing here calls the CUDA path)."""

import numpy as np
import scipy.sparse as sp

from oracle.generator import GenParams, generate


def oracle_instance(params):
    return generate(GenParams.from_dict(params))


def round_bf16(a):
    """Round FP64 values to bfloat16 (round to nearest even) through FP32, as doubles."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


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
