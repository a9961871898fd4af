"""The allocation-free A^T y (l1ls_rmatvec_noalloc) against l1ls_rmatvec and the oracle.

Some callers cannot allocate device memory: real-time loops that must not stall on the
device-wide synchronisation of cudaMalloc / cudaFree, and host applications that own all
device memory and hand libraries none.  The variant keeps its one m-vector of scratch in a
fixed array inside the library (m <= 2^20).  It launches the same gather and product kernels
as l1ls_rmatvec on the same data, so the two results are equal bit for bit.

Collected last so that a run stopping at the first failure has already run every other test.
Passes alone in a fresh process and after the other tests (the first call on a device looks
the array up)."""

import ctypes

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance, stored_values

pytestmark = pytest.mark.gpu

MAX_ROWS = 2 ** 20


def _check_against_oracle(A, y, x, dt):
    """Entry-wise rounding bound of a sum of at most kmax products (as in the product tests)."""
    eps = 2.3e-16 if dt == "f64" else 6e-8
    kmax = 4 * 2 + 2
    ref = A.T @ y
    bound = kmax * eps * (abs(A).T @ np.abs(y)) + (eps * np.abs(ref) if dt != "f64" else 0) + 1e-300
    assert np.all(np.abs(x - ref) <= bound)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_rmatvec_matches_rmatvec_twice(dt):
    import torch

    import paper_1503_03520_gb300 as l1
    params = W.params(m=20002, n=10001, right_stages=2, kappa=1e3, value_dtype=dt, seed=8)
    ref = oracle_instance(params)
    A = stored_values(ref.A, dt)
    ctx = l1.Context(0)
    try:
        inst = ctx.generate(params)
        vt = torch.float64 if dt == "f64" else torch.float32
        for call in range(2):
            y = torch.tensor(W.random_vector(inst.m, 10 + call), dtype=vt, device="cuda")
            want = inst.rmatvec(y)
            out = torch.full((inst.n,), float("nan"), dtype=vt, device="cuda")
            inst.rmatvec_noalloc(y, out)
            torch.cuda.synchronize()
            assert torch.equal(out, want), call
            _check_against_oracle(A, y.double().cpu().numpy(), out.double().cpu().numpy(), dt)
        inst.free()
    finally:
        ctx.close()


def test_noalloc_at_the_row_limit():
    """m = 2^20 exactly, the largest instance the fixed array serves."""
    import torch

    import paper_1503_03520_gb300 as l1
    params = W.params(m=MAX_ROWS, n=MAX_ROWS // 2, right_stages=2, kappa=1e3, value_dtype="f32", seed=9)
    ref = oracle_instance(params)
    A = stored_values(ref.A, "f32")
    ctx = l1.Context(0)
    try:
        inst = ctx.generate(params)
        assert inst.m == MAX_ROWS
        for call in range(2):
            y = torch.tensor(W.random_vector(inst.m, 30 + call), dtype=torch.float32, device="cuda")
            want = inst.rmatvec(y)
            out = torch.full((inst.n,), float("nan"), dtype=torch.float32, device="cuda")
            inst.rmatvec_noalloc(y, out)
            torch.cuda.synchronize()
            assert torch.equal(out, want), call
            _check_against_oracle(A, y.double().cpu().numpy(), out.double().cpu().numpy(), "f32")
        inst.free()
    finally:
        ctx.close()


def test_noalloc_rejects_too_many_rows():
    import torch

    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        inst = ctx.generate(W.params(m=MAX_ROWS + 2, n=MAX_ROWS // 2 + 1, right_stages=1, value_dtype="f32"))
        y = torch.zeros(inst.m, dtype=torch.float32, device="cuda")
        x = torch.zeros(inst.n, dtype=torch.float32, device="cuda")
        with pytest.raises(l1.L1LSError) as e:
            inst.rmatvec_noalloc(y, x)
        assert e.value.status == 1 and "1048576" in str(e.value)
        inst.free()
    finally:
        ctx.close()


def test_noalloc_refuses_host_pointers():
    """Through the C ABI directly: host buffers are refused with EINVAL before anything runs."""
    import torch

    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        inst = ctx.generate(W.params(m=2048, n=1024, right_stages=1, value_dtype="f32"))
        yh = np.zeros(inst.m, np.float32)
        xh = np.zeros(inst.n, np.float32)
        yd = torch.zeros(inst.m, dtype=torch.float32, device="cuda")
        xd = torch.zeros(inst.n, dtype=torch.float32, device="cuda")
        for yp, xp in ((yh.ctypes.data, xd.data_ptr()), (yd.data_ptr(), xh.ctypes.data)):
            st = l1.lib.l1ls_rmatvec_noalloc(inst._h, ctypes.c_void_p(yp), l1.F32, ctypes.c_void_p(xp), None)
            assert st == 1
            assert "device pointers" in l1.lib.l1ls_last_error().decode()
        inst.free()
    finally:
        ctx.close()
