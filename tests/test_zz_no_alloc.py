"""The allocation-free A^T y (l1ls_rmatvec_noalloc) against l1ls_rmatvec.

Some callers cannot allocate device memory (graph capture, real-time loops, fixed budgets);
the variant keeps its scratch in a fixed array inside the library.  Collected last so that a
run stopping at the first failure has already run every other test.  Passes alone in a fresh
process and after the other tests (the first call on a device sets the array up)."""

import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_rmatvec_matches_rmatvec_twice(dt):
    import torch

    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        inst = ctx.generate(W.params(m=20002, n=10001, right_stages=2, kappa=1e3, value_dtype=dt, seed=8))
        vt = torch.float64 if dt == "f64" else torch.float32
        for call in range(2):
            y = torch.tensor(W.random_vector(inst.m, 10 + call), dtype=vt, device="cuda")
            ref = inst.rmatvec(y)
            out = torch.full((inst.n,), float("nan"), dtype=vt, device="cuda")
            inst.rmatvec_noalloc(y, out)
            torch.cuda.synchronize()
            tol = 1e-12 if dt == "f64" else 1e-5
            assert torch.allclose(out, ref, rtol=tol, atol=tol), call
        inst.free()
    finally:
        ctx.close()


def test_noalloc_rejects_too_many_rows():
    import torch

    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        inst = ctx.generate(W.params(m=2 ** 21 + 2, n=2 ** 20, right_stages=1, value_dtype="f32"))
        y = torch.zeros(inst.m, dtype=torch.float32, device="cuda")
        x = torch.zeros(inst.n, dtype=torch.float32, device="cuda")
        with pytest.raises(l1.L1LSError) as e:
            inst.rmatvec_noalloc(y, x)
        assert e.value.status == 1 and "1048576" in str(e.value)
        inst.free()
    finally:
        ctx.close()
