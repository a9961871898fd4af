"""The largest instances of the C2 recipe, checked by properties that hold at any size.

Stored: n = 2^27 (m = 2^28, nnz = 2^30 - 8, about 40 GB) is the largest n whose nonzero count
fits the 32-bit offsets; n = 2^28 (nnz = 2^31 - 8) is rejected with EINVAL.  Matrix-free:
n = 2^29 (m = 2^30, O(m + n) memory).  Properties: the adjoint identity y^T (A x) = (A^T y)^T x
with the library's two products on random vectors, and the generator's optimum x*
certifying at once (its duality gap is within the tolerance, so FISTA stops after zero
iterations), which exercises b, e and both products together at full size."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1503_03520_gb300 as l1
    c = l1.Context(0)
    yield c
    c.close()


def _adjoint_gap(inst, seed):
    """|y^T A x - (A^T y)^T x| relative to |y|^T |A| |x|-sized scales (FP32 products)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(inst.n, generator=g, device="cuda", dtype=torch.float32)
    y = torch.randn(inst.m, generator=g, device="cuda", dtype=torch.float32)
    ax = inst.matvec(x)
    aty = inst.rmatvec(y)
    lhs = float(torch.dot(y.double(), ax.double()))
    rhs = float(torch.dot(aty.double(), x.double()))
    scale = float(torch.linalg.vector_norm(y.double()) * torch.linalg.vector_norm(ax.double()))
    return abs(lhs - rhs) / scale


@pytest.mark.parametrize("log2n,matrix_free", [(27, 0), (29, 1)])
def test_largest_instances(ctx, log2n, matrix_free):
    params = dict(W.c2_scaled(log2n), matrix_free=matrix_free)
    inst = ctx.generate(params)
    try:
        n = inst.n
        assert inst.m == 2 * n and 7.5 * n <= inst.nnz <= 8 * n
        assert _adjoint_gap(inst, 1) <= 1e-5
        xs = inst.xstar()
        _, r = inst.solve_fista(x0=xs, tau=1.0, tol=W.C2_TOL, max_iter=4)
        assert r["status"] == 0 and r["iters"] == 0, r
        assert r["f"] == pytest.approx(inst.info["f_star"], rel=1e-6)
    finally:
        inst.free()


def test_nnz_beyond_32_bit_offsets_is_rejected(ctx):
    import paper_1503_03520_gb300 as l1
    with pytest.raises(l1.L1LSError) as e:
        ctx.generate(W.c2_scaled(28))
    assert e.value.status == 1 and ("32-bit" in str(e.value) or "2^31" in str(e.value))
