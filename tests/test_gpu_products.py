"""Products y = A x and x = A^T y (Algorithms MvPA / MvPAt; A stored) against the oracle."""

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance, stored_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1503_03520_gb300 as l1
    c = l1.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", [(2048, 1024, 1), (20002, 10001, 2), (9000, 4500, 4), (6002, 3001, 8)])
def test_products_match_oracle(ctx, dt, shape):
    """Entry-wise rounding bounds against the oracle's A.  In paired storage a tile of 32 row
    pairs holds about 2 (w + 1) entries per pair, so w = 8 (and w >= 2 with FP64 values) makes
    tiles longer than one shared-memory stage: those are staged in several pieces."""
    import torch
    m, n, w = shape
    params = W.params(m=m, n=n, right_stages=w, kappa=1e3, value_dtype=dt, seed=2)
    ref = oracle_instance(params)
    A = stored_values(ref.A, dt)
    absA = abs(A)
    inst = ctx.generate(params)
    try:
        x = W.random_vector(n, 1)
        y = W.random_vector(m, 2)
        vt = torch.float64 if dt == "f64" else torch.float32
        xd = torch.tensor(x, dtype=vt, device="cuda")
        yd = torch.tensor(y, dtype=vt, device="cuda")
        xr = xd.double().cpu().numpy()
        yr = yd.double().cpu().numpy()
        ax = inst.matvec(xd).double().cpu().numpy()
        aty = inst.rmatvec(yd).double().cpu().numpy()
        torch.cuda.synchronize()
        eps = 2.3e-16 if dt == "f64" else 6e-8
        kmax = 4 * w + 2
        bound_y = kmax * eps * (absA @ np.abs(xr)) + (eps * np.abs(A @ xr) if dt != "f64" else 0) + 1e-300
        bound_x = kmax * eps * (absA.T @ np.abs(yr)) + (eps * np.abs(A.T @ yr) if dt != "f64" else 0) + 1e-300
        assert np.all(np.abs(ax - A @ xr) <= bound_y)
        assert np.all(np.abs(aty - A.T @ yr) <= bound_x)
        # host buffers through the same entry points (staged by the library)
        ax_h = inst.matvec(x.astype(np.float64 if dt == "f64" else np.float32))
        assert np.array_equal(ax_h.astype(np.float64), ax)
        aty_h = inst.rmatvec(y.astype(np.float64 if dt == "f64" else np.float32))
        assert np.array_equal(aty_h.astype(np.float64), aty)
    finally:
        inst.free()


def test_empty_rows_and_edge_sizes(ctx):
    """No left stage: rows n..m-1 of A are empty (A = Sigma G^T, Sec. 8)."""
    import torch
    params = W.params(m=3000, n=1001, right_stages=3, left_stages=0, kappa=10.0, value_dtype="f64")
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        x = torch.ones(1001, dtype=torch.float64, device="cuda")
        y = inst.matvec(x).cpu().numpy()
        assert np.array_equal(y[1001:], np.zeros(3000 - 1001))
        assert np.allclose(y, ref.A @ np.ones(1001), rtol=1e-14, atol=1e-14)
    finally:
        inst.free()
