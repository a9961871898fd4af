"""Batched FISTA along tau paths (the tau study of Sec. 8.8 as a workload) against the oracle.

Each instance's path is also solved by the oracle's FISTA on the stored problem (values
rounded once to FP32), warm-started the same way (the next tau starts from the iterate one
prox-gradient step past the certified one).  An instance solved alone and inside a batch must
give identical results (every reduction order depends only on the instance)."""

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance, stored_values
from oracle import solvers

pytestmark = pytest.mark.gpu

SIZES = [(1024, 512), (2000, 1000), (4096, 2048), (6002, 3001), (10000, 5000), (16384, 8192)]
NTAU = 4


def _params(k, m, n):
    return W.params(m=m, n=n, seed=40 + k, kappa=10.0 ** (2 + 0.2 * k), right_stages=2, left_stages=1,
                    xstar_frac=0.02, value_dtype="f32")


def _taus(lam_max):
    return [0.9 * lam_max * 10.0 ** (-j / 1.5) for j in range(NTAU)]


@pytest.fixture(scope="module")
def setup():
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    params = [_params(k, m, n) for k, (m, n) in enumerate(SIZES)]
    refs = [oracle_instance(p) for p in params]
    insts = [ctx.generate(p) for p in params]
    taus = np.array([_taus(r.lam_max) for r in refs])
    yield ctx, params, refs, insts, taus
    for i in insts:
        i.free()
    ctx.close()


def test_batch_path_matches_oracle(setup):
    import paper_1503_03520_gb300 as l1
    ctx, params, refs, insts, taus = setup
    batch = l1.Batch(ctx, insts)
    xs = [np.zeros(i.n) for i in insts]
    res = batch.solve_path(taus, x_out=xs, tol=1e-6, max_iter=100000, restart=1)
    sch = batch.schedule()
    assert (sch["block"], sch["entries_per_lane"]) in sch["candidates"]
    for k, ref in enumerate(refs):
        A = stored_values(ref.A, "f32")
        b = ref.b.astype(np.float32).astype(np.float64)
        x0 = None
        for j in range(NTAU):
            r = res[k][j]
            assert r["status"] == 0 and r["rel_gap"] <= 1e-6, (k, j, r)
            o = solvers.fista(A, b, taus[k, j], 1.0, 1e-6, 100000, x0=x0, restart=True)
            # restarts are decided on rounded sums, so the paths may part after a restart
            assert abs(r["iters"] - o["iters"]) <= max(5, 0.15 * o["iters"]), (k, j, r["iters"], o["iters"])
            assert abs(r["f"] - o["P"]) <= 2e-6 * o["P"], (k, j)
            x0 = o["x_next"]
        # the certificate of the returned solution, recomputed by the oracle on the stored problem
        P, D, gap, rel = solvers.certificate(A, b, taus[k, -1], xs[k])
        assert rel <= 1e-5
    batch.free()


def test_alone_equals_in_the_mix(setup):
    import paper_1503_03520_gb300 as l1
    ctx, params, refs, insts, taus = setup
    full = l1.Batch(ctx, insts)
    xs_full = [np.zeros(i.n) for i in insts]
    res_full = full.solve_path(taus, x_out=xs_full, tol=1e-6, max_iter=100000, restart=1)
    full.free()
    for k in (0, 3, 5):
        alone = l1.Batch(ctx, [insts[k]])
        x_alone = [np.zeros(insts[k].n)]
        res_alone = alone.solve_path(taus[k:k + 1], x_out=x_alone, tol=1e-6, max_iter=100000, restart=1)
        alone.free()
        for j in range(NTAU):
            a, f = res_alone[0][j], res_full[k][j]
            assert (a["iters"], a["f"], a["gap"], a["rel_gap"]) == (f["iters"], f["f"], f["gap"], f["rel_gap"])
        assert np.array_equal(x_alone[0], xs_full[k])


def test_batch_rejects_mixed_or_unpaired(setup):
    import paper_1503_03520_gb300 as l1
    ctx, params, refs, insts, taus = setup
    plain = ctx.generate(W.params(m=512, n=256, left_stages=0, value_dtype="f32"))
    f64 = ctx.generate(W.params(m=512, n=256, value_dtype="f64"))
    try:
        for bad in ([insts[0], plain], [insts[0], f64]):
            with pytest.raises(l1.L1LSError) as e:
                l1.Batch(ctx, bad)
            assert e.value.status == 1
    finally:
        plain.free()
        f64.free()


def test_bounded_barrier_expires_and_the_context_survives(setup):
    """Failure detection without a GPU fault: the self-test's barrier never fills, every block's
    bounded wait runs out and the kernel returns; the status reaches the host and the next solve
    runs normally."""
    import paper_1503_03520_gb300 as l1
    ctx, params, refs, insts, taus = setup
    batch = l1.Batch(ctx, insts[:2])
    try:
        st, msg, sec = batch.barrier_selftest(max_polls=1 << 12)
        assert st == 3 and "barrier expired" in msg
        assert sec < 30.0
        res = batch.solve_path(taus[:2], tol=1e-6, max_iter=100000, restart=1)
        assert all(r["status"] == 0 for rr in res for r in rr)
    finally:
        batch.free()


def test_batch_with_more_segments_than_warps():
    """Six C2-recipe instances at n = 2^19: 6 x 1024 segments of 16 tiles per phase against at
    most 152 SMs x 24 warps = 3648 warps, so warps draw several segments from the phase counters
    and run the staged traversal over several tiles each.  Both sides run at most 30 FISTA
    iterations at each of two tau (the caps end every tau) from x = 0 with the same warm start;
    the batch's float-float products (about 44 bits) against the oracle's FP64 FISTA on the
    stored FP32 problem.  The device's FP32 values of A may differ from the oracle's rounding of
    its FP64 values by one unit (the generator's value parity), so x, whose components along the
    weak singular directions move by up to about kappa times such a perturbation, is compared
    within 1e-6 max|x| for kappa <= 1e3 and kappa / 1e3 times that above; f, insensitive to it,
    within 1e-9.  (Measured at n = 2^19: 4e-12 at kappa 1e2, 7e-5 at kappa 1e4 with
    max|x| = 51; the same x with segments of 8 or 16 tiles.)  One instance alone equals itself in
    the batch bit for bit."""
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    insts = []
    try:
        params = [W.c2_scaled(19, seed=70 + k, kappa=10.0 ** (2 + 0.5 * k)) for k in range(6)]
        refs = [oracle_instance(p) for p in params]
        insts = [ctx.generate(p) for p in params]
        # at these tau 30 iterations leave gaps far above the tolerance, so the caps end both
        # sides' runs (a gap rounded to <= 0 would end a run at tol = 0)
        taus = np.array([[0.3 * r.lam_max, 0.1 * r.lam_max] for r in refs])
        batch = l1.Batch(ctx, insts)
        xs = [np.zeros(i.n) for i in insts]
        res = batch.solve_path(taus, x_out=xs, tol=1e-12, max_iter=30, restart=0)
        batch.free()
        for k, ref in enumerate(refs):
            A = stored_values(ref.A, "f32")
            b = ref.b.astype(np.float32).astype(np.float64)
            x0 = None
            for j in range(2):
                o = solvers.fista(A, b, taus[k, j], 1.0, 1e-12, 30, x0=x0)
                assert o["status"] == 5
                r = res[k][j]
                assert r["status"] == 5 and r["iters"] == 30, (k, j, r)
                assert abs(r["f"] - o["P"]) <= 1e-9 * o["P"], (k, j, r["f"], o["P"])
                x0 = o["x_next"]
            kappa = params[k]["kappa"]
            assert np.abs(xs[k] - o["x"]).max() <= 1e-6 * max(1.0, kappa / 1e3) * max(1.0, np.abs(o["x"]).max()), k
        alone = l1.Batch(ctx, [insts[4]])
        x_alone = [np.zeros(insts[4].n)]
        res_alone = alone.solve_path(taus[4:5], x_out=x_alone, tol=1e-12, max_iter=30, restart=0)
        alone.free()
        for j in range(2):
            a, f = res_alone[0][j], res[4][j]
            assert (a["iters"], a["f"], a["gap"]) == (f["iters"], f["f"], f["gap"])
        assert np.array_equal(x_alone[0], xs[4])
    finally:
        for i in insts:
            i.free()
        ctx.close()
