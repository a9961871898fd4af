"""Serving loop on the device: results alone equal results in the mix, admission by footprint,
cancellation, and agreement with the oracle."""

import time

import numpy as np
import pytest

import workloads as W
from gpu_util import oracle_instance
from oracle import solvers

pytestmark = pytest.mark.gpu

REQS = [
    (dict(m=2048, n=1024, kappa=1e2, seed=1, right_stages=1, left_stages=1, value_dtype="f64"), "fista", 0.5),
    (dict(m=4000, n=2000, kappa=3e2, seed=2, right_stages=2, left_stages=1, value_dtype="f32"), "fista", 0.2),
    (dict(m=1024, n=2048, kappa=1e2, seed=3, right_stages=2, left_stages=1, value_dtype="f64"), "fista", 0.3),
    (dict(m=3000, n=1500, kappa=1e3, seed=4, right_stages=2, left_stages=0, value_dtype="f64"), "pdncg", 0.1),
    (dict(m=8192, n=4096, kappa=1e2, seed=5, right_stages=2, left_stages=1, value_dtype="f32"), "pdncg", 0.05),
    (dict(m=2000, n=3001, kappa=50.0, seed=6, right_stages=1, left_stages=0, value_dtype="f32",
          n_nnz_per_col=4), "fista", 1.0),
    (dict(m=16384, n=8192, kappa=1e2, seed=7, right_stages=2, left_stages=1, value_dtype="bf16"), "fista", 0.5),
    (dict(m=512, n=256, kappa=10.0, seed=8, right_stages=1, left_stages=1, value_dtype="f64"), "pdncg", 0.8),
    # A by its factors (Algorithms MvPA / MvPAt): pdNCG and FISTA on matrix-free instances
    (dict(m=6000, n=3000, kappa=1e3, seed=9, right_stages=2, left_stages=1, value_dtype="f32", matrix_free=1),
     "pdncg", 0.1),
    (dict(m=5000, n=2500, kappa=1e2, seed=10, right_stages=2, left_stages=0, value_dtype="f32", matrix_free=1),
     "fista", 0.3),
]
OPTS = dict(tol=1e-6, max_iter=20000, restart=1)


def _params(d):
    return W.params(xstar_frac=0.02, **d)


def _solve_alone(l1, ctx, params, method, frac):
    inst = ctx.generate(params)
    try:
        tau = frac * inst.info["lam_max"]
        solve = inst.solve_fista if method == "fista" else inst.solve_pdncg
        x, r = solve(tau=tau, **OPTS)
        return x, r, tau
    finally:
        inst.free()


def _wait(ctx, t, n, limit_s=120.0):
    t0 = time.time()
    while True:
        out = ctx.poll(t, wait_ms=200, n=n)
        if out is not None:
            return out
        assert time.time() - t0 < limit_s, "request did not finish"


def test_results_alone_equal_results_in_the_mix():
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        ctx.serve_config(slots=6)
        tickets = [ctx.submit(_params(p), method=m, tau=-frac, **OPTS) for p, m, frac in REQS]
        served = [_wait(ctx, t, p["n"]) for t, (p, m, frac) in zip(tickets, REQS)]
        st = ctx.serve_stats()
        assert st["completed"] == len(REQS) and st["running"] == 0
        assert st["peak_running"] >= 2                     # requests overlapped
        assert st["peak_reserved_bytes"] <= st["capacity_bytes"]
        for (p, m, frac), (status, res, x) in zip(REQS, served):
            if m == "fista" or p["value_dtype"] == "f64" or p.get("matrix_free"):
                assert status == 0 and res["rel_gap"] <= 1e-6, (p, res)
            assert res["latency_s"] >= res["queue_s"] >= 0.0
            xa, ra, tau = _solve_alone(l1, ctx, _params(p), m, frac)
            # the same arithmetic alone and in the mix: bit-identical
            assert np.array_equal(x, xa)
            assert (res["iters"], res["f"], res["gap"]) == (ra["iters"], ra["f"], ra["gap"])
    finally:
        ctx.close()


def test_served_solutions_match_the_oracle():
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        for p, m, frac in (REQS[0], REQS[2], REQS[3]):
            params = _params(p)
            ref = oracle_instance(params)
            tau = frac * ref.lam_max
            t = ctx.submit(params, method=m, tau=tau, **OPTS)
            status, res, x = _wait(ctx, t, p["n"])
            assert status == 0
            P, D, gap, rel = solvers.certificate(ref.A, ref.b, tau, x)
            assert rel <= 2e-6
            o = solvers.fista(ref.A, ref.b, tau, ref.lipschitz, 1e-9, 200000, restart=True)
            assert abs(P - o["P"]) <= 2e-6 * o["P"]
    finally:
        ctx.close()


def test_admission_by_footprint_and_cancel():
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        p = _params(REQS[6][0])
        fp = l1.footprint(p)
        ctx.serve_config(slots=8, capacity_bytes=int(2.5 * fp))
        # a request larger than the whole capacity is refused at once
        big = dict(p, m=4 * p["m"], n=4 * p["n"])
        with pytest.raises(l1.L1LSError) as e:
            ctx.submit(big, tau=-0.5, **OPTS)
        assert e.value.status == 7
        tickets = [ctx.submit(p, tau=-0.5, **OPTS) for _ in range(6)]
        ctx.cancel(tickets[-1])
        outs = [_wait(ctx, t, p["n"]) for t in tickets]
        assert outs[-1][0] == 9                       # cancelled before it ran (or while running)
        for status, res, x in outs[:-1]:
            assert status == 0
        # identical requests, identical results
        for status, res, x in outs[1:-1]:
            assert np.array_equal(x, outs[0][2])
        st = ctx.serve_stats()
        assert st["peak_running"] <= 2                 # two footprints fit, three do not
        assert st["peak_reserved_bytes"] <= st["capacity_bytes"]
        with pytest.raises(l1.L1LSError) as e:
            ctx.poll(tickets[0], n=p["n"])             # released ticket
        assert e.value.status == 8
    finally:
        ctx.close()


def test_footprint_bounds_the_device_memory_of_a_request():
    import paper_1503_03520_gb300 as l1
    ctx = l1.Context(0)
    try:
        for p, m, frac in REQS:
            params = _params(p)
            inst = ctx.generate(params)
            try:
                solve = inst.solve_fista if m == "fista" else inst.solve_pdncg
                solve(tau=frac * inst.info["lam_max"], tol=1e-3, max_iter=50)
                assert inst.refresh_info()["device_bytes"] <= l1.footprint(params, m), (p, m)
            finally:
                inst.free()
    finally:
        ctx.close()
