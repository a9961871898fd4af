"""Device generator against the oracle: integer structure bit-exact, values within rounding.

Procedures IGen / OsGen and Eq. (bd8) with the stages of Sec. 4.1-4.2; recipes with one and
with no left stage; sizes that span several 256-row tiles with ragged tails."""

import numpy as np
import pytest

import workloads as W
from gpu_util import csr_from_export, oracle_instance, ulp

pytestmark = pytest.mark.gpu

CASES = [
    dict(m=2048, n=1024, right_stages=1, left_stages=1, kappa=1e2, value_dtype="f64"),
    dict(m=10010, n=5003, right_stages=2, left_stages=1, kappa=1e4, value_dtype="f64", seed=3),
    dict(m=6000, n=3000, right_stages=4, left_stages=1, kappa=1e6, value_dtype="f32", seed=5, xstar_frac=0.02),
    dict(m=4098, n=2049, right_stages=3, left_stages=0, kappa=1e3, value_dtype="f64", seed=7),
    dict(m=3000, n=3000, right_stages=2, left_stages=1, kappa=50.0, value_dtype="bf16", seed=9),
    dict(m=512, n=8, right_stages=1, left_stages=1, kappa=10.0, value_dtype="f64", seed=1, xstar_frac=0.25),
]


@pytest.fixture(scope="module")
def ctx():
    import paper_1503_03520_gb300 as l1
    c = l1.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "m%d_n%d_w%d_l%d_%s" % (c["m"], c["n"], c["right_stages"],
                                                                            c["left_stages"], c["value_dtype"]))
def test_generator_matches_oracle(ctx, case):
    params = W.params(**case)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        m, n = params["m"], params["n"]
        assert inst.nnz == ref.A.nnz
        ex = inst.export()
        A = csr_from_export(ex, m, n)
        # integer structure: bit-exact
        assert np.array_equal(ex["indptr"], ref.A.indptr.astype(np.int64))
        assert np.array_equal(ex["indices"], ref.A.indices.astype(np.int32))
        if params["left_stages"]:
            assert np.array_equal(ex["perm"], ref.perm)
        assert np.array_equal(np.flatnonzero(ex["xstar"]), ref.support)
        # x*: the same arithmetic on both sides
        assert np.array_equal(ex["xstar"], ref.xstar)
        # sigma: exp of the same argument (device and host exp may differ by an ulp)
        assert np.allclose(ex["sigma"], ref.sigma, rtol=4e-16, atol=0)
        # values: FP64 entries agree to rounding; stored types to one unit in the last place
        dt = params["value_dtype"]
        diff = np.abs(A.data - ref.A.data)
        if dt == "f64":
            assert diff.max() <= 1e-14 * np.abs(ref.A.data).max()
        else:
            assert np.all(diff <= ulp(ref.A.data, dt) * 1.0 + 1e-15)
        # b: e by different but equivalent routes (Sec. 4); agreement to kappa * eps
        scale = np.abs(ref.b).max()
        assert np.abs(ex["b"] - ref.b).max() <= 50 * params["kappa"] * 2.2e-16 * scale
        info = inst.info
        assert info["f_star"] == pytest.approx(ref.f_star, rel=1e-12)
        # the oracle reaches A^T b through e = tau A G Sigma^-2 G^T g, whose rounding grows like
        # kappa^2 eps; the device evaluates R Sigma^2 R^T x* + tau g directly
        assert info["lam_max"] == pytest.approx(ref.lam_max, rel=max(1e-10, 10 * params["kappa"] ** 2 * 2.2e-16))
        # transposed storage: the same matrix
        et = inst.export_t()
        At = ref.A.tocsc()
        At.sort_indices()
        assert np.array_equal(et["indptr"], At.indptr.astype(np.int64))
        assert np.array_equal(et["indices"], At.indices.astype(np.int32))
        Ag = A.tocsc()
        Ag.sort_indices()
        assert np.array_equal(et["data"], Ag.data)        # exact transposes of each other
    finally:
        inst.free()


def test_generation_is_deterministic(ctx):
    params = W.params(m=4096, n=2048, right_stages=2, seed=11, value_dtype="f32")
    a = ctx.generate(params)
    b = ctx.generate(params)
    try:
        ea, eb = a.export(), b.export()
        for k in ea:
            assert np.array_equal(ea[k], eb[k]), k
    finally:
        a.free()
        b.free()


def test_invalid_parameters_are_rejected(ctx):
    import paper_1503_03520_gb300 as l1
    for bad in [dict(m=2047, n=1024), dict(m=2048, n=1024, kappa=0.5), dict(m=2048, n=1024, right_stages=9),
                dict(m=2048, n=1024, left_stages=2), dict(m=2048, n=1024, tau=-1.0)]:
        with pytest.raises(l1.L1LSError) as e:
            ctx.generate(W.params(**bad))
        assert e.value.status == 1


IGEN2_CASES = [
    dict(m=1024, n=2048, right_stages=2, left_stages=1, kappa=1e2, value_dtype="f64", seed=11),
    dict(m=3001, n=6007, right_stages=1, left_stages=0, kappa=1e3, value_dtype="f32", seed=12, n_nnz_per_col=5),
    dict(m=4096, n=5000, right_stages=3, left_stages=1, kappa=1e4, value_dtype="bf16", seed=13, n_nnz_per_col=16),
]


@pytest.mark.parametrize("case", IGEN2_CASES, ids=lambda c: "m%d_n%d_%s" % (c["m"], c["n"], c["value_dtype"]))
def test_igen2_generator_matches_oracle(ctx, case):
    """Procedure IGen2 (Sec. 3.2): A = [B, N~] with the square part of Eq. (bd8)."""
    params = W.params(**case)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        m, n = params["m"], params["n"]
        info = inst.info
        assert info["igen2"] == 1 and inst.nnz == ref.A.nnz
        ex = inst.export()
        A = csr_from_export(ex, m, n)
        assert np.array_equal(ex["indptr"], ref.A.indptr.astype(np.int64))
        assert np.array_equal(ex["indices"], ref.A.indices.astype(np.int32))
        assert np.array_equal(np.flatnonzero(ex["xstar"]), ref.support)
        assert ref.support.max() < m
        assert np.array_equal(ex["xstar"], ref.xstar)
        assert len(ex["sigma"]) == m
        # values: the scale of a column of N~ divides by N_i^T e, summed in another order on the
        # device than by the oracle's dot product: agreement to a few FP64 ulps before storage
        dt = params["value_dtype"]
        diff = np.abs(A.data - ref.A.data)
        if dt == "f64":
            assert np.all(diff <= 1e-13 * np.abs(ref.A.data) + 1e-14 * np.abs(ref.A.data).max())
        else:
            assert np.all(diff <= ulp(ref.A.data, dt) + 1e-15)
        scale = np.abs(ref.b).max()
        assert np.abs(ex["b"] - ref.b).max() <= 50 * params["kappa"] * 2.2e-16 * scale
        assert info["f_star"] == pytest.approx(ref.f_star, rel=1e-12)
        # a bound built from the values of N~, whose scale divides by a cancelling dot product
        assert info["lipschitz"] == pytest.approx(ref.lipschitz, rel=1e-11)
        assert info["lam_max"] == pytest.approx(ref.lam_max, rel=max(1e-10, 10 * params["kappa"] ** 2 * 2.2e-16))
        et = inst.export_t()
        At = ref.A.tocsc()
        At.sort_indices()
        assert np.array_equal(et["indptr"], At.indptr.astype(np.int64))
        assert np.array_equal(et["indices"], At.indices.astype(np.int32))
        if dt == "f64":
            # Eq. (bd10): A^T (b - A x*) = tau g with |g_i| <= 1, g_i = sign(x*_i) on the support
            tau = params["tau"]
            gt = A.T @ (ex["b"] - A @ ex["xstar"]) / tau
            S = ref.support
            assert np.abs(gt[S] - np.sign(ex["xstar"][S])).max() <= 1e-9 * params["kappa"]
            assert np.abs(gt).max() <= 1.0 + 1e-9 * params["kappa"]
    finally:
        inst.free()


def test_igen2_rejects_bad_column_counts(ctx):
    import paper_1503_03520_gb300 as l1
    for d in (0, 65):
        with pytest.raises(l1.L1LSError) as e:
            ctx.generate(W.params(m=256, n=512, n_nnz_per_col=d))
        assert e.value.status == 1


def test_sec89_generator_matches_oracle(ctx):
    """Sec. 8.9's instance shape (alternating singular values, x* of -1e4 and 0.1) on the device."""
    params = dict(W.sec89(13, value_dtype="f64"), xstar_frac=2.0 ** -6)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        ex = inst.export()
        assert np.array_equal(ex["indptr"], ref.A.indptr.astype(np.int64))
        assert np.array_equal(ex["indices"], ref.A.indices.astype(np.int32))
        assert np.array_equal(ex["sigma"], ref.sigma)
        assert np.array_equal(ex["xstar"], ref.xstar)
        A = csr_from_export(ex, params["m"], params["n"])
        assert np.abs(A.data - ref.A.data).max() <= 1e-14 * np.abs(ref.A.data).max()
        assert inst.info["lipschitz"] == ref.lipschitz == 1e4
        assert inst.info["f_star"] == pytest.approx(ref.f_star, rel=1e-12)
        assert np.abs(ex["b"] - ref.b).max() <= 1e-12 * np.abs(ref.b).max()
    finally:
        inst.free()


@pytest.mark.parametrize("m,n,w,frac,kappa", [(8198, 4099, 2, 0.1, 1e3), (2000, 1000, 3, 1.0, 30.0),
                                             (6002, 3001, 8, 0.37, 1e4), (64, 33, 1, 0.01, 10.0)])
def test_osgen3_generator_matches_oracle(ctx, m, n, w, frac, kappa):
    """Procedure OsGen3 (Sec. 6) on the device: the same support as the oracle (both sides sort
    FP64 |x| values that differ at most by the ulp of exp in sigma, far below the gaps between
    neighbouring |x_i|), x* and b to 1e-13, f*; kappa_rho of Eq. (bd12) on the device against
    the oracle's at thresholds between distinct sigma_i^2 and outside the spectrum, to the
    rounding of R^T x* amplified by kappa_rho itself."""
    from oracle.generator import kappa_rho
    params = W.params(m=m, n=n, right_stages=w, left_stages=1, kappa=kappa, value_dtype="f64", seed=11,
                      xstar_mode=2, gamma=100.0, xstar_frac=frac)
    ref = oracle_instance(params)
    inst = ctx.generate(params)
    try:
        ex = inst.export()
        assert np.allclose(ex["sigma"], ref.sigma, rtol=4e-16, atol=0)
        assert np.array_equal(np.flatnonzero(ex["xstar"]), np.flatnonzero(ref.xstar))
        assert np.allclose(ex["xstar"], ref.xstar, rtol=1e-13, atol=0)
        assert inst.info["s"] == np.count_nonzero(ref.xstar)
        assert np.abs(ex["b"] - ref.b).max() <= 1e-12 * np.abs(ref.b).max()
        assert inst.info["f_star"] == pytest.approx(ref.f_star, rel=1e-12)
        s2 = np.unique(ref.sigma ** 2)
        k = len(s2) // 3
        for rho in (0.0, 0.5 * s2[0], 0.5 * (s2[k] + s2[k + 1]), 0.5 * (s2[-2] + s2[-1]), 2.0 * s2[-1]):
            want = kappa_rho(ref.sigma, ref.R, ref.xstar, rho)
            got = inst.kappa_rho(rho)
            if np.isinf(want):
                assert np.isinf(got)
            else:
                # ||P_rho x*|| = ||x*|| / kappa_rho: the rounding of R^T x* (about (w + 1) eps ||x*||
                # per entry, different orders of operations on the two sides) relative to it
                assert got == pytest.approx(want, rel=1e-12 + 8 * (w + 1) * 2.2e-16 * want)
    finally:
        inst.free()


def test_kappa_rho_rejections(ctx):
    import paper_1503_03520_gb300 as l1
    inst = ctx.generate(W.params(m=300, n=600, value_dtype="f64"))   # IGen2
    try:
        with pytest.raises(l1.L1LSError) as e:
            inst.kappa_rho(1.0)
        assert e.value.status == 1
    finally:
        inst.free()
    with pytest.raises(l1.L1LSError) as e:
        ctx.generate(W.params(m=300, n=600, xstar_mode=2))
    assert e.value.status == 1
