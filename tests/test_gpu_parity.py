"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Integer states bit-exact; theta_N^m within the tolerance
|d| <= 1e-4 max(|theta_oracle|, theta_scale) (theta_scale = the at-the-money
caplet of the same maturity), FP64 paths far tighter."""
import numpy as np
import pytest

import oracle as O
import oracle_par
from paper_1408_5526_gb300 import inputs

JK = inputs.joe_kuo_table()
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    rqmc.load()
    return rqmc


def _to_np(t):
    import torch
    if t.dtype == torch.int64:
        return t.cpu().numpy().view(np.uint64)
    return t.cpu().numpy()


# ------------------------------------------------------------------ point stream
@pytest.mark.parametrize("seq,s", [(O.HALTON_RS, 8), (O.RASRAP, 8), (O.RASRAP, 360), (O.SOBOL_DS, 40),
                                   (O.SOBOL_LMS, 40), (O.SOBOL_LMS, 360),
                                   (O.SOBOL_DS, 360), (O.PHILOX, 10)])
@pytest.mark.parametrize("offset,N", [(0, 3001), (12345, 3001), (0, 3000), (12344, 4096)])
def test_points_raw_bit_exact(R, seq, s, offset, N):
    """N and the offset multiples of 8 take the run kernel (runs of 8 consecutive points per
    lane, vector stores), the others the per-point kernel."""
    M = 3
    gpu = _to_np(R.rqmc_points(s, N, M, seq, 7, offset=offset, transform="raw"))
    ora = O.Sequence(seq, s, M, 7, joe_kuo=JK).points(N, offset, transform=O.RAW)
    assert gpu.shape == ora.shape
    assert np.array_equal(gpu, ora)


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
@pytest.mark.parametrize("prec,transform", [("fp32", "normal"), ("fp64", "uniform"), ("fp32", "raw")])
def test_points_plan_matches_one_shot(R, seq, prec, transform):
    """The point-stream plan (tables built once) writes exactly what rqmc_points writes,
    on every execute, with a point offset."""
    N, M, s, off = 2049, 2, 24, 777
    ref = _to_np(R.rqmc_points(s, N, M, seq, 9, offset=off, prec=prec, transform=transform))
    p = R.Plan.points(s, N, M, seq, 9, prec=prec, transform=transform, offset=off)
    assert p.output_size() == M * s * N and p.launches() == 1
    a = _to_np(p.execute())
    b = _to_np(p.execute())
    p.close()
    assert a.shape == ref.shape and np.array_equal(a, ref) and np.array_equal(b, ref)


@pytest.mark.parametrize("seq", [O.HALTON_RS, O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
@pytest.mark.parametrize("N", [2500, 2504])
def test_points_fp64_uniform_and_normal(R, seq, N):
    M, s = 2, 16
    q = O.Sequence(seq, s, M, 11, joe_kuo=JK)
    u = _to_np(R.rqmc_points(s, N, M, seq, 11, prec="fp64", transform="uniform"))
    np.testing.assert_allclose(u, q.points(N, transform=O.UNIFORM), rtol=0, atol=4e-16)
    z = _to_np(R.rqmc_points(s, N, M, seq, 11, prec="fp64", transform="normal"))
    zo = q.points(N, transform=O.NORMAL)
    np.testing.assert_allclose(z, zo, rtol=0, atol=2e-14 * np.maximum(1, np.abs(zo)).max())


@pytest.mark.parametrize("seq", [O.HALTON_RS, O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
@pytest.mark.parametrize("N", [2500, 2504])
def test_points_fp32_uniform_and_normal(R, seq, N):
    M, s = 2, 40
    q = O.Sequence(seq, s, M, 13, joe_kuo=JK)
    u = _to_np(R.rqmc_points(s, N, M, seq, 13, prec="fp32", transform="uniform"))
    uo = q.points(N, transform=O.UNIFORM)
    np.testing.assert_allclose(u, uo, rtol=4e-7, atol=1e-30)
    z = _to_np(R.rqmc_points(s, N, M, seq, 13, prec="fp32", transform="normal")).astype(np.float64)
    zo = q.points(N, transform=O.NORMAL)
    assert np.max(np.abs(z - zo) / np.maximum(1.0, np.abs(zo))) < 1e-6


def test_points_halton_tail_normals_fp32(R):
    # Halton numerators reach q ~ 1e-19: the FP32 normal keeps its relative accuracy there
    N, M, s = 4096, 4, 8
    q = O.Sequence(O.RASRAP, s, M, 5)
    z = _to_np(R.rqmc_points(s, N, M, O.RASRAP, 5, prec="fp32", transform="normal")).astype(np.float64)
    zo = q.points(N, transform=O.NORMAL)
    assert np.abs(zo).max() > 3.5
    assert np.max(np.abs(z - zo) / np.maximum(1.0, np.abs(zo))) < 1e-6


# ------------------------------------------------------------------ product integrand
@pytest.mark.parametrize("seq", [O.HALTON_RS, O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
def test_product_theta(R, seq):
    cfg = inputs.CONFIGS["product_s8"]
    s, N, M = cfg["s"], cfg["N"], cfg["M"]
    a = inputs.product_weights(s)
    th_o = O.product_theta(O.Sequence(seq, s, M, 1, joe_kuo=JK), N, a)
    th64, rq, sd = R.rqmc_integrate_product(s, N, M, seq, 1, a, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-13)
    th32, _, _ = R.rqmc_integrate_product(s, N, M, seq, 1, a, prec="fp32")
    np.testing.assert_allclose(th32, th_o, rtol=2e-6)
    assert abs(rq - 1.0) < 4 * sd / np.sqrt(M) + 1e-12


# ------------------------------------------------------------------ LMM caplets
def _caplet_tol(theta_o, nK):
    """1e-4 max(|theta|, theta_scale) with theta_scale the middle (at-the-money) strike."""
    t = theta_o.reshape(theta_o.shape[0], -1, nK)
    scale = np.maximum(np.abs(t), np.abs(t[:, :, nK // 2:nK // 2 + 1]))
    return 1e-4 * scale.reshape(theta_o.shape)


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.HALTON_RS, O.SOBOL_LMS])
def test_caplets_small(R, seq):
    lm = inputs.lmm_flat(40)
    K = inputs.LMM_STRIKES
    N, M = 2500, 2
    th_o = O.lmm_caplets(O.Sequence(seq, 40, M, 3, joe_kuo=JK), lm, K, N)
    th64, _, _ = R.price_caplets(lm, K, N, M, seq, 3, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-11, atol=1e-15)
    th32, _, _ = R.price_caplets(lm, K, N, M, seq, 3, prec="fp32")
    assert np.all(np.abs(th32 - th_o) <= _caplet_tol(th_o, len(K)))


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
def test_caplets_treasury_curve(R, seq):
    """Sec. 5's Treasury-curve study inputs (non-flat curve, delta = 0.5, sigma = 4 %,
    K = 1 %) against the oracle in FP64 and FP32."""
    st = inputs.TREASURY_STUDY
    lm = inputs.lmm_treasury(st["T"], st["delta"], st["vol"])
    K = np.array([st["K"]])
    N, M = 3000, 3
    th_o = O.lmm_caplets(O.Sequence(seq, lm["n_fwd"], M, 5, joe_kuo=JK), lm, K, N)
    th64, _, _ = R.price_caplets(lm, K, N, M, seq, 5, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-11, atol=1e-15)
    th32, _, _ = R.price_caplets(lm, K, N, M, seq, 5, prec="fp32")
    assert np.all(np.abs(th32 - th_o) <= 1e-4 * np.abs(th_o) + 1e-9)


@pytest.mark.parametrize("nf", [1, 7, 16, 23, 80, 160])
def test_caplets_bucket_edges(R, nf):
    lm = inputs.lmm_flat(nf, vol=0.2)
    lm["L0"] = np.linspace(0.04, 0.06, nf + 1)
    K = np.array([0.05])
    N, M = 700, 2
    th_o = O.lmm_caplets(O.Sequence(O.SOBOL_DS, nf, M, 4, joe_kuo=JK), lm, K, N)
    th64, _, _ = R.price_caplets(lm, K, N, M, O.SOBOL_DS, 4, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-11, atol=1e-15)
    th32, _, _ = R.price_caplets(lm, K, N, M, O.SOBOL_DS, 4, prec="fp32")
    assert np.all(np.abs(th32 - th_o) <= 1e-4 * np.abs(th_o) + 1e-9)


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
def test_caplets_full_size_sampled(R, seq):
    """The 40-forward, N = 65536, M = 64 workload as the bench runs it; the oracle
    recomputes two replications at full N."""
    cfg = inputs.CONFIGS["lmm_caplets_40"]
    lm = inputs.lmm_flat(cfg["n_fwd"])
    K = inputs.LMM_STRIKES
    N, M = cfg["N"], cfg["M"]
    th32, rq, sd = R.price_caplets(lm, K, N, M, seq, cfg["seed"], prec="fp32")
    q = O.Sequence(seq, 40, M, cfg["seed"], joe_kuo=JK)
    for m in (0, M - 1):
        th_o = O.lmm_caplets(q, lm, K, N, m_range=(m, m + 1))
        assert np.all(np.abs(th32[m:m + 1] - th_o) <= _caplet_tol(th_o, len(K)))


@pytest.mark.parametrize("seq,nf", [(O.RASRAP, 40), (O.SOBOL_DS, 40), (O.PHILOX, 40), (O.SOBOL_LMS, 16),
                                    (O.SOBOL_DS, 80), (O.RASRAP, 160), (O.HALTON_RS, 7)])
def test_caplets_euler_scheme(R, seq, nf):
    """The Euler scheme of eq. (L_n_discrete) (delta L carried linearly, X *= 1 + sigma W)
    against the oracle's Euler branch, FP64 and FP32, across the register buckets."""
    lm = inputs.lmm_flat(nf, vol=0.2, scheme=1)
    lm["L0"] = np.linspace(0.045, 0.055, nf + 1)
    K = inputs.LMM_STRIKES
    N, M = 2000, 2
    th_o = O.lmm_caplets(O.Sequence(seq, nf, M, 6, joe_kuo=JK), lm, K, N)
    th64, _, _ = R.price_caplets(lm, K, N, M, seq, 6, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-11, atol=1e-15)
    th32, _, _ = R.price_caplets(lm, K, N, M, seq, 6, prec="fp32")
    assert np.all(np.abs(th32 - th_o) <= _caplet_tol(th_o, len(K)))
    # the log-Euler result differs: the scheme is really switched
    le, _, _ = R.price_caplets(dict(lm, scheme=0), K, N, M, seq, 6, prec="fp64")
    assert np.max(np.abs(le - th64)) > 1e-6 * np.abs(th64).max()


def test_caplets_euler_zero_volatility_and_refusals(R):
    # sigma = 0: the Euler step is the identity, the closed form of eq. BL
    nf, dl = 12, 0.25
    lm = inputs.lmm_flat(nf, vol=0.0, scheme=1)
    lm["L0"] = np.linspace(0.03, 0.07, nf + 1)
    K = inputs.LMM_STRIKES
    th, _, _ = R.price_caplets(lm, K, 1000, 2, "sobol_ds", 1, prec="fp64")
    B = np.concatenate([[1.0], np.cumprod(1.0 / (1.0 + dl * lm["L0"]))])
    want = np.array([[dl * B[n + 1] * max(lm["L0"][n] - k, 0.0) for k in K] for n in range(1, nf + 1)]).reshape(-1)
    np.testing.assert_allclose(th[0], want, rtol=1e-13, atol=1e-15)
    with pytest.raises(R.RqmcError) as e:   # the adjoint runs log-Euler only
        R.price_adjoint(inputs.lmm_flat(8, scheme=1), [0.05], np.ones(8), 64, 1, "philox", 1)
    assert e.value.status == 5
    with pytest.raises(R.RqmcError) as e:   # unknown scheme
        R.price_caplets(inputs.lmm_flat(8, scheme=7), [0.05], 64, 1, "philox", 1)
    assert e.value.status == 1


def test_caplets_from_bond_prices(R):
    """The initial curve given as bond prices B_0(0)..B_nf+1(0) (rqmc_lmm_params.init = 1): the
    library's eq. BL conversion gives the forwards the inputs module computes, so caplets and
    Greeks are bit-identical to the forwards-given call, and match the oracle."""
    st = inputs.TREASURY_STUDY
    B = inputs.treasury_bonds(11, st["delta"])
    lm_f = inputs.lmm_from_bonds(B, st["delta"], st["vol"])
    lm_b = dict(lm_f, B0=B)
    K = np.array([st["K"]])
    for prec in ("fp64", "fp32"):
        a, _, _ = R.price_caplets(lm_f, K, 2048, 3, "sobol_ds", 4, prec=prec)
        b, _, _ = R.price_caplets(lm_b, K, 2048, 3, "sobol_ds", 4, prec=prec)
        assert np.array_equal(a, b), prec
    th_o = O.lmm_caplets(O.Sequence(O.SOBOL_DS, 10, 3, 4, joe_kuo=JK), lm_f, K, 2048)
    np.testing.assert_allclose(b, th_o, rtol=1e-4, atol=1e-9)
    w = np.ones(10)
    ga = R.price_adjoint(lm_f, K, w, 1024, 2, "philox", 4)
    gb = R.price_adjoint(lm_b, K, w, 1024, 2, "philox", 4)
    for x, y in zip(ga, gb):
        assert np.array_equal(x, y)
    bad = dict(lm_b, B0=np.concatenate([B[:5], [-1.0], B[6:]]))
    with pytest.raises(R.RqmcError) as e:
        R.price_caplets(bad, K, 64, 1, "philox", 1)
    assert e.value.status == 1


# ------------------------------------------------------------------ MBS
@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.HALTON_RS, O.SOBOL_LMS])
def test_mbs_small(R, seq):
    mb = inputs.mbs_paper(360)
    N, M = 1500, 2
    th_o = O.mbs_theta(O.Sequence(seq, 360, M, 5, joe_kuo=JK), mb, N)
    th64, _, _ = R.price_mbs(mb, N, M, seq, 5, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-12)
    th32, _, _ = R.price_mbs(mb, N, M, seq, 5, prec="fp32")
    np.testing.assert_allclose(th32, th_o, rtol=1e-4)


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.SOBOL_LMS])
def test_mbs_full_size_sampled(R, seq):
    """The 360-month, N = 65536, M = 64 MBS workload; the oracle recomputes the last
    replication at full N (point ranges on host threads)."""
    cfg = inputs.CONFIGS["mbs_360"]
    mb = inputs.mbs_paper(cfg["months"])
    N, M = cfg["N"], cfg["M"]
    th32, rq, sd = R.price_mbs(mb, N, M, seq, cfg["seed"], prec="fp32")
    m = M - 1
    q = O.Sequence(seq, 360, M, cfg["seed"], joe_kuo=JK)
    th_o = oracle_par.over_points(lambda off, n: O.mbs_theta(q, mb, n, offset=off, m_range=(m, m + 1), threads=1), N)
    np.testing.assert_allclose(th32[m], th_o[0], rtol=1e-4)


# ------------------------------------------------------------------ RQ_{M,N} and the sample std
def _stats_tol(tol_theta, M):
    """A change of at most e in every theta_N^m moves their mean by at most e and their
    sample standard deviation by at most e sqrt(M / (M - 1)) (triangle inequality on the
    centred vector)."""
    return tol_theta, tol_theta * np.sqrt(M / (M - 1.0))


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.PHILOX])
def test_rq_and_sd_match_the_oracle(R, seq):
    """RQ_{M,N} (Sec. 1) and the sample standard deviation over the M replications (the
    error measure of Sec. 5) that the one-shot calls return, against the oracle's
    rq_stats of its own theta (M >= 2), for the product integrand, caplets and MBS."""
    # the library's statistics are those of its own theta, to rounding
    a = inputs.product_weights(8)
    th, rq, sd = R.rqmc_integrate_product(8, 4096, 32, seq, 1, a, prec="fp64")
    rq_g, sd_g = O.rq_stats(th)
    np.testing.assert_allclose(rq, rq_g[0], rtol=1e-14)
    np.testing.assert_allclose(sd, sd_g[0], rtol=1e-12)
    # product integrand, FP64 (theta within 1e-13 relative)
    th_o = O.product_theta(O.Sequence(seq, 8, 32, 1, joe_kuo=JK), 4096, a)
    rq_o, sd_o = O.rq_stats(th_o)
    e_rq, e_sd = _stats_tol(1e-13 * np.abs(th_o).max(), 32)
    assert abs(rq - rq_o[0]) <= e_rq and abs(sd - sd_o[0]) <= e_sd
    # caplets, FP64 and FP32, M = 8
    lm = inputs.lmm_flat(40)
    K = inputs.LMM_STRIKES
    M = 8
    th_o = O.lmm_caplets(O.Sequence(seq, 40, M, 3, joe_kuo=JK), lm, K, 1500)
    rq_o, sd_o = O.rq_stats(th_o)
    for prec in ("fp64", "fp32"):
        th, rq, sd = R.price_caplets(lm, K, 1500, M, seq, 3, prec=prec)
        tol = (1e-11 * np.abs(th_o) + 1e-15) if prec == "fp64" else _caplet_tol(th_o, len(K))
        e_rq, e_sd = _stats_tol(tol.max(axis=0), M)
        assert np.all(np.abs(rq - rq_o) <= e_rq) and np.all(np.abs(sd - sd_o) <= e_sd), prec
        rq_g, sd_g = O.rq_stats(th)
        np.testing.assert_allclose(rq, rq_g, rtol=1e-14)
        np.testing.assert_allclose(sd, sd_g, rtol=1e-11)
    # MBS, FP32, M = 8
    mb = inputs.mbs_paper(360)
    th_o = O.mbs_theta(O.Sequence(seq, 360, M, 5, joe_kuo=JK), mb, 700)
    rq_o, sd_o = O.rq_stats(th_o)
    th, rq, sd = R.price_mbs(mb, 700, M, seq, 5, prec="fp32")
    e_rq, e_sd = _stats_tol(1e-4 * np.abs(th_o).max(), M)
    assert abs(rq - rq_o[0]) <= e_rq and abs(sd - sd_o[0]) <= e_sd


# ------------------------------------------------------------------ plans and sharding
def test_offset_shards_add_up(R):
    import torch
    lm = inputs.lmm_flat(16)
    K = inputs.LMM_STRIKES
    N, M = 4096, 3
    full = R.Plan.caplets(lm, K, N, M, O.SOBOL_DS, 9, prec="fp64")
    a = R.Plan.caplets(lm, K, N // 2, M, O.SOBOL_DS, 9, prec="fp64", offset=0)
    b = R.Plan.caplets(lm, K, N // 2, M, O.SOBOL_DS, 9, prec="fp64", offset=N // 2)
    tf = full.execute().cpu().numpy()
    ta, tb = a.execute().cpu().numpy(), b.execute().cpu().numpy()
    torch.cuda.synchronize()
    np.testing.assert_allclose(0.5 * (ta + tb), tf, rtol=1e-13, atol=1e-17)


def test_plan_is_deterministic_and_launch_knobs_do_not_change_results(R):
    mb = inputs.mbs_paper(120)
    p = R.Plan.mbs(mb, 3000, 4, O.RASRAP, 2, prec="fp32")
    t1 = p.execute().cpu().numpy()
    t2 = p.execute().cpu().numpy()
    assert np.array_equal(t1, t2)
    p.set_launch(threads=128, paths_per_thread=3)
    t3 = p.execute().cpu().numpy()
    np.testing.assert_allclose(t3, t1, rtol=1e-5)
    p.check()
