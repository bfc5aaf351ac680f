"""Edge cases of the CUDA path against the oracle: single points and single replications,
sizes below and just above a warp, zero volatility (the closed form), very many dimensions
(tables too large for shared memory, read from global memory), and the range checks that
refuse work before any launch."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

JK = inputs.joe_kuo_table()
pytestmark = pytest.mark.gpu
SEQS = [O.RASRAP, O.SOBOL_DS, O.PHILOX, O.HALTON_RS, O.SOBOL_LMS]


@pytest.fixture(scope="module")
def R():
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    rqmc.load()
    return rqmc


@pytest.mark.parametrize("seq", SEQS)
@pytest.mark.parametrize("N", [1, 31, 33])
def test_tiny_point_counts_single_replication(R, seq, N):
    lm = inputs.lmm_flat(5, vol=0.2)
    K = inputs.LMM_STRIKES
    th_o = O.lmm_caplets(O.Sequence(seq, 5, 1, 2, joe_kuo=JK), lm, K, N)
    th64, rq, sd = R.price_caplets(lm, K, N, 1, seq, 2, prec="fp64")
    np.testing.assert_allclose(th64, th_o, rtol=1e-11, atol=1e-15)
    assert np.all(sd == 0.0) and np.array_equal(rq, th64[0])          # one replication: no spread
    th32, _, _ = R.price_caplets(lm, K, N, 1, seq, 2, prec="fp32")
    assert np.all(np.abs(th32 - th_o) <= 1e-4 * np.abs(th_o) + 1e-9)
    mb = inputs.mbs_paper(12)
    v_o = O.mbs_theta(O.Sequence(seq, 12, 1, 2, joe_kuo=JK), mb, N)
    v32, _, _ = R.price_mbs(mb, N, 1, seq, 2, prec="fp32")
    np.testing.assert_allclose(v32, v_o.reshape(v32.shape), rtol=1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zero_volatility_gives_the_closed_form(R, prec):
    # sigma = 0: no drift, no noise; caplet n = delta B_{n+1}(0) (L_n(0) - K)^+ (eq. BL).
    # FP64 to rounding; FP32 carries L to a few 1e-7 relative, which the payoff L - K turns
    # into an absolute error of that size times delta L: bound it by 1e-6 delta max L.
    nf, dl = 12, 0.25
    lm = inputs.lmm_flat(nf, vol=0.0)
    lm["L0"] = np.linspace(0.03, 0.07, nf + 1)
    K = inputs.LMM_STRIKES
    th, _, _ = R.price_caplets(lm, K, 1000, 2, "sobol_ds", 1, prec=prec)
    B = np.concatenate([[1.0], np.cumprod(1.0 / (1.0 + dl * lm["L0"]))])
    want = np.array([[dl * B[n + 1] * max(lm["L0"][n] - k, 0.0) for k in K] for n in range(1, nf + 1)]).reshape(-1)
    for m in range(2):
        if prec == "fp64":
            np.testing.assert_allclose(th[m], want, rtol=1e-13, atol=1e-15)
        else:
            np.testing.assert_allclose(th[m], want, rtol=0, atol=1e-6 * dl * lm["L0"].max())


@pytest.mark.parametrize("seq", [O.RASRAP, O.SOBOL_DS, O.SOBOL_LMS])
def test_very_many_dimensions_read_tables_from_global_memory(R, seq):
    # 2048 dimensions: the per-replication tables (164 KB Halton, 270 KB Sobol') exceed
    # what the kernels stage in shared memory, so they read them where they are
    s, N, M = 2048, 96, 1
    a = inputs.product_weights(s)
    q = O.Sequence(seq, s, M, 4, joe_kuo=JK)
    th_o = O.product_theta(q, N, a)
    th, _, _ = R.rqmc_integrate_product(s, N, M, seq, 4, a, prec="fp64")
    np.testing.assert_allclose(th.reshape(-1), th_o.reshape(-1), rtol=1e-11)
    mb = inputs.mbs_paper(s)
    v_o = O.mbs_theta(q, mb, N)
    v64, _, _ = R.price_mbs(mb, N, M, seq, 4, prec="fp64")
    np.testing.assert_allclose(v64.reshape(-1), v_o.reshape(-1), rtol=1e-12)
    v32, _, _ = R.price_mbs(mb, N, M, seq, 4, prec="fp32")
    np.testing.assert_allclose(v32.reshape(-1), v_o.reshape(-1), rtol=1e-4)
    mb1 = inputs.mbs_paper(1)
    v1_o = O.mbs_theta(O.Sequence(seq, 1, 2, 4, joe_kuo=JK), mb1, 500)
    v1, _, _ = R.price_mbs(mb1, 500, 2, seq, 4, prec="fp64")
    np.testing.assert_allclose(v1.reshape(-1), v1_o.reshape(-1), rtol=1e-12)


def test_out_of_range_requests_are_refused_before_any_launch(R):
    with pytest.raises(R.RqmcError) as e:                       # Sobol' index beyond 32 bits
        R.Plan.points(4, 1 << 20, 1, "sobol_ds", 1, offset=(1 << 32) - 1000)
    assert "2^32" in str(e.value)
    with pytest.raises(R.RqmcError):                            # more forwards than the buckets hold
        R.price_caplets(inputs.lmm_flat(161), [0.05], 64, 1, "philox", 1)
    with pytest.raises(R.RqmcError):                            # adjoint strips up to 80 forwards
        R.price_adjoint(inputs.lmm_flat(81), [0.05], np.ones(81), 64, 1, "philox", 1)
    with pytest.raises(R.RqmcError):                            # one replication at least
        R.price_caplets(inputs.lmm_flat(8), [0.05], 64, 0, "philox", 1)
    # a refused request leaves the library usable
    th, _, _ = R.price_caplets(inputs.lmm_flat(8), [0.05], 64, 1, "philox", 1, prec="fp64")
    assert np.all(np.isfinite(th)) and math.isfinite(float(th.sum()))


def test_pipe_probe_reports_plausible_rates(R):
    r = R.probe_pipes()
    assert set(r) == {"ex2", "rcp", "lg2", "ex2_rcp_pair", "ffma", "dfma", "fp64_pair", "sm_mhz"}
    assert all(math.isfinite(v) and v > 0 for v in r.values())
    # per SM per clock: at most the 128 FP32 lanes; the pair is no faster than its rcp; FP64
    # slower than FP32; the measured clock within the part's range
    assert r["ffma"] <= 140 and r["ex2"] <= 140 and r["ex2_rcp_pair"] <= r["rcp"] * 1.05
    assert r["dfma"] < r["ffma"] and r["fp64_pair"] < r["dfma"]
    assert 200 < r["sm_mhz"] < 2300
