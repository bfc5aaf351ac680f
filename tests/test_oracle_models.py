"""Pins of the oracle's estimators and path models (Sec. 1, Sec. 5, Sec. 6).

Closed forms (product integrand, zero-volatility LMM, sigma = 0 MBS),
quadrature of the exact discrete model on short horizons (first two
caplets, two- and three-month MBS), the Black formula within a measured
discretization budget, and finite differences for the pathwise adjoint.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

JK = inputs.joe_kuo_table()


# ------------------------------------------------------------------ product integrand
def _product_var(a):
    return float(np.prod((4.0 / 3.0 + 2 * a + a * a) / (1 + a) ** 2) - 1.0)


def test_product_variance_closed_form():
    assert abs(_product_var(inputs.product_weights(8)) - 0.19193) < 5e-5


@pytest.mark.parametrize("seq", [O.HALTON_RS, O.RASRAP, O.SOBOL_DS])
def test_product_integral_rqmc(seq):
    cfg = inputs.CONFIGS["product_s8"]
    a = inputs.product_weights(cfg["s"])
    q = O.Sequence(seq, cfg["s"], cfg["M"], cfg["seed"], joe_kuo=JK)
    theta = O.product_theta(q, cfg["N"], a)
    rq, sd = O.rq_stats(theta)
    assert abs(rq[0] - 1.0) <= 4 * sd[0] / math.sqrt(cfg["M"]) + 1e-12
    mc_sd = math.sqrt(_product_var(a) / cfg["N"])
    assert sd[0] < 0.25 * mc_sd          # RQMC beats the MC rate at this N


def test_product_integral_philox_matches_mc_variance():
    a = inputs.product_weights(8)
    M, N = 64, 4096
    q = O.Sequence(O.PHILOX, 8, M, 1)
    theta = O.product_theta(q, N, a)
    rq, sd = O.rq_stats(theta)
    var = _product_var(a)
    ratio = sd[0] ** 2 / (var / N)
    assert 0.55 < ratio < 1.55           # chi^2_63 / 63, two-sided ~0.998
    assert abs(rq[0] - 1.0) <= 4 * math.sqrt(var / (N * M))


# ------------------------------------------------------------------ LMM
def _black(L, K, sigma, T, B):
    d1 = (math.log(L / K) + 0.5 * sigma * sigma * T) / (sigma * math.sqrt(T))
    d2 = d1 - sigma * math.sqrt(T)
    Phi = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
    return B * (L * Phi(d1) - K * Phi(d2))


@pytest.mark.parametrize("scheme", [0, 1])
def test_lmm_zero_vol_is_deterministic(scheme):
    # sigma = 0: no drift, no noise; price = delta B_{n+1}(0) (L_n(0) - K)^+ (eq. BL)
    lm = inputs.lmm_flat(n_fwd=12, vol=0.0, scheme=scheme)
    lm["L0"] = np.linspace(0.03, 0.06, 13)
    K = np.array([0.02, 0.045, 0.07])
    q = O.Sequence(O.SOBOL_DS, 12, 3, 1, joe_kuo=JK)
    theta = O.lmm_caplets(q, lm, K, 64)
    dl = lm["delta"]
    B = np.cumprod(1.0 / (1.0 + dl * lm["L0"]))          # B_1, B_2, ...
    for n in range(1, 13):
        for k in range(3):
            want = dl * B[n] * max(lm["L0"][n] - K[k], 0.0)
            np.testing.assert_allclose(theta[:, (n - 1) * 3 + k], want, rtol=1e-13, atol=1e-17)


def _quad_kinked(f, kink):
    from scipy import integrate
    dens = lambda z: math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    g = lambda z: f(z) * dens(z)
    a = integrate.quad(g, -12.0, kink, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    b = integrate.quad(g, kink, 12.0, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return a + b


def test_lmm_first_two_caplets_match_quadrature():
    pytest.importorskip("scipy")
    r, sig, dl, K = 0.05, 0.3, 0.25, 0.05
    lm = inputs.lmm_flat(n_fwd=6, vol=sig, rate=r, delta=dl)
    h, sh = dl, math.sqrt(dl)
    L0 = r
    a0 = dl * L0 / (1 + dl * L0)

    def L1(z0):
        mu = sig * sig * a0
        return L0 * math.exp((mu - 0.5 * sig * sig) * h + sig * sh * z0)

    def L2_after0(z0):
        mu = sig * sig * 2 * a0
        return L0 * math.exp((mu - 0.5 * sig * sig) * h + sig * sh * z0)

    zk1 = (math.log(K / L0) - (sig * sig * a0 - 0.5 * sig * sig) * h) / (sig * sh)
    cap1 = _quad_kinked(lambda z: dl * max(L1(z) - K, 0.0) / ((1 + dl * r) * (1 + dl * L1(z))), zk1)

    xs, ws = np.polynomial.hermite_e.hermegauss(120)
    ws = ws / math.sqrt(2 * math.pi)
    cap2 = 0.0
    for z0, w0 in zip(xs, ws):
        l1, l2 = L1(z0), L2_after0(z0)
        a = dl * l2 / (1 + dl * l2)
        e = (sig * sig * a - 0.5 * sig * sig) * h
        zk = (math.log(K / l2) - e) / (sig * sh)
        f = lambda z1: dl * max(l2 * math.exp(e + sig * sh * z1) - K, 0.0) / (
            (1 + dl * r) * (1 + dl * l1) * (1 + dl * l2 * math.exp(e + sig * sh * z1)))
        cap2 += w0 * _quad_kinked(f, zk)

    for seq in (O.SOBOL_DS, O.RASRAP):
        q = O.Sequence(seq, 6, 16, 3, joe_kuo=JK)
        theta = O.lmm_caplets(q, lm, [K], 8192)
        rq, sd = O.rq_stats(theta)
        assert abs(rq[0] - cap1) <= 4 * sd[0] / 4 + 1e-9 * cap1, (rq[0], cap1, sd[0])
        assert abs(rq[1] - cap2) <= 4 * sd[1] / 4 + 1e-9 * cap2, (rq[1], cap2, sd[1])


def test_lmm_euler_first_two_caplets_match_quadrature():
    """The Euler scheme of eq. (L_n_discrete), L_n <- L_n + mu_n L_n h + L_n sqrt(h) sigma_n Z with
    mu_n = sum_{j<=n} delta L_j sigma_n sigma_j / (1 + delta L_j): the first two caplets of a
    flat one-factor curve against quadrature of the same discrete model (one and two steps)."""
    pytest.importorskip("scipy")
    r, sig, dl, K = 0.05, 0.3, 0.25, 0.05
    lm = inputs.lmm_flat(n_fwd=6, vol=sig, rate=r, delta=dl, scheme=1)
    h, sh = dl, math.sqrt(dl)
    L0 = r
    a0 = dl * L0 / (1 + dl * L0)

    def L1(z0):                      # forward 1 after step 0 (alive: forwards 1.., prefix a_1)
        return L0 * (1.0 + sig * sig * a0 * h + sig * sh * z0)

    def L2_after0(z0):               # forward 2 after step 0 (prefix a_1 + a_2)
        return L0 * (1.0 + sig * sig * 2 * a0 * h + sig * sh * z0)

    zk1 = (K / L0 - 1.0 - sig * sig * a0 * h) / (sig * sh)
    cap1 = _quad_kinked(lambda z: dl * max(L1(z) - K, 0.0) / ((1 + dl * r) * (1 + dl * L1(z))), zk1)

    xs, ws = np.polynomial.hermite_e.hermegauss(120)
    ws = ws / math.sqrt(2 * math.pi)
    cap2 = 0.0
    for z0, w0 in zip(xs, ws):
        l1, l2 = L1(z0), L2_after0(z0)
        a = dl * l2 / (1 + dl * l2)
        g = lambda z1: l2 * (1.0 + sig * sig * a * h + sig * sh * z1)
        zk = (K / l2 - 1.0 - sig * sig * a * h) / (sig * sh)
        f = lambda z1: dl * max(g(z1) - K, 0.0) / ((1 + dl * r) * (1 + dl * l1) * (1 + dl * g(z1)))
        cap2 += w0 * _quad_kinked(f, zk)

    for seq in (O.SOBOL_DS, O.RASRAP):
        q = O.Sequence(seq, 6, 16, 3, joe_kuo=JK)
        theta = O.lmm_caplets(q, lm, [K], 8192)
        rq, sd = O.rq_stats(theta)
        assert abs(rq[0] - cap1) <= 4 * sd[0] / 4 + 1e-9 * cap1, (rq[0], cap1, sd[0])
        assert abs(rq[1] - cap2) <= 4 * sd[1] / 4 + 1e-9 * cap2, (rq[1], cap2, sd[1])
    # and the scheme is not log-Euler: the two discretizations differ by more than the noise
    q = O.Sequence(O.SOBOL_DS, 6, 16, 3, joe_kuo=JK)
    le = O.rq_stats(O.lmm_caplets(q, dict(lm, scheme=0), [K], 8192))
    eu = O.rq_stats(O.lmm_caplets(q, lm, [K], 8192))
    assert abs(le[0][1] - eu[0][1]) > 10 * (le[1][1] + eu[1][1]) / 4


def test_lmm_black_formula_within_discretization_budget():
    # Black caplet (read with delta in front, as eq. black_cap must be), spot-measure
    # log-Euler bias measured by halving the step (Richardson): |P_h - P_{h/2}| ~ bias / 2.
    nf, dl, r, sig = 8, 0.25, 0.05, 0.15
    Ks = inputs.LMM_STRIKES
    M, N = 16, 8192
    lm1 = inputs.lmm_flat(n_fwd=nf, vol=sig, rate=r, delta=dl)
    lm2 = dict(lm1, substeps=2)
    q1 = O.Sequence(O.SOBOL_DS, nf, M, 1, joe_kuo=JK)
    q2 = O.Sequence(O.SOBOL_DS, 2 * nf, M, 1, joe_kuo=JK)
    rq1, sd1 = O.rq_stats(O.lmm_caplets(q1, lm1, Ks, N))
    rq2, sd2 = O.rq_stats(O.lmm_caplets(q2, lm2, Ks, N))
    B = (1.0 / (1.0 + dl * r)) ** np.arange(nf + 2)
    for n in range(1, nf + 1):
        for k, K in enumerate(Ks):
            o = (n - 1) * len(Ks) + k
            black = dl * _black(r, K, sig, n * dl, B[n + 1])
            budget = 3 * (sd1[o] + sd2[o]) / math.sqrt(M) + 3 * abs(rq1[o] - rq2[o]) + 1e-8
            assert abs(rq1[o] - black) <= budget, (n, K, rq1[o], rq2[o], black)
            assert abs(rq1[o] - black) < 0.01 * black + 2e-7


def test_treasury_curve_inputs_reproduce_table_3():
    # the spline passes through the table: at 6 months, 1, 2, 3 and 5 years the bond prices
    # are exactly the bond-equivalent discount factors of the quoted yields
    B = inputs.treasury_bonds(10, 0.5)
    for T, y in ((0.5, 0.14), (1.0, 0.18), (2.0, 0.31), (3.0, 0.43), (5.0, 0.89)):
        k = int(round(T / 0.5))
        assert abs(B[k] - (1 + y / 200.0) ** (-2 * T)) < 1e-15
    lm = inputs.lmm_treasury()
    assert lm["n_fwd"] == 10 and len(lm["L0"]) == 11
    # eq. BL inverted: the forwards rebuild the bond prices
    Bn = np.concatenate([[1.0], np.cumprod(1.0 / (1.0 + 0.5 * lm["L0"]))])
    np.testing.assert_allclose(Bn, inputs.treasury_bonds(11, 0.5), rtol=1e-14)


def test_treasury_study_caplet_matches_black():
    # Sec. 5's study, (t, T, delta, K, sigma) = (0, 5, 0.5, 0.01, 0.04): the caplet on L_10
    # against Black on the same initial curve, within the measured discretization budget
    st = inputs.TREASURY_STUDY
    lm1 = inputs.lmm_treasury(st["T"], st["delta"], st["vol"])
    lm2 = dict(lm1, substeps=2)
    nf = lm1["n_fwd"]
    M, N = 16, 8192
    q1 = O.Sequence(O.SOBOL_DS, nf, M, 2, joe_kuo=JK)
    q2 = O.Sequence(O.SOBOL_DS, 2 * nf, M, 2, joe_kuo=JK)
    rq1, sd1 = O.rq_stats(O.lmm_caplets(q1, lm1, [st["K"]], N))
    rq2, sd2 = O.rq_stats(O.lmm_caplets(q2, lm2, [st["K"]], N))
    B = inputs.treasury_bonds(nf + 1, st["delta"])
    for n in (1, 5, nf):
        black = st["delta"] * _black(lm1["L0"][n], st["K"], st["vol"], n * st["delta"], B[n + 1])
        o = n - 1
        budget = 3 * (sd1[o] + sd2[o]) / math.sqrt(M) + 3 * abs(rq1[o] - rq2[o]) + 1e-9
        assert abs(rq1[o] - black) <= budget, (n, rq1[o], rq2[o], black)


# ------------------------------------------------------------------ MBS
def _mbs_deterministic(mb):
    Mm, i0 = mb["months"], mb["i0"]
    w = mb["K1"] + mb["K2"] * math.atan(mb["K3"] * i0 + mb["K4"])
    v = 1.0 / (1.0 + i0)
    pv = 0.0
    for k in range(1, Mm + 1):
        ck = (1 - v ** (Mm - k + 1)) / (1 - v)       # geometric sum_{j=0}^{M-k} v^j
        pv += v ** k * (1 - w) ** (k - 1) * ((1 - w) + w * ck) * mb["c"]
    return pv


@pytest.mark.parametrize("months", [1, 12, 360])
def test_mbs_sigma_zero_closed_form(months):
    mb = dict(inputs.mbs_paper(months), sigma=0.0)
    q = O.Sequence(O.RASRAP, months, 2, 1)
    theta = O.mbs_theta(q, mb, 16)
    np.testing.assert_allclose(theta, _mbs_deterministic(mb), rtol=1e-13)


def _mbs_expect_short(mb, months):
    """E[PV] for 2 or 3 months by Gauss-Hermite quadrature over z_1 (, z_2)."""
    i0, s = mb["i0"], mb["sigma"]
    K0 = math.exp(-0.5 * s * s)
    v = 1.0 / (1.0 + i0)
    w_of = lambda i: mb["K1"] + mb["K2"] * math.atan(mb["K3"] * i + mb["K4"])
    ck = [None] + [sum(v ** j for j in range(months - k + 1)) for k in range(1, months + 1)]
    xs, ws = np.polynomial.hermite_e.hermegauss(60)
    ws = ws / math.sqrt(2 * math.pi)

    def pv(z1, z2):
        i1 = K0 * math.exp(s * z1) * i0
        w1 = w_of(i1)
        u1, r1 = v, 1.0
        tot = u1 * mb["c"] * r1 * ((1 - w1) + w1 * ck[1])
        u2, r2 = u1 / (1 + i1), r1 * (1 - w1)
        i2 = K0 * math.exp(s * z2) * i1
        w2 = w_of(i2)
        tot += u2 * mb["c"] * r2 * ((1 - w2) + w2 * ck[2])
        if months == 3:
            u3, r3 = u2 / (1 + i2), r2 * (1 - w2)
            tot += u3 * mb["c"] * r3     # c_3 = 1, so (1-w_3) + w_3 c_3 = 1
        return tot

    if months == 2:
        return sum(w1 * pv(z1, 0.0) for z1, w1 in zip(xs, ws))
    return sum(w1 * w2 * pv(z1, z2) for z1, w1 in zip(xs, ws) for z2, w2 in zip(xs, ws))


@pytest.mark.parametrize("months", [2, 3])
def test_mbs_short_horizon_matches_quadrature(months):
    mb = dict(inputs.mbs_paper(months), sigma=0.4, K3=100.0)   # make the stochastic part visible
    exact = _mbs_expect_short(mb, months)
    det = _mbs_deterministic(dict(mb, sigma=0.0))
    assert abs(exact - det) > 1e-6
    for seq in (O.SOBOL_DS, O.RASRAP, O.PHILOX):
        q = O.Sequence(seq, months, 16, 2, joe_kuo=JK)
        theta = O.mbs_theta(q, mb, 4096)
        rq, sd = O.rq_stats(theta)
        assert abs(rq[0] - exact) <= 4 * sd[0] / 4 + 1e-13, (seq, rq[0], exact, sd[0])


# ------------------------------------------------------------------ adjoint
def test_adjoint_matches_central_differences():
    nf, M, N = 6, 2, 512
    lm = inputs.lmm_two_factor(n_fwd=nf, seed=4)
    lm["L0"] = np.linspace(0.04, 0.06, nf + 1)
    K = np.array([0.045, 0.052])
    w = np.random.default_rng(2).uniform(0.5, 1.5, size=nf * len(K))
    q = O.Sequence(O.SOBOL_DS, nf * 2, M, 9, joe_kuo=JK)
    value, delta, vega = O.lmm_adjoint(q, lm, K, w, N)
    price = lambda lmx: O.lmm_caplets(q, lmx, K, N) @ w
    np.testing.assert_allclose(value, price(lm), rtol=1e-13)
    h = 1e-7     # small enough that no path crosses a payoff kink between the bumps
    for n in range(nf):
        up, dn = dict(lm, L0=lm["L0"].copy()), dict(lm, L0=lm["L0"].copy())
        up["L0"][n + 1] += h
        dn["L0"][n + 1] -= h
        fd = (price(up) - price(dn)) / (2 * h)
        np.testing.assert_allclose(delta[:, n], fd, rtol=2e-5, atol=1e-9)
        up, dn = dict(lm, vol=lm["vol"].copy()), dict(lm, vol=lm["vol"].copy())
        up["vol"][n] += h
        dn["vol"][n] -= h
        fd = (price(up) - price(dn)) / (2 * h)
        np.testing.assert_allclose(vega[:, n], fd, rtol=2e-5, atol=1e-9)


# ------------------------------------------------------------------ RQ_{M,N} and the sample std (Sec. 1, Sec. 5)
def test_rq_stats_closed_forms():
    """RQ_{M,N} is the mean of the M estimates theta_N^m (Sec. 1); the error measure of
    Sec. 5 is their sample standard deviation (divisor M - 1).  Closed forms: two values
    a, b give |a - b| / sqrt 2; the integers 0..M-1 give mean (M-1)/2 and variance
    M (M+1) / 12; a constant column has zero spread; one replication reports zero."""
    rq, sd = O.rq_stats(np.array([[1.0, 5.0], [3.0, 5.0]]))
    np.testing.assert_allclose(rq, [2.0, 5.0], rtol=0, atol=0)
    np.testing.assert_allclose(sd, [math.sqrt(2.0), 0.0], rtol=1e-15, atol=0)
    for M in (2, 3, 10, 64):
        rq, sd = O.rq_stats(np.arange(M, dtype=np.float64))
        assert rq[0] == (M - 1) / 2
        assert abs(sd[0] - math.sqrt(M * (M + 1) / 12.0)) <= 1e-14 * sd[0]
    rq, sd = O.rq_stats(np.array([[0.25, -1.0, 7.0]]))
    np.testing.assert_array_equal(rq, [0.25, -1.0, 7.0])
    np.testing.assert_array_equal(sd, [0.0, 0.0, 0.0])


def test_rq_stats_match_numpy():
    """Against numpy's mean and std(ddof=1) on random estimates, column by column."""
    th = np.random.default_rng(5).normal(0.01, 1e-4, size=(64, 120))
    rq, sd = O.rq_stats(th)
    np.testing.assert_allclose(rq, th.mean(axis=0), rtol=1e-14)
    np.testing.assert_allclose(sd, th.std(axis=0, ddof=1), rtol=1e-12)
