"""Pathwise adjoint Greeks of the caplet strip (GPU, FP32 paths) against the FP64
oracle's adjoint on identical points (each Greek within 1e-4 relative), including the
80-forward two-factor Greeks workload at full N, and against central finite differences of
the GPU's own strip value on common points (bump 1e-4)."""
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


def _assert_greeks(got, ref, rtol=1e-4):
    """Each Greek within rtol of the oracle's value of that Greek."""
    err = np.abs(got - ref) / np.abs(ref)
    assert np.all(err <= rtol), (float(err.max()), np.unravel_index(int(err.argmax()), err.shape))


@pytest.mark.parametrize("seq,d,nf", [(O.SOBOL_DS, 2, 10), (O.RASRAP, 2, 13), (O.PHILOX, 1, 9), (O.SOBOL_DS, 1, 45),
                                      (O.SOBOL_LMS, 2, 17), (O.HALTON_RS, 1, 24)])
def test_adjoint_matches_oracle(R, seq, d, nf):
    """Value, deltas and vegas per replication within 1e-4 relative of the FP64 oracle's
    adjoint on identical points.  N = 2^16: the FP32 paths decide the payoff indicator
    1{L > K} in single precision, and a path within rounding of a strike can take the other
    branch than in FP64, moving a Greek by about w delta / N; at this N that stays well
    below 1e-4 of every Greek."""
    lm = inputs.lmm_two_factor(n_fwd=nf, seed=3) if d == 2 else inputs.lmm_flat(nf, vol=0.2)
    lm["L0"] = np.linspace(0.045, 0.055, nf + 1)
    K = np.array([0.048, 0.052])
    w = np.random.default_rng(1).uniform(0.5, 1.5, size=nf * len(K))
    N, M = 1 << 16, 2
    q = O.Sequence(seq, nf * d, M, 21, joe_kuo=JK)
    v_o, d_o, g_o = oracle_par.over_points(
        lambda off, n: O.lmm_adjoint(q, lm, K, w, n, offset=off, threads=1), N)
    v, dl, vg = R.price_adjoint(lm, K, w, N, M, seq, 21)
    np.testing.assert_allclose(v, v_o, rtol=1e-4)
    _assert_greeks(dl, d_o)
    _assert_greeks(vg, g_o)


@pytest.mark.parametrize("seq", [O.SOBOL_DS, O.RASRAP, O.PHILOX])
def test_adjoint_greeks_workload_full_size_sampled(R, seq):
    """The Greeks workload as the bench runs it -- two-factor strip of 80 quarterly forwards
    (correlation exp(-0.1|i-j|) reduced to 2 factors, vols drawn per seed), strike 5 %,
    N = 2^18, M = 32 -- with the last replication's value, 80 deltas and 80 vegas recomputed
    by the FP64 oracle's adjoint at full N (point ranges on host threads)."""
    cfg = inputs.CONFIGS["adjoint_2f_80"]
    lm = inputs.lmm_two_factor(cfg["n_fwd"], seed=cfg["seed"])
    K = np.array([0.05])
    w = np.ones(cfg["n_fwd"])
    N, M = cfg["N"], cfg["M"]
    v, dl, vg = R.price_adjoint(lm, K, w, N, M, seq, cfg["seed"])
    m = M - 1
    q = O.Sequence(seq, 2 * cfg["n_fwd"], M, cfg["seed"], joe_kuo=JK)
    v_o, d_o, g_o = oracle_par.over_points(
        lambda off, n: O.lmm_adjoint(q, lm, K, w, n, offset=off, m_range=(m, m + 1), threads=1), N)
    np.testing.assert_allclose(v[m], v_o[0], rtol=1e-4)
    _assert_greeks(dl[m:m + 1], d_o)
    _assert_greeks(vg[m:m + 1], g_o)


def test_adjoint_prices_match_caplet_kernel(R):
    lm = inputs.lmm_flat(40)
    K = inputs.LMM_STRIKES
    N, M = 4096, 3
    p = R.Plan.adjoint(lm, K, np.zeros(120), N, M, O.SOBOL_DS, 2)
    out = p.execute().cpu().numpy().reshape(M, -1)
    th, _, _ = R.price_caplets(lm, K, N, M, O.SOBOL_DS, 2, prec="fp32")
    prices = out[:, 1 + 80:]
    assert np.all(np.abs(prices - th) <= 1e-4 * np.maximum(np.abs(th), 1e-6))


def test_adjoint_matches_central_differences_two_factor(R):
    """The 80-forward two-factor strip of the Greeks workload at reduced N: deltas and
    vegas of sampled forwards against central differences (bump 1e-4) of the strip
    value, all on the same points."""
    lm = inputs.lmm_two_factor(80, seed=1)
    K = np.array([0.05])
    w = np.ones(80)
    N, M, seq, seed = 1 << 14, 2, O.SOBOL_DS, 1
    v, dl, vg = R.price_adjoint(lm, K, w, N, M, seq, seed)

    def value(l):
        p = R.Plan.adjoint(l, K, w, N, M, seq, seed)
        out = p.execute().cpu().numpy().reshape(M, -1)
        p.close()
        return out[:, 0]

    h = 1e-4
    for n in (0, 9, 39, 79):
        up, dn = dict(lm, L0=lm["L0"].copy()), dict(lm, L0=lm["L0"].copy())
        up["L0"][n + 1] += h
        dn["L0"][n + 1] -= h
        fd = (value(up) - value(dn)) / (2 * h)
        np.testing.assert_allclose(dl[:, n], fd, rtol=2e-3, atol=2e-3 * np.abs(dl).max())
        up, dn = dict(lm, vol=lm["vol"].copy()), dict(lm, vol=lm["vol"].copy())
        up["vol"][n] += h
        dn["vol"][n] -= h
        fd = (value(up) - value(dn)) / (2 * h)
        np.testing.assert_allclose(vg[:, n], fd, rtol=2e-3, atol=2e-3 * np.abs(vg).max())


def test_autograd_backward_is_the_adjoint(R):
    import torch
    lm = inputs.lmm_two_factor(12, seed=5)
    K = np.array([0.05])
    L0 = torch.tensor(lm["L0"][1:], dtype=torch.float64, requires_grad=True)
    vol = torch.tensor(lm["vol"], dtype=torch.float64, requires_grad=True)
    prices = R.caplet_strip(L0, vol, lm, K, 2048, 2, O.SOBOL_DS, 7)
    assert prices.shape == (12,)
    prices.sum().backward()
    _, dl, vg = R.price_adjoint(lm, K, np.ones(12), 2048, 2, O.SOBOL_DS, 7)
    np.testing.assert_allclose(L0.grad.numpy(), dl.mean(axis=0), rtol=1e-12)
    np.testing.assert_allclose(vol.grad.numpy(), vg.mean(axis=0), rtol=1e-12)
