"""Pathwise adjoint Greeks of the caplet strip (GPU, FP32 paths) against the FP64
oracle's adjoint on identical points, and against central finite differences of the
GPU's own strip value on common points (bump 1e-4)."""
import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

JK = inputs.joe_kuo_table()
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    rqmc.load()
    return rqmc


@pytest.mark.parametrize("seq,d,nf", [(O.SOBOL_DS, 2, 10), (O.RASRAP, 2, 13), (O.PHILOX, 1, 9), (O.SOBOL_DS, 1, 45),
                                      (O.SOBOL_LMS, 2, 17)])
def test_adjoint_matches_oracle(R, seq, d, nf):
    lm = inputs.lmm_two_factor(n_fwd=nf, seed=3) if d == 2 else inputs.lmm_flat(nf, vol=0.2)
    lm["L0"] = np.linspace(0.045, 0.055, nf + 1)
    K = np.array([0.048, 0.052])
    w = np.random.default_rng(1).uniform(0.5, 1.5, size=nf * len(K))
    N, M = 4001, 2
    q = O.Sequence(seq, nf * d, M, 21, joe_kuo=JK)
    v_o, d_o, g_o = O.lmm_adjoint(q, lm, K, w, N)
    v, dl, vg = R.price_adjoint(lm, K, w, N, M, seq, 21)
    np.testing.assert_allclose(v, v_o, rtol=1e-4)
    # The payoff indicator 1{L > K} is decided in FP32 on the GPU and in FP64 in the
    # oracle; a path that sits on a kink can flip, moving one Greek by about w delta / N.
    # Allow at most two such flips on top of 2e-4 of the Greek's scale, and require 95 %
    # of the Greeks within the tight bound.
    flip = 2 * w.max() * lm["delta"] / N
    for got, ref in ((dl, d_o), (vg, g_o)):
        scale = np.abs(ref).max()
        err = np.abs(got - ref)
        assert np.all(err <= 2e-4 * scale + flip), (err.max() / scale)
        assert np.mean(err <= 2e-4 * scale) >= 0.95


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
