"""Statistical regression of the paper's convergence claims on GPU-computed estimates: the
sample standard deviation of M independent estimates falls like N^rate (the fitted slope of
log std against log N over N = 2^10..2^16, M = 64; a weak, statistical pin).  The paper
reports for its GPU runs (Sec. 5: LIBOR caplet, Philox 0.52, Rasrap 0.86, Sobol' 0.95;
Sec. 6: MBS, MC 0.5, Rasrap 0.68, Sobol' 0.86).  The pseudorandom stream must show the
Monte Carlo rate (0.5 +- 0.1); each quasi-random sequence must converge clearly faster than
Monte Carlo and no slower than the paper's rate (0.15 of slack).  Measured on GB300, the
MBS Rasrap rate is 0.87, faster than the paper's 0.68; the others agree within 0.15."""
import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    rqmc.load()
    return rqmc


def _rate(price, Ns):
    std = [float(np.std(price(N), ddof=1)) for N in Ns]
    return float(np.polyfit(np.log(Ns), np.log(std), 1)[0])


def _check(seq, rate, paper):
    if seq == O.PHILOX:
        assert abs(rate + 0.5) <= 0.1, (seq, rate)
    else:
        assert rate <= -0.6 and rate <= paper + 0.15, (seq, rate)


NS = [1 << e for e in range(10, 17, 2)]


@pytest.mark.parametrize("seq,paper", [(O.PHILOX, -0.52), (O.RASRAP, -0.86), (O.SOBOL_DS, -0.95)])
def test_caplet_std_rate_matches_the_paper(R, seq, paper):
    st = inputs.TREASURY_STUDY
    lm = inputs.lmm_treasury(st["T"], st["delta"], st["vol"])
    nf = lm["n_fwd"]

    def price(N):
        th, _, _ = R.price_caplets(lm, [st["K"]], N, 64, seq, 3, prec="fp32")
        return th[:, nf - 1]

    _check(seq, _rate(price, NS), paper)


@pytest.mark.parametrize("seq,paper", [(O.PHILOX, -0.5), (O.RASRAP, -0.68), (O.SOBOL_DS, -0.86)])
def test_mbs_std_rate_matches_the_paper(R, seq, paper):
    mb = inputs.mbs_paper(360)

    def price(N):
        th, _, _ = R.price_mbs(mb, N, 64, seq, 3, prec="fp32")
        return th.reshape(-1)

    _check(seq, _rate(price, NS), paper)
