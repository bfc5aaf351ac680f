"""The generators at the top of their index ranges, bit-exact against the oracle.

Philox counts points with 48 bits (low word n_lo32, then n_hi16 in the second counter
word): ranges near 2^40 that cross a 2^32 boundary, and the last points below 2^48.
Sobol' indices are 32-bit: the last N points below 2^32.  Halton/Rasrap split the index at
digit L with p^L <= 2^31 for every base (the low part lo0 + i stays below 2^32): runs at
exactly the largest N this allows for s = 1 (N = 2^31), s = 2 (N = 3^19) and s = 360
(N = 1291^2, and one point less, a multiple of 8 that the run kernel takes), checked on
windows at the start, the end and inside the range.  One more
point than each limit is refused before any launch.  The caplet kernel's own generator (a
separate code path from the point stream) runs at the same large offsets."""
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


def _raw(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("offset,N", [((1 << 40) + (1 << 32) - 1500, 3001), ((1 << 40) + (1 << 32) - 1500, 3000),
                                      ((1 << 48) - 3001, 3001), ((1 << 48) - 3000, 3000)])
def test_philox_points_at_large_offsets(R, offset, N):
    M, s = 2, 10
    gpu = _raw(R.rqmc_points(s, N, M, O.PHILOX, 7, offset=offset, transform="raw"))
    ora = O.Sequence(O.PHILOX, s, M, 7).points(N, offset, transform=O.RAW)
    assert np.array_equal(gpu, ora)


def test_philox_refuses_beyond_48_bits(R):
    with pytest.raises(R.RqmcError) as e:
        R.Plan.points(4, 3001, 1, "philox", 1, offset=(1 << 48) - 3000)
    assert "2^48" in str(e.value)


@pytest.mark.parametrize("seq", [O.SOBOL_DS, O.SOBOL_LMS])
@pytest.mark.parametrize("N", [3001, 3000])
def test_sobol_points_up_to_two_to_the_32(R, seq, N):
    M, s = 2, 40
    offset = (1 << 32) - N
    gpu = _raw(R.rqmc_points(s, N, M, seq, 7, offset=offset, transform="raw"))
    ora = O.Sequence(seq, s, M, 7, joe_kuo=JK).points(N, offset, transform=O.RAW)
    assert np.array_equal(gpu, ora)


def _windows(N):
    rng = np.random.default_rng(3)
    mids = sorted(int(x) for x in rng.integers(2048, N - 2048 - 256, size=6))
    return [(0, 2048), (N - 2048, 2048)] + [(a, 256) for a in mids]


@pytest.mark.parametrize("seq,s,N", [(O.RASRAP, 1, 1 << 31), (O.HALTON_RS, 2, 3 ** 19), (O.RASRAP, 2, 3 ** 19),
                                     (O.RASRAP, 360, 1291 ** 2), (O.RASRAP, 360, 1291 ** 2 - 1)])
def test_halton_at_the_digit_split_limit(R, seq, s, N):
    import torch
    M = 1
    p = R.Plan.points(s, N, M, seq, 5, transform="raw")
    out = p.execute()
    q = O.Sequence(seq, s, M, 5)
    for a, c in _windows(N):
        gpu = out[:, :, a:a + c].cpu().numpy().view(np.uint64)
        ora = q.points(c, a, transform=O.RAW)
        assert np.array_equal(gpu, ora), (a, c)
    p.close()
    del out
    torch.cuda.empty_cache()
    if N in (1 << 31, 3 ** 19, 1291 ** 2):   # the largest N of its s: one more point is refused
        with pytest.raises(R.RqmcError):
            R.Plan.points(s, N + 1, M, seq, 5, transform="raw")


@pytest.mark.parametrize("seq,offset", [(O.PHILOX, (1 << 40) + (1 << 32) - 1500), (O.PHILOX, (1 << 48) - 3001),
                                        (O.SOBOL_DS, (1 << 32) - 3001)])
def test_caplet_kernel_at_large_offsets(R, seq, offset):
    lm = inputs.lmm_flat(16, vol=0.2)
    K = inputs.LMM_STRIKES
    N, M = 3001, 2
    th_o = O.lmm_caplets(O.Sequence(seq, 16, M, 9, joe_kuo=JK), lm, K, N, offset=offset)
    for prec, rtol in (("fp64", 1e-11), ("fp32", 1e-4)):
        p = R.Plan.caplets(lm, K, N, M, seq, 9, prec=prec, offset=offset)
        th = p.execute().cpu().numpy().reshape(M, -1)
        p.close()
        t = th_o.reshape(M, -1, len(K))
        scale = np.maximum(np.abs(t), np.abs(t[:, :, 1:2])).reshape(M, -1)
        assert np.all(np.abs(th - th_o) <= rtol * scale + 1e-15), prec
