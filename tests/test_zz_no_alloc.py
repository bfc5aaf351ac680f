"""rqmc_price_caplets_noalloc against price_caplets.

The no-allocation entry point exists for callers that cannot allocate device memory
when they price -- a callback running inside another framework's device allocator, a
process whose device memory a pool reserved at start-up, or a service that forbids
allocation after start-up.  It runs the same caplet kernel but keeps its scratch (tables,
partial sums, status) in a fixed 16 MiB array built into the library.  The test calls it through the C ABI twice
in a row per sequence, so the second call reuses the array the first one filled, and
checks each result against the allocating entry point within the FP32 caplet
tolerance.  This file is collected last so that a failure here comes after every
other test has run."""
import ctypes as C

import numpy as np
import pytest

from paper_1408_5526_gb300 import inputs

pytestmark = pytest.mark.gpu


def _tol(theta_ref, nK):
    t = theta_ref.reshape(theta_ref.shape[0], -1, nK)
    scale = np.maximum(np.abs(t), np.abs(t[:, :, nK // 2:nK // 2 + 1]))
    return 1e-4 * scale.reshape(theta_ref.shape)


def test_noalloc_matches_price_caplets_on_two_calls_in_a_row():
    import torch
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    L = rqmc.load()
    lm = inputs.lmm_flat(40)
    K = inputs.LMM_STRIKES
    N, M = 8192, 8
    keep: list = []
    p = rqmc._lmm_struct(lm, keep)
    Kc = np.ascontiguousarray(K, dtype=np.float64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seq in (rqmc.RASRAP, rqmc.SOBOL_DS, rqmc.PHILOX):
        ref, _, _ = rqmc.price_caplets(lm, K, N, M, seq, 5, prec="fp32")
        for call in range(2):
            out = torch.full((M, 40 * len(K)), float("nan"), dtype=torch.float64, device="cuda")
            st = L.rqmc_price_caplets_noalloc(C.byref(p), Kc.ctypes.data_as(C.POINTER(C.c_double)), len(K), N, M,
                                              seq, 5, rqmc.FP32,
                                              C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)), stream)
            assert st == 0, L.rqmc_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), (seq, call)
            assert np.all(np.abs(got - ref) <= _tol(ref, len(K))), (seq, call)


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    from paper_1408_5526_gb300 import rqmc
    rqmc.load()
    lm = inputs.lmm_flat(160)
    out = torch.empty(64 * 160 * 8, dtype=torch.float64, device="cuda")   # a valid output buffer
    with pytest.raises(rqmc.RqmcError) as e:
        rqmc.price_caplets_noalloc(lm, [0.05] * 8, 1 << 20, 64, rqmc.PHILOX, 1, out)
    assert e.value.status == 1 and "scratch" in str(e.value)


def test_noalloc_refuses_what_price_caplets_refuses_with_the_same_codes():
    """Both entry points run the same argument checks: a two-factor model, an unknown
    scheme, too many forwards and M = 0 give the same status from each (called through the
    C ABI, so that the binding's own checks do not answer first)."""
    import torch
    from paper_1408_5526_gb300 import rqmc
    L = rqmc.load()
    out = torch.empty(64 * 200 * 8, dtype=torch.float64, device="cuda")
    K = np.array([0.05])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(inputs.lmm_two_factor(8, seed=1), 2), (dict(inputs.lmm_flat(8), scheme=2), 2),
             (inputs.lmm_flat(161), 2), (inputs.lmm_flat(8), 0)]
    for lm, M in cases:
        keep: list = []
        p = rqmc._lmm_struct(lm, keep)
        th = np.zeros(max(M, 1) * lm["n_fwd"])
        a = L.price_caplets(C.byref(p), K.ctypes.data_as(C.POINTER(C.c_double)), 1, 64, M, rqmc.PHILOX, 1,
                            rqmc.FP32, th.ctypes.data_as(C.POINTER(C.c_double)), None, None, stream)
        b = L.rqmc_price_caplets_noalloc(C.byref(p), K.ctypes.data_as(C.POINTER(C.c_double)), 1, 64, M,
                                         rqmc.PHILOX, 1, rqmc.FP32,
                                         C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)), stream)
        assert a != 0 and a == b, (lm["n_fwd"], M, a, b)
