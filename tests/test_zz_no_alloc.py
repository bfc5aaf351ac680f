"""rqmc_price_caplets_noalloc against price_caplets.

The no-allocation entry point exists for callers that cannot allocate device memory
when they price -- code running inside a CUDA graph capture, inside another
framework's allocator callback, or under a no-allocation-after-start-up policy.  It
runs the same caplet kernel but keeps its scratch (tables, partial sums, status) in a
fixed 16 MiB array built into the library.  The test calls it through the C ABI twice
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
