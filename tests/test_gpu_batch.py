"""The batched persistent launch (graph-captured, autotuned tiles) against the FP64
oracle, instrument by instrument (instrument i uses index i in its Philox counters)."""
import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

JK = inputs.joe_kuo_table()
pytestmark = pytest.mark.gpu

INSTS = [
    {"kind": "lmm", "n_fwd": 8, "N": 3000, "rate": 0.05, "vol": 0.15, "strike": 0.05},
    {"kind": "mbs", "months": 120, "N": 1000},
    {"kind": "lmm", "n_fwd": 23, "N": 1024, "rate": 0.04, "vol": 0.2, "strike": 0.042},
    {"kind": "lmm", "n_fwd": 40, "N": 777, "rate": 0.05, "vol": 0.15, "strike": 0.05},
    {"kind": "mbs", "months": 13, "N": 4096},
    {"kind": "lmm", "n_fwd": 97, "N": 600, "rate": 0.05, "vol": 0.15, "strike": 0.05},
    {"kind": "lmm", "n_fwd": 160, "N": 300, "rate": 0.03, "vol": 0.1, "strike": 0.03},
]


@pytest.fixture(scope="module")
def R(tmp_path_factory):
    import os
    os.environ["RQMC_AUTOTUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "autotune.json")
    from paper_1408_5526_gb300 import _build, rqmc
    _build.build()
    rqmc.load()
    return rqmc


def _oracle(seq, M, seed, insts=INSTS):
    out = []
    for i, d in enumerate(insts):
        if d["kind"] == "lmm":
            lm = inputs.lmm_flat(d["n_fwd"], delta=0.25, rate=d["rate"], vol=d["vol"])
            q = O.Sequence(seq, d["n_fwd"], M, seed, inst=i, joe_kuo=JK)
            out.append(O.lmm_caplets(q, lm, [d["strike"]], d["N"]))
        else:
            q = O.Sequence(seq, d["months"], M, seed, inst=i, joe_kuo=JK)
            out.append(O.mbs_theta(q, inputs.mbs_paper(d["months"]), d["N"])[:, None])
    return out


@pytest.mark.parametrize("seq", [O.SOBOL_DS, O.RASRAP, O.PHILOX, O.SOBOL_LMS])
def test_batch_matches_oracle_per_instrument(R, seq):
    M, seed = 2, 11
    got = R.price_batch(INSTS, M, seq, seed)
    ref = _oracle(seq, M, seed)
    for d, g, r in zip(INSTS, got, ref):
        assert g.shape == r.shape
        tol = 1e-4 * np.maximum(np.abs(r), np.abs(r).max(axis=1, keepdims=True) * 1e-2) + 1e-12
        assert np.all(np.abs(g - r) <= tol), (d, np.max(np.abs(g - r) / tol))


def test_batch_graph_replay_is_deterministic_and_cached(R):
    import os
    import torch
    p = R.Plan.batch(INSTS, 3, O.SOBOL_DS, 5)
    a = p.execute().cpu().numpy()
    b = p.execute().cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(a, b)
    # one persistent kernel per work class present (160-forward strips, MBS, smaller
    # strips: all three here) and the theta kernel
    assert p.launches() == 4
    assert os.path.exists(os.environ["RQMC_AUTOTUNE_CACHE"])
    parts = p.split_batch(a)
    assert [x.shape for x in parts] == [(3, d["n_fwd"] if d["kind"] == "lmm" else 1) for d in INSTS]


@pytest.mark.parametrize("subset", [[1, 4], [0, 2, 3], [5, 6], [6, 1]])
def test_batch_with_some_work_classes_empty(R, subset):
    """Batches that leave one or two of the three work classes empty (MBS only, small
    strips only, 160-forward strips only, and no small strips) still match the oracle."""
    insts = [INSTS[k] for k in subset]
    M, seed = 2, 3
    got = R.price_batch(insts, M, O.SOBOL_DS, seed)
    ref = _oracle(O.SOBOL_DS, M, seed, insts)
    for d, g, r in zip(insts, got, ref):
        tol = 1e-4 * np.maximum(np.abs(r), np.abs(r).max(axis=1, keepdims=True) * 1e-2) + 1e-12
        assert np.all(np.abs(g - r) <= tol), (d, np.max(np.abs(g - r) / tol))
