"""The batched persistent launch (graph-captured, autotuned tiles) against the FP64
oracle, instrument by instrument (instrument i uses index i in its Philox counters).
Every caplet and MBS value within 1e-4 of the oracle's, relative to that value: the batch's
caplets are at or in the money, so the at-the-money scale of the caplet tolerance is the
value itself."""
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


def _oracle_one(seq, M, seed, i, d):
    if d["kind"] == "lmm":
        lm = inputs.lmm_flat(d["n_fwd"], delta=0.25, rate=d["rate"], vol=d["vol"])
        q = O.Sequence(seq, d["n_fwd"], M, seed, inst=i, joe_kuo=JK)
        return O.lmm_caplets(q, lm, [d["strike"]], d["N"], threads=1)
    q = O.Sequence(seq, d["months"], M, seed, inst=i, joe_kuo=JK)
    return O.mbs_theta(q, inputs.mbs_paper(d["months"]), d["N"], threads=1)[:, None]


def _oracle(seq, M, seed, insts=INSTS):
    """Oracle theta of every instrument (instruments on host threads, one each)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(O.max_threads(), 16)) as ex:
        return list(ex.map(lambda a: _oracle_one(seq, M, seed, *a), list(enumerate(insts))))


@pytest.mark.parametrize("seq", [O.SOBOL_DS, O.RASRAP, O.PHILOX, O.SOBOL_LMS])
def test_batch_matches_oracle_per_instrument(R, seq):
    M, seed = 2, 11
    got = R.price_batch(INSTS, M, seq, seed)
    ref = _oracle(seq, M, seed)
    for d, g, r in zip(INSTS, got, ref):
        assert g.shape == r.shape
        assert np.all(np.abs(g - r) <= 1e-4 * np.abs(r)), (d, np.max(np.abs(g - r) / np.abs(r)))


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


def test_batch_autotuner_keeps_the_fastest_tile_and_reuses_its_cache(R, tmp_path, monkeypatch):
    """The autotuner times the three candidate tiles, keeps the fastest (recorded in its cache
    with every candidate's time) and a later plan of the same batch takes the cached tile."""
    import json
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("RQMC_AUTOTUNE_CACHE", str(cache))
    monkeypatch.delenv("RQMC_AUTOTUNE", raising=False)
    insts = INSTS[:3]
    p = R.Plan.batch(insts, 2, O.SOBOL_DS, 7)
    threads, ppt = p.launch_shape()
    p.close()
    kv = json.loads(cache.read_text())
    keys = [k for k in kv if "|us_ppt" not in k]
    assert len(keys) == 1 and kv[keys[0]] == ppt and threads == 256
    times = {int(k.rsplit("ppt", 1)[1]): v for k, v in kv.items() if k.startswith(keys[0] + "|us_ppt")}
    assert sorted(times) == [4, 8, 16]
    assert times[ppt] == min(times.values())
    # a different tile written into the cache is taken as it stands: no tuning, same batch key
    other = next(c for c in (16, 8, 4) if c != ppt)
    kv[keys[0]] = other
    cache.write_text(json.dumps(kv, indent=2))   # the cache keeps one "key": value entry per line
    q = R.Plan.batch(insts, 2, O.SOBOL_DS, 7)
    assert q.launch_shape() == (256, other)
    got = q.split_batch(q.execute())
    q.close()
    ref = _oracle(O.SOBOL_DS, 2, 7, insts)
    for d, g, r in zip(insts, got, ref):
        assert np.all(np.abs(g - r) <= 1e-4 * np.abs(r)), (d, np.max(np.abs(g - r) / np.abs(r)))


@pytest.mark.parametrize("subset", [[1, 4], [0, 2, 3], [5, 6], [6, 1]])
def test_batch_with_some_work_classes_empty(R, subset):
    """Batches that leave one or two of the three work classes empty (MBS only, small
    strips only, 160-forward strips only, and no small strips) still match the oracle."""
    insts = [INSTS[k] for k in subset]
    M, seed = 2, 3
    got = R.price_batch(insts, M, O.SOBOL_DS, seed)
    ref = _oracle(O.SOBOL_DS, M, seed, insts)
    for d, g, r in zip(insts, got, ref):
        assert np.all(np.abs(g - r) <= 1e-4 * np.abs(r)), (d, np.max(np.abs(g - r) / np.abs(r)))


@pytest.mark.parametrize("seq,M", [(O.SOBOL_DS, 2), (O.RASRAP, 1)])
def test_batch_512_instrument_draw_with_capped_N(R, seq, M):
    """The 512-instrument draw of the batch workload (384 caplet strips of 8..160 forwards
    and 128 MBS of 120..360 months, sizes as drawn from seed 1) with every instrument's N
    capped at 2^11 so that the oracle prices all 512 in well under a minute on the host.
    All three work classes and the full ticket queues run; each instrument's values are
    checked against the oracle."""
    desc = inputs.batch_instruments(1)
    insts = [dict(d, N=min(d["N"], 1 << 11), rate=0.05, vol=0.15, strike=0.05) if d["kind"] == "lmm"
             else dict(d, N=min(d["N"], 1 << 11)) for d in desc]
    got = R.price_batch(insts, M, seq, 1)
    ref = _oracle(seq, M, 1, insts)
    worst = max(float(np.max(np.abs(g - r) / np.abs(r))) for g, r in zip(got, ref))
    assert worst <= 1e-4, worst


def test_batch_stats_report_the_load_balance(R):
    """The per-CTA timing records of the persistent kernels: the busiest SM over the mean SM
    is at least 1, every non-empty work class has a positive span within the whole span, and
    an empty class reports 0."""
    p = R.Plan.batch([INSTS[k] for k in (0, 1, 2, 3)], 3, O.SOBOL_DS, 5)   # no strip beyond 80 forwards
    p.execute()
    st = p.batch_stats()
    p.close()
    assert st["imbalance"] >= 1.0 and st["span_ms"] > 0.0
    assert st["class_160_ms"] == 0.0
    assert 0.0 < st["class_mbs_ms"] <= st["span_ms"] * 1.0001 and 0.0 < st["class_small_ms"] <= st["span_ms"] * 1.0001
