"""Host logic of the multi-rank path: point-range sharding and the theta combination.

The counter-based generators let the points of one replication be split into contiguous
ranges (the plans' `offset`); the estimator of Sec. 1 is then recovered by the
count-weighted mean of the per-rank estimates.  Two gloo ranks on the CPU price their
ranges with the oracle and combine through `shard.combine_theta`; the result must equal
the unsharded oracle estimate up to summation order.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1408_5526_gb300 import inputs, shard

JK = inputs.joe_kuo_table()


@pytest.mark.parametrize("n_total,world", [(0, 1), (7, 1), (3001, 2), (4096, 4), (5, 8), (65536, 3)])
def test_point_range_partitions_contiguously(n_total, world):
    ranges = [shard.point_range(r, world, n_total) for r in range(world)]
    pos = 0
    for off, cnt in ranges:
        assert off == pos and cnt >= 0
        pos += cnt
    assert pos == n_total
    counts = [c for _, c in ranges]
    assert max(counts) - min(counts) <= 1


def test_point_range_rejects_bad_arguments():
    for args in ((2, 2, 10), (-1, 2, 10), (0, 0, 10), (0, 2, -1)):
        with pytest.raises(ValueError):
            shard.point_range(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_total, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, cnt = shard.point_range(rank, world, n_total)
        lm = inputs.lmm_flat(8)
        K = inputs.LMM_STRIKES
        out = {}
        for name, seq in (("rasrap", O.RASRAP), ("sobol_ds", O.SOBOL_DS), ("philox", O.PHILOX)):
            q = O.Sequence(seq, 8, 3, 5, joe_kuo=JK)
            th = O.lmm_caplets(q, lm, K, cnt, offset=off, threads=1)
            out[name] = shard.combine_theta(torch.from_numpy(np.ascontiguousarray(th)), cnt).numpy()
            out[name + "_known_total"] = shard.combine_theta(torch.from_numpy(np.ascontiguousarray(th)), cnt,
                                                             total=n_total).numpy()
            q8 = O.Sequence(seq, 8, 3, 5, joe_kuo=JK)
            tp = O.product_theta(q8, cnt, inputs.product_weights(8), offset=off, threads=1)
            out[name + "_product"] = shard.combine_theta(torch.from_numpy(np.ascontiguousarray(tp)), cnt).numpy()
        if rank == 0:
            np.savez(result_path, **out)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsharded_estimate(tmp_path):
    O.build()
    n_total, world = 3001, 2            # uneven split: 1501 + 1500 points
    path = str(tmp_path / "combined.npz")
    mp.spawn(_worker, args=(world, _free_port(), n_total, path), nprocs=world, join=True)
    got = np.load(path)
    lm = inputs.lmm_flat(8)
    for name, seq in (("rasrap", O.RASRAP), ("sobol_ds", O.SOBOL_DS), ("philox", O.PHILOX)):
        q = O.Sequence(seq, 8, 3, 5, joe_kuo=JK)
        ref = O.lmm_caplets(q, lm, inputs.LMM_STRIKES, n_total, threads=1)
        np.testing.assert_allclose(got[name], ref, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(got[name + "_known_total"], ref, rtol=1e-12, atol=1e-15)
        q8 = O.Sequence(seq, 8, 3, 5, joe_kuo=JK)
        refp = O.product_theta(q8, n_total, inputs.product_weights(8), threads=1)
        np.testing.assert_allclose(got[name + "_product"], refp, rtol=1e-12, atol=1e-15)


def test_combine_theta_single_process_is_identity():
    th = torch.arange(12, dtype=torch.float64).reshape(3, 4)
    assert torch.equal(shard.combine_theta(th, 17), th)
    with pytest.raises(TypeError):
        shard.combine_theta(th.float(), 17)


def test_point_range_threads_reproduce_the_oracle():
    """The test-side helper that runs the oracle over contiguous point ranges on host
    threads (tests/oracle_par.py) returns the estimate of one sequential call."""
    import oracle_par
    lm = inputs.lmm_two_factor(6, seed=2)
    K = np.array([0.05])
    w = np.ones(6)
    for seq in (O.RASRAP, O.SOBOL_DS, O.PHILOX):
        q = O.Sequence(seq, 12, 2, 3, joe_kuo=JK)
        ref = O.lmm_adjoint(q, lm, K, w, 1001, threads=1)
        got = oracle_par.over_points(lambda off, n: O.lmm_adjoint(q, lm, K, w, n, offset=off, threads=1), 1001,
                                     threads=5)
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-17)
        mb = inputs.mbs_paper(24)
        q = O.Sequence(seq, 24, 2, 3, joe_kuo=JK)
        np.testing.assert_allclose(
            oracle_par.over_points(lambda off, n: O.mbs_theta(q, mb, n, offset=off, threads=1), 777, threads=4),
            O.mbs_theta(q, mb, 777, threads=1), rtol=1e-13)
