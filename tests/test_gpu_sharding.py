"""Point-range sharding through the CUDA path: two gloo ranks, each a process on the one
GPU, price their own contiguous range of every replication's points through plans with an
`offset` and combine with shard.combine_theta (with the counts exchanged, and with the
total known on the host).  The combined theta must equal the unsharded FP64 oracle within
the tolerances of the single-GPU parity tests.  The ranks' kernels never wait on one
another; the one exchange is the all-reduce of theta on the host (gloo)."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

JK = inputs.joe_kuo_table()
pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n_total, path):
    import torch
    import torch.distributed as dist
    from paper_1408_5526_gb300 import rqmc, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        rqmc.load()
        off, cnt = shard.point_range(rank, world, n_total)
        lm = inputs.lmm_flat(16, vol=0.2)
        mb = inputs.mbs_paper(120)
        out = {}
        for name, seq in (("rasrap", "rasrap"), ("sobol_ds", "sobol_ds"), ("philox", "philox")):
            for prec in ("fp64", "fp32"):
                with rqmc.Plan.caplets(lm, inputs.LMM_STRIKES, cnt, 3, seq, 5, prec=prec, offset=off) as p:
                    th = p.execute().cpu()
                out[f"{name}_caplets_{prec}"] = shard.combine_theta(th, cnt).numpy()
                out[f"{name}_caplets_{prec}_known"] = shard.combine_theta(th, cnt, total=n_total).numpy()
            with rqmc.Plan.mbs(mb, cnt, 3, seq, 5, prec="fp32", offset=off) as p:
                th = p.execute().cpu()
            out[f"{name}_mbs"] = shard.combine_theta(th, cnt, total=n_total).numpy()
        torch.cuda.synchronize()
        if rank == 0:
            np.savez(path, **out)
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_the_cuda_path_reproduce_the_unsharded_oracle(tmp_path):
    import torch.multiprocessing as mp
    from paper_1408_5526_gb300 import _build
    _build.build()                     # once, before the ranks load the library
    n_total, world = 3001, 2           # uneven split: 1501 + 1500 points
    path = str(tmp_path / "combined.npz")
    mp.spawn(_rank, args=(world, _free_port(), n_total, path), nprocs=world, join=True)
    got = np.load(path)
    lm = inputs.lmm_flat(16, vol=0.2)
    mb = inputs.mbs_paper(120)
    K = inputs.LMM_STRIKES
    for name, seq in (("rasrap", O.RASRAP), ("sobol_ds", O.SOBOL_DS), ("philox", O.PHILOX)):
        ref = O.lmm_caplets(O.Sequence(seq, 16, 3, 5, joe_kuo=JK), lm, K, n_total).reshape(-1)
        t = ref.reshape(3, 16, 3)
        scale = np.maximum(np.abs(t), np.abs(t[:, :, 1:2])).reshape(-1)
        for suffix in ("", "_known"):
            np.testing.assert_allclose(got[f"{name}_caplets_fp64{suffix}"], ref, rtol=1e-11, atol=1e-15)
            assert np.all(np.abs(got[f"{name}_caplets_fp32{suffix}"] - ref) <= 1e-4 * scale)
        ref_m = O.mbs_theta(O.Sequence(seq, 120, 3, 5, joe_kuo=JK), mb, n_total)
        np.testing.assert_allclose(got[f"{name}_mbs"].reshape(-1), ref_m, rtol=1e-4)
