"""Single workloads for profiler captures and quick timings.

Each case builds one device-resident plan, executes it a few times (warm-up, then timed
with CUDA events) and prints the median time, so that a profiler can pick a launch of one
kernel by its position (``ncu -k regex:<kernel> -s <warm-up launches> -c 1``).

    python -m paper_1408_5526_gb300.cases caplets --n-fwd 160 --seq sobol_ds --N 65536 --M 8
    python -m paper_1408_5526_gb300.cases batch --n-fwd 160 --N 65536 --M 8
    python -m paper_1408_5526_gb300.cases adjoint --N 65536 --M 8
    python -m paper_1408_5526_gb300.cases mbs --months 360 --N 65536 --M 8 --seq rasrap
    python -m paper_1408_5526_gb300.cases points --s 360 --N 65536 --M 4 --seq rasrap

Every case runs the product path only (the CUDA library through the C ABI).
"""
from __future__ import annotations

import argparse
import statistics

import numpy as np


def _time(fn, reps: int, warm: int) -> float:
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def main(argv=None) -> None:
    import torch

    from . import inputs, rqmc

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=["caplets", "batch", "adjoint", "mbs", "points"])
    ap.add_argument("--n-fwd", type=int, default=40)
    ap.add_argument("--seq", default="sobol_ds")
    ap.add_argument("--N", type=int, default=65536)
    ap.add_argument("--M", type=int, default=8)
    ap.add_argument("--s", type=int, default=360, help="dimensions of the point stream")
    ap.add_argument("--months", type=int, default=360)
    ap.add_argument("--strikes", type=int, default=1, choices=[1, 3], help="ATM only, or 4.5/5/5.5 %%")
    ap.add_argument("--transform", default="normal", choices=["uniform", "normal"])
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    rqmc.load()
    K = inputs.LMM_STRIKES if a.strikes == 3 else np.array([0.05])
    if a.case == "caplets":
        plan = rqmc.Plan.caplets(inputs.lmm_flat(a.n_fwd), K, a.N, a.M, a.seq, 1, prec="fp32")
        what = f"{a.n_fwd}-forward caplets, {a.seq}"
        work = a.n_fwd * (a.n_fwd + 1) // 2 * a.N * a.M
    elif a.case == "batch":
        # one instrument: its items (replication, tile) make up one work class of the batch
        plan = rqmc.Plan.batch([{"kind": "lmm", "n_fwd": a.n_fwd, "N": a.N}], a.M, a.seq, 1)
        what = f"batch of one {a.n_fwd}-forward strip, {a.seq}"
        work = a.n_fwd * (a.n_fwd + 1) // 2 * a.N * a.M
    elif a.case == "adjoint":
        lm = inputs.lmm_two_factor(80, seed=1)
        plan = rqmc.Plan.adjoint(lm, [0.05], np.ones(80), a.N, a.M, a.seq, 1)
        what = f"two-factor 80-forward adjoint, {a.seq}"
        work = 80 * 81 // 2 * a.N * a.M
    elif a.case == "mbs":
        plan = rqmc.Plan.mbs(inputs.mbs_paper(a.months), a.N, a.M, a.seq, 1, prec="fp32")
        what = f"MBS, {a.months} months, {a.seq}"
        work = a.months * a.N * a.M
    else:
        plan = rqmc.Plan.points(a.s, a.N, a.M, a.seq, 1, transform=a.transform)
        what = f"point stream s={a.s}, {a.seq} {a.transform}"
        work = a.s * a.N * a.M
    dtype = torch.float32 if a.case == "points" else torch.float64
    out = torch.empty(plan.output_size(), dtype=dtype, device="cuda")
    ms = _time(lambda: plan.execute(out), a.reps, a.warmup)
    unit = {"points": "coordinates", "mbs": "path-months"}.get(a.case, "forward updates")
    print(f"{what}, N={a.N}, M={a.M}: {ms:.3f} ms per execute, {work / ms / 1e9:.3f} T {unit}/s "
          f"({plan.launches()} launches per execute)", flush=True)
    plan.close()


if __name__ == "__main__":
    main()
