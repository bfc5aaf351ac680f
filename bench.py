#!/usr/bin/env python3
"""Throughput of the RQMC hot path on GB300: path-steps/s.

Workload (default): LIBOR-market-model caplets, one factor, 40 quarterly
forwards, flat 5 % curve, 15 % vol, strikes 4.5/5/5.5 %, log-Euler spot-measure
steps (s = 40), N = 65536 points per replication, M = 64 replications, on the
three sequences of the comparison (Rasrap, digitally shifted Sobol', Philox),
FP32 paths with Kahan sums.  One step = one plan execute per sequence
(3 x N x M x 40 = 503M path-steps).  The result of every timed configuration is
checked against the FP64 oracle (two replications at full N) before timing.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the oracle is the reference implementation).
Under torchrun each rank prices its own contiguous range of N points of every
replication (plan offset = rank x N, weak scaling); each step ends with the one
exchange of the estimator, an all-reduce of the M x 120 theta values per sequence.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_FWD, N_PATHS, M_REPL, SEED = 40, 65536, 64, 1
SEQS = ("rasrap", "sobol_ds", "philox")
L2_FLUSH_BYTES = 512 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one lmm_caplet_kernel<40, 1, float> launch
# (Rasrap) of this workload, from an ncu capture of the kernel as committed; set to None
# whenever that kernel changes until it is captured again.
LMM_TRAFFIC_BYTES = 714.8e3


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def lmm_algorithmic_ops(nf, nK, paths):
    """Source-level operations of one fused caplet launch.
    MUFU: ex2 + rcp per forward update; per step lg2 (inverse CDF) and ex2 + rcp
    (fixed forward and numeraire).  Returned as SFU issue slots: on GB300 ex2 issues at
    32 per SM per clock and rcp/lg2 at 16, so an ex2 counts half a slot.
    FP32 pipe: 4 per forward update (1 + e, drift, state), 16 per inverse CDF, 4 per step,
    4 per strike."""
    upd = nf * (nf + 1) // 2
    n_ex2, n_rcp, n_lg2 = upd + nf, upd + nf, nf
    slots = 0.5 * n_ex2 + n_rcp + n_lg2
    fma = 4 * upd + nf * (16 + 4 + 4 * nK)
    return slots * paths, fma * paths


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for k, v in zip(names, c[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(k)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args, rank, world):
    import torch
    from paper_1408_5526_gb300 import inputs, rqmc, shard

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rqmc.load()
    lm = inputs.lmm_flat(N_FWD)
    K = inputs.LMM_STRIKES
    seed = SEED
    offset, n_local = shard.point_range(rank, world, N_PATHS * world)
    plans = [rqmc.Plan.caplets(lm, K, n_local, M_REPL, s, seed, prec="fp32", offset=offset) for s in SEQS]
    outs = [torch.empty(p.output_size(), dtype=torch.float64, device=dev) for p in plans]
    stream = torch.cuda.current_stream()

    # parity gate: the timed configuration must match the oracle (rank 0 checks)
    parity = None
    if rank == 0 and not args.skip_parity:
        import oracle as O
        worst = 0.0
        for p, s, o in zip(plans, SEQS, outs):
            p.execute(o)
            th = o.cpu().numpy().reshape(M_REPL, -1)
            q = O.Sequence(rqmc._SEQ[s], N_FWD, M_REPL, seed, joe_kuo=inputs.joe_kuo_table())
            th_o = O.lmm_caplets(q, lm, K, N_PATHS, m_range=(M_REPL - 1, M_REPL))
            t = th_o.reshape(1, N_FWD, len(K))
            scale = np.maximum(np.abs(t), np.abs(t[:, :, 1:2])).reshape(1, -1)
            worst = max(worst, float(np.max(np.abs(th[M_REPL - 1:] - th_o) / scale)))
        parity = {"max_scaled_err": worst, "tol": 1e-4, "ok": worst <= 1e-4, "checked": "m=63, all 120 outputs"}

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        for p, o in zip(plans, outs):
            p.execute(o, stream)
            if world > 1:
                shard.combine_theta(o, n_local)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in SEQS]
           for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))   # L2 flush outside the timed intervals
            ev[k][0].record(stream)
            for j, (p, o) in enumerate(zip(plans, outs)):
                kev[k][j][0].record(stream)
                p.execute(o, stream)
                kev[k][j][1].record(stream)
                if world > 1:
                    shard.combine_theta(o, n_local)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        time.sleep(0.25)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launch_ms = [a.elapsed_time(b) for row in kev for a, b in row]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    units = N_PATHS * M_REPL * N_FWD * len(SEQS) * args.steps * world
    value = units / (total_ms / 1e3)

    # e2e: the one-shot C-ABI call with host buffers (tables, H2D, kernels, D2H, stats) per sequence
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in SEQS:
            rqmc.price_caplets(lm, K, N_PATHS, M_REPL, s, seed, prec="fp32")
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = N_PATHS * M_REPL * N_FWD * len(SEQS) * world / (statistics.median(e2e_ms) / 1e3)
    h2d = 40 * 64 + 40 * 32 * 4   # Halton base constants (Rasrap) + Sobol' direction numbers
    d2h = len(SEQS) * (M_REPL * N_FWD * len(K) * 8 + 16)

    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    mufu_peak = 16 * 152 * sm_max * 1e6           # SFU issue slots/s: 16 per SM per clock
    fma_peak = 128 * 152 * sm_max * 1e6           # FP32 lane-ops/s: 128 per SM per clock
    mufu, fma = lmm_algorithmic_ops(N_FWD, len(K), N_PATHS * M_REPL)
    per_launch_s = statistics.mean(launch_ms) / 1e3
    a_mufu, a_fma = mufu / per_launch_s, fma / per_launch_s
    roof = {"bound": "alu", "pipe": "sfu" if a_mufu / mufu_peak >= a_fma / fma_peak else "fma",
            "achieved": round(a_mufu / 1e12, 4), "peak": round(mufu_peak / 1e12, 4),
            "unit": "T SFU issue slots/s (ex2 = 1/2 slot, rcp/lg2 = 1 slot)",
            "frac": round(a_mufu / mufu_peak, 4), "traffic": LMM_TRAFFIC_BYTES,
            "traffic_unit": "DRAM bytes per launch (ncu, Rasrap launch; tables only)",
            "fma_achieved": round(a_fma / 1e12, 3), "fma_peak": round(fma_peak / 1e12, 3),
            "fma_frac": round(a_fma / fma_peak, 4),
            "kernel": "lmm_caplet_kernel<40,float> + theta_kernel",
            "launch_ms": round(per_launch_s * 1e3, 4),
            "peak_source": "derived: 16 SFU slots / 128 FP32 lanes per SM per clock x 152 SMs x sm_max_mhz"}
    if rank == 0:
        # the same pipes measured on this GPU (rqmc_probe_pipes), next to the derived peak
        probe = rqmc.probe_pipes()
        # one SFU issue slot = one rcp or lg2 = two ex2, as the roofline counts them
        slot_rate = min(probe["rcp"], probe["lg2"], 0.5 * probe["ex2"])
        roof["probe_per_sm_clk"] = {k: round(v, 2) for k, v in probe.items()}
        roof["frac_of_probed_sfu"] = round(a_mufu / (slot_rate * 152 * sm_max * 1e6), 4) if slot_rate else None
    extra = other_workloads(args, dev, seed) if (rank == 0 and not args.no_extra) else None
    cpu = cpu_baseline(args) if (rank == 0 and not args.no_cpu) else None
    cpu_gen = cpu_generators() if (rank == 0 and not args.no_cpu) else None
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": "path-steps/s", "value": value, "unit": "path-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "lmm_caplets_40fwd_N65536_M64_rasrap+sobol_ds+philox", "n_fwd": N_FWD,
                       "N": N_PATHS, "M": M_REPL, "strikes": list(map(float, K)), "sequences": list(SEQS),
                       "precision": "fp32 paths, Kahan sums, fp64 replication reduction",
                       "path_steps_per_step": N_PATHS * M_REPL * N_FWD * len(SEQS) * world,
                       "parallelism": (f"point ranges x{world}: offset = rank x N, "
                                       "theta all-reduced per sequence per step") if world > 1 else "1 GPU",
                       "l2": "flushed (512 MiB write) before every timed step, outside its interval",
                       "timing": "sum of per-step CUDA-event intervals"},
            "parity": parity,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "path-steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms": statistics.median(e2e_ms),
                    "api": "price_caplets (host buffers) x 3 sequences"},
            "gpu_launches": args.steps * sum(p.launches() for p in plans),
            "clocks": clocks,
            "workloads": extra,
            "cpu_generators_table1": cpu_gen,
        }
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


def _time_plan(execute, reps, flush):
    import torch
    for _ in range(3):
        execute()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        execute()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def other_workloads(args, dev, seed):
    """The other configurations of the scope, one timed figure each (median of a few
    launches, L2 flushed before each, inputs resident): product integrand (FP64),
    LMM caplets in FP64, MBS (FP32), two-factor adjoint Greeks (FP32), the
    512-instrument batch (FP32, graph launch), the Treasury-curve study of Sec. 5 (std, time
    and efficiency against N) and the point stream (HBM write GB/s)."""
    import torch
    from paper_1408_5526_gb300 import inputs, rqmc
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    # product integrand, s = 8, N = 4096, M = 32, random-start Halton, FP64
    p = rqmc.Plan.product(8, 4096, 32, "halton_rs", seed, inputs.product_weights(8), prec="fp64")
    o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
    ms = _time_plan(lambda: p.execute(o), 10, flush)
    th = o.cpu().numpy()
    out["product_s8_N4096_M32_fp64"] = {"ms": ms, "path_steps_per_s": 8 * 4096 * 32 / (ms / 1e3),
                                        "rq": float(th.mean()), "exact": 1.0}
    p.close()
    # LMM caplets in FP64 (same 40-forward workload), Rasrap
    lm = inputs.lmm_flat(N_FWD)
    p = rqmc.Plan.caplets(lm, inputs.LMM_STRIKES, N_PATHS, M_REPL, "rasrap", seed, prec="fp64")
    o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
    ms = _time_plan(lambda: p.execute(o), 2, flush)
    out["lmm_caplets_40_N65536_M64_fp64_rasrap"] = {"ms": ms,
                                                    "path_steps_per_s": N_PATHS * M_REPL * N_FWD / (ms / 1e3)}
    p.close()
    # MBS, 360 months, N = 65536, M = 64, FP32 + Kahan
    mb = inputs.mbs_paper(360)
    res = {}
    for s_ in SEQS:
        p = rqmc.Plan.mbs(mb, N_PATHS, M_REPL, s_, seed, prec="fp32")
        o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
        ms = _time_plan(lambda: p.execute(o), 3, flush)
        res[s_] = {"ms": ms, "path_steps_per_s": N_PATHS * M_REPL * 360 / (ms / 1e3), "rq": float(o.mean())}
        p.close()
    out["mbs_360_N65536_M64_fp32"] = res
    # adjoint Greeks: two-factor 80-forward strip, N = 2^18, M = 32, FP32 paths
    l2 = inputs.lmm_two_factor(80, seed=seed)
    p = rqmc.Plan.adjoint(l2, [0.05], np.ones(80), 1 << 18, 32, "sobol_ds", seed)
    o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
    ms = _time_plan(lambda: p.execute(o), 2, flush)
    out["adjoint_2f_80_N262144_M32_fp32_sobol"] = {"ms": ms,
                                                   "path_steps_per_s": (1 << 18) * 32 * 160 / (ms / 1e3)}
    p.close()
    # 512-instrument batch, one graph launch
    desc = inputs.batch_instruments(seed)
    insts = [dict(d, rate=0.05, vol=0.15, strike=0.05) if d["kind"] == "lmm" else d for d in desc]
    p = rqmc.Plan.batch(insts, 32, "sobol_ds", seed)
    o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
    ms = _time_plan(lambda: p.execute(o), 1, flush)
    steps = sum(d["N"] * 32 * (d["n_fwd"] if d["kind"] == "lmm" else d["months"]) for d in desc)
    out["batch_512_M32_fp32_sobol"] = {"ms": ms, "path_steps_per_s": steps / (ms / 1e3), "path_steps": steps}
    p.close()
    # Sec. 5's Treasury-curve study: caplet on L_10 (T = 5, delta = 0.5, K = 1 %, sigma = 4 %)
    # from the 24 Feb 2012 curve; std of M = 100 independent estimates, time and efficiency
    # (std x time) against N, and the fitted convergence rate of the std
    st = inputs.TREASURY_STUDY
    lmt = inputs.lmm_treasury(st["T"], st["delta"], st["vol"])
    study = {}
    for s_ in SEQS + ("sobol_lms",):
        rows = []
        for e in range(10, 21, 2):
            pt = rqmc.Plan.caplets(lmt, [st["K"]], 1 << e, st["M"], s_, seed, prec="fp32")
            ot = torch.empty(pt.output_size(), dtype=torch.float64, device=dev)
            ms = _time_plan(lambda: pt.execute(ot), 3, flush)
            th = ot.cpu().numpy().reshape(st["M"], -1)[:, lmt["n_fwd"] - 1]
            pt.close()
            rows.append({"N": 1 << e, "rq": float(th.mean()), "std": float(th.std(ddof=1)), "ms": ms,
                         "efficiency": float(th.std(ddof=1)) * ms})
        lx = np.log([r["N"] for r in rows])
        ly = np.log([r["std"] for r in rows])
        study[s_] = {"rate": float(np.polyfit(lx, ly, 1)[0]), "by_N": rows}
    out["lmm_treasury_study_T5_M100_fp32"] = study
    # Matousek-scrambled Sobol' on the headline caplet workload (same kernel, scrambled tables)
    pl_ = rqmc.Plan.caplets(inputs.lmm_flat(N_FWD), inputs.LMM_STRIKES, N_PATHS, M_REPL, "sobol_lms", seed,
                            prec="fp32")
    o_ = torch.empty(pl_.output_size(), dtype=torch.float64, device=dev)
    ms = _time_plan(lambda: pl_.execute(o_), 3, flush)
    pl_.close()
    out["lmm_caplets_40_N65536_M64_fp32_sobol_lms"] = {"ms": ms,
                                                       "path_steps_per_s": N_PATHS * M_REPL * N_FWD / (ms / 1e3)}
    # point stream: s = 360, N = 65536, M = 64 FP32 normals, written to HBM
    buf = torch.empty((M_REPL, 360, N_PATHS), dtype=torch.float32, device=dev)
    res = {}
    peaks = _peaks()
    for s_ in SEQS:
        pp = rqmc.Plan.points(360, N_PATHS, M_REPL, s_, seed, prec="fp32", transform="normal")
        ms = _time_plan(lambda: pp.execute(buf), 3, flush)   # kernel only: tables built once
        pp.close()
        ms1 = _time_plan(lambda: rqmc.rqmc_points(360, N_PATHS, M_REPL, s_, seed, transform="normal", out=buf), 2,
                         flush)   # one-shot call: tables + kernel
        gbs = buf.numel() * 4 / (ms / 1e3) / 1e9
        res[s_] = {"ms": ms, "GB_per_s": gbs, "frac_of_measured_hbm": gbs / float(peaks.get("hbm_gbs", 6800.0)),
                   "gnumbers_per_s": buf.numel() / (ms / 1e3) / 1e9, "one_shot_ms": ms1}
    out["points_s360_N65536_M64_fp32_normal"] = res
    del buf
    return out


def cpu_baseline(args, seconds_hint=True):
    """The FP64 oracle as it stands, OpenMP over replications, on a bounded sample:
    Rasrap, full N, one replication per host thread (capped at 16)."""
    import oracle as O
    from paper_1408_5526_gb300 import inputs
    cores = min(O.max_threads(), 16)
    lm = inputs.lmm_flat(N_FWD)
    K = inputs.LMM_STRIKES
    q = O.Sequence(O.RASRAP, N_FWD, M_REPL, SEED)
    t0 = time.perf_counter()
    O.lmm_caplets(q, lm, K, N_PATHS, m_range=(0, cores), threads=cores)
    dt = time.perf_counter() - t0
    return {"value": cores * N_PATHS * N_FWD / dt, "unit": "path-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"rasrap, {cores} replications x N={N_PATHS} x 40 steps ({dt:.1f} s)"}


def cpu_generators():
    """Table 1 style CPU generator throughput on this host, for context beside the GPU point
    stream: the recursive generators (Algorithm 2 for Rasrap, Gray-code order for Sobol')
    and the counter-based forms (Algorithm 3, binary-order Sobol', Philox) of the oracle,
    raw integer states of s = 40 dimensions, M = 8, N = 65536, one thread and all threads
    (capped at 16)."""
    import oracle as O
    from paper_1408_5526_gb300 import inputs
    jk = inputs.joe_kuo_table()
    cores = min(O.max_threads(), 16)
    out = {"cores": cores, "unit": "GNumbers/s", "sample": "s=40, M=8, N=65536 raw states"}
    for name, seq in (("rasrap", O.RASRAP), ("sobol_ds", O.SOBOL_DS), ("philox", O.PHILOX)):
        q = O.Sequence(seq, 40, 8, SEED, joe_kuo=jk if seq == O.SOBOL_DS else None)
        row = {}
        for th in (1, cores):
            t0 = time.perf_counter()
            a = q.stream(0, 65536, threads=th)
            row[f"recursive_{th}t"] = a.size / (time.perf_counter() - t0) / 1e9
        t0 = time.perf_counter()
        b = q.points(65536, transform=O.RAW, threads=cores)
        row[f"counter_based_{cores}t"] = b.size / (time.perf_counter() - t0) / 1e9
        out[name] = row
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    from paper_1408_5526_gb300 import inputs
    cores = min(O.max_threads(), 16)
    lm = inputs.lmm_flat(N_FWD)
    K = inputs.LMM_STRIKES
    n_sample = 8192
    for _ in range(args.warmup):
        pass
    t = []
    for k in range(args.steps):
        s = SEQS[k % len(SEQS)]
        q = O.Sequence({"rasrap": O.RASRAP, "sobol_ds": O.SOBOL_DS, "philox": O.PHILOX}[s], N_FWD, M_REPL, SEED,
                       joe_kuo=inputs.joe_kuo_table())
        t0 = time.perf_counter()
        O.lmm_caplets(q, lm, K, n_sample, m_range=(0, cores), threads=cores)
        t.append(time.perf_counter() - t0)
    units = cores * n_sample * N_FWD
    value = units * len(t) / sum(t)
    line = {"impl": "reference", "metric": "path-steps/s", "value": value, "unit": "path-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lmm_caplets_40fwd_N65536_M64_rasrap+sobol_ds+philox",
                       "sample": f"{cores} replications x N={n_sample} per step, sequences cycled"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "path-steps/s",
                             "sample": f"{cores} replications x N={n_sample} x 40 steps per step"},
            "e2e": {"value": value, "unit": "path-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--skip-parity", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other-configuration figures")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
