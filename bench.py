#!/usr/bin/env python3
"""Throughput of the RQMC hot path on GB300: path-steps/s.

Workload (default): LIBOR-market-model caplets, one factor, 40 quarterly
forwards, flat 5 % curve, 15 % vol, strikes 4.5/5/5.5 %, log-Euler spot-measure
steps (s = 40), N = 65536 points per replication, M = 64 replications, on the
three sequences of the comparison (Rasrap, digitally shifted Sobol', Philox),
FP32 paths with Kahan sums.  One step = one plan execute per sequence
(3 x N x M x 40 = 503M path-steps).

A result counts only when it matches the FP64 oracle in the same run: the
`cpu_baseline` leg runs the oracle on the host cores over the whole headline
workload (all 64 replications of all three sequences at full N) and the parity
block compares every theta_N^m with it (tolerance 1e-4 of the larger of the
value and the at-the-money caplet of the same maturity).  The other
configurations of the scope each carry their own timed oracle sample, parity
check, roofline fraction and error against the oracle.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the oracle is the reference implementation).
Under torchrun each rank prices its own contiguous range of N points of every
replication (plan offset = rank x N, weak scaling); each step ends with the one
exchange of the estimator, a single all-reduce of the 3 x M x 120 theta values
of the three sequences (the combined counts are known on the host, so nothing is
read back inside the step).
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
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_FWD, N_PATHS, M_REPL, SEED = 40, 65536, 64, 1
SEQS = ("rasrap", "sobol_ds", "philox")
L2_FLUSH_BYTES = 512 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one plan execute of this workload (Rasrap:
# points_run_kernel 0.7 + 609.9 MB, lmm_caplet_kernel<40> 671.2 + 11.7 MB, theta_kernel 7.9 MB),
# from an ncu capture of the kernels as committed (profiles/lmm_caplet_kernel_40fwd_N65536_M64.md);
# None whenever one of them has changed since the capture.
LMM_TRAFFIC_BYTES = 1301.4e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def lmm_algorithmic_ops(nf, nK, paths):
    """Source-level operations of one caplet plan execute (normals, paths, payoffs).
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


def lmm_fp64_pairs(nf, paths):
    """FP64 forward updates of one caplet launch: one exp + one reciprocal per forward update
    and per fixing (the pair the probe's FP64 update measures)."""
    return (nf * (nf + 1) // 2 + nf) * paths


def mbs_algorithmic_ops(months, paths):
    """Per month and path: SFU lg2 (inverse CDF), ex2 (rate), rcp (arctangent reflection),
    rcp (discount) = 3.5 slots; FP32 17 (inverse CDF) + 15 (arctangent) + 16 (rate, prepayment,
    cash flow, Kahan sum, discount and survival factors) = 48."""
    return 3.5 * months * paths, 48.0 * months * paths


def adjoint_algorithmic_ops(nf, d, paths):
    """Pathwise adjoint of a d-factor strip, per path: the forward sweep's nf(nf+1)/2 forward
    updates (ex2 + rcp, 2 + 3d FP32), the reverse sweep's as many steps back (the pre-step state
    reconstructed from the post-step one, 2 + d FP32, and its drift factor again, ex2 + rcp)
    with their adjoint updates (3 + 7d FP32), the fixings' ex2 + rcp in both sweeps, and 2 nf d
    inverse CDFs (the normals drawn in the forward sweep and regenerated in the reverse one,
    lg2 + 17 FP32 each).  SFU slots and FP32 operations."""
    upd = nf * (nf + 1) // 2
    slots = 1.5 * (2 * upd + 2 * nf) + 2 * nf * d
    fma = (2 + 3 * d) * upd + (2 + d) * upd + (3 + 7 * d) * upd + 2 * nf * d * 17
    return slots * paths, fma * paths


def caplet_scaled_err(th, th_o, nK):
    """|theta - theta_oracle| / max(|theta_oracle|, theta_ATM of the same maturity)."""
    M = th_o.shape[0]
    t = th_o.reshape(M, -1, nK)
    scale = np.maximum(np.abs(t), np.abs(t[:, :, nK // 2:nK // 2 + 1])).reshape(M, -1)
    return np.abs(th.reshape(M, -1) - th_o.reshape(M, -1)) / scale


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


class Peaks:
    """Roofline denominators on this GPU: SFU issue slots and FP32 lanes derived from the unit
    counts (16 and 128 per SM per clock) at the maximum SM clock, FP64 rates from the library's
    own probe, HBM from MEASURED_PEAKS.json."""

    def __init__(self, sms, probe):
        pk = _peaks()
        self.sms = sms
        self.mhz = float(pk.get("sm_max_mhz", 2070.0))
        self.hbm_gbs = float(pk.get("hbm_gbs", 6800.0))
        self.hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in pk else "fallback 6.8 TB/s"
        self.probe = probe
        self.sfu = 16 * sms * self.mhz * 1e6
        self.fp32 = 128 * sms * self.mhz * 1e6
        self.fp64_pair = probe["fp64_pair"] * sms * self.mhz * 1e6
        self.dfma = probe["dfma"] * sms * self.mhz * 1e6

    def alu(self, slots, fma, seconds, kernel):
        """Fraction of the busier of the SFU (slots) and FP32 (lanes) pipes."""
        a_s, a_f = slots / seconds, fma / seconds
        fs, ff = a_s / self.sfu, a_f / self.fp32
        sfu = fs >= ff
        return {"bound": "alu", "pipe": "sfu" if sfu else "fp32",
                "achieved": round((a_s if sfu else a_f) / 1e12, 4), "peak": round((self.sfu if sfu else self.fp32) / 1e12, 4),
                "unit": "T SFU issue slots/s" if sfu else "T FP32 lane-ops/s", "frac": round(max(fs, ff), 4),
                "sfu_frac": round(fs, 4), "fp32_frac": round(ff, 4), "kernel": kernel,
                "peak_source": f"derived: 16 SFU slots / 128 FP32 lanes per SM per clock x {self.sms} SMs x "
                               f"{self.mhz:.0f} MHz"}


def _oracle_points(fn, N, threads):
    """An oracle estimate over N points as contiguous point ranges on host threads (ctypes
    releases the GIL); each part is a mean over its points, weighted by its count."""
    cuts = np.linspace(0, N, threads + 1).astype(np.int64)
    rs = [(int(a), int(b - a)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    with ThreadPoolExecutor(len(rs)) as ex:
        parts = list(ex.map(lambda r: fn(*r), rs))
    if isinstance(parts[0], tuple):
        return tuple(sum(p[k] * c for p, (_, c) in zip(parts, rs)) / N for k in range(len(parts[0])))
    return sum(p * c for p, (_, c) in zip(parts, rs)) / N


def run_ours(args, rank, world):
    import torch
    from paper_1408_5526_gb300 import inputs, rqmc, shard

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rqmc.load()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    lm = inputs.lmm_flat(N_FWD)
    K = inputs.LMM_STRIKES
    nK = len(K)
    seed = SEED
    offset, n_local = shard.point_range(rank, world, N_PATHS * world)
    plans = [rqmc.Plan.caplets(lm, K, n_local, M_REPL, s, seed, prec="fp32", offset=offset) for s in SEQS]
    nout = plans[0].output_size()
    buf = torch.empty(len(SEQS) * nout, dtype=torch.float64, device=dev)   # the three theta blocks
    outs = [buf[j * nout:(j + 1) * nout] for j in range(len(SEQS))]
    stream = torch.cuda.current_stream()

    # headline results for the parity gate (the timed loop recomputes them, bit for bit)
    for p, o in zip(plans, outs):
        p.execute(o, stream)
    if world > 1:
        shard.combine_theta(buf, n_local, total=N_PATHS * world)
    th_gpu = buf.cpu().numpy().reshape(len(SEQS), M_REPL, -1)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        for p, o in zip(plans, outs):
            p.execute(o, stream)
        if world > 1:
            shard.combine_theta(buf, n_local, total=N_PATHS * world)

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
                shard.combine_theta(buf, n_local, total=N_PATHS * world)
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
    th_last = buf.cpu().numpy().reshape(len(SEQS), M_REPL, -1)
    replay_identical = bool(np.array_equal(th_last, th_gpu))

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
    d2h = len(SEQS) * (M_REPL * N_FWD * nK * 8 + 16)

    probe = rqmc.probe_pipes()
    pk = Peaks(sms, probe)
    mufu, fma = lmm_algorithmic_ops(N_FWD, nK, N_PATHS * M_REPL)
    per_launch_s = statistics.mean(launch_ms) / 1e3
    roof = pk.alu(mufu, fma, per_launch_s, "one plan execute: points_run_kernel normals + "
                  "lmm_caplet_kernel<40,float> (normals loaded) + theta_kernel")
    roof.update({"traffic": LMM_TRAFFIC_BYTES,
                 "traffic_unit": ("DRAM bytes per plan execute (ncu, Rasrap, kernels replayed cold): the FP32 "
                                  "normals' round trip through HBM, 0 algorithmic bytes") if LMM_TRAFFIC_BYTES
                 else "not captured since the kernels last changed",
                 "launch_ms": round(per_launch_s * 1e3, 4),
                 "probe_per_sm_clk": {k: round(v, 2) for k, v in probe.items()}})
    # the same pipes measured on this GPU: one slot = one rcp or lg2 = two ex2
    slot_rate = min(probe["rcp"], probe["lg2"], 0.5 * probe["ex2"])
    roof["frac_of_probed_sfu"] = round(mufu / per_launch_s / (slot_rate * sms * pk.mhz * 1e6), 4)

    cpu, parity = None, None
    if rank == 0 and not args.no_cpu:
        cpu, parity = headline_oracle(th_gpu, lm, K, args.threads)
        parity["replay_bit_identical"] = replay_identical
    extra = other_workloads(args, dev, seed, pk) if (rank == 0 and not args.no_extra) else None
    cpu_gen = cpu_generators(args.threads) if (rank == 0 and not args.no_cpu) else None
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
                                       "one all-reduce of the three theta blocks per step") if world > 1 else "1 GPU",
                       "sms": sms,
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


def headline_oracle(th_gpu, lm, K, threads):
    """The oracle over the whole headline workload (every replication of every sequence at
    full N, OpenMP over replications): its timing is the CPU baseline and its theta the
    parity reference of every GPU theta_N^m."""
    import oracle as O
    from paper_1408_5526_gb300 import inputs
    jk = inputs.joe_kuo_table()
    ids = {"rasrap": O.RASRAP, "sobol_ds": O.SOBOL_DS, "philox": O.PHILOX}
    per_seq, t_total = {}, 0.0
    worst = 0.0
    for j, s in enumerate(SEQS):
        q = O.Sequence(ids[s], N_FWD, M_REPL, SEED, joe_kuo=jk)
        t0 = time.perf_counter()
        th_o = O.lmm_caplets(q, lm, K, N_PATHS, threads=threads)
        t_total += time.perf_counter() - t0
        e = caplet_scaled_err(th_gpu[j], th_o, len(K))
        rel = np.abs(th_gpu[j] - th_o) / np.abs(th_o)
        per_seq[s] = {"max_scaled_err": float(e.max()), "max_rel_err": float(rel.max()),
                      "median_rel_err": float(np.median(rel)), "theta_checked": int(e.size)}
        worst = max(worst, float(e.max()))
    steps = len(SEQS) * M_REPL * N_PATHS * N_FWD
    cpu = {"value": steps / t_total, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
           "sample": f"the whole workload: 3 sequences x {M_REPL} replications x N={N_PATHS} x {N_FWD} steps "
                     f"({t_total:.1f} s, OpenMP over replications)"}
    parity = {"ok": worst <= 1e-4, "tol": 1e-4, "max_scaled_err": worst, "per_sequence": per_seq,
              "checked": f"every theta_N^m: {M_REPL} replications x {N_FWD * len(K)} outputs x 3 sequences at full N",
              "scale": "max(|theta_oracle|, theta_oracle of the at-the-money strike, same maturity)"}
    return cpu, parity


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


def _timed_oracle(fn):
    t0 = time.perf_counter()
    r = fn()
    return r, time.perf_counter() - t0


def other_workloads(args, dev, seed, pk):
    """The other configurations of the scope, one timed figure each (median of a few
    launches, L2 flushed before each, inputs resident), each with a timed oracle sample
    (cpu_baseline), the parity of the GPU result on that sample, the largest error against
    the oracle, and a roofline fraction: product integrand (FP64), LMM caplets in FP64,
    MBS (FP32), two-factor adjoint Greeks (FP32), the 512-instrument batch (FP32, graph
    launch), the Treasury-curve study of Sec. 5 and the MBS study of Sec. 6 (std, time and
    efficiency against N), the Matousek-scrambled Sobol' caplets and the point stream (HBM
    write GB/s)."""
    import torch

    import oracle as O
    from paper_1408_5526_gb300 import inputs, rqmc
    jk = inputs.joe_kuo_table()
    T = args.threads
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    chosen = set(args.extra.split(",")) if args.extra != "all" else None

    def want(name):
        return chosen is None or name in chosen

    lm = inputs.lmm_flat(N_FWD)
    K = inputs.LMM_STRIKES
    ids = {"rasrap": O.RASRAP, "sobol_ds": O.SOBOL_DS, "philox": O.PHILOX}

    # ---- product integrand, s = 8, N = 4096, M = 32, random-start Halton, FP64
    if want("product"):
        s, N, M = 8, 4096, 32
        a = inputs.product_weights(s)
        p = rqmc.Plan.product(s, N, M, "halton_rs", seed, a, prec="fp64")
        o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
        ms = _time_plan(lambda: p.execute(o), 10, flush)
        th = o.cpu().numpy()
        p.close()
        th_o, t_o = _timed_oracle(lambda: O.product_theta(O.Sequence(O.HALTON_RS, s, M, seed), N, a, threads=T))
        rel = float(np.max(np.abs(th - th_o) / np.abs(th_o)))
        out["product_s8_N4096_M32_fp64"] = {
            "ms": ms, "path_steps_per_s": s * N * M / (ms / 1e3), "rq": float(th.mean()), "exact": 1.0,
            "parity": {"ok": rel <= 1e-11, "tol": 1e-11, "max_rel_err": rel, "checked": "all 32 replications"},
            "cpu_baseline": {"value": s * N * M / t_o, "unit": "point-dims/s", "cores": T, "kind": "oracle",
                             "sample": "the whole workload"},
            "roofline": {"bound": "latency", "note": "one launch of 1M point-dims plus the theta reduction; at "
                         f"{ms * 1e3:.0f} us the launch and tail dominate", "frac": None}}

    # ---- LMM caplets in FP64 (same 40-forward workload), Rasrap
    if want("fp64"):
        p = rqmc.Plan.caplets(lm, K, N_PATHS, M_REPL, "rasrap", seed, prec="fp64")
        o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
        ms = _time_plan(lambda: p.execute(o), 2, flush)
        th = o.cpu().numpy().reshape(M_REPL, -1)
        p.close()
        mr = 4
        th_o, t_o = _timed_oracle(lambda: O.lmm_caplets(O.Sequence(O.RASRAP, N_FWD, M_REPL, seed), lm, K, N_PATHS,
                                                        m_range=(0, mr), threads=T))
        rel = float(np.max(np.abs(th[:mr] - th_o) / np.abs(th_o)))
        pairs = lmm_fp64_pairs(N_FWD, N_PATHS * M_REPL)
        out["lmm_caplets_40_N65536_M64_fp64_rasrap"] = {
            "ms": ms, "path_steps_per_s": N_PATHS * M_REPL * N_FWD / (ms / 1e3),
            "parity": {"ok": rel <= 1e-11, "tol": 1e-11, "max_rel_err": rel, "checked": f"replications 0..{mr - 1}, full N"},
            "cpu_baseline": {"value": mr * N_PATHS * N_FWD / t_o, "unit": "path-steps/s", "cores": min(T, mr),
                             "kind": "oracle", "sample": f"{mr} replications x N={N_PATHS}"},
            "roofline": {"bound": "fp64", "pipe": "fp64 update pair (exp + reciprocal)",
                         "achieved": round(pairs / (ms / 1e3) / 1e9, 3), "peak": round(pk.fp64_pair / 1e9, 3),
                         "unit": "G FP64 update pairs/s", "frac": round(pairs / (ms / 1e3) / pk.fp64_pair, 4),
                         "peak_source": f"probed: {pk.probe['fp64_pair']:.3f} pairs per SM per clock x {pk.sms} SMs x "
                                        f"{pk.mhz:.0f} MHz"}}

    # ---- MBS, 360 months, N = 65536, M = 64, FP32 + Kahan
    if want("mbs"):
        mb = inputs.mbs_paper(360)
        res = {}
        for s_ in SEQS:
            p = rqmc.Plan.mbs(mb, N_PATHS, M_REPL, s_, seed, prec="fp32")
            o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
            ms = _time_plan(lambda: p.execute(o), 3, flush)
            th = o.cpu().numpy()
            p.close()
            q = O.Sequence(ids[s_], 360, M_REPL, seed, joe_kuo=jk)
            th_o, t_o = _timed_oracle(lambda: _oracle_points(
                lambda off, n: O.mbs_theta(q, mb, n, offset=off, m_range=(0, 1), threads=1), N_PATHS, T))
            rel = float(abs(th[0] - th_o[0]) / abs(th_o[0]))
            slots, fma = mbs_algorithmic_ops(360, N_PATHS * M_REPL)
            res[s_] = {"ms": ms, "path_steps_per_s": N_PATHS * M_REPL * 360 / (ms / 1e3), "rq": float(th.mean()),
                       "parity": {"ok": rel <= 1e-4, "tol": 1e-4, "max_rel_err": rel,
                                  "checked": "replication 0 at full N"},
                       "cpu_baseline": {"value": N_PATHS * 360 / t_o, "unit": "path-steps/s", "cores": T,
                                        "kind": "oracle", "sample": f"replication 0 x N={N_PATHS} (point ranges)"},
                       "roofline": pk.alu(slots, fma, ms / 1e3, f"mbs_kernel<float,{s_}>")}
        out["mbs_360_N65536_M64_fp32"] = res

    # ---- adjoint Greeks: two-factor 80-forward strip, N = 2^18, M = 32, FP32 paths
    if want("adjoint"):
        cfg = inputs.CONFIGS["adjoint_2f_80"]
        l2 = inputs.lmm_two_factor(cfg["n_fwd"], seed=cfg["seed"])
        Na, Ma, nfa = cfg["N"], cfg["M"], cfg["n_fwd"]
        w = np.ones(nfa)
        p = rqmc.Plan.adjoint(l2, [0.05], w, Na, Ma, "sobol_ds", seed)
        o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
        ms = _time_plan(lambda: p.execute(o), 2, flush)
        ad = o.cpu().numpy().reshape(Ma, -1)
        p.close()
        q = O.Sequence(O.SOBOL_DS, 2 * nfa, Ma, seed, joe_kuo=jk)
        (v_o, d_o, g_o), t_o = _timed_oracle(lambda: _oracle_points(
            lambda off, n: O.lmm_adjoint(q, l2, [0.05], w, n, offset=off, m_range=(0, 1), threads=1), Na, T))
        e_v = float(abs(ad[0, 0] - v_o[0]) / abs(v_o[0]))
        e_d = float(np.max(np.abs(ad[0, 1:1 + nfa] - d_o[0]) / np.abs(d_o[0])))
        e_g = float(np.max(np.abs(ad[0, 1 + nfa:1 + 2 * nfa] - g_o[0]) / np.abs(g_o[0])))
        slots, fma = adjoint_algorithmic_ops(nfa, 2, Na * Ma)
        out["adjoint_2f_80_N262144_M32_fp32_sobol"] = {
            "ms": ms, "path_steps_per_s": Na * Ma * 2 * nfa / (ms / 1e3),
            "parity": {"ok": max(e_v, e_d, e_g) <= 1e-4, "tol": 1e-4, "value_rel_err": e_v, "max_delta_rel_err": e_d,
                       "max_vega_rel_err": e_g, "checked": "replication 0 at full N: value, 80 deltas, 80 vegas"},
            "cpu_baseline": {"value": Na * 2 * nfa / t_o, "unit": "path-steps/s", "cores": T, "kind": "oracle",
                             "sample": f"replication 0 x N={Na} (point ranges)"},
            "roofline": pk.alu(slots, fma, ms / 1e3, "lmm_adjoint_kernel<80,2,sobol>")}

    # ---- 512-instrument batch, one graph launch
    if want("batch"):
        desc = inputs.batch_instruments(seed)
        insts = [dict(d, rate=0.05, vol=0.15, strike=0.05) if d["kind"] == "lmm" else d for d in desc]
        Mb = 32
        p = rqmc.Plan.batch(insts, Mb, "sobol_ds", seed)
        o = torch.empty(p.output_size(), dtype=torch.float64, device=dev)
        ms = _time_plan(lambda: p.execute(o), 1, flush)
        parts = p.split_batch(o.cpu().numpy())
        bstats = p.batch_stats()   # of the last timed execute
        p.close()
        steps = sum(d["N"] * Mb * (d["n_fwd"] if d["kind"] == "lmm" else d["months"]) for d in desc)
        slots = fma = 0.0
        for d in desc:
            if d["kind"] == "lmm":
                s_, f_ = lmm_algorithmic_ops(d["n_fwd"], 1, d["N"] * Mb)
            else:
                s_, f_ = mbs_algorithmic_ops(d["months"], d["N"] * Mb)
            slots, fma = slots + s_, fma + f_
        sample = list(range(0, len(desc), 32))   # every 32nd instrument, replication 0, full N

        def one(i):
            d = insts[i]
            if d["kind"] == "lmm":
                lmi = inputs.lmm_flat(d["n_fwd"], delta=0.25, rate=d["rate"], vol=d["vol"])
                return O.lmm_caplets(O.Sequence(O.SOBOL_DS, d["n_fwd"], Mb, seed, inst=i, joe_kuo=jk), lmi, [d["strike"]],
                                     d["N"], m_range=(0, 1), threads=1)[0]
            return O.mbs_theta(O.Sequence(O.SOBOL_DS, d["months"], Mb, seed, inst=i, joe_kuo=jk),
                               inputs.mbs_paper(d["months"]), d["N"], m_range=(0, 1), threads=1)

        def run_sample():
            with ThreadPoolExecutor(T) as ex:
                return list(ex.map(one, sample))
        ref, t_o = _timed_oracle(run_sample)
        rel = max(float(np.max(np.abs(parts[i][0] - r) / np.abs(r))) for i, r in zip(sample, ref))
        o_steps = sum(desc[i]["N"] * (desc[i]["n_fwd"] if desc[i]["kind"] == "lmm" else desc[i]["months"]) for i in sample)
        out["batch_512_M32_fp32_sobol"] = {
            "ms": ms, "path_steps_per_s": steps / (ms / 1e3), "path_steps": steps,
            "imbalance_max_sm_busy_over_mean": bstats["imbalance"], "class_spans_ms": bstats,
            "parity": {"ok": rel <= 1e-4, "tol": 1e-4, "max_rel_err": rel,
                       "checked": f"{len(sample)} instruments (every 32nd), replication 0, full N"},
            "cpu_baseline": {"value": o_steps / t_o, "unit": "path-steps/s", "cores": T, "kind": "oracle",
                             "sample": f"{len(sample)} instruments x replication 0"},
            "roofline": pk.alu(slots, fma, ms / 1e3, "batch_kernel<sobol, 3 work classes>")}

    # ---- Sec. 5's Treasury-curve study: caplet on L_10 (T = 5, delta = 0.5, K = 1 %, sigma = 4 %)
    if want("treasury"):
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
                th_all = ot.cpu().numpy().reshape(st["M"], -1)
                th = th_all[:, lmt["n_fwd"] - 1]
                pt.close()
                rows.append({"N": 1 << e, "rq": float(th.mean()), "std": float(th.std(ddof=1)), "ms": ms,
                             "efficiency": float(th.std(ddof=1)) * ms})
                if e == 14:   # parity at N = 2^14: every replication, the study's caplet and the whole strip
                    sid = {"rasrap": O.RASRAP, "sobol_ds": O.SOBOL_DS, "philox": O.PHILOX, "sobol_lms": O.SOBOL_LMS}[s_]
                    th_o = O.lmm_caplets(O.Sequence(sid, lmt["n_fwd"], st["M"], seed, joe_kuo=jk), lmt, [st["K"]],
                                         1 << e, threads=T)
                    c = lmt["n_fwd"] - 1
                    rel14 = float(np.max(np.abs(th_all[:, c] - th_o[:, c]) / np.abs(th_o[:, c])))
                    abs14 = float(np.max(np.abs(th_all - th_o)))
                    ok14 = rel14 <= 1e-4 and bool(np.all(np.abs(th_all - th_o) <= 1e-4 * np.abs(th_o) + 1e-9))
            lx = np.log([r["N"] for r in rows])
            ly = np.log([r["std"] for r in rows])
            study[s_] = {"rate": float(np.polyfit(lx, ly, 1)[0]), "by_N": rows,
                         "parity": {"ok": ok14, "tol": "1e-4 relative on the study's caplet (L_10); 1e-4 |theta| + 1e-9 "
                                    "on every caplet of the strip (the early ones are worth 0 at K = 1 %)",
                                    "study_caplet_max_rel_err": rel14, "strip_max_abs_err": abs14,
                                    "checked": "N = 2^14, all 100 replications, all 10 caplets"}}
        out["lmm_treasury_study_T5_M100_fp32"] = study

    if want("mbs_study"):
        # Sec. 6 study: std of M = 64 independent MBS estimates (360 months), time and efficiency
        # (std x time) against N, and the fitted convergence rate of the std (the paper's GPU rates:
        # Philox ~0.5, Rasrap 0.68, Sobol' 0.86)
        mbs = inputs.mbs_paper(360)
        Ms = 64
        study = {}
        for s_ in SEQS + ("sobol_lms",):
            rows = []
            for e in range(10, 19, 2):
                pt = rqmc.Plan.mbs(mbs, 1 << e, Ms, s_, seed, prec="fp32")
                ot = torch.empty(pt.output_size(), dtype=torch.float64, device=dev)
                ms = _time_plan(lambda: pt.execute(ot), 3, flush)
                th = ot.cpu().numpy()
                pt.close()
                rows.append({"N": 1 << e, "rq": float(th.mean()), "std": float(th.std(ddof=1)), "ms": ms,
                             "efficiency": float(th.std(ddof=1)) * ms})
                if e == 12:   # parity at N = 2^12 on the first 8 replications
                    sid = {"rasrap": O.RASRAP, "sobol_ds": O.SOBOL_DS, "philox": O.PHILOX, "sobol_lms": O.SOBOL_LMS}[s_]
                    th_o = O.mbs_theta(O.Sequence(sid, 360, Ms, seed, joe_kuo=jk), mbs, 1 << e, m_range=(0, 8),
                                       threads=T)[:8]
                    rel12 = float(np.max(np.abs(th[:8] - th_o) / np.abs(th_o)))
            lx = np.log([r["N"] for r in rows])
            ly = np.log([r["std"] for r in rows])
            study[s_] = {"rate": float(np.polyfit(lx, ly, 1)[0]), "by_N": rows,
                         "parity": {"ok": rel12 <= 1e-4, "tol": 1e-4, "max_rel_err": rel12,
                                    "checked": "N = 2^12, replications 0..7"}}
        out["mbs_study_360m_M64_fp32"] = study

    # ---- Matousek-scrambled Sobol' on the headline caplet workload (same kernel, scrambled tables)
    if want("lms"):
        pl_ = rqmc.Plan.caplets(lm, K, N_PATHS, M_REPL, "sobol_lms", seed, prec="fp32")
        o_ = torch.empty(pl_.output_size(), dtype=torch.float64, device=dev)
        ms = _time_plan(lambda: pl_.execute(o_), 3, flush)
        th = o_.cpu().numpy().reshape(M_REPL, -1)
        pl_.close()
        th_o, t_o = _timed_oracle(lambda: O.lmm_caplets(O.Sequence(O.SOBOL_LMS, N_FWD, M_REPL, seed, joe_kuo=jk), lm, K,
                                                        N_PATHS, m_range=(0, 4), threads=T))
        e = float(caplet_scaled_err(th[:4], th_o, len(K)).max())
        mufu, fma = lmm_algorithmic_ops(N_FWD, len(K), N_PATHS * M_REPL)
        out["lmm_caplets_40_N65536_M64_fp32_sobol_lms"] = {
            "ms": ms, "path_steps_per_s": N_PATHS * M_REPL * N_FWD / (ms / 1e3),
            "parity": {"ok": e <= 1e-4, "tol": 1e-4, "max_scaled_err": e, "checked": "replications 0..3, full N"},
            "cpu_baseline": {"value": 4 * N_PATHS * N_FWD / t_o, "unit": "path-steps/s", "cores": min(T, 4),
                             "kind": "oracle", "sample": f"4 replications x N={N_PATHS}"},
            "roofline": pk.alu(mufu, fma, ms / 1e3, "lmm_caplet_kernel<40,sobol,float>")}

    # ---- point stream: s = 360, N = 65536, M = 64 FP32 normals and uniforms, written to HBM
    if want("points"):
        Mp = args.points_m
        buf = torch.empty((Mp, 360, N_PATHS), dtype=torch.float32, device=dev)
        res = {}
        for s_ in SEQS:
            row = {}
            for tr in ("normal", "uniform"):
                pp = rqmc.Plan.points(360, N_PATHS, Mp, s_, seed, prec="fp32", transform=tr)
                ms = _time_plan(lambda: pp.execute(buf), 3, flush)   # kernel only: tables built once
                pp.close()
                gbs = buf.numel() * 4 / (ms / 1e3) / 1e9
                q = O.Sequence(ids[s_], 360, 1, seed, joe_kuo=jk)
                ref = q.points(4096, transform=O.NORMAL if tr == "normal" else O.UNIFORM, threads=T)[0, :, :]
                got = buf[0, :, :4096].cpu().numpy().astype(np.float64)
                err = float(np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref)))) if tr == "normal" else \
                    float(np.max(np.abs(got - ref) / ref))
                tol = 1e-6 if tr == "normal" else 4e-7
                row[tr] = {"ms": ms, "GB_per_s": gbs, "gnumbers_per_s": buf.numel() / (ms / 1e3) / 1e9,
                           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": pk.hbm_gbs, "unit": "GB/s",
                                        "frac": round(gbs / pk.hbm_gbs, 4), "peak_source": pk.hbm_src},
                           "parity": {"ok": err <= tol, "tol": tol, "max_err": err,
                                      "checked": "replication 0, all 360 dimensions, points 0..4095"}}
            ms1 = _time_plan(lambda: rqmc.rqmc_points(360, N_PATHS, Mp, s_, seed, transform="normal", out=buf), 2,
                             flush)   # one-shot call: tables + kernel
            row["one_shot_normal_ms"] = ms1
            res[s_] = row
        out[f"points_s360_N65536_M{Mp}_fp32"] = res
        del buf
    return out


def cpu_generators(threads):
    """Table 1 style CPU generator throughput on this host, for context beside the GPU point
    stream: the recursive generators (Algorithm 2 for Rasrap, Gray-code order for Sobol')
    and the counter-based forms (Algorithm 3, binary-order Sobol', Philox) of the oracle,
    raw integer states of s = 40 dimensions, M = 8, N = 65536, one thread and all threads."""
    import oracle as O
    from paper_1408_5526_gb300 import inputs
    jk = inputs.joe_kuo_table()
    out = {"cores": threads, "unit": "GNumbers/s", "sample": "s=40, M=8, N=65536 raw states"}
    for name, seq in (("rasrap", O.RASRAP), ("sobol_ds", O.SOBOL_DS), ("philox", O.PHILOX)):
        q = O.Sequence(seq, 40, 8, SEED, joe_kuo=jk if seq == O.SOBOL_DS else None)
        row = {}
        for th in (1, threads):
            t0 = time.perf_counter()
            a = q.stream(0, 65536, threads=th)
            row[f"recursive_{th}t"] = a.size / (time.perf_counter() - t0) / 1e9
        t0 = time.perf_counter()
        b = q.points(65536, transform=O.RAW, threads=threads)
        row[f"counter_based_{threads}t"] = b.size / (time.perf_counter() - t0) / 1e9
        out[name] = row
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    from paper_1408_5526_gb300 import inputs
    cores = args.threads
    lm = inputs.lmm_flat(N_FWD)
    K = inputs.LMM_STRIKES
    n_sample = 8192
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
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (cpu_baseline and parity)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other-configuration figures")
    ap.add_argument("--extra", default="all",
                    help="comma-separated subset of the other configurations: product, fp64, mbs, adjoint, batch, "
                         "treasury, mbs_study, lms, points (default all)")
    ap.add_argument("--points-m", type=int, default=M_REPL,
                    help="replications of the point-stream figure (default 64; smaller for profiler captures)")
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
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    args.threads = max(1, min(cores, 16))   # host threads of the oracle legs
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
