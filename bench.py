#!/usr/bin/env python3
"""Benchmark of the stochastic Chebyshev (KPM) density-of-states hot path.

Workload (one "step" = the whole DOS path on one batch of synthetic input):
  honeycomb lattice 4096 x 4096 cells (33.5M orbitals), t = -2.7 eV, Anderson disorder
  W = 2 eV, 0.5 % seeded vacancies, Gershgorin bounds, M = 2048 moments, R = 8
  random-phase vectors, complex FP32 recursion with FP64 moment accumulation, then the
  FP64 Jackson reconstruction of the DOS on a 1024-point energy grid.
Metric: orbital * moment * vector updates per second (N_eff * M * R / step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kite|reference]

N > 1 runs under torchrun, one rank per GPU; each rank runs its own disorder
realisation (independent samples, no data-path collective) and `value` is the total
over ranks divided by the slowest rank's time ("weak" scaling).  `--impl reference`
times the FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site·moment·vector updates/s, FP32 vs FP64 at stated error; % of HBM peak"
UNIT = "updates/s"
WORKLOAD = dict(lattice="honeycomb", Lx=4096, Ly=4096, t=-2.7, W=2.0, p_vac=0.005, M=2048, R=8,
                precision="fp32 recursion, fp64 moment accumulation", K_energies=1024,
                kernel="jackson")
WORKLOAD_NAME = ("large_dos_honeycomb_4096x4096_W2_vac0.005_M2048_R8_fp32 + "
                 "jackson_dos_1024pts")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="kite", choices=["kite", "reference"])
    p.add_argument("--Lx", type=int, default=WORKLOAD["Lx"])
    p.add_argument("--Ly", type=int, default=WORKLOAD["Ly"])
    p.add_argument("--M", type=int, default=WORKLOAD["M"])
    p.add_argument("--R", type=int, default=WORKLOAD["R"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-doubling", action="store_true")
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--no-learned", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


STEP_SOURCES = ("kite_kpm1d.cu", "kite_step.cuh", "kite_step2.cuh", "kite_device.cuh")


def kernel_source_hash():
    """Hash of the sources the 1D step kernels (one-step and two-step) are built from."""
    h = hashlib.sha1()
    for fn in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1910_05194_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(updates_per_launch: float, steps_per_pass: int):
    """DRAM bytes per launch of the dominant step kernel (one-step, or the two-step pass)
    from the committed ncu summary, scaled per update of the launch, if the kernel source
    still matches the one profiled (else None)."""
    name = "kpm_step2_traffic.json" if steps_per_pass == 2 else "kpm_step_traffic.json"
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_update"]) * updates_per_launch


def job_throughput(updates_local: float, ms_local: float, dist=None, device="cpu"):
    """Whole-job rate over N ranks: the updates of all ranks (summed) over the slowest rank's
    time per step (max), as (updates/s, ms per step).  dist: torch.distributed or None."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([updates_local], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return float(u.item()) / (ms * 1e-3), ms


def run_reference(args, rank, world):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    cores = os.cpu_count() or 1
    sysd = dict(lattice=0, Lx=args.Lx, Ly=args.Ly, t=WORKLOAD["t"], W=WORKLOAD["W"],
                p_vac=WORKLOAD["p_vac"], seed=2)
    sample_M, sample_R = 8, 1
    s = oracle.make_system(**sysd)
    n = oracle.norb(s)
    _, vac = oracle.disorder(s)
    n_eff = int((vac == 0).sum())
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.moments_1d(s, sample_M, sample_R, threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    upd = n_eff * sample_M * sample_R
    value = upd / float(np.mean(times))
    sample = (f"oracle FP64 (C, OpenMP) on the full {args.Lx}x{args.Ly} lattice with "
              f"M={sample_M}, R={sample_R} per step (bounded sample; metric per update)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, **WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _median_time(fn, runs=3):
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def cpu_baseline_leg(args, kite, ctx, n_eff_gpu):
    """The oracle timed on the host cores on a bounded sample of the workload (median of
    three runs on all cores and on one core), the GPU's error against the oracle on that
    sample in FP32 and FP64, and the FP32 error at the workload's full order M = 2048 on a
    lattice the oracle finishes in seconds."""
    import oracle
    cores = os.cpu_count() or 1
    sysd = dict(lattice=0, Lx=args.Lx, Ly=args.Ly, t=WORKLOAD["t"], W=WORKLOAD["W"],
                p_vac=WORKLOAD["p_vac"], seed=2)
    s = oracle.make_system(**sysd)
    _, vac = oracle.disorder(s)
    n_eff = int((vac == 0).sum())
    M, R = 8, 2
    res = {}
    dt = _median_time(lambda: res.__setitem__("mu", oracle.moments_1d(s, M, R, threads=cores)))
    mu_ref = res["mu"]
    M1, R1 = 2, 1
    dt1 = _median_time(lambda: oracle.moments_1d(s, M1, R1, threads=1))
    ks = kite.make_system(lattice=0, Lx=args.Lx, Ly=args.Ly, t=WORKLOAD["t"], W=WORKLOAD["W"],
                          p_vac=WORKLOAD["p_vac"], seed=2)
    mu = np.zeros(M)
    kite.moments_1d(ctx, ks, kite.make_kpm(M, R, 1, kite.FP32), mu)
    mu64 = np.zeros(M)
    kite.moments_1d(ctx, ks, kite.make_kpm(M, R, 1, kite.FP64), mu64)
    # DOS error of the GPU path on the sample: L1 distance of the Jackson DOS (per orbital
    # per eV) from the GPU's FP32 moments and from the oracle's FP64 moments
    lo, hi = kite.bounds(ks)
    E = np.linspace(lo * 0.999, hi * 0.999, 2001)
    rho = np.zeros(E.size)
    kite.reconstruct_dos(ctx, mu, M, M, kite.KERNEL_JACKSON, 0.0, lo, hi, E, E.size, rho)
    rho_ref = oracle.dos(mu_ref.real.mean(0), E, lo, hi, oracle.kernel_jackson(M))
    l1 = float(np.sum(np.abs(rho - rho_ref)[:-1] * np.diff(E)))
    # the full order on a 256 x 256 lattice of the same kind (FP32 rounding grows with n)
    d256 = dict(sysd, Lx=256, Ly=256)
    M2, R2 = WORKLOAD["M"], WORKLOAD["R"]
    ref2 = oracle.moments_1d(oracle.make_system(**d256), M2, R2, threads=cores).real.mean(0)
    mu2 = np.zeros(M2)
    st2 = kite.moments_1d(ctx, kite.make_system(**d256), kite.make_kpm(M2, R2, 1, kite.FP32), mu2)
    return {"value": n_eff * M * R / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full {args.Lx}x{args.Ly} lattice, M={M}, R={R}, FP64 oracle (C, OpenMP), "
                      f"median of 3 runs: {dt:.2f} s",
            "value_1core": n_eff * M1 * R1 / dt1,
            "sample_1core": f"full {args.Lx}x{args.Ly} lattice, M={M1}, R={R1}, one thread, median of 3: {dt1:.2f} s",
            "max_abs_dmu_gpu_fp32_vs_oracle_on_sample": float(np.max(np.abs(mu - mu_ref.real.mean(0)))),
            "max_abs_dmu_gpu_fp64_vs_oracle_on_sample": float(np.max(np.abs(mu64 - mu_ref.real.mean(0)))),
            "dos_l1_gpu_fp32_vs_oracle_on_sample": l1,
            "fp32_error_at_full_order": {
                "lattice": "honeycomb 256x256, same W, vacancies and seed", "M": M2, "R": R2,
                "max_abs_dmu_vs_oracle": float(np.max(np.abs(mu2 - ref2))),
                "steps_per_pass": st2.steps_per_pass},
            "n_eff_match": bool(n_eff == n_eff_gpu)}


def cpu_baselines_per_config(kite, ctx):
    """The oracle on every other configuration, all host cores and one core (median of
    three where a run takes seconds), on bounded samples extrapolated linearly in the work
    (the paper's moment-scaling table shows run time linear in M); each entry says what it
    ran and which values are extrapolated."""
    import oracle
    import synth
    from paper_1910_05194_gb300 import learned
    cores = os.cpu_count() or 1
    out = {}
    # small FP64 DOS: the whole workload
    b = (3 * 2.7 + 0.5) * 1.01
    s1 = oracle.make_system(lattice=0, Lx=64, Ly=64, t=-2.7, W=1.0, seed=1)
    upd1 = 8192 * 256 * 4
    t_all = _median_time(lambda: oracle.moments_1d(s1, 256, 4, e_min=-b, e_max=b, threads=cores))
    t_one = _median_time(lambda: oracle.moments_1d(s1, 256, 4, e_min=-b, e_max=b, threads=1))
    out["small_dos_honeycomb_64x64_M256_R4_fp64"] = {
        "seconds_per_call_all_cores": t_all, "seconds_per_call_1core": t_one,
        "updates_per_s_all_cores": upd1 / t_all, "updates_per_s_1core": upd1 / t_one,
        "sample": "the whole call (median of 3)"}
    # batched: three systems of the workload at M = 64, extrapolated to the workload's updates
    specs = synth.batched_square_systems(256, seed=3)
    total = float(sum(sp["L"] ** 2 * sp["M"] * 4 for sp in specs))
    pick = specs[:3]
    sy = [oracle.make_system(lattice=1, Lx=sp["L"], Ly=sp["L"], t=-1.0, W=sp["W"], seed=sp["seed"]) for sp in pick]
    upd3 = float(sum(sp["L"] ** 2 * 64 * 4 for sp in pick))
    t3 = _median_time(lambda: [oracle.moments_1d(x, 64, 4, threads=cores) for x in sy])
    t3_1 = _median_time(lambda: oracle.moments_1d(sy[0], 16, 4, threads=1), runs=1)
    rate1 = pick[0]["L"] ** 2 * 16 * 4 / t3_1
    out["batched_256_square_systems_R4"] = {
        "updates_per_s_all_cores": upd3 / t3, "updates_per_s_1core": rate1,
        "workload_updates": total, "extrapolated_workload_s_all_cores": total / (upd3 / t3),
        "extrapolated_workload_s_1core": total / rate1,
        "sample": f"systems L={[sp['L'] for sp in pick]} at M=64, R=4 (median of 3); one core: the first at "
                  "M=16; workload time extrapolated linearly in updates"}
    # Kubo-Bastin 1024 x 1024, M = 1024: the oracle's 8-row + 8-column panels per vector
    s4 = oracle.make_system(lattice=0, Lx=1024, Ly=1024, t=-2.7, W=1.0, seed=4)
    t0 = time.perf_counter()
    rows = [0, 1, 127, 128, 511, 640, 1000, 1023]
    cols = [0, 2, 129, 255, 256, 513, 767, 1023]
    pr, pc = oracle.moments_2d_panels(s4, 1024, 1, rows, cols, threads=cores)
    t4 = time.perf_counter() - t0
    full4 = t4 * (1024 / 16) * 4
    out["kubo_bastin_honeycomb_1024x1024_M1024_R4"] = {
        "panel_s_all_cores": t4, "panel_sample": "8 rows + 8 columns of mu_nm, M=1024, one vector (one run)",
        "extrapolated_full_s_all_cores": full4,
        "extrapolation": "full M x M: the panels' dot products dominate, so M/16 panel runs per vector, 4 vectors; "
                         "one core: scaled by the all-cores/one-core ratio of the large-DOS samples"}
    # learned DOS workload: the plain FP64 high-M path per sample (one 256 x 256 system)
    e_min, e_max = learned.window(1.0, 4.0)
    sp5 = synth.learned_dos_systems(1, 5_000_000, L=256)[0]
    s5 = oracle.make_system(lattice=0, Lx=256, Ly=256, t=learned.T_HOP, W=sp5["W"], delta=sp5["delta"],
                            p_vac=sp5["p_vac"], seed=sp5["seed"])
    t5 = _median_time(lambda: oracle.moments_1d(s5, 1024, 4, e_min=e_min, e_max=e_max, threads=cores))
    t5_1 = _median_time(lambda: oracle.moments_1d(s5, 64, 4, e_min=e_min, e_max=e_max, threads=1), runs=1)
    out["learned_dos_honeycomb_256x256_plain_fp64_per_sample"] = {
        "seconds_M1024_R4_all_cores": t5, "extrapolated_seconds_M4096_R4_all_cores": 4 * t5,
        "seconds_M64_R4_1core": t5_1, "extrapolated_seconds_M4096_R4_1core": 64 * t5_1,
        "sample": "one held-out-distribution system, oracle moments at M=1024 (median of 3) and M=64 on one core, "
                  "extrapolated linearly in M"}
    return out, (rows, cols, pr, pc)


def secondary_legs(kite, ctx, peaks):
    """The other hot-path configurations, each in its own launch configuration: the small
    FP64 DOS call (latency-bound, microseconds per call), the 256-system batched
    persistent launch, and the 2D Kubo-Bastin moments (families + tensor-core
    contraction).  Parity of each lives in the tests; here only their timings."""
    import synth
    out = {}
    # small FP64 DOS: honeycomb 64x64, W = 1, bounds +-(3|t| + 0.5) * 1.01, M = 256, R = 4
    b = (3 * 2.7 + 0.5) * 1.01
    s1 = kite.make_system(kite.HONEYCOMB, 64, 64, -2.7, 1.0, 0.0, 0.0, 1)
    mu1 = np.zeros(256)
    res = {}
    # the autotuner's choice (the on-chip cluster sweep when it is measured faster), then
    # the streaming step kernels alone (KITE_CLUSTER=0) for comparison
    for suffix, pin in (("", None), ("_streaming", "0")):
        old = os.environ.pop("KITE_CLUSTER", None)
        if pin is not None:
            os.environ["KITE_CLUSTER"] = pin
        try:
            for name, dbl in (("plain", False), ("doubling", True)):
                kpm1 = kite.make_kpm(256, 4, 1, kite.FP64, -b, b, doubling=dbl)
                for _ in range(3):
                    kite.moments_1d(ctx, s1, kpm1, mu1)
                t0 = time.perf_counter()
                for _ in range(20):
                    st = kite.moments_1d(ctx, s1, kpm1, mu1)
                res[name + suffix + "_us_per_call"] = 1e6 * (time.perf_counter() - t0) / 20
                res[name + suffix + "_step_us"] = 1e6 * st.step_seconds
                if pin is None:
                    res[name + "_cluster_ctas"] = st.cluster_ctas
        finally:
            os.environ.pop("KITE_CLUSTER", None)
            if old is not None:
                os.environ["KITE_CLUSTER"] = old
    out["small_dos_honeycomb_64x64_M256_R4_fp64"] = res
    # batched: 256 square systems, L 64..1024, W 0..4, M in {512..4096}, R = 4, one launch
    specs = synth.batched_square_systems(256, seed=3)
    systems = [kite.make_system(kite.SQUARE, sp["L"], sp["L"], -1.0, sp["W"], 0.0, 0.0, sp["seed"])
               for sp in specs]
    mus = [np.zeros(sp["M"]) for sp in specs]
    res = {}
    for name, dbl in (("plain", False), ("doubling", True)):
        kpms = [kite.make_kpm(sp["M"], 4, 1, kite.FP32, doubling=dbl) for sp in specs]
        st = kite.moments_1d_batched(ctx, systems, kpms, mus)
        res[name] = {"updates_per_s": st.updates / st.seconds, "seconds": st.seconds,
                     "hbm_gbs": st.bytes_moved / st.seconds / 1e9, "grid": st.grid,
                     "autotuned": {"ring_stages": st.ring_stages, "ctas_per_sm": st.ctas_per_sm, "steps_per_pass": st.steps_per_pass}}
    res["updates"] = st.updates
    out["batched_256_square_systems_R4_fp32_one_graph_launch"] = res
    import torch
    # FP64 recursion on the full lattice (fewer moments to bound the time): HBM bytes and
    # FP64 arithmetic against their measured peaks (FP64: a cuBLAS DGEMM through torch)
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, a)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        torch.matmul(a, a)
    torch.cuda.synchronize()
    fp64_tflops = 3 * 2 * 4096.0 ** 3 / (time.perf_counter() - t0) / 1e12
    del a
    s2 = kite.make_system(kite.HONEYCOMB, WORKLOAD["Lx"], WORKLOAD["Ly"], WORKLOAD["t"], WORKLOAD["W"], 0.0,
                          WORKLOAD["p_vac"], 2)
    mu2 = torch.zeros(256, dtype=torch.float64, device="cuda")
    kpm2 = kite.make_kpm(256, WORKLOAD["R"], 1, kite.FP64)
    kite.moments_1d(ctx, s2, kpm2, mu2)  # tunes
    st64 = kite.moments_1d(ctx, s2, kpm2, mu2)
    upd = st64.n_eff * 255.0 * WORKLOAD["R"]
    # per update: the stencil (2 adds and 2 FMA per component: 2t~ s + (2V~ r_n - r_{n-1}))
    # and the real part of the moment (2 FMA; the imaginary part vanishes for a Hermitian H~
    # and is not formed) = 2 * 6 + 4 = 16 FP64 flops in 10 FP64 operations
    gbs = st64.step_bytes / st64.step_seconds / 1e9
    tfl = 16.0 * upd / st64.step_seconds / 1e12
    out["large_dos_honeycomb_4096x4096_M256_R8_fp64"] = {
        "updates_per_s": upd / st64.step_seconds, "step_seconds": st64.step_seconds,
        "hbm_gbs": gbs, "hbm_frac": gbs / peaks.get("hbm_gbs", 6800.0), "fp64_tflops": tfl,
        "fp64_peak_tflops_dgemm": fp64_tflops, "fp64_frac": tfl / fp64_tflops,
        "bound": "fp64" if tfl / fp64_tflops > gbs / peaks.get("hbm_gbs", 6800.0) else "hbm",
        "autotuned": {"ring_stages": st64.ring_stages, "ctas_per_sm": st64.ctas_per_sm,
                      "steps_per_pass": st64.steps_per_pass}}
    # 2D Kubo-Bastin moments: honeycomb 1024x1024, W = 1, M = 1024, R = 4 (xx)
    s4 = kite.make_system(kite.HONEYCOMB, 1024, 1024, -2.7, 1.0, 0.0, 0.0, 4)
    mu_nm = torch.zeros((1024, 1024, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = kite.moments_2d(ctx, s4, kite.make_kpm(1024, 4, 1, kite.FP32), mu_nm)
    wall = time.perf_counter() - t0
    tflops = st.gemm_flops / st.gemm_seconds / 1e12
    fam_gbs = st.step_bytes / st.step_seconds / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    out["kubo_bastin_honeycomb_1024x1024_M1024_R4"] = {
        "wall_s": wall, "families_s": st.step_seconds, "contraction_s": st.gemm_seconds,
        "families_bytes": st.step_bytes, "families_gbs": fam_gbs, "families_frac_of_hbm": fam_gbs / hbm,
        "families_bytes_note": "per orbital and step: A step 32 B per vector (r_n-1, r_n, r_n+1, a_n+1 as BF16 hi+lo), "
                               "B step 40 B per vector (b_n and -i b_n as hi+lo), plus 4 B of on-site term per step",
        "contraction_tflops": tflops, "bf16_peak_tflops": peaks.get("bf16_tflops"),
        "contraction_frac_of_burst": tflops / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None,
        "contraction_frac_of_sustained": (tflops / peaks["bf16_tflops_sustained"]
                                          if peaks.get("bf16_tflops_sustained") else None)}
    return out


def kubo_bastin_panel_error(kite, ctx, panels):
    """mu_nm of the full-size Kubo-Bastin workload (one vector) against the oracle's eight
    rows and eight columns (computed in the CPU baseline): max |error| / max |mu|."""
    import torch
    rows, cols, pr, pc = panels
    s4 = kite.make_system(kite.HONEYCOMB, 1024, 1024, -2.7, 1.0, 0.0, 0.0, 4)
    mu = torch.zeros((1024, 1024, 2), dtype=torch.float64, device="cuda")
    kite.moments_2d(ctx, s4, kite.make_kpm(1024, 1, 1, kite.FP32), mu)
    m = mu.cpu().numpy()
    m = m[..., 0] + 1j * m[..., 1]
    scale = float(np.max(np.abs(m)))
    err = max(float(np.max(np.abs(m[rows, :] - pr))), float(np.max(np.abs(m[:, cols] - pc))))
    return {"max_abs_err_over_max_mu": err / scale, "rows": rows, "cols": cols, "M": 1024, "R": 1,
            "oracle": "FP64 plain recursion, each row/column dotted against stored a_n or b_m"}


def learned_leg(kite, ctx):
    """A bounded run of the learned-DOS workload (its sizes in the result): dataset, training
    on the GPU, held-out L1 of the network against Jackson-128 and the targets' noise floor,
    the plain order reaching the network's L1, and the wall time of the learned path (FP32
    moments + network + gate + fallback) against the plain FP64 path and the batched FP32
    path at that order."""
    from paper_1910_05194_gb300 import learned
    t0 = time.perf_counter()
    out = learned.run(ctx, n_train=2000, n_test=200, L=256, M_hi=4096, R=4, epochs=200, batch=256, lr=1e-3,
                      chunk=2200, time_sample=200, noise_sample=50)
    out["leg_wall_s"] = time.perf_counter() - t0
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import paper_1910_05194_gb300 as kite
    from paper_1910_05194_gb300 import _build
    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    ctx = kite.Context(local, stream)
    M, R = args.M, args.R
    system = kite.make_system(kite.HONEYCOMB, args.Lx, args.Ly, WORKLOAD["t"], WORKLOAD["W"], 0.0,
                              WORKLOAD["p_vac"], seed=2 + 1000003 * rank)
    # realisation of this rank: different seed per rank (independent samples)
    kpm = kite.make_kpm(M, R, 1, kite.FP32)
    e_min, e_max = kite.bounds(system)
    K = WORKLOAD["K_energies"]
    E = torch.linspace(e_min, e_max, K + 2, dtype=torch.float64, device="cuda")[1:-1].contiguous()
    mu = torch.zeros(M, dtype=torch.float64, device="cuda")
    rho = torch.zeros(K, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()  # the context's stream does not wait on torch's stream

    def step():
        st = kite.moments_1d(ctx, system, kpm, mu)
        kite.reconstruct_dos(ctx, mu, M, M, kite.KERNEL_JACKSON, 0.0, e_min, e_max, E, K, rho)
        return st

    for _ in range(args.warmup):
        st = step()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step_s, step_n, step_bytes = 0.0, 0, 0.0
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        st = step()
        step_s += st.step_seconds
        step_n += st.step_launches
        step_bytes += st.step_bytes
    ev1.record(stream)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    updates_per_step = float(st.n_eff) * M * R  # this rank's
    value, ms = job_throughput(updates_per_step, ms, dist, device="cuda")
    # onsite, init, recursion launches, reduce, average, dos x2
    launches_per_step = 1 + 1 + step_n // args.steps + 1 + 1 + 2
    roofline = None
    if step_n > 0:
        peak, peak_kind = measured_peaks()
        achieved = step_bytes / step_s / 1e9
        two = st.steps_per_pass == 2
        # updates of one launch: orbitals x vectors x recursion steps of the launch
        upd_per_launch = float(st.n_eff) * R * (2 if two else 1)
        traffic = profiled_traffic(upd_per_launch, st.steps_per_pass)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": ("k_step2<float, honeycomb, 4 chunks> (two recursion steps per pass)" if two
                               else "k_step<float, honeycomb, 4 chunks>"),
                    "algorithmic_bytes_per_launch": step_bytes / step_n,
                    "avg_launch_us": 1e6 * step_s / step_n, "peak_kind": peak_kind + " (copy test)",
                    "note": ("a pass reads r_n-1, r_n, r_0 and writes r_n+1, r_n+2 (5 vector streams "
                             "for 2 steps: 20.25 B/update at R=8, against 32.5 for one step per "
                             "launch); frac is that smaller traffic over the copy peak" if two else
                             "a step reads r_n-1, r_n, r_0 and writes r_n+1 (32.5 B/update at R=8)")}

    # ---- moment doubling on the same workload (two moments per recursion step) --------
    doubling = None
    if not args.no_doubling:
        kpm_d = kite.make_kpm(M, R, 1, kite.FP32, doubling=True)
        mu_d = torch.zeros(M, dtype=torch.float64, device="cuda")

        def step_d():
            st_d = kite.moments_1d(ctx, system, kpm_d, mu_d)
            kite.reconstruct_dos(ctx, mu_d, M, M, kite.KERNEL_JACKSON, 0.0, e_min, e_max, E, K, rho)
            return st_d

        for _ in range(args.warmup):
            step_d()
        barrier()
        ev0.record(stream)
        ds, dn, db = 0.0, 0, 0.0
        for _ in range(args.steps):
            st_d = step_d()
            ds += st_d.step_seconds
            dn += st_d.step_launches
            db += st_d.step_bytes
        ev1.record(stream)
        barrier()
        v_d, ms_d = job_throughput(updates_per_step, ev0.elapsed_time(ev1) / args.steps, dist, device="cuda")
        peak, _ = measured_peaks()
        doubling = {"value": v_d, "unit": UNIT, "ms_per_step": ms_d,
                    "step_launches_per_step": dn // args.steps,
                    "step_gbs": db / ds / 1e9, "step_frac": db / ds / 1e9 / peak,
                    "max_abs_diff_vs_plain": float((mu_d - mu).abs().max().item()),
                    "autotuned": {"ring_stages": st_d.ring_stages, "ctas_per_sm": st_d.ctas_per_sm,
                                  "steps_per_pass": st_d.steps_per_pass},
                    "note": "mu_2n = 2<r_n|r_n> - mu_0, mu_2n+1 = 2<r_n|r_n+1> - mu_1: ceil(M/2) "
                            "steps, r_0 not re-read (with two steps per pass: four vector streams per "
                            "two steps); same M moments, same unit"}

    # ---- real +-1 vectors (16 per batch, half the bytes per vector), with doubling -------
    realvec = None
    if not args.no_doubling:
        R2 = 2 * R
        kpm_r = kite.make_kpm(M, R2, 1, kite.FP32, doubling=True, real_vectors=True)
        mu_r = torch.zeros(M, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            kite.moments_1d(ctx, system, kpm_r, mu_r)
        barrier()
        ev0.record(stream)
        rs, rb = 0.0, 0.0
        for _ in range(args.steps):
            st_r = kite.moments_1d(ctx, system, kpm_r, mu_r)
            rs += st_r.step_seconds
            rb += st_r.step_bytes
        ev1.record(stream)
        barrier()
        v_r, ms_r = job_throughput(float(st_r.n_eff) * M * R2, ev0.elapsed_time(ev1) / args.steps, dist,
                                   device="cuda")
        peak, _ = measured_peaks()
        realvec = {"value": v_r, "unit": UNIT, "R": R2,
                   "ms_per_step": ms_r, "step_gbs": rb / rs / 1e9, "step_frac": rb / rs / 1e9 / peak,
                   "max_abs_diff_vs_complex_plain": float((mu_r - mu).abs().max().item()),
                   "autotuned": {"ring_stages": st_r.ring_stages, "ctas_per_sm": st_r.ctas_per_sm,
                                 "steps_per_pass": st_r.steps_per_pass},
                   "note": "real +-1 vectors (Sec. 2c white noise) with moment doubling; a real vector "
                           "has twice the trace-estimate variance of a unit-phase one, so R=16 real "
                           "carries the statistical weight of R=8 complex at the same bytes"}

    # ---- end to end through the C ABI with host buffers -------------------------------
    e2e = None
    if not args.no_e2e:
        import synth
        n = int(args.Lx) * int(args.Ly) * 2
        r0_host = torch.empty((R, n, 2), dtype=torch.float64, pin_memory=True)
        for r in range(R):  # seeded unit-phase start vectors, one vector at a time
            z = synth.unit_phase_vectors(n, 1, seed=12345 + 1000 * rank + r)[0]
            r0_host[r, :, 0] = torch.from_numpy(z.real)
            r0_host[r, :, 1] = torch.from_numpy(z.imag)
            del z
        mu_h = torch.zeros(M, dtype=torch.float64).pin_memory()
        E_h = E.cpu().pin_memory()
        rho_h = torch.zeros(K, dtype=torch.float64).pin_memory()
        kpm_h = kite.make_kpm(M, R, 1, kite.FP32, r0=r0_host)
        torch.cuda.synchronize()

        def e2e_step():
            kite.moments_1d(ctx, system, kpm_h, mu_h)
            kite.reconstruct_dos(ctx, mu_h, M, M, kite.KERNEL_JACKSON, 0.0, e_min, e_max, E_h, K, rho_h)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            e2e_step()
        barrier()
        t_e2e = (time.perf_counter() - t0) / e2e_steps
        v_e2e, _ = job_throughput(updates_per_step, 1e3 * t_e2e, dist, device="cuda")
        h2d = r0_host.numel() * 8 + mu_h.numel() * 8 + E_h.numel() * 8
        d2h = mu_h.numel() * 8 + rho_h.numel() * 8
        e2e = {"value": v_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "path": "kite_moments_1d(host start vectors, host mu) + kite_reconstruct_dos(host E, host rho)"}

    cpu = None
    panels = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args, kite, ctx, st.n_eff)
        cpu["per_config"], panels = cpu_baselines_per_config(kite, ctx)
        kb = cpu["per_config"]["kubo_bastin_honeycomb_1024x1024_M1024_R4"]
        one_core_ratio = cpu["value"] / cpu["value_1core"]
        kb["extrapolated_full_s_1core"] = kb["extrapolated_full_s_all_cores"] * one_core_ratio
    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except Exception:
            peaks = {}
        secondary = secondary_legs(kite, ctx, peaks)
        if cpu is not None:
            secondary["large_dos_honeycomb_4096x4096_M256_R8_fp64"]["max_abs_dmu_vs_oracle_on_sample"] = \
                cpu["max_abs_dmu_gpu_fp64_vs_oracle_on_sample"]
            secondary["large_dos_honeycomb_4096x4096_M256_R8_fp64"]["oracle_sample"] = cpu["sample"]
        if panels is not None:
            secondary["kubo_bastin_honeycomb_1024x1024_M1024_R4"]["mu_nm_panel_error"] = \
                kubo_bastin_panel_error(kite, ctx, panels)
        if not args.no_learned:
            secondary["learned"] = learned_leg(kite, ctx)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, **WORKLOAD, "Lx": args.Lx, "Ly": args.Ly,
                           "M": M, "R": R, "n_eff": int(st.n_eff),
                           "l2": "inputs larger than L2 (three 2.1 GB vector buffers per step)",
                           "parallelism": f"{world} independent realisations" if world > 1 else "single GPU",
                           "grid": st.grid, "block": st.block,
                           "autotuned": {"ring_stages": st.ring_stages, "ctas_per_sm": st.ctas_per_sm, "steps_per_pass": st.steps_per_pass}},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "moment_doubling": doubling, "real_vectors": realvec, "secondary": secondary,
                "gpu_launches": launches_per_step * args.steps,
                "wall_s_timed": wall}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
