"""Benchmark: batched Monte Carlo Kelvin-Helmholtz on one GB300.

Workload (one "step" = one pass of the whole hot path over one batch): 4096 seeded samples of the
2D Kelvin-Helmholtz problem on a 256^2 periodic grid, FP32 state, WENO3 + HLLC + SSP-RK3 at CFL
0.4 to T = 1 with a per-sample CFL step (about 1,500 RK steps per sample), then the FP64 Welford
mean/variance of (rho, u, v, p) per cell and the FP64 conservation totals. Metric: cell-updates/s
(one cell advanced one full RK step, summed over samples) and samples/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The state (4.3 GB) and stage buffers exceed L2 (129 MB), so no L2 flush is needed between steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
M = 4096
T_END = 1.0
SEED = 12345
METRIC = "cell-updates/s & % HBM roofline; MC samples/s batched-FP32 vs plain FP64"
# Algorithmic floating-point operations per cell-update of 2D WENO3 (primitive) + HLLC + SSP-RK3,
# counted on the oracle's counting scalar (a CPU test checks this constant against that count).
FLOPS_PER_CELL_UPDATE_2D_WENO3_HLLC_RK3 = 1980
# FP32 (non-tensor) peak from the unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops (FMA)
# x 2.07 GHz (maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
STAGE_KERNEL_NAMES = {0: "k_stage<float, Euler, 2D, WENO3, HLLC, 32x16>",
                      1: "k_stage<float, Euler, 2D, WENO3, HLLC, 32x8>",
                      2: "k_stage<float, Euler, 2D, WENO3, HLLC, 32x32>",
                      3: "k_stage2d_col<WENO3, HLLC>",
                      4: "k_stage2d_pair<WENO3, HLLC, 32x16>",
                      5: "k_stage2d_pair<WENO3, HLLC, 32x8>",
                      6: "k_stage2d_pair<WENO3, HLLC, 32x16, sample halves>",
                      7: "k_stage2d_pair<WENO3, HLLC, 32x8, sample halves>",
                      8: "k_stage2d_pair2<WENO3, HLLC, 32x16>",
                      9: "k_stage2d_pair2<WENO3, HLLC, 32x16, reads in flight>",
                      10: "k_stage2d_pair2<WENO3, HLLC, 32x16, sample halves>",
                      11: "k_stage2d_pair2<WENO3, HLLC, 32x16, sample halves, reads in flight>",
                      12: "k_stage2d_pair2<WENO3, HLLC, 32x16, reads in flight, x-fluxes by shuffle>",
                      13: "k_stage2d_pair2<WENO3, HLLC, 32x16, sample halves, reads in flight, x-fluxes by shuffle>"}
WORKLOAD = "kh2d_256x256_mc4096_weno3_hllc_ssprk3_fp32_T1"
# compulsory HBM bytes per 2D SSP-RK3 cell-update in FP32: per variable read U^n + write U1,
# read U1 + U^n + write U2, read U2 + U^n + write U^{n+1} = 8 words, x 4 variables x 4 bytes
BYTES_PER_CELL_UPDATE = 8 * 4 * 4


def desc_kwargs(batch=M, seed=SEED):
    return dict(ndim=2, n=(N, N), lo=(0, 0), hi=(1, 1), batch=batch, eq="euler", gamma=1.4, recon="weno3",
                rvars="prim", flux="hllc", rk="ssprk3", bc="periodic", cfl=0.4, precision="fp32", seed=seed)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        # the raw samples go to BENCH_CLOCK_DIR when set (to keep them), else to a temporary folder
        d = os.environ.get("BENCH_CLOCK_DIR") or tempfile.mkdtemp(prefix="bench_clocks_")
        self.path = os.path.join(d, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def _parse(self, lines):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return sm, mx, reasons

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = self._parse(open(self.path))
        if not sm:
            # a region shorter than the sampler's start-up: one sample right after it
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
                sm, mx, reasons = self._parse(out.stdout.splitlines())
            except Exception:
                pass
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_step(S, alsv, world=1):
    """One pass of the hot path on device-resident inputs: init from the seed, evolve to T,
    statistics, totals; with several ranks, the per-rank statistics are all-gathered and merged
    in rank order (the one exchange of the sharded ensemble). Returns per-sample step counts."""
    S.set_initial_data("kh")
    S.evolve_to(T_END)
    alsv.alsv_stats_reset(S.ctx, S.stats)
    alsv.alsv_stats_accumulate(S.ctx, S.stats)
    alsv.alsv_conservation_totals(S.ctx, S.tot)
    if world > 1:
        from paper_1912_07645_gb300.parallel import gather, merge_in_rank_order
        S.sync()
        S.merged = merge_in_rank_order(S, gather(S.stats))
    _, nstep = S.time()
    return nstep


def plain_fp64_loop(alsv, torch, steps_per_sample, variant, T_short=0.066):
    """The plain per-sample FP64 path on the same GPU: sample 0 of the batch alone (B = 1) in FP64,
    timed over the CFL steps to T_short and extrapolated to the sample's full step count. Its
    relative L1 difference from the batched FP32 result for the same sample at T_short (the batch's
    stage schedule; a sample's result does not depend on the batch around it) states the error at
    which the two throughputs compare. Returns (line entry, FP32 state, FP64 state) at T_short."""
    kw = desc_kwargs(batch=1)
    S64 = alsv.Solver(alsv.make_desc(**dict(kw, precision="fp64")))
    S64.set_initial_data("kh")
    S64.step(3)
    S64.sync()
    S64.set_initial_data("kh")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = S64.evolve_to(T_short)
    el = time.perf_counter() - t0
    u64 = S64.to_host(S64.U).double()
    S64.close()
    S32 = alsv.Solver(alsv.make_desc(**kw))
    S32.set_initial_data("kh")
    alsv.alsv_set_tile_variant(S32.ctx, variant)
    S32.evolve_to(T_short)
    u32 = S32.to_host(S32.U).double()
    S32.close()
    rel = float((u32 - u64).abs().sum() / u64.abs().sum())
    ms_step = 1000.0 * el / max(n, 1)
    return ({"samples_per_s": 1000.0 / (ms_step * steps_per_sample), "ms_per_rk_step": ms_step, "steps_timed": n,
             "T_timed": T_short, "steps_per_sample": int(steps_per_sample), "precision": "fp64",
             "fp32_batched_vs_fp64_rel_l1": rel}, u32.numpy(), u64.numpy())


def errors_vs_oracle(u32, u64, T_short=0.066):
    """The cpu_baseline leg's second use of the oracle: sample 0 of the workload evolved by the FP64
    oracle to T_short, and the relative L1 differences of the GPU's FP32 (batched schedule) and FP64
    results for that sample from it - the error each result states against the FP64 oracle."""
    import numpy as np
    import oracle
    d = oracle.make_desc(**desc_kwargs(batch=1))
    th = oracle.theta_splitmix(SEED, 1, 20)
    uo, _, _ = oracle.evolve(d, oracle.init(d, "kh", 1, th), T=T_short)
    den = np.abs(uo).sum()
    return {"T": T_short, "sample": 0, "fp32_batched_vs_oracle_rel_l1": float(np.abs(u32.reshape(uo.shape) - uo).sum() / den),
            "fp64_vs_oracle_rel_l1": float(np.abs(u64.reshape(uo.shape) - uo).sum() / den),
            "fp64_vs_oracle_max_rel": float(np.abs(u64.reshape(uo.shape) - uo).max() / np.abs(uo).max())}


def stage_traffic(variant, cell_updates, launches):
    """DRAM bytes per stage launch from the committed ncu summary, scaled from its per-cell-update
    figure; None once the kernel sources no longer match the profiled ones or another schedule
    was chosen."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "stage_traffic.txt")
    if not os.path.exists(path) or launches <= 0:
        return None, None
    rec, per_variant = {}, {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            if f[0] == "variant":   # variant V bytes_per_cell_update B thread_inst_per_cell_stage I
                per_variant[f[1]] = dict(zip(f[2::2], f[3::2]))
            else:
                rec[f[0]] = f[1]
    if str(variant) not in per_variant:
        return None, None
    rec.update(per_variant[str(variant)], variant=str(variant))
    csrc = os.path.join(ROOT, "paper_1912_07645_gb300", "csrc")
    h = hashlib.sha256()
    kernel_src = "fv_pair2.cuh" if variant in (8, 9, 10, 11, 12, 13) else "fv_pair.cuh"
    for f in (kernel_src, "fv_packed.cuh", "fv_physics.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    if h.hexdigest()[:16] != rec.get("sources_sha256_prefix") or str(variant) != rec.get("variant"):
        return None, None
    pcu = float(rec["bytes_per_cell_update"])
    stage_traffic.inst_per_cell_stage = float(rec["thread_inst_per_cell_stage"]) if "thread_inst_per_cell_stage" in rec else None
    return pcu * cell_updates / launches, pcu


def cpu_baseline_oracle(budget_s=15.0):
    """Time the FP64 oracle as it stands on this host's cores on a bounded sample of the same
    workload (one sample of the batch, as many CFL steps as fit in the budget)."""
    import oracle
    import numpy as np
    kw = desc_kwargs(batch=1)
    d = oracle.make_desc(**kw)
    th = oracle.theta_splitmix(SEED, 1, 20)
    U = oracle.init(d, "kh", 1, th)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and steps < 10000:
        U, s, _ = oracle.evolve(d, U, T=math.inf, max_steps=1)
        steps += 1
    el = time.perf_counter() - t0
    cu = steps * N * N
    return {"value": cu / el, "unit": "cell-updates/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1 of {M} samples, first {steps} CFL steps of T=1 on 256^2 (FP64 oracle, {el:.1f} s)",
            "elapsed_s": el, "cell_updates": cu}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    per_step = max(3.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline_oracle(budget_s=min(per_step, 3.0))
    vals, tot_cu, tot_t = [], 0, 0.0
    last = None
    for _ in range(args.steps):
        last = cpu_baseline_oracle(budget_s=per_step)
        tot_cu += last["cell_updates"]
        tot_t += last["elapsed_s"]
    value = tot_cu / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded KH parameters, SplitMix64)",
            "config": {"workload": WORKLOAD, "grid": [N, N], "samples": M, "T": T_END,
                       "reference_sample": "one sample per step, CFL steps within a time budget"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# Other configurations (1D Sod, KH 2D 1024^2, uneven and coupled MLMC levels, the adjoint, the 3D
# slab): same JSON contract, one GPU.
# bytes per cell-update: per variable read U^n + write U1 (stage 1), read U^(s) + U^n + write (later
# stages): RK2 = 5 words, RK3 = 8 words.
WORKLOADS = {
    "sod1024_fp64": dict(desc=dict(ndim=1, n=(1024,), batch=1, eq="euler", recon="mc", flux="hllc", rvars="prim",
                                   rk="ssprk2", bc="outflow", cfl=0.45, precision="fp64"), init="sod", T=0.2,
                         words=5, nv=3, esize=8),
    "kh2d1024_fp32": dict(desc=dict(ndim=2, n=(1024, 1024), batch=1, eq="euler", recon="weno3", flux="hllc",
                                    rvars="prim", rk="ssprk3", bc="periodic", cfl=0.4, precision="fp32", seed=0),
                          init="kh", T=2.0, words=8, nv=4, esize=4),
    # the batched KH workload's scheme on 512 samples to T = 0.2, each sample resident in one
    # thread-block cluster for its whole evolution (16 CTAs, 256 threads each)
    "kh2d256_resident_fp32": dict(desc=dict(ndim=2, n=(256, 256), batch=512, eq="euler", recon="weno3", flux="hllc",
                                            rvars="prim", rk="ssprk3", bc="periodic", cfl=0.4, precision="fp32",
                                            seed=SEED), init="kh", T=0.2, words=8, nv=4, esize=4, resident=True),
    # the further numerics of Sec. 2.1 (Roe, Godunov, ENO2, the entropy-conservative fluxes and
    # TECNO2) on the KH data, each on the default tile schedule (the only one they run on), beside
    # HLLC + WENO3 on the same schedule: 20 RK3 steps of 256 (FP32) / 32 (FP64) samples of 256^2
    "schemes_kh2d256": dict(desc=dict(ndim=2, n=(256, 256), eq="euler", rvars="prim", rk="ssprk3", bc="periodic",
                                      cfl=0.4, seed=SEED), init="kh", steps=20, schemes=True,
                            batch={"fp32": 256, "fp64": 32},
                            list=[("hllc", "weno3"), ("roe", "weno3"), ("godunov", "weno3"), ("hllc", "eno2"),
                                  ("ec", "pc"), ("ec4", "pc"), ("tecno2", "pc")]),
    "kh2d1024_fp64": dict(desc=dict(ndim=2, n=(1024, 1024), batch=1, eq="euler", recon="weno3", flux="hllc",
                                    rvars="prim", rk="ssprk3", bc="periodic", cfl=0.4, precision="fp64", seed=0),
                          init="kh", T=0.02, words=8, nv=4, esize=8),
    "mlmc_fp32": dict(desc=dict(ndim=2, levels=[((64, 64), 4096), ((128, 128), 1024), ((256, 256), 256),
                                                ((512, 512), 64)], eq="euler", recon="weno3", flux="hllc",
                                rvars="prim", rk="ssprk3", bc="periodic", cfl=0.4, precision="fp32", seed=SEED),
                      init="kh", T=1.0, words=8, nv=4, esize=4),
    "mlmc_coupled_fp32": dict(desc=dict(ndim=2, levels=[((64, 64), 4096), ((128, 128), 1024), ((64, 64), 1024, 1),
                                                        ((256, 256), 256), ((128, 128), 256, 3), ((512, 512), 64),
                                                        ((256, 256), 64, 5)], eq="euler", recon="weno3",
                                        flux="hllc", rvars="prim", rk="ssprk3", bc="periodic", cfl=0.4,
                                        precision="fp32", seed=SEED),
                              init="kh", T=1.0, words=8, nv=4, esize=4, mlmc=True),
    "kh3d512_fp32": dict(desc=dict(ndim=3, n=(512, 512, 512), batch=1, eq="euler", recon="weno3", flux="hllc",
                                   rvars="prim", rk="ssprk3", bc="periodic", cfl=0.3, precision="fp32", seed=0),
                         init="kh", steps=100, words=8, nv=5, esize=4),
    # a quarter-size slab for profiler captures (state 0.34 GB, above L2)
    "kh3d256_fp32": dict(desc=dict(ndim=3, n=(256, 256, 256), batch=1, eq="euler", recon="weno3", flux="hllc",
                                   rvars="prim", rk="ssprk3", bc="periodic", cfl=0.3, precision="fp32", seed=0),
                         init="kh", steps=10, words=8, nv=5, esize=4),
    # one 1024^3 sample (5.4e9 elements, above one context's 2^31) as four z-blocks on one GPU with
    # halo exchange between RK stages; the same scheme at 512^3 whole and as four blocks gives the
    # decomposition's overhead, (t_blocks - t_whole) / t_whole per step (Sec. 3.1)
    "kh3d1024_blocks_fp32": dict(desc=dict(ndim=3, n=(1024, 1024, 1024), batch=1, eq="euler", recon="weno3",
                                           flux="hllc", rvars="prim", rk="ssprk3", bc="periodic", cfl=0.3,
                                           precision="fp32", seed=0),
                                 init="kh", steps=20, parts=(1, 1, 4), words=8, nv=5, esize=4, blocks=True,
                                 overhead_n=(512, 512, 512), overhead_steps=40),
    # the same at 256^3 (state 0.34 GB), for profiler captures
    "kh3d256_blocks_fp32": dict(desc=dict(ndim=3, n=(256, 256, 256), batch=1, eq="euler", recon="weno3",
                                          flux="hllc", rvars="prim", rk="ssprk3", bc="periodic", cfl=0.3,
                                          precision="fp32", seed=0),
                                init="kh", steps=10, parts=(1, 1, 4), words=8, nv=5, esize=4, blocks=True,
                                overhead_n=(256, 256, 256), overhead_steps=20),
    "adjoint512_fp32": dict(desc=dict(ndim=2, n=(512, 512), batch=64, eq="euler", recon="mc", flux="rusanov",
                                      rvars="prim", rk="ssprk2", bc="periodic", cfl=0.4, precision="fp32", seed=SEED),
                            adjoint=True, T=1.0),
    # the same at T = 0.01 (31 fixed steps), for profiler captures
    "adjoint512_fp32_short": dict(desc=dict(ndim=2, n=(512, 512), batch=64, eq="euler", recon="mc", flux="rusanov",
                                            rvars="prim", rk="ssprk2", bc="periodic", cfl=0.4, precision="fp32",
                                            seed=SEED), adjoint=True, T=0.01),
    "adjoint512_fp64": dict(desc=dict(ndim=2, n=(512, 512), batch=64, eq="euler", recon="mc", flux="rusanov",
                                      rvars="prim", rk="ssprk2", bc="periodic", cfl=0.4, precision="fp64", seed=SEED),
                            adjoint=True, T=1.0),
    # agreement of the FP64 adjoint gradient with central differences formed inside one batch
    # (sample 0 of the ensemble, +-h on six of the 20 parameters: 13 samples) at growing horizons
    "adjoint512_fp64_fd": dict(desc=dict(ndim=2, n=(512, 512), batch=13, eq="euler", recon="mc", flux="rusanov",
                                         rvars="prim", rk="ssprk2", bc="periodic", cfl=0.4, precision="fp64",
                                         seed=SEED), adjoint=True, fd_check=(0.01, 0.1, 0.3, 0.6, 1.0),
                               fd_params=(0, 3, 7, 10, 13, 17), fd_h=(1e-6,)),
    # the same at the two horizons where h = 1e-6 straddles limiter kinks, with smaller steps
    "adjoint512_fp64_fd_h": dict(desc=dict(ndim=2, n=(512, 512), batch=13, eq="euler", recon="mc", flux="rusanov",
                                           rvars="prim", rk="ssprk2", bc="periodic", cfl=0.4, precision="fp64",
                                           seed=SEED), adjoint=True, fd_check=(0.3, 0.6),
                                 fd_params=(0, 3, 7, 10, 13, 17), fd_h=(1e-7, 1e-8)),
}


# Algorithmic floating-point operations per cell-update of each workload's scheme, counted on the
# oracle's counting scalar (a CPU test checks them), and the ALU peaks: FP32 from the unit counts
# (152 SMs x 128 lanes x 2 x 2.07 GHz), FP64 the GB300's nominal 1.25 TFLOP/s.
WORKLOAD_FLOPS = {"sod1024_fp64": 287, "kh2d1024_fp32": 1980, "kh2d1024_fp64": 1980, "mlmc_fp32": 1980,
                  "mlmc_coupled_fp32": 1980, "kh3d512_fp32": 3591, "kh3d256_fp32": 3591,
                  "kh3d1024_blocks_fp32": 3591, "kh3d256_blocks_fp32": 3591}
FP64_PEAK_TFLOPS = 1.25
ISSUE_CLOCK_GHZ = 2.07


def run_adjoint_fd_check(name, W, S, alsv, torch):
    """FP64 adjoint gradient of the kinetic energy at T against central differences formed inside
    one batch (h = h_rel max(1, |theta_j|)), for each step h_rel and horizon T of the workload: the largest
    |g_j - fd_j| over the checked parameters relative to max_j |g_j|, with the plan used."""
    import numpy as np
    P = W["fd_params"]
    B = 1 + 2 * len(P)
    S.set_initial_data("kh")
    th0 = torch.empty((S.samples, 20), dtype=torch.float64, device="cuda")
    alsv.alsv_get_parameters(S.ctx, th0)
    S.sync()
    base = th0[0].cpu().numpy()
    rows = []
    for hrel, T in [(h, T) for h in W["fd_h"] for T in W["fd_check"]]:
        th = np.tile(base, (B, 1))
        hs = hrel * np.maximum(1.0, np.abs(base))
        for i, j in enumerate(P):
            th[1 + 2 * i, j] += hs[j]
            th[2 + 2 * i, j] -= hs[j]
        tth = torch.from_numpy(th).cuda()
        t0 = time.perf_counter()
        J, g = S.adjoint(tth, T)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        J, g = J.cpu().numpy(), g.cpu().numpy()
        nst, dt_fixed, passes = alsv.alsv_adjoint_get_plan(S.ctx)
        fd = np.array([(J[1 + 2 * i] - J[2 + 2 * i]) / (2 * hs[j]) for i, j in enumerate(P)])
        gsel = g[0, list(P)]
        rows.append({"T": T, "h": hrel, "steps": int(nst), "passes": int(passes), "J": float(J[0]),
                     "max_abs_grad": float(np.abs(g[0]).max()),
                     "rel_diff_vs_fd": float(np.abs(gsel - fd).max() / np.abs(g[0]).max()),
                     "per_param_rel": [float(abs(a - b) / max(abs(b), 1e-300)) for a, b in zip(gsel, fd)],
                     "seconds": el})
    line = {"metric": "adjoint gradient vs central differences (FP64, KE, 512^2 KH)", "value": rows[-1]["rel_diff_vs_fd"],
            "unit": "max |g - fd| / max |g|", "higher_is_better": False, "n_gpus": 1,
            "config": {"workload": name, "grid": [512, 512], "samples": B, "params_checked": list(P)},
            "horizons": rows, "gpu_launches": alsv.alsv_get_launch_count(S.ctx)}
    print(json.dumps(line), flush=True)
    S.close()
    return 0


def run_blocks_workload(name, W, args):
    """A single sample decomposed into blocks on one GPU (halo exchange between RK stages)."""
    import numpy as np
    import torch
    import paper_1912_07645_gb300 as alsv
    from paper_1912_07645_gb300.decomp import Decomposition
    peaks, peak_kind = measured_peaks()
    cfg = W["desc"]
    dec = Decomposition(parts=W["parts"], **cfg)
    dec.set_initial_data(W["init"])
    b0 = dec.blocks[0]
    if args.tile_variant >= 0:
        chosen, ms_var = args.tile_variant, []
    else:
        chosen, ms_var = b0.autotune(3)
    for b in dec.blocks:
        b.set_tile_variant(chosen)
    cells = int(np.prod(cfg["n"]))

    def one():
        dec.set_initial_data(W["init"])
        dec.step(W["steps"])
        dec.sync()
        return W["steps"] * cells

    for _ in range(args.warmup):
        one()
    dec.set_profiling(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cu = 0
    for _ in range(args.steps):
        cu += one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    stage_ms, stage_launches = dec.stage_ms()
    dec.set_profiling(False)
    launches = sum(alsv.alsv_get_launch_count(b.ctx) for b in dec.blocks)
    dec.close()
    del dec
    torch.cuda.empty_cache()

    # overhead of the decomposition: the same scheme at a size one context holds, whole vs blocks
    def per_step(parts, overlap=False):
        kw = dict(cfg, n=W["overhead_n"])
        if parts is None:
            S = alsv.Solver(alsv.make_desc(**kw))
            S.set_tile_variant(chosen)
            S.set_initial_data(W["init"])
            run = (lambda k: (S.step(k), S.sync()))
            close = S.close
        else:
            D = Decomposition(parts=parts, tile_variant=chosen, overlap=overlap, **kw)
            D.set_initial_data(W["init"])
            run = (lambda k: (D.step(k), D.sync()))
            close = D.close
        run(3)
        torch.cuda.synchronize()
        t = time.perf_counter()
        run(W["overhead_steps"])
        torch.cuda.synchronize()
        ms = 1000 * (time.perf_counter() - t) / W["overhead_steps"]
        close()
        return ms

    ms_whole = per_step(None)
    ms_blocks = per_step(W["parts"], overlap=False)
    ms_blocks_split = per_step(W["parts"], overlap=True)
    bpc = W["words"] * W["nv"] * W["esize"]
    # the blocks' stage launches run concurrently on their own streams, so their event times
    # overlap: the achieved rates use the wall time of the timed steps (stages, halo packs and time
    # control), a lower bound of the stage kernels' own rate
    achieved = cu * bpc / el / 1e9
    tflops = cu * WORKLOAD_FLOPS[name] / el / 1e12
    line = {"metric": METRIC, "value": cu / el, "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": cfg["precision"], "data": "synthetic",
            "config": {"workload": name, "grid": list(cfg["n"]), "blocks": list(W["parts"]),
                       "rk_steps_per_pass": W["steps"], "samples": 1, "tile_variant": chosen,
                       "autotune_ms": ms_var},
            "ms_per_rk_step": 1000 * el / (args.steps * W["steps"]),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"] if achieved else None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_cell_update": bpc, "time_basis": "wall time of the timed steps",
                         "stage_event_ms_sum": stage_ms, "stage_launches": stage_launches,
                         "step_ms_total": 1000 * el},
            "alu_roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": tflops / FP32_PEAK_TFLOPS,
                             "flops_per_cell_update": WORKLOAD_FLOPS[name],
                             "peak_kind": "nominal: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
            "decomposition_overhead": {"grid": list(W["overhead_n"]), "blocks": list(W["parts"]),
                                       "ms_per_step_whole": ms_whole, "ms_per_step_blocks": ms_blocks,
                                       "overhead": (ms_blocks - ms_whole) / ms_whole,
                                       "ms_per_step_blocks_split_stages": ms_blocks_split,
                                       "overhead_split_stages": (ms_blocks_split - ms_whole) / ms_whole},
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    return 0


def run_schemes_workload(name, W, args):
    """Cell-updates/s of each listed scheme in FP32 and FP64 on the default tile schedule."""
    import numpy as np
    import torch
    import paper_1912_07645_gb300 as alsv
    rows, launches = [], 0
    only = tuple(args.scheme.split(",")) if args.scheme else None   # flux,recon,precision
    for precision in ("fp32", "fp64"):
        for flux, recon in W["list"]:
            if only and (flux, recon, precision) != only:
                continue
            cfg = dict(W["desc"], flux=flux, recon=recon, precision=precision, batch=W["batch"][precision])
            S = alsv.Solver(alsv.make_desc(**cfg))
            alsv.alsv_set_tile_variant(S.ctx, 0)
            cells = cfg["batch"] * int(np.prod(cfg["n"]))

            def one():
                S.set_initial_data(W["init"])
                S.step(W["steps"])
                S.sync()

            for _ in range(args.warmup):
                one()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                one()
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            _, ns = S.time()   # sync() above raised if a sample went non-physical
            launches += alsv.alsv_get_launch_count(S.ctx)
            rows.append({"flux": flux, "recon": recon, "precision": precision, "samples": cfg["batch"],
                         "cell_updates_per_s": cells * W["steps"] * args.steps / el,
                         "ms_per_rk_step": 1000 * el / (args.steps * W["steps"]), "steps_done": int(ns.max())})
            S.close()
    tec = ([r for r in rows if r["flux"] == "tecno2" and r["precision"] == "fp32"] or rows)[0]
    line = {"metric": "cell-updates/s per scheme (default tile schedule)", "value": tec["cell_updates_per_s"],
            "value_is": f"{tec['flux']} + {tec['recon']}, {tec['precision']}", "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32 and fp64", "data": "synthetic (seeded KH perturbation parameters, SplitMix64)",
            "config": {"workload": name, "grid": list(W["desc"]["n"]), "rk_steps": W["steps"],
                       "samples": W["batch"], "tile_variant": 0},
            "schemes": rows, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    return 0


def run_workload(name, args):
    import numpy as np
    import torch
    from paper_1912_07645_gb300 import build
    build.build()
    import paper_1912_07645_gb300 as alsv
    W = WORKLOADS[name]
    if W.get("blocks"):
        return run_blocks_workload(name, W, args)
    if W.get("schemes"):
        return run_schemes_workload(name, W, args)
    desc = alsv.make_desc(**W["desc"])
    S = alsv.Solver(desc)
    peaks, peak_kind = measured_peaks()
    if W.get("fd_check"):
        return run_adjoint_fd_check(name, W, S, alsv, torch)
    if W.get("adjoint"):
        S.set_initial_data("kh")
        # the forward sweeps run the context's stage schedule: pick the fastest for this shape
        if args.tile_variant >= 0:
            alsv.alsv_set_tile_variant(S.ctx, args.tile_variant)
            chosen, ms_var = args.tile_variant, []
        else:
            chosen, ms_var = alsv.alsv_autotune(S.ctx, 3) if alsv.alsv_num_tile_variants(S.ctx) > 1 else (0, [])
        th = torch.empty((S.samples, 20), dtype=torch.float64, device="cuda")
        alsv.alsv_get_parameters(S.ctx, th)
        S.sync()
        for _ in range(args.warmup):
            S.adjoint(th, min(W["T"], 0.01))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            J, g = S.adjoint(th, W["T"])
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        nst, dt_fixed, passes = alsv.alsv_adjoint_get_plan(S.ctx)
        grads = S.samples * args.steps / el
        line = {"metric": "adjoint gradients/s (KE at T w.r.t. 20 KH parameters)", "value": grads,
                "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": W["desc"]["precision"], "data": "synthetic (SplitMix64 KH parameters)",
                "config": {"workload": name, "grid": [512, 512], "samples": S.samples, "T": W["T"],
                           "fixed_steps": nst, "fixed_dt": dt_fixed, "forward_passes": passes,
                           "tile_variant": chosen, "autotune_ms": ms_var},
                "forward_cell_updates_per_s": S.samples * 512 * 512 * nst * args.steps / el,
                "gpu_launches": alsv.alsv_get_launch_count(S.ctx)}
        print(json.dumps(line), flush=True)
        S.close()
        return 0
    chosen, ms_var = (0, [])
    S.set_initial_data(W["init"])
    if args.tile_variant >= 0:
        alsv.alsv_set_tile_variant(S.ctx, args.tile_variant)
        chosen = args.tile_variant
    elif alsv.alsv_num_tile_variants(S.ctx) > 1:
        chosen, ms_var = alsv.alsv_autotune(S.ctx, 3)
    cells = [int(np.prod(desc.level_n[l][:desc.ndim])) for l in range(desc.n_levels)] if desc.n_levels > 1 else \
        [int(np.prod(list(desc.n)[:desc.ndim]))]

    est = {}

    def one():
        S.set_initial_data(W["init"])
        if "steps" in W:
            S.step(W["steps"])
            S.sync()
        elif W.get("resident"):
            S.evolve_resident(W["T"])
        else:
            S.evolve_to(W["T"])
        if W.get("mlmc"):
            S.mlmc_init()
            S.mlmc_accumulate()
            est["counts"], _, _, lev = S.mlmc_read()
            est["level_sums"] = lev.cpu().numpy()
        _, ns = S.time()
        if desc.n_levels > 1:
            cu, s0 = 0, 0
            for l in range(desc.n_levels):
                B = desc.level_batch[l]
                cu += int(ns[s0:s0 + B].sum()) * cells[l]
                s0 += B
            return cu
        return int(ns.sum()) * cells[0]

    for _ in range(args.warmup):
        one()
    alsv.alsv_set_profiling(S.ctx, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cu = 0
    for _ in range(args.steps):
        cu += one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    prof = alsv.alsv_get_profile(S.ctx)
    alsv.alsv_set_profiling(S.ctx, False)
    bpc = W["words"] * W["nv"] * W["esize"]
    achieved = cu * bpc / (prof["stage_ms"] / 1000.0) / 1e9 if prof["stage_ms"] > 0 else None
    line = {"metric": METRIC, "value": cu / el, "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": W["desc"]["precision"], "data": "synthetic",
            "config": {"workload": name, "T": W.get("T"), "fixed_steps": W.get("steps"), "samples": S.samples,
                       "tile_variant": chosen, "autotune_ms": ms_var},
            "samples_per_s": S.samples * args.steps / el,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"] if achieved else None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_cell_update": bpc, "stage_ms_total": prof["stage_ms"],
                         "stage_launches": prof["stage_launches"], "step_ms_total": 1000 * el},
            "gpu_launches": alsv.alsv_get_launch_count(S.ctx)}
    if W.get("resident"):
        # the whole run is one launch per pass; its rate against the batched tile schedule of the
        # same samples (the state would move to HBM and back every stage there)
        line["config"]["schedule"] = "resident: one thread-block cluster per sample, distributed shared memory"
        t0 = time.perf_counter()
        cu_tile = 0
        for _ in range(args.steps):
            S.set_initial_data(W["init"])
            S.evolve_to(W["T"])
            _, ns = S.time()
            cu_tile += int(ns.sum()) * cells[0]
        torch.cuda.synchronize()
        line["batched_tile_schedule"] = {"value": cu_tile / (time.perf_counter() - t0), "unit": "cell-updates/s",
                                         "tile_variant": chosen}
        line["roofline"] = None
    if name in WORKLOAD_FLOPS and prof["stage_ms"] > 0:
        fp64 = W["desc"]["precision"] == "fp64"
        peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
        tflops = cu * WORKLOAD_FLOPS[name] / (prof["stage_ms"] / 1000.0) / 1e12
        line["alu_roofline"] = {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                                "frac": tflops / peak, "flops_per_cell_update": WORKLOAD_FLOPS[name],
                                "peak_kind": "nominal FP64" if fp64 else "nominal: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    if W.get("mlmc"):
        # per level: samples, grid, mean steps per sample of the pair, and for rho the integrals of
        # the mean correction |E[Y_l]| and of its variance Var[Y_l] (the variance decay)
        _, ns = S.time()
        lv = S.mlmc_levels()
        rows = []
        for k, l in enumerate(lv):
            s0 = sum(desc.level_batch[j] for j in range(l))
            rows.append({"level": k, "grid": list(desc.level_n[l])[:2], "samples": est["counts"][k],
                         "steps_per_sample": float(ns[s0:s0 + desc.level_batch[l]].mean()),
                         "rho_abs_mean_correction": float(est["level_sums"][k, 0, 1]),
                         "rho_var_correction": float(est["level_sums"][k, 0, 2])})
        line["mlmc_levels"] = rows
    print(json.dumps(line), flush=True)
    S.close()
    return 0


def main():
    global T_END
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="alsv")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--samples", type=int, default=M, help="samples per GPU (default 4096; fewer for profiling runs)")
    ap.add_argument("--T", type=float, default=T_END, help="end time (default 1; shorter for profiling runs)")
    ap.add_argument("--tile-variant", type=int, default=-1,
                    help="skip the autotuner and run this stage schedule (profiler runs, where timing the "
                         "candidates under the profiler would pick another one)")
    ap.add_argument("--scheme", default="", help="schemes_kh2d256 only: run one 'flux,recon,precision'")
    ap.add_argument("--workload", default="mc", choices=["mc"] + sorted(WORKLOADS),
                    help="mc (default): batched Monte Carlo KH 256^2 x 4096; others: the remaining configurations")
    args = ap.parse_args()
    T_END = args.T
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload != "mc":
        return run_workload(args.workload, args)

    import torch
    import torch.distributed as dist
    from paper_1912_07645_gb300 import build
    build.build()
    import paper_1912_07645_gb300 as alsv

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    Mr = args.samples
    # weak scaling: every rank advances its own contiguous shard of Mr samples of one ensemble
    kw = dict(desc_kwargs(batch=Mr), sample_offset=rank * Mr)
    S = alsv.Solver(alsv.make_desc(**kw))
    S.stats_init()
    with torch.cuda.stream(S.stream):
        S.tot = torch.empty((Mr, 4), dtype=torch.float64, device=dev)
    S.set_initial_data("kh")
    if args.tile_variant >= 0:
        alsv.alsv_set_tile_variant(S.ctx, args.tile_variant)
        chosen, ms_var = args.tile_variant, []
    else:
        chosen, ms_var = alsv.alsv_autotune(S.ctx, 3)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        run_step(S, alsv, world)
    barrier()
    # ---- device-timed region (inputs resident in HBM)
    clocks = ClockSampler(local)
    clocks.start()
    alsv.alsv_set_profiling(S.ctx, True)
    l0 = alsv.alsv_get_launch_count(S.ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(S.stream)
    cell_updates = 0
    for _ in range(args.steps):
        nstep = run_step(S, alsv, world)
        cell_updates += int(nstep.sum()) * N * N
    ev1.record(S.stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = alsv.alsv_get_launch_count(S.ctx) - l0
    prof = alsv.alsv_get_profile(S.ctx)
    alsv.alsv_set_profiling(S.ctx, False)
    ck = clocks.stop()
    t_rank = torch.tensor([ms], dtype=torch.float64, device=dev)
    cu_rank = torch.tensor([float(cell_updates)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_rank, op=dist.ReduceOp.MAX)
        dist.all_reduce(cu_rank, op=dist.ReduceOp.SUM)
    ms_max = float(t_rank.item())
    cu_all = float(cu_rank.item())
    value = cu_all / (ms_max / 1000.0)
    samples_per_s = world * Mr * args.steps / (ms_max / 1000.0)

    # ---- end-to-end through the public API with host buffers (pinned)
    th_host = torch.empty((Mr, 20), dtype=torch.float64).pin_memory()
    th_host.copy_(torch.from_numpy(__import__("numpy").random.default_rng(rank).uniform(0, 1, (Mr, 20))))
    th_host[:, 10:] *= 2 * math.pi
    mean_host = torch.empty((4, 1, N, N), dtype=torch.float64).pin_memory()
    var_host = torch.empty_like(mean_host)
    with torch.cuda.stream(S.stream):
        th_dev = torch.empty((Mr, 20), dtype=torch.float64, device=dev)
        mean_dev = torch.empty((4, 1, N, N), dtype=torch.float64, device=dev)
        var_dev = torch.empty_like(mean_dev)
    barrier()
    t0 = time.perf_counter()
    cu_e2e = 0
    for _ in range(args.steps):
        with torch.cuda.stream(S.stream):
            th_dev.copy_(th_host, non_blocking=True)
        alsv.alsv_set_initial_data(S.ctx, "kh", th_dev, 20, S.U)
        S.evolve_to(T_END)
        alsv.alsv_stats_reset(S.ctx, S.stats)
        alsv.alsv_stats_accumulate(S.ctx, S.stats)
        alsv.alsv_stats_read(S.ctx, S.stats, mean_dev, var_dev)
        with torch.cuda.stream(S.stream):
            mean_host.copy_(mean_dev, non_blocking=True)
            var_host.copy_(var_dev, non_blocking=True)
        S.stream.synchronize()
        _, nstep = S.time()
        cu_e2e += int(nstep.sum()) * N * N
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    e2e_cu = torch.tensor([float(cu_e2e)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e2e_cu, op=dist.ReduceOp.SUM)
    e2e = {"value": float(e2e_cu.item()) / float(e2e_t.item()), "unit": "cell-updates/s",
           "h2d_bytes_per_step": Mr * 20 * 8, "d2h_bytes_per_step": 2 * 4 * N * N * 8,
           "samples_per_s": world * Mr * args.steps / float(e2e_t.item())}

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        stage_bytes = cell_updates * BYTES_PER_CELL_UPDATE
        achieved = stage_bytes / (prof["stage_ms"] / 1000.0) / 1e9 if prof["stage_ms"] > 0 else None
        traffic, traffic_pcu = stage_traffic(chosen, cell_updates, prof["stage_launches"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (achieved / peaks["hbm_gbs"]) if achieved else None, "peak_kind": peak_kind,
                "kernel": STAGE_KERNEL_NAMES.get(chosen, str(chosen)),
                "algorithmic_bytes_per_cell_update": BYTES_PER_CELL_UPDATE,
                "stage_ms_total": prof["stage_ms"], "stage_launches": prof["stage_launches"],
                "stage_share_of_step": prof["stage_ms"] / ms if ms > 0 else None,
                "traffic": traffic, "traffic_bytes_per_cell_update": traffic_pcu,
                "traffic_source": "profiles/stage_traffic.txt (the 256-sample capture of this schedule's kernel, "
                                  "per cell-update, scaled to this run's cell-updates per stage launch)"}
        line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "fp32 (stencil); fp64 (statistics, totals, time)",
                "data": "synthetic (seeded KH perturbation parameters, SplitMix64)",
                "config": {"workload": WORKLOAD if (Mr == M and T_END == 1.0) else f"kh2d_256x256_mc{Mr}_weno3_hllc_ssprk3_fp32_T{T_END:g}",
                           "grid": [N, N], "samples_per_gpu": Mr, "T": T_END, "cfl": 0.4,
                           "scheme": "WENO3 (primitive) + HLLC + SSP-RK3", "parallelism": f"samples sharded x{world} (rank-ordered statistics merge)",
                           "l2": "inputs larger than L2 (4.3 GB state), no flush",
                           "tile_variant": chosen, "autotune_ms": ms_var},
                "samples_per_s": samples_per_s, "gpu_launches": launches, "e2e": e2e, "roofline": roof,
                "clocks": ck}
        ipcs = getattr(stage_traffic, "inst_per_cell_stage", None) if traffic is not None else None
        if achieved and ipcs:
            # issue-slot roofline: the profiled thread instructions per cell-stage at this run's
            # cell-stage rate against one warp instruction per cycle per SM sub-partition
            cell_stages = 3 * cell_updates
            warp_inst_rate = cell_stages * ipcs / 32.0 / (prof["stage_ms"] / 1000.0) / 1e9
            issue_peak = 152 * 4 * ISSUE_CLOCK_GHZ
            line["issue_roofline"] = {"bound": "issue", "achieved": warp_inst_rate, "peak": issue_peak,
                                      "unit": "G warp-instructions/s", "frac": warp_inst_rate / issue_peak,
                                      "thread_inst_per_cell_stage": ipcs,
                                      "peak_kind": "nominal: 152 SMs x 4 schedulers x 1 instruction/cycle x 2.07 GHz",
                                      "hbm_frac_at_full_issue": roof["frac"] / (warp_inst_rate / issue_peak)}
        if achieved:
            # the same stage time against the FP32 ALU: algorithmic flops per cell-update
            tflops = cell_updates * FLOPS_PER_CELL_UPDATE_2D_WENO3_HLLC_RK3 / (prof["stage_ms"] / 1000.0) / 1e12
            line["alu_roofline"] = {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                    "frac": tflops / FP32_PEAK_TFLOPS,
                                    "flops_per_cell_update": FLOPS_PER_CELL_UPDATE_2D_WENO3_HLLC_RK3,
                                    "peak_kind": "nominal: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
        steps0 = float(nstep[0]) if len(nstep) else 1.0
        line["plain_fp64"], u32, u64 = plain_fp64_loop(alsv, torch, steps0, chosen)
        line["batched_vs_plain_fp64_samples_per_s"] = samples_per_s / line["plain_fp64"]["samples_per_s"]
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = {k: v for k, v in cpu_baseline_oracle().items() if k not in ("elapsed_s", "cell_updates")}
            line["error_vs_oracle"] = errors_vs_oracle(u32, u64)
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        dist.barrier()       # rank 0 may still be timing the CPU baseline: tear down together
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
