#!/usr/bin/env python3
"""Benchmark: voxels/s of the two gradient-domain steps solved to a 1e-6
relative residual on a 1024 x 1024 x 128 synthetic EM stack.

One step = anisotropic diffusion along z (beta = (1, 1, 10)) followed by the
per-slice screened Poisson solve (alpha = 0.01), each V(2,2)-cycled down to a
16 x 16 coarsest grid until ||b - A x|| / ||b|| <= 1e-6, on inputs resident
in HBM.  Every array (537 MB in float32) is larger than the 126 MB L2, so no
L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own stack (independent problems, no collective on the data path) and the
value is all ranks' voxels over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxels/s to 1e-6 rel. residual (plain vs mixed-prec+learned); % of HBM peak"
UNIT = "voxels/s"
NX, NY, NZ = 1024, 1024, 128
BETA = (1.0, 1.0, 10.0)
ALPHA = 0.01
TOL = 1e-6      # AD: max |d| vs the exact solution ~3e-4 at this tolerance
TOL_SP = 1e-7   # SP: alpha = 0.01 makes the slice-smooth error ~100x the residual;
                # 1e-7 keeps max |d| <= 1e-3 (at 1e-6 it is ~1e-2)
SEED = 2
WORKLOAD = "gd_ad_then_sp_1024x1024x128"
# NPR filter workload (Sec. 7's video example)
NPR_NX, NPR_NY, NPR_NZ = 1920, 1080, 742
NPR_W = (0.001, 1.0, 1.0, 0.1)   # alpha, W = Diag(1, 1, 0.1)
NPR_LAMBDA, NPR_SIGMA = 1.25, 5.0
NPR_TOL = 1e-8
# batched screened Poisson on independent slices of different sizes
BATCH_N, BATCH_LO, BATCH_HI = 512, 256, 4096
BATCH_TOL = 1e-7

# DRAM traffic of the dominant kernel class from one ncu capture: the ratio of
# dram__bytes_read.sum + dram__bytes_write.sum to the algorithmic bytes over the
# four fine-level sweeps of one AD V-cycle (zero start, plain, prolongation,
# plain) of the 1024 x 1024 x 64 case (bench.py --ncu-case; 268 MB arrays, twice
# the L2); the traffic of a full-size launch is that ratio times its algorithmic
# bytes.  Valid only while the kernel source is the one it was taken from.
NCU_TRAFFIC = {
    "rb_sweep_fine": {"dram_over_alg": 3158.1 / 3087.0, "src_sha256": "4c47b9570ba99876172827ff38f5def62927c51d8c361ec50dd4bd8983b5067c"},
}


def kernel_src_sha() -> str:
    p = os.path.join(ROOT, "paper_1310_0041_gb300", "csrc", "gd_zmarch.cu")
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a scalar over ranks (identity when world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        # the timed region starts once the sampler is producing rows
        t0 = time.perf_counter()
        while not self.rows and time.perf_counter() - t0 < 3.0:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th is not None:
            self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample_step(I0c: np.ndarray) -> tuple:
    """AD then SP with the oracle's V-cycle (red-black Gauss-Seidel, OpenMP),
    each to 1e-6, on a crop of the workload; returns (seconds, voxels)."""
    import oracle
    t0 = time.perf_counter()
    I1, _ = oracle.ad_solve(I0c, BETA[0], BETA[1], BETA[2], method="mg", tol=TOL, max_cycles=400)
    oracle.sp_solve(I0c, I1, ALPHA, method="mg", tol=TOL_SP, max_cycles=400)
    return time.perf_counter() - t0, I0c.size


def oracle_crop():
    import gdsynth
    # 256 x 256 x 32 window of the 1024 x 1024 x 128 stack, solved as its own problem
    return gdsynth.em_stack(NX, NY, NZ, seed=SEED, ncells=2000,
                            window=(384, 512, 48, 256, 256, 32)).astype(np.float64)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    I0c = oracle_crop()
    for _ in range(args.warmup):
        oracle_sample_step(I0c)
    times = []
    for _ in range(args.steps):
        t, vox = oracle_sample_step(I0c)
        times.append(t)
    sec = sum(times) / len(times)
    value = I0c.size / sec
    sample = "AD (to 1e-6) + SP (to 1e-7) with the FP64 oracle V-cycle on a 256x256x32 crop of the stack"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nz": NZ, "beta": BETA,
                   "alpha": ALPHA, "rel_tol": TOL, "rel_tol_sp": TOL_SP, "sample": "256x256x32 crop"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_bounded() -> dict:
    """The oracle timed once on the bounded sample (about 10-30 s of CPU work)
    on all host cores, then one run of the sample on a single thread."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        res = pool.apply(_cpu_baseline_child)
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"  # read by the spawned child's OpenMP runtime
    try:
        with ctx.Pool(1) as pool:
            t1, v1, thr = pool.apply(_cpu_single_thread_child)
    finally:
        if old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = old
    res["single_thread"] = {"value": v1 / t1, "unit": UNIT, "seconds": t1, "threads": thr,
                            "sample": "one run of the same sample"}
    return res


def _cpu_single_thread_child():
    import oracle
    t, v = oracle_sample_step(oracle_crop())
    return t, v, oracle.threads()


def _cpu_baseline_child():
    import oracle
    I0c = oracle_crop()
    # repeat the sample until about 10 s of wall time (at most 30 s)
    total, vox, runs = 0.0, 0, 0
    while total < 10.0 and runs < 64:
        t, v = oracle_sample_step(I0c)
        total += t
        vox += v
        runs += 1
        if total + t > 30.0:
            break
    return {"value": vox / total, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "AD (to 1e-6) + SP (to 1e-7) with the FP64 oracle V-cycle (red-black GS, "
                      "OpenMP) on a 256x256x32 crop of the 1024x1024x128 stack, %d runs (%.1f s)"
                      % (runs, total)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    world, rank, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import gdsynth
    import paper_1310_0041_gb300 as gd
    gd.build()

    # the oracle baseline runs first in a spawned process (before heavy GPU work)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base = cpu_baseline_bounded()

    dev = torch.device("cuda", torch.cuda.current_device())
    I0h = gdsynth.em_stack(NX, NY, NZ, seed=SEED + rank, ncells=2000)
    I0 = torch.from_numpy(I0h).to(dev).float()
    I1 = torch.empty_like(I0)
    I2 = torch.empty_like(I0)
    stream = torch.cuda.current_stream()
    s = gd.gd_stack_create(NX, NY, NZ, stream=stream.cuda_stream)
    ctl = gd.solve_ctl(40, TOL, 2, 2, 16)
    ctl_sp = gd.solve_ctl(40, TOL_SP, 2, 2, 16)
    w_ad = (0.0, BETA[0], BETA[1], BETA[2])
    reps = []

    def step():
        r1 = gd.gd_diffuse_z(s, I0, I1, w_ad, ctl)
        r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, ALPHA, ctl_sp)
        reps.append((r1, r2))

    for _ in range(max(args.warmup, 0)):
        step()
    reps.clear()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local if world > 1 else 0)
    clocks.start()
    launches0 = gd.gd_launch_count(s)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    launches = gd.gd_launch_count(s) - launches0
    # per-kernel durations: the same K steps again with a CUDA event pair
    # around every launch (event nodes in the captured V-cycles); the events
    # stretch the step, so this pass gives the kernel figures, not the value
    reps.clear()
    gd.gd_profile_reset(s)
    gd.gd_profile_enable(s, True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    gd.gd_profile_enable(s, False)
    prof = gd.gd_profile_all(s)
    clk = clocks.stop()
    ms_max = reduce_max(ms_local, world, dev)
    voxels = NX * NY * NZ
    value = world * voxels * args.steps / (ms_max * 1e-3)

    # the mixed-precision mode (bfloat16 levels, float32 arithmetic, the same
    # float-pair refinement and tolerances), timed the same way
    sm = gd.gd_stack_create(NX, NY, NZ, prec=gd.GD_PREC_MIXED, stream=stream.cuda_stream)
    mreps = []

    def mstep():
        r1 = gd.gd_diffuse_z(sm, I0, I1, w_ad, ctl)
        r2 = gd.gd_screened_poisson_slices(sm, I0, I1, I2, ALPHA, ctl_sp)
        mreps.append((r1, r2))

    for _ in range(max(args.warmup, 1)):
        mstep()
    mreps.clear()
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        mstep()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    mms = reduce_max(e0.elapsed_time(e1), world, dev)
    gd.gd_destroy(sm)
    m1, m2 = mreps[-1]
    mixed = {"value": world * voxels * args.steps / (mms * 1e-3), "unit": UNIT,
             "ms_per_step": mms / args.steps,
             "storage": "bfloat16 levels between the fine and the coarsest, float32 arithmetic, "
                        "float-pair outer refinement",
             "ad_cycles": m1["cycles"], "ad_rel_residual": m1["rel_residual"],
             "sp_cycles": m2["cycles"], "sp_rel_residual": m2["rel_residual"]}

    # The NPR gradient filter of Sec. 7 on a video-sized synthetic stack (the
    # paper's 1920 x 1080 x 742 example; moving Voronoi cells stand in for
    # the video): filtered right-hand side, then the general screened Poisson
    # solve to 1e-8 (alpha = 0.001 magnifies smooth error ~1000x), timed
    # like the main workload.
    npr = None
    if not args.no_npr:
        V0 = torch.from_numpy(gdsynth.em_stack(NPR_NX, NPR_NY, NPR_NZ, seed=SEED + 100 + rank,
                                               ncells=NPR_NX * NPR_NY // 524)).to(dev).float()
        Vb = torch.empty_like(V0)
        Vx = torch.empty_like(V0)
        sn = gd.gd_stack_create(NPR_NX, NPR_NY, NPR_NZ, stream=stream.cuda_stream)
        ctl_npr = gd.solve_ctl(40, NPR_TOL, 2, 2, 16)
        nreps = []

        def nstep():
            gd.gd_npr_rhs(sn, V0, Vb, NPR_W, NPR_LAMBDA, NPR_SIGMA)
            nreps.append(gd.gd_screened_poisson(sn, NPR_W, Vb, Vx, ctl_npr, x0=V0))

        for _ in range(max(1, min(args.warmup, 2))):
            nstep()
        nreps.clear()
        nsteps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(nsteps):
            nstep()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        nms = reduce_max(e0.elapsed_time(e1), world, dev)
        gd.gd_destroy(sn)
        rn = nreps[-1]
        nvox = NPR_NX * NPR_NY * NPR_NZ
        npr = {"workload": "npr_filter_%dx%dx%d" % (NPR_NX, NPR_NY, NPR_NZ),
               "value": world * nvox * nsteps / (nms * 1e-3), "unit": UNIT,
               "ms_per_step": nms / nsteps, "steps": nsteps,
               "params": {"alpha": NPR_W[0], "W": list(NPR_W[1:]), "lambda": NPR_LAMBDA,
                          "sigma": NPR_SIGMA, "rel_tol": NPR_TOL, "x0": "I0"},
               "cycles": rn["cycles"], "rel_residual": rn["rel_residual"], "levels": rn["levels"]}
        del V0, Vb, Vx
        torch.cuda.empty_cache()

    # The Hybrid discretisation (Sec. 4.2: 6-point fine operator, first-order
    # B-spline transfers, Galerkin 27-point coarse operators) on the same
    # stack and tolerances.
    def profiled_step(stk, fn):
        """Kernel-class times (ms) of one more step with a CUDA event pair
        around every launch (not part of any timed value)."""
        gd.gd_profile_reset(stk)
        gd.gd_profile_enable(stk, True)
        fn()
        torch.cuda.synchronize()
        gd.gd_profile_enable(stk, False)
        return {name: round(ms, 3) for name, n, ms, _ in gd.gd_profile_all(stk) if n > 0}

    hybrid = None
    if not args.no_hybrid:
        sh = gd.gd_stack_create(NX, NY, NZ, disc=gd.GD_DISC_HYBRID, stream=stream.cuda_stream)
        hreps = []

        # AD to 1e-7: the Hybrid hierarchy leaves a smoother residual, and at
        # 1e-6 max |d| against the exact solution is ~5e-3 (1e-3 needs 1e-7)
        ctl_h = gd.solve_ctl(40, TOL_SP, 2, 2, 16)

        def hstep():
            h1 = gd.gd_diffuse_z(sh, I0, I1, w_ad, ctl_h)
            h2 = gd.gd_screened_poisson_slices(sh, I0, I1, I2, ALPHA, ctl_sp)
            hreps.append((h1, h2))

        for _ in range(max(1, min(args.warmup, 2))):
            hstep()
        hreps.clear()
        hsteps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(hsteps):
            hstep()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        hms = reduce_max(e0.elapsed_time(e1), world, dev)
        h1, h2 = hreps[-1]
        hkern = profiled_step(sh, hstep)
        gd.gd_destroy(sh)
        hybrid = {"value": world * voxels * hsteps / (hms * 1e-3), "unit": UNIT,
                  "ms_per_step": hms / hsteps, "steps": hsteps,
                  "discretisation": "hybrid: 6-point fine, B-spline transfers, Galerkin 27-point coarse",
                  "rel_tol_ad": TOL_SP, "rel_tol_sp": TOL_SP,
                  "ad_cycles": h1["cycles"], "ad_rho_per_cycle": h1["rho_per_cycle"],
                  "ad_rel_residual": h1["rel_residual"], "sp_cycles": h2["cycles"],
                  "sp_rho_per_cycle": h2["rho_per_cycle"], "sp_rel_residual": h2["rel_residual"],
                  "constant_ad_rho_per_cycle": reps[-1][0]["rho_per_cycle"],
                  "constant_sp_rho_per_cycle": reps[-1][1]["rho_per_cycle"],
                  "kernel_ms_profiled_step": hkern}

    # The Linear discretisation (Sec. 4.2, trilinear finite elements: a
    # 27-point fine operator, FP64 residuals) on the same stack.
    linear = None
    if not args.no_hybrid:
        sl = gd.gd_stack_create(NX, NY, NZ, disc=gd.GD_DISC_LINEAR, stream=stream.cuda_stream)
        lreps = []

        def lstep():
            l1 = gd.gd_diffuse_z(sl, I0, I1, w_ad, ctl)
            l2 = gd.gd_screened_poisson_slices(sl, I0, I1, I2, ALPHA, ctl_sp)
            lreps.append((l1, l2))

        lstep()
        lreps.clear()
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        lstep()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        lms = reduce_max(e0.elapsed_time(e1), world, dev)
        l1, l2 = lreps[-1]
        lkern = profiled_step(sl, lstep)
        gd.gd_destroy(sl)
        linear = {"value": world * voxels / (lms * 1e-3), "unit": UNIT, "ms_per_step": lms, "steps": 1,
                  "discretisation": "linear: trilinear elements, 27-point fine operator",
                  "ad_cycles": l1["cycles"], "ad_rho_per_cycle": l1["rho_per_cycle"],
                  "ad_rel_residual": l1["rel_residual"], "sp_cycles": l2["cycles"],
                  "sp_rho_per_cycle": l2["rho_per_cycle"], "sp_rel_residual": l2["rel_residual"],
                  "kernel_ms_profiled_step": lkern}

    # Batched screened Poisson on 512 independent slices, square, sides
    # log-uniform in [256, 4096], alpha ~ U(0.001, 0.1) per slice; every
    # slice to 1e-7 relative residual, timed like the main workload.
    batch = None
    if not args.no_batch:
        bseed = SEED + 200 + rank
        sides = gdsynth.batch_sides(BATCH_N, BATCH_LO, BATCH_HI, seed=bseed)
        bal = gdsynth.batch_alphas(BATCH_N, seed=bseed)
        B0s, B1s = gdsynth.batch_slices(sides, sides, seed=bseed)
        BI0 = torch.from_numpy(gdsynth.pack(B0s)).to(dev)
        BI1 = torch.from_numpy(gdsynth.pack(B1s)).to(dev)
        del B0s, B1s
        BO = torch.empty_like(BI0)
        bh = gd.gd_batch_create(sides, sides, bal, stream=stream.cuda_stream)
        bchunk = gd.gd_batch_tune(bh)
        bctl = gd.solve_ctl(40, BATCH_TOL, 2, 2, 16)
        breps = []
        for _ in range(max(1, min(args.warmup, 2))):
            breps.append(gd.gd_batch_screened_poisson(bh, BI0, BI1, BO, bctl))
        breps.clear()
        bsteps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        barrier(world)
        bl0 = gd.gd_batch_launch_count(bh)
        e0.record(stream)
        for _ in range(bsteps):
            breps.append(gd.gd_batch_screened_poisson(bh, BI0, BI1, BO, bctl))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        bms = reduce_max(e0.elapsed_time(e1), world, dev)
        blaunch = gd.gd_batch_launch_count(bh) - bl0
        bvox = int(BI0.numel())
        rb_ = breps[-1]
        # the bytes each solve's passes actually move (slices at tolerance
        # leave the later cycles)
        alg = gd.gd_batch_last_traffic(bh)
        batch = {"workload": "sp_batch_%d_slices_%d_to_%d" % (BATCH_N, BATCH_LO, BATCH_HI),
                 "value": world * bvox * bsteps / (bms * 1e-3), "unit": UNIT,
                 "ms_per_step": bms / bsteps, "steps": bsteps, "voxels": bvox, "slices": BATCH_N,
                 "params": {"alpha": [0.001, 0.1], "rel_tol": BATCH_TOL, "x0": "I0",
                            "tolerance_per": "slice"},
                 "cycles": rb_["cycles"], "rel_residual_max": rb_["rel_residual"],
                 "levels": rb_["levels"], "gpu_launches": blaunch,
                 "alg_bytes_per_step": alg, "achieved_GBps": alg / (bms / bsteps * 1e-3) / 1e9}
        gd.gd_batch_destroy(bh)
        batch["rows_per_item"] = bchunk
        # the same slices solved one at a time with the stack solver (one
        # stack of nz = 1 per slice, its own plan and graph): per-slice launches
        stacks = [gd.gd_stack_create(n, n, 1, stream=stream.cuda_stream) for n in sides]
        offs = np.cumsum([0] + [n * n for n in sides])
        PO = torch.empty_like(BI0)
        views = [(BI0[offs[k]:offs[k + 1]], BI1[offs[k]:offs[k + 1]], PO[offs[k]:offs[k + 1]])
                 for k in range(BATCH_N)]
        prel = []

        def pstep():
            prel.clear()
            for k in range(BATCH_N):
                r_ = gd.gd_screened_poisson_slices(stacks[k], *views[k], bal[k], bctl)
                prel.append(r_["rel_residual"])

        pstep()
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        pstep()
        e1.record(stream)
        torch.cuda.synchronize()
        pms = reduce_max(e0.elapsed_time(e1), world, dev)
        for st_ in stacks:
            gd.gd_destroy(st_)
        batch["per_slice_launches"] = {
            "method": "one stack (nz = 1) per slice, gd_screened_poisson_slices each, same tolerance",
            "ms_per_step": pms, "value": world * bvox / (pms * 1e-3), "unit": UNIT,
            "rel_residual_max": max(prel), "batch_speedup": pms / (bms / bsteps)}
        del BI0, BI1, BO, PO, views
        torch.cuda.empty_cache()

    # The learned initial guess (the 2048 x 2048 x 512 workload): the
    # encoder-decoder is trained here on the GPU (untimed) on 20k
    # (256 x 256 x 16 tile, AD solution) pairs that the solver produces from
    # fresh stacks, then the plain FP32 method (zero start) is timed against
    # mixed precision with the learned start (network inference over the whole
    # stack + exact projection of its lowest xy modes), AD to 1e-6 and SP to
    # 1e-7 each, inference included in the timed region.
    # The mixed-precision workload (4096 x 4096 x 256, 4.3 G voxels): AD then
    # SP in the float32 and the mixed mode, timed like the main workload, with
    # the per-level effect of 16-bit storage measured on a 1024 x 1024 x 64
    # crop solved as its own problem.
    config3 = None
    if not args.no_config3:
        config3 = bench_config3(args, gd, gdsynth, torch, stream, world, dev, e0, e1)
        torch.cuda.empty_cache()

    learned = None
    if not args.no_learned:
        learned = bench_learned(args, gd, gdsynth, torch, stream, world, rank, dev, e0, e1)
        torch.cuda.empty_cache()

    # end to end through the C ABI with pinned host buffers, the one call a
    # user makes for the two steps (gd_ad_then_sp): H2D of I0 and D2H of I2
    # inside the timed region
    I0p = torch.from_numpy(I0h.astype(np.float32)).pin_memory()
    I2p = torch.empty(I0p.shape, dtype=torch.float32).pin_memory()
    for _ in range(1):
        gd.gd_ad_then_sp(s, I0p, I2p, w_ad, ALPHA, ctl, ctl_sp)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    esteps = max(1, min(args.steps, 10))  # host wall clock: average over several steps
    for _ in range(esteps):
        gd.gd_ad_then_sp(s, I0p, I2p, w_ad, ALPHA, ctl, ctl_sp)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
    e2e_value = world * voxels * esteps / e2e_s
    gd.gd_destroy(s)

    if rank == 0:
        peaks = measured_peaks()
        peak = peaks.get("hbm_gbs")
        peak_src = "measured" if peak else "fallback"
        if not peak:
            peak = 6800.0
        dom = max(prof, key=lambda q: q[2]) if prof else None
        roof = None
        if dom and dom[1] > 0 and dom[2] > 0:
            name, nl, ms, by = dom
            achieved = by / (ms * 1e-3) / 1e9
            tr = NCU_TRAFFIC.get(name)
            traffic = None
            if tr and tr.get("src_sha256") == kernel_src_sha():
                traffic = tr["dram_over_alg"] * (by / nl)
            roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                    "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "launches": nl, "avg_launch_ms": ms / nl,
                    "alg_bytes_per_launch": by / nl}
        if batch is not None:
            batch["frac_of_hbm"] = batch["achieved_GBps"] / peak
        r1, r2 = reps[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "nz": NZ, "beta": BETA,
                       "alpha": ALPHA, "rel_tol": TOL, "rel_tol_sp": TOL_SP, "cycle": "V(2,2)", "coarsest_xy": 16,
                       "precision": "fp32 kernels, float-pair fine iterate",
                       "l2": "inputs larger than L2 (537 MB per array), no flush",
                       "kernel_timing": "a second pass of the same steps with a CUDA event pair "
                                        "around every launch",
                       "parallelism": "replicas" if world > 1 else "single"},
            "solver": {"ad_cycles": r1["cycles"], "ad_rel_residual": r1["rel_residual"],
                       "ad_levels": r1["levels"], "sp_cycles": r2["cycles"],
                       "sp_rel_residual": r2["rel_residual"], "sp_levels": r2["levels"]},
            "roofline": roof,
            "kernels": [{"name": q[0], "launches": q[1], "ms": q[2], "alg_GBps":
                         (q[3] / (q[2] * 1e-3) / 1e9) if q[2] > 0 else None} for q in prof],
            "cpu_baseline": cpu_base,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": voxels * 4,
                    "d2h_bytes_per_step": voxels * 4, "call": "gd_ad_then_sp, pinned host arrays"},
            "gpu_launches": launches,
            "mixed": mixed,
            "npr": npr,
            "batch": batch,
            "hybrid": hybrid,
            "linear": linear,
            "learned": learned,
            "mixed_config3": config3,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def level_operator(info: dict) -> np.ndarray:
    """Dense FP64 matrix of a level's operator from gd_level_info:
    wx Kx(x)My(x)Mz + wy Mx(x)Ky(x)Mz + wz Mx(x)My(x)Kz + wm Mx(x)My(x)Mz, K the
    1D Neumann Laplacian, M = diag(children counts); x fastest (z outermost)."""
    def K(n):
        A = np.zeros((n, n))
        for i in range(n - 1):
            A[i, i] += 1
            A[i + 1, i + 1] += 1
            A[i, i + 1] -= 1
            A[i + 1, i] -= 1
        return A

    def M(n, s_, l_):
        d = np.full(n, float(s_))
        d[-1] = l_
        return np.diag(d)
    nx, ny, nz = info["dims"]
    Kx, Ky, Kz = K(nx), K(ny), K(nz)
    Mx, My, Mz = (M(n, s_, l_) for n, s_, l_ in zip((nx, ny, nz), info["s"], info["l"]))
    wx, wy, wz, wm = info["weights"]
    kr = lambda a, b, c: np.kron(a, np.kron(b, c))
    return wx * kr(Mz, My, Kx) + wy * kr(Mz, Ky, Mx) + wz * kr(Kz, My, Mx) + wm * kr(Mz, My, Mx)


def mixed_level_errors(gd, torch, I0, w, stream=None) -> dict:
    """What 16-bit storage does to each level: one AD V-cycle from the zero
    start (the same input) on a float32-storage stack and on a mixed stack;
    per level, max and RMS of the difference of the stored corrections
    relative to the float32 hierarchy's, both taken modulo the AD operator's
    null space (the constants: mass-weighted mean removed); and the coarsest
    solve (float32 fast diagonalisation on the device) against an FP64 dense
    solve of the same coarsest system on the host."""
    nz, ny, nx = I0.shape
    out = torch.empty_like(I0)
    levels = {}
    coarse = None
    for prec in (gd.GD_PREC_FP32, gd.GD_PREC_MIXED):
        s = gd.gd_stack_create(nx, ny, nz, prec=prec, stream=stream)
        try:
            gd.gd_diffuse_z(s, I0, out, w, gd.solve_ctl(1, 1e-30), raise_on_error=False)
            L = gd.gd_level_count(s)
            for lv in range(1, L):
                info = gd.gd_level_info(s, lv)
                buf = np.empty(int(np.prod(info["dims"])), np.float32)
                gd.gd_level_fetch(s, lv, 0, buf)
                levels.setdefault(lv, {})[prec] = (info, buf.astype(np.float64))
            if prec == gd.GD_PREC_FP32:
                info = gd.gd_level_info(s, L - 1)
                bL = np.empty(int(np.prod(info["dims"])), np.float32)
                gd.gd_level_fetch(s, L - 1, 1, bL)
                coarse = (info, bL.astype(np.float64), levels[L - 1][prec][1])
        finally:
            gd.gd_destroy(s)
    def masses(info):
        (nxl, nyl, nzl), s_, l_ = info["dims"], info["s"], info["l"]
        ax = [np.r_[[s_[d]] * (n - 1), l_[d]].astype(np.float64) for d, n in enumerate((nxl, nyl, nzl))]
        return np.kron(ax[2], np.kron(ax[1], ax[0]))

    def null_free(info, v):
        # the AD operator (no screening term) is singular: a level's correction
        # is defined up to a constant, which the fine level's mean fix removes
        if info["weights"][3] != 0.0:
            return v
        m = masses(info)
        return v - np.dot(m, v) / m.sum()

    rows = []
    for lv in sorted(levels):
        (i32, x32), (imx, xmx) = levels[lv][gd.GD_PREC_FP32], levels[lv][gd.GD_PREC_MIXED]
        x32, xmx = null_free(i32, x32), null_free(imx, xmx)
        d = xmx - x32
        scale = max(np.abs(x32).max(), 1e-30)
        rows.append({"level": lv, "dims": list(i32["dims"]), "storage": "bf16" if imx["bytes"] == 2 else "fp32",
                     "rel_max_diff": float(np.abs(d).max() / scale),
                     "rel_rms_diff": float(np.sqrt(np.mean(d * d)) / max(np.sqrt(np.mean(x32 * x32)), 1e-30))})
    info, bL, xL = coarse
    A = level_operator(info)
    xref = np.linalg.lstsq(A, bL, rcond=None)[0]
    m = masses(info)
    mf = lambda v: v - np.dot(m, v) / m.sum()
    e = mf(xL) - mf(xref)
    coarsest = {"dims": list(info["dims"]), "device": "fp32 fast diagonalisation",
                "rel_max_err_vs_fp64": float(np.abs(e).max() / max(np.abs(mf(xref)).max(), 1e-30)),
                "rel_residual_fp32_solve": float(np.linalg.norm(bL - A @ xL) / max(np.linalg.norm(bL), 1e-30))}
    return {"levels": rows, "coarsest": coarsest}


C3_NX, C3_NY, C3_NZ = 4096, 4096, 256


def bench_config3(args, gd, gdsynth, torch, stream, world, dev, e0, e1):
    gdsynth.build_cuda()
    nx, ny, nz = C3_NX, C3_NY, C3_NZ
    I0 = gdsynth.em_stack_cuda(nx, ny, nz, seed=SEED + 400).float()
    I1 = torch.empty_like(I0)
    I2 = torch.empty_like(I0)
    w_ad = (0.0, BETA[0], BETA[1], BETA[2])
    ctl = gd.solve_ctl(40, TOL, 2, 2, 16)
    ctl_sp = gd.solve_ctl(40, TOL_SP, 2, 2, 16)
    nsteps = max(1, min(args.steps, 2))
    out = {"workload": "mixed_precision_%dx%dx%d" % (nx, ny, nz), "steps": nsteps}
    for name, prec in (("fp32", gd.GD_PREC_FP32), ("mixed", gd.GD_PREC_MIXED)):
        s = gd.gd_stack_create(nx, ny, nz, prec=prec, stream=stream.cuda_stream)
        reps = []

        def one():
            r1 = gd.gd_diffuse_z(s, I0, I1, w_ad, ctl)
            r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, ALPHA, ctl_sp)
            reps.append((r1, r2))

        one()
        reps.clear()
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(nsteps):
            one()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = reduce_max(e0.elapsed_time(e1), world, dev) / nsteps
        gd.gd_destroy(s)
        r1, r2 = reps[-1]
        out[name] = {"value": world * nx * ny * nz / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "ad_cycles": r1["cycles"], "ad_rel_residual": r1["rel_residual"],
                     "sp_cycles": r2["cycles"], "sp_rel_residual": r2["rel_residual"]}
    out["mixed_speedup"] = out["fp32"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    del I0, I1, I2
    torch.cuda.empty_cache()
    crop = gdsynth.em_stack_cuda(nx, ny, nz, seed=SEED + 400, window=(1536, 1024, 96, 1024, 1024, 64)).float()
    out["per_level"] = mixed_level_errors(gd, torch, crop, w_ad, stream=stream.cuda_stream)
    out["per_level"]["measured_on"] = "one AD V-cycle on a 1024x1024x64 crop solved as its own problem"
    return out


LEARN_NX, LEARN_NY, LEARN_NZ = 2048, 2048, 512
LEARN_LOWMODES = 4


def bench_learned(args, gd, gdsynth, torch, stream, world, rank, dev, e0, e1):
    from paper_1310_0041_gb300 import guess, learn
    gdsynth.build_cuda()
    t0 = time.perf_counter()
    net = learn.gd_learn_create(16, 16, (16, 32, 64, 128), 256, 256, 32, seed=1,
                                stream=stream.cuda_stream)
    tr = guess.train_on_solver_pairs(
        net, lambda sd: gdsynth.em_stack_cuda(1024, 1024, 128, seed=sd), args.learned_pairs,
        passes=4, lr=2e-3, seed0=100000 + 1000 * rank)
    train_s = time.perf_counter() - t0
    nx, ny, nz = LEARN_NX, LEARN_NY, LEARN_NZ
    I0 = gdsynth.em_stack_cuda(nx, ny, nz, seed=SEED + 300 + rank).float()
    I1 = torch.empty_like(I0)
    I2 = torch.empty_like(I0)
    x0 = torch.empty_like(I0)
    w_ad = (0.0, BETA[0], BETA[1], BETA[2])
    ctl = gd.solve_ctl(40, TOL, 2, 2, 16)
    ctl_sp = gd.solve_ctl(40, TOL_SP, 2, 2, 16)
    nsteps = max(1, min(args.steps, 2))
    out = {}
    for mode, prec, use_net in (("plain_fp32", gd.GD_PREC_FP32, False),
                                ("mixed", gd.GD_PREC_MIXED, False),
                                ("mixed_learned", gd.GD_PREC_MIXED, True)):
        s = gd.gd_stack_create(nx, ny, nz, prec=prec, stream=stream.cuda_stream)
        reps = []
        parts = {"network_ms": 0.0, "lowmodes_ms": 0.0}
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

        def one(timed_parts):
            xs = None
            if use_net:
                ev[0].record(stream)
                guess.learned_start(net, I0, x0)
                ev[1].record(stream)
                learn.gd_learn_lowmodes(net, I0, x0, nx, ny, nz, w_ad, LEARN_LOWMODES)
                ev[2].record(stream)
                xs = x0
            r1 = gd.gd_diffuse_z(s, I0, I1, w_ad, ctl, x0=xs)
            r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, ALPHA, ctl_sp)
            reps.append((r1, r2))
            if use_net and timed_parts:
                torch.cuda.synchronize()
                parts["network_ms"] += ev[0].elapsed_time(ev[1])
                parts["lowmodes_ms"] += ev[1].elapsed_time(ev[2])

        one(False)
        reps.clear()
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(nsteps):
            one(False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = reduce_max(e0.elapsed_time(e1), world, dev) / nsteps
        if use_net:  # a separate pass for the split (the events synchronise)
            one(True)
        gd.gd_destroy(s)
        r1, r2 = reps[-1]
        out[mode] = {"value": world * nx * ny * nz / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "ad_cycles": r1["cycles"], "ad_rel_residual": r1["rel_residual"],
                     "ad_history": r1["history"], "sp_cycles": r2["cycles"],
                     "sp_rel_residual": r2["rel_residual"]}
        if use_net:
            out[mode]["network_ms"] = parts["network_ms"]
            out[mode]["lowmodes_ms"] = parts["lowmodes_ms"]
    launches = learn.gd_learn_launch_count(net)
    learn.gd_learn_destroy(net)
    del I0, I1, I2, x0
    p, m = out["plain_fp32"], out["mixed_learned"]
    return {"workload": "learned_guess_%dx%dx%d" % (nx, ny, nz), "steps": nsteps,
            "network": "3x3 encoder-decoder 16-32-64-128, bf16 tcgen05 convolutions, fp32 accumulation, "
                       "256x256x16 tiles (slices as channels), predicts I1 - I0",
            "start": "x0 = I0 + net(I0), then its %dx%d lowest xy cosine modes per slice replaced by the "
                     "exact AD solution's (gd_learn_lowmodes)" % (LEARN_LOWMODES, LEARN_LOWMODES),
            "training": {"pairs": tr["pairs"], "stacks": tr["stacks"], "steps": tr["steps"],
                         "stack": "1024x1024x128", "seconds": train_s,
                         "loss_first": float(np.mean(tr["losses"][:20])),
                         "loss_last": float(np.mean(tr["losses"][-20:]))},
            "plain_fp32": p, "mixed": out["mixed"], "mixed_learned": m,
            "ad_cycles_saved": p["ad_cycles"] - m["ad_cycles"],
            "speedup_vs_plain": p["ms_per_step"] / m["ms_per_step"],
            "network_launches": launches}


def run_ncu_case(args):
    """A small case for detailed ncu captures (not a benchmark): one AD
    V-cycle on a 1024 x 1024 x 64 stack (arrays of 268 MB, twice the L2;
    about 4 GB on the device), or 1024 x 512 x 64 with --ncu-case-ny 512."""
    import torch
    import gdsynth
    import paper_1310_0041_gb300 as gd
    gd.build()
    nx, ny, nz = 1024, args.ncu_case_ny, 64
    I0 = torch.from_numpy(gdsynth.em_stack(nx, ny, nz, seed=SEED, ncells=nx * ny // 524)).cuda().float()
    I1 = torch.empty_like(I0)
    s = gd.gd_stack_create(nx, ny, nz)
    rep = gd.gd_diffuse_z(s, I0, I1, (0.0,) + BETA, gd.solve_ctl(1, TOL), raise_on_error=False)
    gd.gd_destroy(s)
    print(json.dumps({"ncu_case": "ad_%dx%dx%d_one_vcycle" % (nx, ny, nz), "status": rep["status"],
                      "cycles": rep["cycles"]}))
    return 0 if rep["status"] in (0, 5) else 1


def run_ncu_linear(args):
    """One AD + SP step of the Linear discretisation on the 1024 x 1024 x 128
    benchmark stack after one warm-up step (for ncu launch lists; not a
    benchmark); 1024 x 512 x 64 with --ncu-linear-small (about 3 GB on the
    device, for multi-pass captures)."""
    import torch
    import gdsynth
    import paper_1310_0041_gb300 as gd
    gd.build()
    nx, ny, nz = (NX, NY // 2, NZ // 2) if args.ncu_linear_small else (NX, NY, NZ)
    I0 = torch.from_numpy(gdsynth.em_stack(nx, ny, nz, seed=SEED, ncells=2000)).cuda().float()
    I1 = torch.empty_like(I0)
    I2 = torch.empty_like(I0)
    s = gd.gd_stack_create(nx, ny, nz, disc=gd.GD_DISC_LINEAR)
    ctl = gd.solve_ctl(30, TOL, 2, 2, 16)
    ctl_sp = gd.solve_ctl(30, TOL_SP, 2, 2, 16)
    for _ in range(2):
        r1 = gd.gd_diffuse_z(s, I0, I1, (0.0,) + BETA, ctl)
        r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, ALPHA, ctl_sp)
    torch.cuda.synchronize()
    gd.gd_destroy(s)
    print(json.dumps({"ncu_linear": "linear_ad_sp_%dx%dx%d" % (nx, ny, nz), "ad_cycles": r1["cycles"],
                      "sp_cycles": r2["cycles"]}))
    return 0 if r1["status"] == 0 and r2["status"] == 0 else 1


def run_ncu_conv(args):
    """The learned guess's forward pass on 32 tiles of 256 x 256 x 16, four
    times (for ncu captures of the convolution kernels; not a benchmark):
    each forward launches e1, pool, e2, pool, e3, pool, e4, d3, d2, d1, y."""
    import torch
    import paper_1310_0041_gb300 as gd
    from paper_1310_0041_gb300 import learn
    gd.build()
    B = 32
    net = learn.gd_learn_create(16, 16, (16, 32, 64, 128), 256, 256, B, seed=0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn((B, 256, 256, 16), device="cuda", generator=g).to(torch.bfloat16)
    yf = torch.empty((B, 256, 256, 16), device="cuda")
    for _ in range(4):
        learn.gd_learn_forward(net, x, B, yf)
    torch.cuda.synchronize()
    learn.gd_learn_destroy(net)
    print(json.dumps({"ncu_conv": "forward_32x256x256x16", "forwards": 4}))
    return 0


def run_ncu_batch(args):
    """One batched solve of the batch workload (for ncu captures; not a
    benchmark): sides log-uniform in [256, 4096], to 1e-7 per slice; 512
    slices unless --ncu-batch-slices says otherwise."""
    import torch
    import gdsynth
    import paper_1310_0041_gb300 as gd
    gd.build()
    bseed = SEED + 200
    nsl = args.ncu_batch_slices
    sides = gdsynth.batch_sides(nsl, BATCH_LO, BATCH_HI, seed=bseed)
    bal = gdsynth.batch_alphas(nsl, seed=bseed)
    B0s, B1s = gdsynth.batch_slices(sides, sides, seed=bseed)
    BI0 = torch.from_numpy(gdsynth.pack(B0s)).cuda()
    BI1 = torch.from_numpy(gdsynth.pack(B1s)).cuda()
    del B0s, B1s
    BO = torch.empty_like(BI0)
    bh = gd.gd_batch_create(sides, sides, bal)
    rep = gd.gd_batch_screened_poisson(bh, BI0, BI1, BO, gd.solve_ctl(40, BATCH_TOL, 2, 2, 16),
                                       raise_on_error=False)
    torch.cuda.synchronize()
    gd.gd_batch_destroy(bh)
    print(json.dumps({"ncu_batch": "sp_batch_%d_slices" % nsl, "status": rep["status"],
                      "cycles": rep["cycles"], "voxels": int(BI0.numel())}))
    return 0 if rep["status"] == 0 else 1


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-npr", action="store_true", help="skip the NPR filter measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-slices measurement")
    ap.add_argument("--no-hybrid", action="store_true",
                    help="skip the Hybrid and Linear discretisation measurements")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 4096x4096x256 float32 / mixed-precision measurement")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-initial-guess measurement (training + 2048x2048x512)")
    ap.add_argument("--learned-pairs", type=int, default=20000,
                    help="training pairs of the learned initial guess")
    ap.add_argument("--ncu-batch", action="store_true",
                    help="one solve of the 512-slice batch for ncu launch lists (no timing)")
    ap.add_argument("--ncu-batch-slices", type=int, default=BATCH_N,
                    help="slices of the --ncu-batch case (fewer for detailed captures)")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run the small profiling case instead of the benchmark")
    ap.add_argument("--ncu-linear", action="store_true",
                    help="one Linear AD + SP step on the benchmark stack after a warm-up (for ncu; not a benchmark)")
    ap.add_argument("--ncu-linear-small", action="store_true",
                    help="--ncu-linear on a 1024 x 512 x 64 stack")
    ap.add_argument("--ncu-case-ny", type=int, default=1024,
                    help="y extent of the --ncu-case stack (1024 x ny x 64)")
    ap.add_argument("--ncu-conv", action="store_true",
                    help="four forward passes of the learned guess's network, for ncu")
    args = ap.parse_args(argv)
    if args.ncu_case:
        return run_ncu_case(args)
    if args.ncu_linear or args.ncu_linear_small:
        return run_ncu_linear(args)
    if args.ncu_conv:
        return run_ncu_conv(args)
    if args.ncu_batch:
        return run_ncu_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
