"""Benchmark of the fused fluctuating central-moment LBM step on GB300.

Workload (one "step" = one lattice update of every site, the whole hot path, with the
statistics reduction on every `stats_every`-th step): D3Q27 256^3 periodic box, FP32
deviations in one AA-pattern array (1.81 GB, far above the 129 MB L2, so no flush is
needed between steps), rho0 = 1 with a seeded 1e-3 uniform density perturbation, drift
u0 = (0.05, 0.02, 0), kBT = 1e-4, shear rate omega = 1.6 (Lambda_7-9), all other modes 1.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). N > 1 runs N independent replicas (one lattice per
GPU, weak scaling, no data exchange) launched by torch.distributed.run. At N = 1 the
line also carries the same workload with BF16 and FP16 deviation storage
("storage_widths"), on the isotropic D3Q27 variant and D3Q19 ("other_lattices"), at
k_BT = 0 ("noise_off": the cost of the noise) and the 256-lattice batched ensemble
("batched_ensemble").
`--impl reference` times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fluctuating D3Q27 GLUPS and fraction of HBM roofline at stated oracle error"
UNIT = "GLUPS"
DIMS = (256, 256, 256)  # overridable with --dims for profiling runs on smaller boxes
STATS_RECORD_BYTES = (32 * 33 // 2 + 1) * 8  # one D3Q27 statistics record on the device
KBT = 1e-4
OMEGA = 1.6
U0 = (0.05, 0.02, 0.0)
AMP = 1e-3
SEED = 0
BYTES_PER_SITE = 27 * 4 * 2  # read + write of 27 FP32 populations (noise is generated, not stored)


def lam_d3q27(omega=OMEGA):
    lam = np.ones(27)
    lam[[7, 8, 9]] = omega
    return lam


def workload_config(stats_every, world, dims=DIMS):
    return {
        "workload": "D3Q27 256^3 periodic fluctuating central-moment LBM, FP32 AA-pattern, "
                    "rho0=1 +1e-3 seeded perturbation, drift (0.05,0.02,0), kBT=1e-4, shear omega=1.6",
        "lattice": "D3Q27",
        "dims": list(dims),
        "storage": "fp32 deviations f_i - w_i rho0, one in-place AA array",
        "kBT": KBT,
        "omega_shear": OMEGA,
        "u0": list(U0),
        "rho_perturb": AMP,
        "stats_every": stats_every,
        "l2": "inputs larger than L2 (1.81 GB state vs 129 MB L2); no flush",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
    }


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Sources the single-lattice step kernels are compiled from (a change to any of them
# invalidates recorded DRAM counters).
STEP_SOURCES = ("step.cu", "step_kernels.cuh", "step_pipe.cu", "async.cuh", "cm.cuh", "collide.cuh", "philox.cuh",
                "lattice.cuh", "vec.cuh", "internal.h")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_16486_gb300", "csrc")
    for name in STEP_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per step-kernel launch from an ncu capture, if it was taken on the
    current kernel sources (profiles/step_traffic.json), else None."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    if rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("bytes_per_launch_256cube")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.seek(0)
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
                "samples": len(sms)}


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks (the job's time is the slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_glups(world, sites_per_rank, steps, elapsed_s):
    """Whole-job throughput: every rank's site updates over the slowest rank's time."""
    return world * sites_per_rank * steps / elapsed_s / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_ours(args):
    import torch

    import paper_2602_16486_gb300 as fl

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    dims = tuple(args.dims)
    sites = dims[0] * dims[1] * dims[2]
    S = args.stats_every

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    lat = fl.Lattice(fl.FLBM_D3Q27, dims, lam_d3q27(), KBT, 1.0, SEED + rank, fl.FLBM_FP32,
                     cuda_stream=stream.cuda_stream)
    fl.flbm_set_sample_capacity(lat.ctx, max(1, (args.steps + args.warmup) // S + 2))
    lat.init_uniform(U0, AMP, SEED + rank)
    if args.variant:
        lat.variant = args.variant
        variant = lat.variant
    else:
        variant = lat.autotune(10)  # launch configuration only; runs on a copy of the state

    def one_step(k):
        lat.step(1)
        if k % S == 0:
            lat.sample()

    for k in range(args.warmup):
        one_step(k)
    lat.fetch_samples()
    stream.synchronize()

    # ---- device-timed region: K steps, inputs resident in HBM ---------------------------
    ev_k = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(dev)).split(",")[dev if world == 1 else local]
    barrier()
    torch.cuda.synchronize()
    launches = 0
    with ClockSampler(gpu_index) as clocks:
        t0.record(stream)
        for k in range(args.steps):
            ev_k[k][0].record(stream)
            lat.step(1)
            ev_k[k][1].record(stream)
            launches += 1
            if k % S == 0:
                lat.sample()
                launches += 1
        t1.record(stream)
        torch.cuda.synchronize()
    barrier()
    elapsed_ms = t0.elapsed_time(t1)
    step_kernel_ms = [a.elapsed_time(b) for a, b in ev_k]
    samples = lat.fetch_samples()
    nonfinite = sum(s["nonfinite"] for s in samples)
    elapsed_ms = max_over_ranks(elapsed_ms, world, "cuda")

    # ---- end to end through the C ABI with host buffers ---------------------------------
    if args.no_e2e:
        lat.close()
        if rank != 0:
            return None
        return {"metric": METRIC, "value": sites * args.steps / (elapsed_ms * 1e-3) / 1e9, "unit": UNIT,
                "dims": list(dims), "avg_step_kernel_ms": float(np.mean(step_kernel_ms)),
                "note": "profiling run (--no-e2e): not a bench line"}
    nbytes = fl.flbm_checkpoint_bytes(lat.ctx)
    host_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    host_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    fl.flbm_save(lat.ctx, host_in.data_ptr(), nbytes)
    n_e2e = args.steps
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    fl.flbm_load(lat.ctx, host_ptr=host_in.data_ptr(), nbytes=nbytes)
    for k in range(n_e2e):
        lat.step(1)
        if k % S == 0:
            lat.sample()
    e2e_samples = lat.fetch_samples()  # every sample's record to the host
    stats_bytes = len(e2e_samples) * STATS_RECORD_BYTES
    fl.flbm_save(lat.ctx, host_out.data_ptr(), nbytes)
    e2e_s = time.perf_counter() - w0
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    lat.close()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return None

    value = job_glups(world, sites, args.steps, elapsed_ms * 1e-3)
    avg_kernel_ms = float(np.mean(step_kernel_ms))
    peaks, peak_kind = measured_peaks()
    achieved = BYTES_PER_SITE * sites / (avg_kernel_ms * 1e-3) / 1e9
    roof = {
        "bound": "hbm",
        "achieved": round(achieved, 1),
        "peak": peaks["hbm_gbs"],
        "unit": "GB/s",
        "frac": round(achieved / peaks["hbm_gbs"], 4),
        "traffic": recorded_traffic(),
        "kernel": f"fused collide + AA stream, D3Q27 fp32 (step variant {variant})",
        "peak_kind": f"{peak_kind} STREAM-style copy (hbm_gbs)",
        "algorithmic_bytes_per_launch": BYTES_PER_SITE * sites,
        "avg_launch_ms": round(avg_kernel_ms, 5),
    }
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded lattice state, no dataset)",
        "config": dict(workload_config(S, world, dims), step_variant=variant),
        "roofline": roof,
        "e2e": {
            "value": round(job_glups(world, sites, n_e2e, e2e_s), 3),
            "unit": UNIT,
            "h2d_bytes_per_step": int(nbytes / n_e2e),
            "d2h_bytes_per_step": int((nbytes + stats_bytes) / n_e2e),
            "what": "flbm_load from pinned host blob, K x flbm_step(1) with flbm_sample every "
                    f"{S} steps, flbm_fetch_samples (D2H of every record), flbm_save to pinned host; "
                    "wall clock",
        },
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "nonfinite_sites_in_samples": int(nonfinite),
    }
    if world == 1 and not args.no_extras:
        line["storage_widths"] = storage_widths(fl, torch, stream, dims, peaks["hbm_gbs"])
        line["other_lattices"] = other_lattices(fl, torch, stream, dims, peaks["hbm_gbs"])
        line["noise_off"] = noise_off(fl, torch, stream, dims, peaks["hbm_gbs"], avg_kernel_ms)
        line["batched_ensemble"] = batched_ensemble(fl, torch, peaks["hbm_gbs"])
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return line


# ---- the two other systems forms: 16-bit storage and batched ensembles -------------------
def draw_ensemble(n=256, seed=0):
    """The batched-ensemble workload: n lattices drawn from `seed`: D2Q9 or D3Q27 with
    probability 1/2, side log-uniform in [32, 256] (D2Q9) or [16, 64] (D3Q27), kBT
    log-uniform in [1e-5, 1e-3], shear relaxation time tau uniform in [0.51, 2.0]
    (Lambda_shear = 1/tau, every other non-conserved mode 1), seed 1000 + j."""
    rng = np.random.default_rng(seed)
    specs = []
    for j in range(n):
        d3 = rng.random() < 0.5
        lo, hi = (16, 64) if d3 else (32, 256)
        side = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        kbt = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-3))))
        tau = float(rng.uniform(0.51, 2.0))
        lam = np.ones(27 if d3 else 9)
        lam[[7, 8, 9] if d3 else [4, 5]] = 1.0 / tau
        specs.append(dict(lattice=1 if d3 else 0, dims=(side, side, side if d3 else 1), lam=lam, kBT=kbt,
                          rho0=1.0, seed=1000 + j))
    return specs


def _event_time(torch, stream, fn, n):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn(n)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


def storage_widths(fl, torch, stream, dims, peak):
    """GLUPS of the same workload with BF16 and FP16 deviation storage (FP32 arithmetic)."""
    out = {}
    sites = dims[0] * dims[1] * dims[2]
    for storage, name in ((fl.FLBM_BF16, "bf16"), (fl.FLBM_FP16, "fp16")):
        with fl.Lattice(fl.FLBM_D3Q27, dims, lam_d3q27(), KBT, 1.0, SEED, storage,
                        cuda_stream=stream.cuda_stream) as lat:
            lat.init_uniform(U0, AMP, SEED)
            variant = lat.autotune(10)
            lat.step(6)
            ms = _event_time(torch, stream, lat.step, 200)
            gbs = 27 * 2 * 2 * sites / (ms * 1e-3) / 1e9
            out[name] = {"value": round(sites / (ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms_per_step": round(ms, 5),
                         "step_variant": variant, "achieved_gbs": round(gbs, 1),
                         "frac_of_hbm": round(gbs / peak, 4), "bytes_per_site": 108}
    return out


def other_lattices(fl, torch, stream, dims, peak):
    """GLUPS of the same workload (drift, perturbation, kBT, shear rate 1.6) on the
    isotropic D3Q27 variant (deviators at the shear rate too) and on D3Q19, FP32."""
    out = {}
    sites = dims[0] * dims[1] * dims[2]
    lam_iso = np.ones(27)
    lam_iso[[5, 6, 7, 8, 9]] = OMEGA
    lam19 = np.ones(19)
    lam19[[7, 8, 9]] = OMEGA
    for lattice, lam, q, name in ((fl.FLBM_D3Q27_ISO, lam_iso, 27, "d3q27_isotropic"), (fl.FLBM_D3Q19, lam19, 19, "d3q19")):
        with fl.Lattice(lattice, dims, lam, KBT, 1.0, SEED, cuda_stream=stream.cuda_stream) as lat:
            lat.init_uniform(U0, AMP, SEED)
            variant = lat.autotune(10)
            lat.step(6)
            ms = _event_time(torch, stream, lat.step, 200)
            gbs = q * 4 * 2 * sites / (ms * 1e-3) / 1e9
            out[name] = {"value": round(sites / (ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms_per_step": round(ms, 5),
                         "step_variant": variant, "achieved_gbs": round(gbs, 1),
                         "frac_of_hbm": round(gbs / peak, 4), "bytes_per_site": q * 8}
    return out


def noise_off(fl, torch, stream, dims, peak, noisy_ms):
    """The headline workload at k_BT = 0 (the kernels' noise-free instantiation: no Philox,
    no Box-Muller, identical loads, transforms, relaxation and stores), FP32, the noisy
    kernel's variant: the difference to the noisy step is the cost of the 23 normals per
    site."""
    sites = dims[0] * dims[1] * dims[2]
    with fl.Lattice(fl.FLBM_D3Q27, dims, lam_d3q27(), 0.0, 1.0, SEED, cuda_stream=stream.cuda_stream) as lat:
        lat.init_uniform(U0, AMP, SEED)
        variant = lat.autotune(10)
        lat.step(6)
        ms = _event_time(torch, stream, lat.step, 200)
    gbs = BYTES_PER_SITE * sites / (ms * 1e-3) / 1e9
    return {"value": round(sites / (ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms_per_step": round(ms, 5),
            "step_variant": variant, "achieved_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
            "noise_share_of_noisy_step": round(max(0.0, 1.0 - ms / noisy_ms), 4)}


FORMS = ["per-step launches", "persistent launch", "per-step launches, 5 blocks/SM (D2Q9: 10)",
         "per-step launches, rolled noise loop"]


def batched_ensemble(fl, torch, peak, steps=200, calls=25):
    """The batched-ensemble workload in one batch (per-step graph-captured launches or one
    persistent launch, as the autotuner picks) against the same lattices stepped one
    context at a time. The timed region is the workload's 5000 steps: `calls` calls of
    `steps` steps, each replaying the same captured graph."""
    specs = draw_ensemble()
    sites = sum(int(np.prod(d["dims"])) for d in specs)
    nbytes = sum(int(np.prod(d["dims"])) * (27 if d["lattice"] else 9) * 8 for d in specs)
    with fl.Batch(specs) as b:
        for i in range(len(specs)):
            b.lattice(i).init_uniform((0.0, 0.0, 0.0), 0.0, 0)
        threads, form = b.autotune(10)
        threads2, form2 = b.type_shape(0)  # the D2Q9 lattices' own shape
        b.step(4)
        b.step(steps)  # capture of the timed call's graph
        b.sync()
        t = time.perf_counter()
        for _ in range(calls):
            b.step(steps)
        b.sync()
        ms = (time.perf_counter() - t) * 1e3 / (steps * calls)
        graph = b.uses_graph
    lats = [fl.Lattice(d["lattice"], d["dims"], d["lam"], d["kBT"], d["rho0"], d["seed"]) for d in specs]
    try:
        for lat in lats:
            lat.init_uniform((0.0, 0.0, 0.0), 0.0, 0)
            lat.step(2)
        for lat in lats:
            lat.sync()
        n = 20
        t = time.perf_counter()
        for _ in range(n):
            for lat in lats:
                lat.step(1)
        for lat in lats:
            lat.sync()
        ms_loop = (time.perf_counter() - t) * 1e3 / n
    finally:
        for lat in lats:
            lat.close()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": "256 lattices drawn from seed 0 (D2Q9 32^2..256^2 / D3Q27 16^3..64^3, kBT 1e-5..1e-3, "
                        "tau 0.51..2.0, seeds 1000+j), FP32",
            "lattices": len(specs), "sites": sites, "value": round(sites / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "ms_per_step": round(ms, 5), "achieved_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
            "steps": steps * calls, "threads": threads, "form": FORMS[form],
            "d2q9_threads": threads2, "d2q9_form": FORMS[form2], "graph": graph,
            "single_context_loop_ms_per_step": round(ms_loop, 5),
            "speedup_vs_single_context_loop": round(ms_loop / ms, 3),
            "timing": "wall clock around synchronised calls (own stream)"}


# ---- the oracle on the host cores ---------------------------------------------------------
def _oracle_sample_dims(target_sites):
    # A cube-ish D3Q27 box of about target_sites sites (same physics as the workload).
    n = max(4, int(round(target_sites ** (1.0 / 3.0))))
    return (n, n, n)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# Lattices the oracle is timed on: the 2-D and 3-D sizes of the statistics ensemble and a
# 32^3 box (the 256^3 workload itself is far too slow for the dense FP64 oracle).
CPU_LEGS = ((0, (512, 512, 1)), (1, (32, 32, 32)), (1, (64, 64, 64)))


def _lam_for(lattice):
    if lattice == 0:
        lam = np.ones(9)
        lam[[4, 5]] = OMEGA
        return lam
    return lam_d3q27()


def cpu_baseline(budget_s=20.0):
    """Time the oracle (as it stands) on bounded samples: D2Q9 512^2 and D3Q27 32^3 and
    64^3 with the workload's physics, each at one thread and at every host thread, about
    budget_s / 6 seconds per leg after a one-step calibration. The headline value is the
    D3Q27 64^3 leg at every thread."""
    import oracle

    oracle.build()
    nproc = os.cpu_count() or 1
    legs = []
    leg_s = budget_s / (2 * len(CPU_LEGS))
    per_site = {}  # (lattice, threads) -> seconds per site update of the first (smaller) box
    for lattice, dims in CPU_LEGS:
        lam = _lam_for(lattice)
        u0 = U0 if lattice else U0[:2] + (0.0,)
        sites = int(np.prod(dims))
        for threads in (1, nproc):
            f = oracle.init_uniform(lattice, dims, 1.0, u0, AMP, SEED)
            if (lattice, threads) not in per_site:  # calibrate with one step
                t = time.perf_counter()
                f = oracle.run(lattice, dims, lam, KBT, SEED, f, 0, 1, threads=threads)
                per_site[(lattice, threads)] = (time.perf_counter() - t) / sites
            steps = max(1, int(round(leg_s / max(per_site[(lattice, threads)] * sites, 1e-6))))
            t = time.perf_counter()
            oracle.run(lattice, dims, lam, KBT, SEED, f, 1, steps, threads=threads)
            dt = time.perf_counter() - t
            legs.append({"lattice": "D2Q9" if lattice == 0 else "D3Q27", "dims": list(dims), "threads": threads,
                         "steps": steps, "seconds": round(dt, 3),
                         "mlups": round(sites * steps / dt / 1e6, 4)})
    head = [g for g in legs if g["lattice"] == "D3Q27" and g["dims"] == [64, 64, 64] and g["threads"] == nproc][0]
    return {"value": head["mlups"] / 1e3, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"D3Q27 64^3 (same physics as the workload), {head['steps']} steps, {head['seconds']} s at "
                      f"{nproc} threads; also D2Q9 512^2 and D3Q27 32^3, each at 1 and {nproc} threads (legs); "
                      "FP64 dense T(u)+LU, OpenMP over sites",
            "legs": legs}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    lam = lam_d3q27()
    cal = (16, 16, 16)
    f = oracle.init_uniform(1, cal, 1.0, U0, AMP, SEED)
    t = time.perf_counter()
    oracle.run(1, cal, lam, KBT, SEED, f, 0, 1, threads=threads)
    per_site = (time.perf_counter() - t) / np.prod(cal)
    total_budget = args.ref_budget
    dims = _oracle_sample_dims(max(512, min(total_budget / max(1, args.steps + args.warmup) / per_site,
                                            64 ** 3)))
    f = oracle.init_uniform(1, dims, 1.0, U0, AMP, SEED)
    for k in range(args.warmup):
        f = oracle.run(1, dims, lam, KBT, SEED, f, k, 1, threads=threads)
    S = args.stats_every
    t = time.perf_counter()
    for k in range(args.steps):
        if k % S == 0:  # the statistics of the state the step reads, as in the GPU arm
            oracle.stats(1, dims, f)
        f = oracle.run(1, dims, lam, KBT, SEED, f, args.warmup + k, 1, threads=threads)
    dt = time.perf_counter() - t
    sites = int(np.prod(dims))
    value = sites * args.steps / dt / 1e9
    sample = (f"D3Q27 {dims[0]}x{dims[1]}x{dims[2]} per step (bounded sample of the 256^3 workload, "
              f"same physics, statistics every {S} steps), FP64 oracle, OpenMP over sites")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded lattice state, no dataset)",
        "config": workload_config(S, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_profile_workload(args):
    """A short run of one kernel family for ncu captures (no timing, no bench line):
    stats: a D3Q27 box of --dims, two steps, two statistics reductions; d3q19: a D3Q19 box
    of --dims with the paper's rates (shear 1.6), four steps of --variant (default 2), with
    --noise-off at k_BT = 0;
    batch: the 256-lattice ensemble, three steps of the per-step form at 128 threads;
    step: the headline physics on a D3Q27 box of --dims in --storage (D2Q9 when the box has
    nz = 1), four steps of --variant (default 5); with --noise-off at k_BT = 0."""
    import torch

    import paper_2602_16486_gb300 as fl

    torch.cuda.set_device(0)
    dims = tuple(args.dims)
    if args.profile == "stats":
        with fl.Lattice(fl.FLBM_D3Q27, dims, lam_d3q27(), KBT, 1.0, SEED) as lat:
            lat.init_uniform(U0, AMP, SEED)
            lat.step(2)
            lat.stats()
            lat.stats()
    elif args.profile == "step":
        lattice = fl.FLBM_D2Q9 if dims[2] == 1 else fl.FLBM_D3Q27
        lam = _lam_for(lattice)
        with fl.Lattice(lattice, dims, lam, 0.0 if args.noise_off else KBT, 1.0, SEED, args.storage) as lat:
            lat.variant = args.variant or 5
            lat.init_uniform(U0 if lattice else U0[:2] + (0.0,), AMP, SEED)
            lat.step(4)
            lat.sync()
    elif args.profile == "d3q19":
        lam = np.ones(19)
        lam[[7, 8, 9]] = OMEGA
        with fl.Lattice(fl.FLBM_D3Q19, dims, lam, 0.0 if args.noise_off else KBT, 1.0, SEED) as lat:
            lat.variant = args.variant or 2
            lat.init_uniform(U0, AMP, SEED)
            lat.step(4)
            lat.sync()
    else:
        specs = draw_ensemble()
        with fl.Batch(specs) as b:
            for i in range(len(specs)):
                b.lattice(i).init_uniform((0.0, 0.0, 0.0), 0.0, 0)
            b.shape = (128, 0)  # the shape the autotuner picks for this ensemble on GB300
            b.step(3)
            b.sync()
    return {"profile": args.profile, "dims": list(dims), "note": "profiling workload: not a bench line"}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--stats-every", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-budget", type=float, default=20.0)
    p.add_argument("--ref-budget", type=float, default=120.0)
    p.add_argument("--dims", type=lambda s: [int(x) for x in s.split(",")], default=list(DIMS),
                   help="box for profiling runs (default 256,256,256: the workload)")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    p.add_argument("--variant", type=int, default=0,
                   help="step-kernel variant (1-6); default 0 = autotune")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the 16-bit storage, other-lattice and batched-ensemble measurements")
    p.add_argument("--noise-off", action="store_true",
                   help="--profile step / d3q19: k_BT = 0 (the kernels' noise-free instantiation)")
    p.add_argument("--storage", type=int, default=0, choices=[0, 1, 2],
                   help="storage of the --profile step workload: 0 FP32, 1 BF16, 2 FP16")
    p.add_argument("--profile", choices=["stats", "d3q19", "batch", "step"], default=None,
                   help="run a short workload of one kernel family for ncu captures and exit")
    args = p.parse_args(argv)
    if args.profile:
        print(json.dumps(run_profile_workload(args)), flush=True)
        return
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    world, _, _ = dist_setup()
    if world != args.gpus and world > 1:
        p.error(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
