#!/usr/bin/env python
"""Throughput benchmark of the two-component D3Q19 Shan-Chen LBM step on GB300.

One "step" is one full time step (moments, Eq. 7 interaction, collision with
forcing, streaming) over the whole lattice.  Default workload: the 512^3
periodic spinodal mixture, FP32 populations, BGK, tau = 1.0.  The metric is
MLUPS (million two-component cell updates per second) for the whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, N > 1): each rank advances its own independent replica
(the benchmark runs replicas only: one GPU per process, no exchange), value =
cells of all ranks x K / (max over ranks of the timed region).

--impl reference times the FP64 CPU oracle (the baseline of this project) on
a bounded 64^3 cut of the same workload, on rank 0 only.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1601_01237_gb300 import workloads as wl  # noqa: E402

METRIC = "MLUPS (2-comp D3Q19)"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_VALUE = {"f64": 8, "f32": 4, "f16_dev": 2, "bf16_dev": 2, "f16_rel": 2, "bf16_rel": 2}


def state_bytes_per_cell(storage):
    """Bytes of one state per cell: 2 components x 19 populations, plus the
    two FP32 reference densities of the relative 16-bit formats."""
    return 2 * 19 * BYTES_PER_VALUE[storage] + (8 if storage.endswith("_rel") else 0)
ORACLE_SAMPLE_SHAPE = (64, 64, 64)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="perf512_spinodal_f32", choices=sorted(wl.CONFIGS))
    ap.add_argument("--storage", default=None, help="override the workload's population storage")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=None,
                    help="steps of the differentiation case (default: its configured 500; shorter for captures)")
    ap.add_argument("--mask", choices=["none", "inclined"], default="none",
                    help="inclined: staircase slab of solid sites (30 degrees, 8 cells thick) on the workload")
    ap.add_argument("--shape", type=int, nargs=3, default=None, metavar=("NZ", "NY", "NX"),
                    help="run the workload's parameters on another lattice (small profiling captures)")
    return ap.parse_args()


def workload_desc(name, cfg, storage):
    nz, ny, nx = cfg["shape"]
    return {
        "workload": "%s%s: %dx%dx%d two-component D3Q19, %s populations, %s, tau=%s, G_eq7=%.3g, %s" % (
            name, " (lattice override)" if cfg.get("shape_override") else "", nx, ny, nz, storage,
            cfg.get("collision", "bgk"), cfg["tau"][0], cfg["G"],
            "periodic" if all(cfg.get("periodic", (1, 1, 1))) else "z walls"),
        "shape_zyx": list(cfg["shape"]),
        "storage": storage,
        "collision": cfg.get("collision", "bgk"),
        "tau": list(cfg["tau"]),
        "G12_eq7": cfg["G"],
    }


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return FALLBACK_HBM_GBS, "fallback (MEASURED_PEAKS.json absent)"
    for key in ("hbm_gbs", "hbm_GBps", "hbm_copy_gbs", "hbm"):
        v = d.get(key)
        if isinstance(v, (int, float)):
            return float(v), "measured (MEASURED_PEAKS.json %s)" % key
        if isinstance(v, dict):
            for k2 in ("gbs", "value", "GBps"):
                if isinstance(v.get(k2), (int, float)):
                    return float(v[k2]), "measured (MEASURED_PEAKS.json %s.%s)" % (key, k2)
    return FALLBACK_HBM_GBS, "fallback (no HBM figure in MEASURED_PEAKS.json)"


# source files that define each timed kernel (a change to any of them voids
# the committed DRAM-traffic figure of that kernel)
KERNEL_SOURCES = {"k_step_fused": ("d3q19.cuh", "lbm_fused_impl.cuh"),
                  "k_density": ("d3q19.cuh", "lbm_forward.cu"),
                  "k_collide": ("d3q19.cuh", "lbm_forward.cu")}


def kernel_source_hash(kernel):
    """Hash of the kernel's sources with comments and blank lines removed
    (editing a comment keeps the committed counters valid)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1601_01237_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        text = open(os.path.join(csrc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(l.rstrip() for l in text.splitlines() if l.strip()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, storage, cells):
    """DRAM bytes per launch from the committed ncu summary, scaled by cells,
    or None when the kernels changed since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = d.get("%s/%s" % (kernel, storage))
    if not e or e.get("kernel_source_sha") != kernel_source_hash(kernel):
        return None
    return e["dram_bytes_per_cell"] * cells


def algorithmic_bytes_per_cell(kernel, storage):
    """Minimum HBM bytes per cell of one launch: every population read once
    and written once (2 components x 19 values x s bytes x 2, and for the
    relative 16-bit formats the cell's two FP32 reference densities read and
    written); the density pass of the two-kernel step reads the state and
    writes 2 densities; the collision pass also reads the 2 densities."""
    b = state_bytes_per_cell(storage)
    r = 8 if storage == "f64" else 4
    if kernel == "k_density":
        return b + 2 * r
    if kernel == "k_collide":
        return b * 2 + 2 * r
    return b * 2


def max_over_ranks(x, device="cpu"):
    """Maximum of a per-rank scalar over all ranks (identity without a
    process group)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_mlups(cells_per_rank, world, steps, max_seconds):
    """Whole-job throughput: every rank advances its own replica of
    cells_per_rank cells by `steps`; the job takes the slowest rank's time."""
    return cells_per_rank * world * steps / max_seconds / 1e6


# --------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands (single-threaded C), timed on the host
    cores: one process per core, each stepping its own copy of a bounded cut
    of the workload from a common start (W warm-up steps, then K timed); the
    value is the aggregate over all processes."""
    if rank != 0:
        return None
    import multiprocessing as mp
    cfg = dict(wl.CONFIGS[args.workload])
    shape = ORACLE_SAMPLE_SHAPE if len(cfg["shape"]) == 3 and cfg["shape"][0] > 1 else cfg["shape"]
    sub = {k: cfg[k] for k in ("tau", "G", "periodic", "collision") if k in cfg}
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        start = time.time() + 5.0 + 0.5 * args.warmup
        res = pool.map(_oracle_sample, [(args.workload, shape, sub, args.steps, start, args.warmup)] * cores)
    total = sum(r[0] for r in res)
    dt = max(r[2] for r in res) - min(r[1] for r in res)
    value = total / dt / 1e6
    storage = args.storage or cfg["storage"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_desc(args.workload, cfg, storage),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": "%dx%dx%d cut of the workload, %d steps after %d warm-up, FP64; one process per "
                                   "core, each on its own copy" % (shape[2], shape[1], shape[0], args.steps,
                                                                   args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def _oracle_sample(job):
    """One process of the CPU baseline and of the reference arm: the oracle on
    its own copy of the sample, warm-up steps, then nsteps from a common start
    time; returns (cell updates, start, end)."""
    workload, shape, cfg, nsteps, t_start = job[:5]
    warmup = job[5] if len(job) > 5 else 1
    import oracle
    oracle.set_threads(1)   # one single-threaded process per core
    r1, r2 = wl.fields_for(workload, shape=shape)
    p = oracle.make_params(shape, tau=cfg["tau"], G12=cfg["G"], periodic=cfg.get("periodic", (1, 1, 1)),
                           collision=cfg.get("collision", "bgk"))
    f = oracle.init(p, r1, r2)
    oracle.step(p, f, warmup)
    while time.time() < t_start:
        time.sleep(0.001)
    t0 = time.time()
    oracle.step(p, f, nsteps)
    return int(np.prod(shape)) * nsteps, t0, time.time()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_baseline(args, cfg):
    """The oracle as it stands (plain single-threaded C) on a bounded 64^3 cut
    of the workload: one process, and one process per host core, each on its
    own copy of the cut and started together (spawned processes: this runs
    after CUDA is initialised).  The all-core aggregate is the reported value."""
    import multiprocessing as mp
    shape = ORACLE_SAMPLE_SHAPE
    n = 30
    sub = {k: cfg[k] for k in ("tau", "G", "periodic", "collision") if k in cfg}
    cells, t0, t1 = _oracle_sample((args.workload, shape, sub, n, 0.0))
    single = cells / (t1 - t0) / 1e6
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        # the common start leaves every process time to build its sample
        start = time.time() + 5.0
        res = pool.map(_oracle_sample, [(args.workload, shape, sub, n, start)] * cores)
    total = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": total / wall / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": single, "cpu_model": cpu_model(),
            "sample": "64x64x64 cut of the workload, %d steps, FP64; one process per core, each on its own copy "
                      "(single_core_value: one process alone)" % n}


def adjoint_ratio(stream, steps=None):
    """Adjoint/forward time ratio on the differentiation case: 96^3 droplet
    (R = 20), FP32, 500 steps, checkpoints every 25.  Forward = lbm_step(500)
    after a warm-up lbm_step(100); reverse = lbm_adjoint over an lbm_record of
    the same 500 steps, including its recomputation of every checkpoint
    segment, after one warm-up lbm_adjoint call over the same recording (both
    warm-ups build the CUDA graphs that the timed calls replay)."""
    import torch
    from paper_1601_01237_gb300 import Lattice
    c = wl.CONFIGS["c3_adjoint96"]
    shape, n, every = c["shape"], steps or c["steps"], c["ckpt_every"]
    r1, r2 = wl.droplet(shape, c["R"])
    tgt, _ = wl.ellipsoid(shape, c["target_axes"])
    lat = Lattice(shape, storage=c["storage"], tau=c["tau"], G12=c["G"], stream=stream.cuda_stream)
    d1, d2 = torch.from_numpy(r1).cuda(), torch.from_numpy(r2).cuda()
    lat.init_fields(d1, d2)
    lat.step(100)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / n
    lat.init_fields(d1, d2)
    lat.record(n, every)
    out1 = torch.empty(shape, dtype=torch.float64, device="cuda")
    lat.moments_device(rho1=out1, out_f64=True)
    g = 2.0 * (out1 - torch.from_numpy(tgt).cuda())
    gr0 = torch.empty(shape, dtype=torch.float64, device="cuda")
    lat.adjoint(g, None, gr0, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    par = lat.adjoint(g, None, gr0, None)
    torch.cuda.synchronize()
    adj_ms = (time.perf_counter() - t0) * 1e3 / n
    lat.close()
    return {"workload": "96^3 droplet R=20, FP32, %d steps, checkpoints every %d" % (n, every),
            "forward_ms_per_step": fwd_ms, "adjoint_ms_per_step": adj_ms, "ratio": adj_ms / fwd_ms,
            "dL_dG12_tied": par[0] + par[1], "dL_dtau1": par[2]}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1601_01237_gb300 import Lattice
    dist = world > 1
    torch.cuda.set_device(local_rank)
    cfg = dict(wl.CONFIGS[args.workload])
    if args.shape:
        cfg["shape"], cfg["shape_override"] = tuple(args.shape), True
    storage = args.storage or cfg["storage"]
    shape = tuple(cfg["shape"])
    cells = int(np.prod(shape))
    g_ext = wl.tilted_gravity(cfg["g_mag"], cfg["tilt_deg"]) if "g_mag" in cfg else (0.0, 0.0, 0.0)
    kw = dict(storage=storage, tau=cfg["tau"], G12=cfg["G"], periodic=cfg.get("periodic", (1, 1, 1)),
              collision=cfg.get("collision", "bgk"), g_ext=g_ext,
              rho0_dev=0.5 if storage.endswith("_dev") else 0.0)
    r1, r2 = wl.fields_for(args.workload, shape=shape)
    stream = torch.cuda.current_stream()
    lat = Lattice(shape, stream=stream.cuda_stream, **kw)
    mask_desc = None
    if args.mask == "inclined":
        solid = wl.inclined_slab(shape)
        lat.set_solid(solid)
        mask_desc = "staircase slab inclined 30 deg, 8 cells thick: %.1f %% solid sites (wall model %s)" % (
            100.0 * solid.mean(), kw.get("wall_model", "mirror"))
        del solid
    d1 = torch.from_numpy(r1).cuda()
    d2 = torch.from_numpy(r2).cuda()
    lat.init_fields(d1, d2)
    del d1, d2
    lat.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-kernel events inside -----------------
    sampler = ClockSampler(local_rank)
    sampler.start()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kern = lat.step_timed(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, device="cuda")
    value = job_mlups(cells, world, args.steps, ms_max / 1e3)
    red = lat.reduce()

    # ---- roofline of the dominant kernel ----------------------------------
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_n = kern[dom]
    per_launch_s = dom_ms / dom_n / 1e3
    alg = algorithmic_bytes_per_cell(dom, storage) * cells
    peak, peak_src = measured_hbm_peak()
    achieved = alg / per_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic(dom, storage, cells), "kernel": dom,
                "algorithmic_bytes_per_launch": alg, "launch_ms": per_launch_s * 1e3,
                "peak_source": peak_src,
                "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                                "share": v[0] / sum(x[0] for x in kern.values())} for k, v in kern.items()}}
    step_bytes = state_bytes_per_cell(storage) * 2 * cells
    roofline["step_frac_of_peak"] = step_bytes / (ms_max / args.steps / 1e3) / 1e9 / peak

    # ---- end to end through the public API with host buffers -------------
    e2e = None
    if not args.no_e2e:
        h1 = torch.from_numpy(r1).pin_memory()
        h2 = torch.from_numpy(r2).pin_memory()
        torch.cuda.synchronize()
        if dist:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        lat.init_fields(h1, h2)          # H2D of the initial fields (pinned host)
        lat.step(args.steps)
        out = lat.reduce()               # D2H of the step's result (FP64 reductions)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, device="cuda")
        e2e = {"value": job_mlups(cells, world, args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": 2 * cells * 8 / args.steps,
               "d2h_bytes_per_step": (1216 * 8 * 8) / args.steps,
               "note": "lbm_init_fields from pinned host + lbm_step(K) + lbm_reduce to host, per step amortised",
               "mass_check": abs(out["mass1"] - red["mass1"]) / red["mass1"] < 1e-3}
    lat.close()

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if storage == "f64" else "f32",
        "data": "synthetic",
        "config": dict(workload_desc(args.workload, cfg, storage),
                       l2="inputs larger than L2: %.1f GB of populations per copy" % (
                           state_bytes_per_cell(storage) * cells / 1e9),
                       parallelism="replicas" if world > 1 else "single GPU",
                       **({"mask": mask_desc} if mask_desc else {})),
        "roofline": roofline,
        # (a mask adds the two wall-density kernels of the mirror model per step)
        "gpu_launches": sum(v[1] for v in kern.values()) * (3 if mask_desc and "k_step_fused" in kern else 1),
        "clocks": clocks,
        "e2e": e2e,
        "mass": [red["mass1"], red["mass2"]],
    }
    if not args.no_adjoint:
        line["adjoint"] = adjoint_ratio(torch.cuda.current_stream(), args.adjoint_steps)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, cfg)
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if line:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
