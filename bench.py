"""Benchmark: fused D3Q19 MRT lattice Boltzmann step with the Smagorinsky closure fed by the
strain rate (Yu's or Chai's formula), FP32 populations, on a 256 x 128 x 128 channel with
halfway bounce-back walls at the y faces and a uniform body force g_x = 1e-6.

One benchmark step is one lattice time step over the whole grid (pull-stream, moments, strain
rate, closure, relaxation, force, store, all in one kernel).  The timed region is one
lbm_step(K) call, which the library's automatic schedule runs as a single multi-step launch on
this lattice (steps overlap tile by tile instead of draining the GPU between them).  The metric
is MLUPS (million lattice node updates per second) and the fraction of the measured HBM bandwidth
that the minimum traffic (19 populations read + 19 written, 152 bytes per node update)
represents.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|fp16s|bf16s|fp64] [--formula yu|chai] [--lattice 19|15]
                  [--closure smag|smag_lagged|smag_dev] [--no-variants] [--quick]

--precision / --formula pick the headline (default fp32 / yu); --quick skips the end-to-end
run, the other variants and the CPU baseline (used for profiler captures).

With N > 1 (torchrun) every rank runs its own replica of the workload (the step has no
cross-GPU exchange), value = all ranks' node updates / the slowest rank's time.
--impl reference times the FP64 CPU oracle (the paper has no implementation) on a bounded
sample of the same workload.
"""
import argparse
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

NX, NY, NZ = 256, 128, 128
TAU0, CS, G = 0.51, 0.17, 1e-6
RATES = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98,
         1.98, 1.98]
RATES15 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98]
BC = ["periodic", "periodic", "wall", "wall", "periodic", "periodic"]
BYTES_PER_LUP = {"fp32": 152, "fp64": 304, "fp16s": 76, "bf16s": 76}
STORAGE_NOTE = {"fp32": "fp32 populations, fp32 arithmetic", "fp64": "fp64 populations, fp64 arithmetic",
                "fp16s": "fp16 populations (delta-rho form), fp32 arithmetic",
                "bf16s": "bf16 populations (delta-rho form), fp32 arithmetic"}
CLOSURE_NOTE = {"smag": "smagorinsky", "smag_lagged": "smagorinsky, tau from the previous step",
                "smag_dev": "smagorinsky on the traceless strain rate, closed form"}
WORKLOAD = "D3Q19 MRT Smagorinsky LES channel 256x128x128, walls at y, g_x=1e-6, Cs=0.17, tau0=0.51"
METRIC = "MLUPS, MRT step + strain rate (Smagorinsky LES channel)"


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def captured_traffic(kernel):
    """DRAM bytes per lattice step of `kernel` from the committed ncu capture (the capture's bytes
    divided by the steps its launch ran), or None when the capture is of another kernel or the
    kernel sources changed since it was taken."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as fh:
            doc = json.load(fh)
        h = hashlib.sha256()
        for src in doc["sources"]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
        if doc["kernel"] == kernel and h.hexdigest() == doc["sources_sha256"]:
            return int(doc["dram_bytes_per_step"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# our arm


def make_lattice(precision="fp32", formula="yu", dims=(NX, NY, NZ), lattice=19, closure="smag"):
    from paper_1704_07559_gb300 import inputs as I
    from paper_1704_07559_gb300 import lbm

    lat = lbm.Lattice(lattice, *dims, rates=RATES if lattice == 19 else RATES15, force=[G, 0.0, 0.0],
                      precision=precision, closure=closure, smag_cs=CS, formula=formula, bc=BC)
    drho, u = I.channel_profile(*dims, u_centre=0.1, noise=0.01, seed=2)
    lat.init(drho, u)
    return lat


def time_steps(lat, steps, warmup, per_launch=False):
    """Device time of `steps` lattice steps (ms) via CUDA events on the library's stream; with
    per_launch, a list of each launch's time (an event pair around every launch)."""
    import torch

    s = lat.stream
    lat.step(warmup)
    torch.cuda.synchronize()
    if per_launch:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            a.record(s)
            lat.step(1)
            b.record(s)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    lat.step(steps)
    t1.record(s)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1)


def time_e2e(lat, steps):
    """End to end through the public API with host buffers: each step uploads the state from
    pinned host memory, advances one step and reads the global sums back to the host."""
    import torch

    host = lat.get_state().cpu().pin_memory()
    torch.cuda.synchronize()
    lat.set_state(host)
    lat.step(1)
    lat.sums()
    t0 = time.perf_counter()
    for _ in range(steps):
        lat.set_state(host)
        lat.step(1)
        lat.sums()
    dt = time.perf_counter() - t0
    h2d = host.numel() * host.element_size()
    return dt / steps, h2d, 8 * (1 + lat.d)


def _oracle_channel_box(nx, ny, nz):
    import oracle as O
    from paper_1704_07559_gb300 import inputs as I

    p = O.make_params(19, RATES, closure=O.SMAG, smag_cs=CS, formula=O.YU,
                      bc=[O.PERIODIC, O.PERIODIC, O.WALL, O.WALL, O.PERIODIC, O.PERIODIC])
    Gr = O.Grid(p, nx, ny, nz)
    drho, u = I.channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2)
    F = np.array([G, 0.0, 0.0])
    return Gr, Gr.init(drho, u, force=F), F


def job_rate(ms_local, updates_local, dist=None, device="cpu"):
    """Whole-job rate of N replicas: the slowest rank's time of the timed region (max over ranks)
    and all ranks' node updates / that time, in MLUPS.  dist: torch.distributed (initialised) or
    None for one process; every rank does the same number of updates."""
    import torch

    world = 1
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_local = float(t.item())
        dist.barrier()
    return ms_local, world * updates_local / (ms_local * 1e-3) / 1e6


FMA_PROBE_SRC = os.path.join(ROOT, "bench_fma_peak.cu")
FMA_PROBE_LIB = os.path.join(ROOT, "libbench_fma_peak.so")


def build_fma_probe(force=False):
    """Compile the benchmark's FMA-throughput probe (bench_fma_peak.cu, not part of the library)
    for sm_103a if its source is newer than the shared object; return the object's path."""
    if not force and os.path.exists(FMA_PROBE_LIB) and os.path.getmtime(FMA_PROBE_LIB) >= os.path.getmtime(FMA_PROBE_SRC):
        return FMA_PROBE_LIB
    import shutil

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = FMA_PROBE_LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC", "-shared", "-o", tmp,
           FMA_PROBE_SRC, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s%s" % (FMA_PROBE_SRC, r.stdout, r.stderr))
    os.replace(tmp, FMA_PROBE_LIB)
    return FMA_PROBE_LIB


def alu_peaks():
    """Measured FP32 and FP64 FMA throughput of this GPU (TFLOP/s, 2 flops per FMA), from the
    benchmark's probe: the arithmetic ceilings beside the HBM roofline."""
    import ctypes

    lib = ctypes.CDLL(build_fma_probe())
    lib.fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, fp64 in (("fp32_fma_tflops", 0), ("fp64_fma_tflops", 1)):
        v = ctypes.c_double()
        out[name] = round(v.value, 3) if lib.fma_peak(fp64, ctypes.byref(v)) == 0 else None
    return out


def host_cpu():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.machine()


def cpu_baseline(steps, warmup, seconds_budget=8.0):
    """The FP64 oracle as it stands, on the host cores, on the reference arm's configuration: one
    spawned process per host core, each stepping its own nx x 32 x 32 sub-box of the channel (same
    rates, closure, force and walls, Yu route; nx as the reference arm picks it for these steps),
    for about seconds_budget of timed steps; value = all processes' node updates / the slowest
    process's timed steps.  Also one thread on the 512^2 D2Q9 power-law cavity (Chai route)."""
    import multiprocessing as mp

    import oracle as O

    O.lib()  # built once before the workers start
    dims, rate = reference_subbox(steps, warmup)
    nodes = dims[0] * dims[1] * dims[2]
    per = max(1, int(rate * seconds_budget / nodes))  # timed steps per process for ~budget seconds
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_reference_worker, [(dims, 1, per)] * cores)
    dt = max(r[1] for r in res)
    allcore = sum(r[0] for r in res) * per / dt / 1e6
    # D2Q9 512^2 lid-driven power-law cavity (n = 0.5), one thread
    L2, U = 512, 0.05
    tau_ref = 0.5 + 3 * U * L2 / 1000.0
    p9 = O.make_params(9, [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / tau_ref, 1 / tau_ref], closure=O.POWERLAW,
                       formula=O.CHAI, pl_n=0.5, pl_k=U ** 1.5 * L2 ** 0.5 / 1000.0,
                       bc=[O.WALL, O.WALL, O.WALL, O.LID, O.PERIODIC, O.PERIODIC],
                       lid_u=[[0, 0, 0]] * 3 + [[U, 0, 0]] + [[0, 0, 0]] * 2)
    G9 = O.Grid(p9, L2, L2, 1)
    f9 = G9.init(np.zeros((1, L2, L2)), np.zeros((2, 1, L2, L2)))
    t0 = time.perf_counter()
    s9 = 0
    while time.perf_counter() - t0 < seconds_budget / 2 and s9 < 50:
        f9, _ = G9.step(f9)
        s9 += 1
    d2q9 = L2 * L2 * s9 / (time.perf_counter() - t0) / 1e6
    return {"value": round(allcore, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": reference_sample(cores, dims) + ", %d timed steps each" % per,
            "single_thread": {"value": round(rate / 1e6, 4), "unit": "MLUPS",
                              "sample": "calibration step of a 16x32x16 sub-box of the channel, one thread"},
            "d2q9_512_cavity": {"value": round(d2q9, 4), "unit": "MLUPS",
                                "sample": "512^2 power-law (n = 0.5) lid cavity, Chai route, %d steps, one thread" % s9},
            "host_cpu": host_cpu()}


def run_ours(args):
    import torch

    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1704_07559_gb300 import build

    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    if args.workload == "cavity":
        lat = cavity_lattice(4096, args.n_index, args.formula)
        lname, bytes_per_lup, grid, force = "D2Q9", 72, [4096, 4096, 1], "noforce"
        workload = ("D2Q9 MRT power-law lid-driven cavity 4096x4096, n=%g, lid velocity %g, Re=%g, fluid at rest "
                    "at t=0" % (args.n_index, CAVITY_U, CAVITY_RE))
        closure, cl_tag, l2 = "power law, n=%g" % args.n_index, "POWERLAW", "two 604 MB population buffers"
    elif args.workload == "box":
        n = args.box_n
        lat = box_lattice(n, args.precision, args.formula, 8, 0.03, 4)
        lname, bytes_per_lup, grid, force = "D3Q19", BYTES_PER_LUP[args.precision], [n, n, n], "noforce"
        workload = ("D3Q19 MRT Smagorinsky periodic box %d^3, divergence-free random Fourier start |k|<=8, "
                    "rms 0.03, Cs=%g, tau0=%g" % (n, CS, TAU0))
        closure, cl_tag = CLOSURE_NOTE["smag"], "SMAG"
        l2 = "two %.0f MB population buffers" % (n ** 3 * bytes_per_lup / 2 / 1e6)
    else:
        lat = make_lattice(args.precision, args.formula, lattice=args.lattice, closure=args.closure)
        lname = "D3Q%d" % args.lattice
        bytes_per_lup = BYTES_PER_LUP[args.precision] * args.lattice // 19
        if args.closure == "smag_lagged":  # the stored tau, read and written
            bytes_per_lup += 16 if args.precision == "fp64" else 8
        grid, force, workload = [NX, NY, NZ], "force", WORKLOAD.replace("D3Q19", lname)
        closure, cl_tag = CLOSURE_NOTE[args.closure], args.closure.upper()
        l2 = "two %.0f MB population buffers" % (NX * NY * NZ * BYTES_PER_LUP[args.precision] * args.lattice // 19 / 2 / 1e6)
    N = lat.N

    # timed region: barrier + synchronize on both sides, max over ranks
    lat.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    steps0, launches0 = lat.stats()
    with ClockSampler(gpu_index) as clk:
        ms = time_steps(lat, args.steps, 0)
        torch.cuda.synchronize()
    steps1, launches1 = lat.stats()
    launches = launches1 - launches0
    assert steps1 - steps0 == args.steps
    local_ms = ms
    ms, value = job_rate(ms, N * args.steps, dist, device="cuda")
    ms_per_step = ms / args.steps

    # kernel time per step for the roofline: the timed region holds only step launches (one per step,
    # or multi-step launches), so its CUDA-event time / steps is the time of one step's work
    k_ms = local_ms / args.steps
    achieved = bytes_per_lup * N / (k_ms * 1e-3) / 1e9
    # one-step launches with an event pair around each (no overlap between launches), for reference
    k_iso = statistics.mean(time_steps(lat, min(args.steps, 500), 0, per_launch=True))

    streamed = launches < args.steps
    pair = args.precision in ("fp16s", "bf16s") and grid[0] % 2 == 0
    kname = ("k_step_stream_pair" if pair else "k_step_stream") if streamed else ("k_step_pair_seq" if pair else "k_step")
    kernel = "%s<%s,%s,%s,%s,%s>" % (kname, lname, args.precision, cl_tag, args.formula.upper(), force)
    out = {
        "metric": METRIC if args.workload == "channel" else METRIC.replace(
            "Smagorinsky LES channel", "power-law cavity" if args.workload == "cavity" else "Smagorinsky box"),
        "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": workload, "lattice": lname, "grid": grid,
                   "formula": args.formula, "closure": closure,
                   "precision": STORAGE_NOTE[args.precision],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (%s per step)" % l2},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4),
                     "traffic": captured_traffic(kernel),
                     "peak_kind": peak_kind, "kernel": kernel,
                     "bytes_per_lup": bytes_per_lup,
                     "per": "lattice step (%d steps per launch)" % round(args.steps / max(launches, 1)),
                     "kernel_ms": round(k_ms, 5), "one_step_launches_ms": round(k_iso, 5)},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and (args.quick or args.workload != "channel"):
        print(json.dumps(out), flush=True)
    elif rank == 0:
        # end to end through the C ABI with host buffers
        e2e_s, h2d, d2h = time_e2e(lat, max(3, min(args.steps, 50)))
        out["e2e"] = {"value": round(world * N / e2e_s / 1e6, 2), "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h}
        out["alu_peaks"] = alu_peaks()
        if not args.no_variants:
            out["variants"] = variants(args, hbm, out["alu_peaks"])
        if world == 1:
            out["cpu_baseline"] = cpu_baseline(args.steps, args.warmup)
        print(json.dumps(out), flush=True)
    lat.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def slab_lattice(precision, formula, rank, world):
    """This rank's z-slab of the channel: the 128 planes split evenly over the ranks, halo z faces
    (the planes of the ranks below and above in the ghost planes), the channel's start."""
    from paper_1704_07559_gb300 import inputs as I
    from paper_1704_07559_gb300 import lbm, slab

    z0, z1 = slab.split_planes(NZ, world, rank)
    lat = lbm.Lattice(19, NX, NY, z1 - z0, rates=RATES, force=[G, 0.0, 0.0], precision=precision, closure="smag",
                      smag_cs=CS, formula=formula, bc=BC[:4] + ["halo", "halo"])
    drho, u = I.channel_profile(NX, NY, NZ, u_centre=0.1, noise=0.01, seed=2)
    planes = np.arange(z0 - 1, z1 + 1) % NZ
    lat.init(np.take(drho, planes, axis=-3), np.take(u, planes, axis=-3))
    return lat


def run_slab(args):
    """--decomp slab: one channel cut into z-slabs, one per rank, halos exchanged after every step
    (NCCL send/recv between the GPUs; one rank exchanges with itself), strong scaling.  The timed
    region holds the steps and the exchanges; value = the channel's node updates / the slowest
    rank's time."""
    import torch

    from paper_1704_07559_gb300 import build, slab

    rank, world = env_int("RANK", 0), env_int("WORLD_SIZE", 1)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    lat = slab_lattice(args.precision, args.formula, rank, world)
    own = lat.N // lat.nz * (lat.nz - 2)
    ex = slab.Slabs(lat, dist)
    ex.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    s = lat.stream
    steps0, launches0 = lat.stats()
    with ClockSampler(local) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        ex.step(args.steps)
        t1.record(s)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
    launches = lat.stats()[1] - launches0 + 2 * args.steps  # step kernels, and a pack and an unpack per step
    local_ms = ms
    ms, value = job_rate(ms, own * args.steps, dist, device="cuda")
    bpl = BYTES_PER_LUP[args.precision]
    achieved = bpl * own / (local_ms / args.steps * 1e-3) / 1e9
    out = {"metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "lattice": "D3Q19", "grid": [NX, NY, NZ], "formula": args.formula,
                      "closure": CLOSURE_NOTE["smag"], "precision": STORAGE_NOTE[args.precision],
                      "parallelism": "z-slabs over %d rank(s), halos exchanged every step" % world,
                      "l2": "inputs larger than L2 (two %.0f MB population buffers per step, split over the ranks)"
                            % (NX * NY * NZ * bpl / 2 / 1e6)},
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(achieved / hbm, 4), "traffic": None, "peak_kind": peak_kind,
                        "kernel": "k_step<D3Q19,%s,SMAG,%s,force> + halo copies + exchange" % (args.precision,
                                                                                           args.formula.upper()),
                        "bytes_per_lup": bpl, "per": "lattice step of this rank's slab, exchange included"},
           "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)
    lat.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def fp64_alu_counts():
    """FP64 flops and FP64-pipe instructions per node update of the FP64 Yu-route step kernel,
    from the committed ncu capture (profiles/fp64_alu.json), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_alu.json")) as fh:
            doc = json.load(fh)
        return float(doc["fp64_flops_per_lup"]), float(doc["fp64_instructions_per_lup"])
    except (OSError, ValueError, KeyError):
        return None


def variants(args, hbm, peaks=None):
    """The other (formula x form) pairs and the other workloads, each with its own timing."""
    import torch

    res = {"channel": {}}
    steps = max(10, min(args.steps, 1000))
    # channel (headline workload): the other formula x precision pairs
    for precision, formula in (("fp32", "chai"), ("fp16s", "yu"), ("fp16s", "chai"), ("bf16s", "yu"),
                               ("bf16s", "chai"), ("fp64", "yu"), ("fp64", "chai")):
        lat = make_lattice(precision, formula)
        n = steps if precision != "fp64" else max(5, steps // 10)
        k_ms = step_ms(lat, n, max(3, args.warmup // 10))
        res["channel"]["%s_%s" % (precision, formula)] = rate(lat.N, k_ms, BYTES_PER_LUP[precision], hbm)
        counts = fp64_alu_counts()
        if precision == "fp64" and formula == "yu" and counts and peaks and peaks.get("fp64_fma_tflops"):
            # the FP64 path is bound by the FP64 pipe: its arithmetic roofline
            mlups = res["channel"]["fp64_yu"]["MLUPS"]
            pk = peaks["fp64_fma_tflops"]
            res["channel"]["fp64_yu"]["alu"] = {
                "bound": "alu", "fp64_flops_per_lup": counts[0], "achieved_tflops": round(mlups * counts[0] / 1e6, 4),
                "peak_tflops": pk, "frac": round(mlups * counts[0] / 1e6 / pk, 4),
                "fp64_pipe_frac": round(mlups * 1e6 * counts[1] / (pk * 1e12 / 2), 4)}
        lat.close()
        torch.cuda.empty_cache()
    # Smagorinsky variants on the same channel: the lagged closure (tau stored from the previous
    # step, 8 more bytes per node update) and the deviatoric closure in closed form; their rate,
    # and their difference from the implicit closure after 1000 steps from the same start
    T = 1000
    for formula in ("yu", "chai"):
        ref = make_lattice("fp32", formula)
        ref.step(T)
        _, u_ref = ref.macroscopic()
        S_ref = ref.strain_rate(formula)
        ref.close()
        for closure, extra in (("smag_lagged", 8), ("smag_dev", 0)):
            lat = make_lattice("fp32", formula, closure=closure)
            k_ms = step_ms(lat, steps, max(3, args.warmup // 10))
            row = rate(lat.N, k_ms, BYTES_PER_LUP["fp32"] + extra, hbm)
            lat.close()
            lat = make_lattice("fp32", formula, closure=closure)
            lat.step(T)
            _, u = lat.macroscopic()
            S = lat.strain_rate(formula)
            row["u_rel_l2_vs_implicit_t1000"] = float((u - u_ref).norm() / u_ref.norm())
            row["S_rel_l2_vs_implicit_t1000"] = float((S - S_ref).norm() / S_ref.norm())
            res["channel"]["fp32_%s_%s" % (formula, closure)] = row
            lat.close()
            del u, S
        del u_ref, S_ref
        torch.cuda.empty_cache()
    # the same channel on D3Q15 (d'Humieres basis; Yu-type formula of the Sec. 5.4 procedure)
    for precision, formula in (("fp32", "yu"), ("fp32", "chai"), ("fp16s", "yu"), ("fp16s", "chai")):
        lat = make_lattice(precision, formula, lattice=15)
        k_ms = step_ms(lat, steps, max(3, args.warmup // 10))
        res["channel"]["d3q15_%s_%s" % (precision, formula)] = rate(lat.N, k_ms, 2 * 15 * (4 if precision == "fp32" else 2),
                                                                    hbm)
        lat.close()
        torch.cuda.empty_cache()
    for name, fn in (("box512", box512), ("precision64", precision64), ("cavity4096", cavity4096),
                     ("adjoint128", adjoint128), ("tgv32", tgv32)):
        try:
            res[name] = fn(args, hbm)
        except Exception as e:  # report, keep the headline line
            res[name] = {"error": repr(e)[:300]}
        torch.cuda.empty_cache()
    return res


def step_ms(lat, steps, warmup):
    """Average time of one step among `steps` back-to-back step launches (ms): the same measure
    as the headline's timed region."""
    return time_steps(lat, steps, warmup) / steps


def rate(N, k_ms, bytes_per_lup, hbm):
    gbs = bytes_per_lup * N / (k_ms * 1e-3) / 1e9
    return {"MLUPS": round(N / (k_ms * 1e-3) / 1e6, 1), "GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4),
            "kernel_ms": round(k_ms, 5)}


def box_lattice(n, precision, formula, kmax, rms, seed, with_force=None, closure="smag"):
    from paper_1704_07559_gb300 import inputs as I
    from paper_1704_07559_gb300 import lbm

    kw = {}
    if with_force is not None:
        kw["force_field"] = with_force
    lat = lbm.Lattice(lbm.D3Q19, n, n, n, rates=RATES, precision=precision, closure=closure, smag_cs=CS,
                      formula=formula, **kw)
    drho, u = I.random_fourier(n, n, n, kmax=kmax, rms=rms, seed=seed, device="cuda")
    lat.init(drho, u)
    del drho, u
    return lat


def box512(args, hbm):
    """Reduced-precision workload: 512^3 periodic Smagorinsky box, divergence-free random Fourier
    start (|k| <= 8, rms 0.03, seed 4); FP32, FP16S and BF16S storage, both routes."""
    import torch

    out = {}
    n = 512
    for precision in ("fp32", "fp16s", "bf16s"):
        for formula in ("yu", "chai"):
            lat = box_lattice(n, precision, formula, 8, 0.03, 4)
            k_ms = step_ms(lat, 30, 5)
            out["%s_%s" % (precision, formula)] = rate(lat.N, k_ms, BYTES_PER_LUP[precision], hbm)
            lat.close()
            torch.cuda.empty_cache()
    return out


def precision64(args, hbm):
    """Error of FP32 / FP16S / BF16S storage against FP64 on a 64^3 instance of the same field:
    relative L2 and max errors of u and S after 100 and 1000 steps (the FP64 path itself matches
    the FP64 oracle to 1e-12 per step, checked by the parity tests)."""
    out = {}
    n = 64
    ref = box_lattice(n, "fp64", "yu", 8, 0.03, 4)
    lats = {p: box_lattice(n, p, "yu", 8, 0.03, 4) for p in ("fp32", "fp16s", "bf16s")}
    done = 0
    for mark in (100, 1000):
        ref.step(mark - done)
        for lat in lats.values():
            lat.step(mark - done)
        done = mark
        _, ur = ref.macroscopic()
        Sr = ref.strain_rate("yu")
        for p, lat in lats.items():
            _, u = lat.macroscopic()
            S = lat.strain_rate("yu")
            eu, eS = u.double() - ur, S.double() - Sr
            out["%s_t%d" % (p, mark)] = {
                "u_rel_l2": float(eu.norm() / ur.norm()), "u_rel_max": float(eu.abs().max() / ur.abs().max()),
                "S_rel_l2": float(eS.norm() / Sr.norm()), "S_rel_max": float(eS.abs().max() / Sr.abs().max())}
    for lat in [ref] + list(lats.values()):
        lat.close()
    return out


CAVITY_U, CAVITY_RE = 0.05, 1000.0


def cavity_lattice(Lc, nidx, formula):
    """D2Q9 power-law lid-driven cavity of side Lc, lid velocity 0.05 on the +y face, consistency
    K = U^(2-n) L^n / Re with Re = 1000, fluid at rest at t = 0, FP32 populations."""
    import torch
    from paper_1704_07559_gb300 import lbm

    U = CAVITY_U
    tau_ref = 0.5 + 3 * U * Lc / CAVITY_RE
    r9 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 1 / tau_ref, 1 / tau_ref]
    K = U ** (2 - nidx) * Lc ** nidx / CAVITY_RE
    lat = lbm.Lattice(lbm.D2Q9, Lc, Lc, 1, rates=r9, precision="fp32", closure="powerlaw", formula=formula,
                      pl_n=nidx, pl_k=K, pl_tau_min=0.505, pl_tau_max=5.0, bc=["wall", "wall", "wall", "lid"],
                      lid_u={3: (U, 0.0, 0.0)})
    lat.init(torch.zeros((1, Lc, Lc), dtype=torch.float64, device="cuda"),
             torch.zeros((2, 1, Lc, Lc), dtype=torch.float64, device="cuda"))
    return lat


def cavity4096(args, hbm):
    """D2Q9 power-law lid-driven cavity, 4096^2, lid velocity 0.05, n in {0.5, 1, 1.5}, consistency
    K = U^(2-n) L^n / Re with Re = 1000, tau solved per node by fixed point, fluid at rest at t = 0."""
    out = {}
    for nidx in (0.5, 1.0, 1.5):
        for formula in ("chai", "yu"):
            lat = cavity_lattice(4096, nidx, formula)
            k_ms = step_ms(lat, 50, 20)
            out["n%.1f_%s" % (nidx, formula)] = rate(lat.N, k_ms, 72, hbm)
            lat.close()
    return out


ADJ_N, ADJ_T, ADJ_SEG = 128, 256, 16


def adjoint_lattice(precision="fp32", g=None):
    """Adjoint workload lattice: 128^3 periodic Smagorinsky box bound to the force field g
    (default N(0, (1e-5)^2), seed 5), started from the random Fourier field |k| <= 4, rms 0.01
    (seed 6)."""
    import torch
    from paper_1704_07559_gb300 import inputs as I

    n = ADJ_N
    if g is None:
        g = torch.from_numpy(I.gaussian_force(3, (n, n, n), std=1e-5, seed=5))
    return box_lattice(n, precision, "yu", 4, 0.01, 6, with_force=g)


def adjoint128(args, hbm):
    """Adjoint workload: 128^3 periodic Smagorinsky box, force field N(0, (1e-5)^2) (seed 5),
    start from the random Fourier field |k| <= 4, rms 0.01 (seed 6); dL/dg of the dissipation
    after T = 256 steps with checkpoints every 16 steps.  Reports the forward time of T steps, the
    time of lbm_adjoint (forward with checkpoints + functional + reverse sweep with recompute),
    and their ratio."""
    import torch

    T, seg = ADJ_T, ADJ_SEG
    lat = adjoint_lattice("fp32")
    f0 = lat.get_state().clone()
    lat.step(5)
    torch.cuda.synchronize()
    s = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fwd = []
    for _ in range(3):
        lat.set_state(f0)
        e0.record(s)
        lat.step(T)
        e1.record(s)
        torch.cuda.synchronize()
        fwd.append(e0.elapsed_time(e1))
    lat.set_state(f0)
    lat.adjoint(T, seg)  # warm-up
    adj = []
    for _ in range(3):
        lat.set_state(f0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, grad = lat.adjoint(T, seg)
        adj.append((time.perf_counter() - t0) * 1e3)
    f_ms, a_ms = min(fwd), min(adj)
    lat.close()
    return {"T": T, "seg": seg, "loss": loss, "grad_rms": float(grad.pow(2).mean().sqrt()),
            "forward_ms": round(f_ms, 3), "adjoint_total_ms": round(a_ms, 3),
            "reverse_over_forward": round((a_ms - f_ms) / f_ms, 3), "total_over_forward": round(a_ms / f_ms, 3)}


TGV_N, TGV_U0, TGV_TAU, TGV_STEPS = 32, 0.02, 0.6, 500


def tgv_rates():
    r = list(RATES)
    for k in (9, 11, 13, 14, 15):
        r[k] = 1 / TGV_TAU
    return r


def tgv_lattice(formula="yu"):
    """D3Q19 FP64 32^3 periodic Taylor-Green vortex, u0 = 0.02, tau = 0.6, Newtonian."""
    from paper_1704_07559_gb300 import inputs as I
    from paper_1704_07559_gb300 import lbm

    lat = lbm.Lattice(lbm.D3Q19, TGV_N, TGV_N, TGV_N, rates=tgv_rates(), precision="fp64", closure="newton",
                      formula=formula)
    drho, u, g = I.taylor_green_3d(TGV_N, u0=TGV_U0)
    lat.init(drho, u, g)
    return lat


def tgv32(args, hbm):
    """Correctness workload: D3Q19 FP64, 32^3 periodic Taylor-Green vortex u0 = 0.02, tau = 0.6,
    500 steps; S by Yu and by Chai, their difference, and the decay of S against the linear
    (Stokes) rate exp(-3 nu k^2 t) of this non-exact flow."""
    n, tau, T = TGV_N, TGV_TAU, TGV_STEPS
    lat = tgv_lattice()
    S0 = lat.strain_rate("yu").abs().max().item()
    k_ms = step_ms(lat, T, 0)
    Sy, Sc = lat.strain_rate("yu"), lat.strain_rate("chai")
    nu, kk = (tau - 0.5) / 3, 2 * np.pi / n
    ratio = Sy.abs().max().item() / S0 / np.exp(-3 * nu * kk * kk * T)
    lat.close()
    return {"steps": T, "MLUPS": round(n ** 3 / (k_ms * 1e-3) / 1e6, 1),
            "yu_minus_chai_rel": float((Sy - Sc).abs().max() / Sy.abs().max()),
            "S_amplitude_over_stokes_decay": round(ratio, 5)}


# ------------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores


def _reference_worker(job):
    """One host process of the reference arm: `warmup` untimed and `steps` timed oracle steps on
    its own copy of a channel sub-box; returns (nodes, seconds of the timed steps)."""
    dims, warmup, steps = job
    Gr, f, F = _oracle_channel_box(*dims)
    for _ in range(warmup):
        f, _ = Gr.step(f, force=F)
    t0 = time.perf_counter()
    for _ in range(steps):
        f, _ = Gr.step(f, force=F)
    return Gr.N, time.perf_counter() - t0


def reference_subbox(steps, warmup):
    """The sub-box each host process of the oracle arms steps, ((nx, 32, 32), one thread's rate in
    node updates per second): nx from a calibration step so that warmup + steps steps take about
    90 s, at most the channel's 256."""
    Gc, fc, F = _oracle_channel_box(16, 32, 16)
    t0 = time.perf_counter()
    Gc.step(fc, force=F)
    rate = Gc.N / (time.perf_counter() - t0)
    nodes = rate * 90.0 / (steps + warmup)
    return (int(max(1, min(NX, nodes // (32 * 32)))), 32, 32), rate


def reference_sample(cores, dims):
    return ("%d processes (one per host core), each an %dx%dx%d sub-box of the channel (walls at y) per step, "
            "FP64 oracle, Yu route" % ((cores,) + tuple(dims)))


def run_reference(args):
    """The oracle as it stands on the host cores: one spawned process per core, each stepping its
    own nx x 32 x 32 sub-box of the channel (walls at y, same rates, closure and force), nx sized
    from a calibration step so that warm-up + timed steps take about 90 s.  Value = all
    processes' node updates / the slowest process's timed steps."""
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle as O

    O.lib()  # built once before the workers start
    dims, _ = reference_subbox(args.steps, args.warmup)
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_reference_worker, [(dims, args.warmup, args.steps)] * cores)
    dt = max(r[1] for r in res)
    value = sum(r[0] for r in res) * args.steps / dt / 1e6
    sample = reference_sample(cores, dims)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "lattice": "D3Q19", "grid": [NX, NY, NZ], "formula": "yu",
                      "closure": "smagorinsky"},
           "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                            "sample": sample, "host_cpu": host_cpu()},
           "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16s", "bf16s", "fp64"])
    ap.add_argument("--formula", default="yu", choices=["yu", "chai"])
    ap.add_argument("--closure", default="smag", choices=["smag", "smag_lagged", "smag_dev"],
                    help="the channel's Smagorinsky closure: implicit (default), lagged or deviatoric closed form")
    ap.add_argument("--lattice", type=int, default=19, choices=[19, 15],
                    help="19: the D3Q19 channel (default); 15: the same channel on D3Q15")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="replicas: one channel per rank (default, weak scaling); slab: one channel cut into "
                         "z-slabs over the ranks, halos exchanged every step (strong scaling)")
    ap.add_argument("--workload", default="channel", choices=["channel", "cavity", "box"],
                    help="channel: the headline (default); cavity: the D2Q9 power-law 4096^2 cavity (FP32); box: "
                         "the periodic Smagorinsky box (--box-n); the last two print the timed line only")
    ap.add_argument("--n-index", type=float, default=0.5, help="the cavity's power-law index n")
    ap.add_argument("--box-n", type=int, default=512, help="the box's side")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--quick", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "cavity" and args.precision != "fp32":
        ap.error("the cavity runs FP32 populations")
    if args.impl == "reference":
        run_reference(args)
    elif args.decomp == "slab":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
