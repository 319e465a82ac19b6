"""Benchmark: fused D3Q19 MRT lattice Boltzmann step with the Smagorinsky closure fed by the
strain rate (Yu's or Chai's formula), FP32 populations, on a 256 x 128 x 128 channel with
halfway bounce-back walls at the y faces and a uniform body force g_x = 1e-6.

One benchmark step is one lattice time step over the whole grid (one kernel launch: pull-stream,
moments, strain rate, closure, relaxation, force, store).  The metric is MLUPS (million lattice
node updates per second) and the fraction of the measured HBM bandwidth that the minimum
traffic (19 populations read + 19 written, 152 bytes per node update) represents.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|fp16s|bf16s|fp64] [--formula yu|chai] [--no-variants] [--quick]

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
BC = ["periodic", "periodic", "wall", "wall", "periodic", "periodic"]
BYTES_PER_LUP = {"fp32": 152, "fp64": 304, "fp16s": 76, "bf16s": 76}
STORAGE_NOTE = {"fp32": "fp32 populations, fp32 arithmetic", "fp64": "fp64 populations, fp64 arithmetic",
                "fp16s": "fp16 populations (delta-rho form), fp32 arithmetic",
                "bf16s": "bf16 populations (delta-rho form), fp32 arithmetic"}
WORKLOAD = "D3Q19 MRT Smagorinsky LES channel 256x128x128, walls at y, g_x=1e-6, Cs=0.17, tau0=0.51"
METRIC = "MLUPS, MRT step + strain rate (Smagorinsky LES channel)"


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


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


def make_lattice(precision="fp32", formula="yu", dims=(NX, NY, NZ)):
    from paper_1704_07559_gb300 import inputs as I
    from paper_1704_07559_gb300 import lbm

    lat = lbm.Lattice(lbm.D3Q19, *dims, rates=RATES, force=[G, 0.0, 0.0], precision=precision, closure="smag",
                      smag_cs=CS, formula=formula, bc=BC)
    drho, u = I.channel_profile(*dims, u_centre=0.1, noise=0.01, seed=2)
    lat.init(drho, u)
    return lat


def time_steps(lat, steps, warmup, per_launch=False):
    """Device time of `steps` lattice steps (ms) via CUDA events on the library's stream."""
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
    for _ in range(steps):
        lat.step(1)
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


def cpu_baseline(seconds_budget=15.0):
    """The FP64 oracle on the host cores, on a 64 x 32 x 32 sub-box of the same channel
    (same rates, closure, force and walls), Yu route, as many steps as fit the budget."""
    import oracle as O
    from paper_1704_07559_gb300 import inputs as I

    nx, ny, nz = 64, 32, 32
    p = O.make_params(19, RATES, closure=O.SMAG, smag_cs=CS, formula=O.YU,
                      bc=[O.PERIODIC, O.PERIODIC, O.WALL, O.WALL, O.PERIODIC, O.PERIODIC])
    Gr = O.Grid(p, nx, ny, nz)
    drho, u = I.channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2)
    F = np.array([G, 0.0, 0.0])
    f = Gr.init(drho, u, force=F)
    t0 = time.perf_counter()
    steps = 0
    while True:
        f, _ = Gr.step(f, force=F)
        steps += 1
        if time.perf_counter() - t0 > seconds_budget or steps >= 200:
            break
    dt = time.perf_counter() - t0
    return {"value": round(nx * ny * nz * steps / dt / 1e6, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%dx%dx%d sub-box of the channel, %d steps, FP64, Yu route, single thread" % (nx, ny, nz, steps)}


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
    lat = make_lattice(args.precision, args.formula)
    N = lat.N

    # timed region: barrier + synchronize on both sides, max over ranks
    lat.step(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    with ClockSampler(gpu_index) as clk:
        ms = time_steps(lat, args.steps, 0)
        torch.cuda.synchronize()
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    ms_per_step = ms / args.steps
    value = world * N * args.steps / (ms * 1e-3) / 1e6

    # kernel duration per launch for the roofline (events around each launch)
    per = time_steps(lat, min(args.steps, 500), 0, per_launch=True)
    k_ms = statistics.mean(per)
    achieved = BYTES_PER_LUP[args.precision] * N / (k_ms * 1e-3) / 1e9

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "D3Q19", "grid": [NX, NY, NZ], "formula": args.formula,
                   "closure": "smagorinsky", "precision": STORAGE_NOTE[args.precision],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (two 319 MB population buffers per step)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None, "peak_kind": peak_kind,
                     "kernel": "k_step<D3Q19,%s,SMAG,%s,force>" % (args.precision, args.formula.upper()),
                     "bytes_per_lup": BYTES_PER_LUP[args.precision],
                     "kernel_ms": round(k_ms, 5)},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and args.quick:
        print(json.dumps(out), flush=True)
    elif rank == 0:
        # end to end through the C ABI with host buffers
        e2e_s, h2d, d2h = time_e2e(lat, max(3, min(args.steps, 50)))
        out["e2e"] = {"value": round(world * N / e2e_s / 1e6, 2), "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h}
        if not args.no_variants:
            out["variants"] = variants(args, hbm)
        if world == 1:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)
    lat.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def variants(args, hbm):
    """The other (formula x form) pairs on the same channel, same timing protocol."""
    import torch

    res = {}
    steps = max(10, min(args.steps, 1000))
    for precision, formula in (("fp32", "chai"), ("fp16s", "yu"), ("fp16s", "chai"), ("bf16s", "yu"),
                               ("bf16s", "chai"), ("fp64", "yu"), ("fp64", "chai")):
        lat = make_lattice(precision, formula)
        n = steps if precision != "fp64" else max(5, steps // 10)
        per = time_steps(lat, n, max(3, args.warmup // 10), per_launch=True)
        k_ms = statistics.mean(per)
        gbs = BYTES_PER_LUP[precision] * lat.N / (k_ms * 1e-3) / 1e9
        res["%s_%s" % (precision, formula)] = {"MLUPS": round(lat.N / (k_ms * 1e-3) / 1e6, 1),
                                              "GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4)}
        lat.close()
        torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores


def run_reference(args):
    """The oracle as it stands, one bounded sub-box of the channel per step, sized from a
    calibration step so that warm-up + timed steps take about 90 s in total."""
    rank = env_int("RANK", 0)
    if rank != 0:
        return
    import oracle as O
    from paper_1704_07559_gb300 import inputs as I

    O.lib()
    p = O.make_params(19, RATES, closure=O.SMAG, smag_cs=CS, formula=O.YU,
                      bc=[O.PERIODIC, O.PERIODIC, O.WALL, O.WALL, O.PERIODIC, O.PERIODIC])
    F = np.array([G, 0.0, 0.0])

    def box(nx, ny, nz):
        Gr = O.Grid(p, nx, ny, nz)
        drho, u = I.channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2)
        return Gr, Gr.init(drho, u, force=F)

    Gc, fc = box(16, 32, 16)
    t0 = time.perf_counter()
    Gc.step(fc, force=F)
    rate = Gc.N / (time.perf_counter() - t0)
    nodes = rate * 90.0 / (args.steps + args.warmup)
    nx = int(max(1, min(NX, nodes // (32 * 32))))
    Gr, f = box(nx, 32, 32)
    for _ in range(args.warmup):
        f, _ = Gr.step(f, force=F)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, _ = Gr.step(f, force=F)
    dt = time.perf_counter() - t0
    value = Gr.N * args.steps / dt / 1e6
    sample = "%dx32x32 sub-box of the channel per step (walls at y), FP64 oracle, Yu route, single thread" % nx
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "lattice": "D3Q19", "grid": [NX, NY, NZ], "formula": "yu",
                      "closure": "smagorinsky"},
           "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                            "sample": sample},
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
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--quick", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
