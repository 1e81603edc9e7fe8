"""Benchmark of the GALS step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload vortex4096|rotation4096|deform512|batch256|surrogate2048]
                    [--layout full|compact]

A bench step is one GALS time step (trace + Jacobian, Hermite evaluation, gradient
write-back and mixed-derivative reconstruction) over the whole grid.  The default
workload is the 4096^2 FP32 single-vortex case (state 4 float32 planes per node, 268 MB
per buffer, larger than the 129 MB L2, so no flush is needed between steps).
The K timed steps are issued as one gals_step call (a CUDA-graph replay), bracketed by
CUDA events on the grid's stream.  Prints ONE JSON line.

--impl reference times the FP64 CPU oracle (the reference of this method) on the host
cores, on bounded row bands of the same workload.
Under torchrun (N > 1) every rank advances an independent replica (the method runs on
one GPU per problem; there is no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GALS node-updates/s and % of HBM roofline; learned vs plain trace at equal error"
UNIT = "node-updates/s"

WORKLOADS = {
    # name: (dim, n, velocity kwargs, dt rule, description)
    "vortex4096": dict(dim=2, n=(4096, 4096), vel=dict(kind="vortex2d", T=8.0), vmax=1.0,
                       desc="2D GALS 4096x4096 nodes on [0,1]^2, FP32, single vortex T=8, "
                            "circle SDF r=0.15 at (0.5,0.75), superconsistent RK3 trace, CFL 1"),
    "rotation4096": dict(dim=2, n=(4096, 4096), vel=dict(kind="rotation", omega=2 * math.pi,
                                                         center=(0.5, 0.5, 0.0)), vmax=math.pi,
                         desc="2D GALS 4096x4096, FP32, Zalesak slotted disk in rigid rotation "
                              "(omega=2pi about (0.5,0.5)), RK3 trace, CFL 1"),
    "deform512": dict(dim=3, n=(512, 512, 512), vel=dict(kind="deform3d", T=3.0), vmax=2.0,
                      desc="3D GALS 512^3 nodes on [0,1]^3, FP32, LeVeque deformation T=3, "
                           "sphere SDF r=0.15 at (0.35,0.35,0.35), RK3 trace, CFL 1"),
    "zalesak512": dict(dim=3, n=(512, 512, 512), vel=dict(kind="rotation", omega=2 * math.pi,
                                                        center=(0.5, 0.5, 0.5)), vmax=math.pi,
                       desc="3D GALS 512^3 nodes on [0,1]^3, FP32, Zalesak's slotted sphere "
                            "(r=0.15 at (0.5,0.75,0.5), slot width 0.05, depth 0.25) in rigid "
                            "rotation about the z-axis through (0.5,0.5) (omega=2pi), RK3 "
                            "trace, CFL 1"),
    "fourier4096": dict(dim=2, n=(4096, 4096), vel=dict(kind="fourier2d"), vmax=None, nmodes=16,
                        desc="2D GALS 4096x4096 nodes on [0,1]^2, FP32, time-periodic (period 1) "
                             "stream-function field of 16 Fourier modes (seed 9053409), circle SDF "
                             "r=0.15 at (0.5,0.75), RK3 trace, CFL 1 (the batched mode's field "
                             "kind on one grid larger than L2, for profiling its tile code)"),
    "batch256": dict(dim=2, n=None, batch=256, vel=dict(kind="fourier2d"), vmax=None,
                     desc="Batched 2D GALS, FP32: 256 independent problems, side lengths uniform "
                          "in [128,1024] (seed 9053409), each an ellipse SDF advected by its own "
                          "steady 8-mode Fourier stream-function field, RK3 trace, CFL 1; one "
                          "launch per step over all problems' tiles, CUDA-graph time loop, "
                          "autotuned launch shape"),
    "surrogate2048": dict(dim=2, n=(2048, 2048), vel=dict(kind="fourier2d"), vmax=None,
                          surrogate=True, nmodes=16,
                          desc="2D GALS 2048x2048 nodes on [0,1]^2, FP32, time-periodic (period 1) "
                               "stream-function field of 16 Fourier modes (seed 9053409), circle "
                               "SDF r=0.15 at (0.5,0.75), CFL 1; learned flow-map trace (MLP "
                               "3-128x4-6 on the tensor cores, FP16 inference, trained on 32-sub-step RK4 "
                               "targets) with per-tile RK3 residual check and fallback, against "
                               "the plain RK3 trace"),
    "waves2048": dict(dim=2, n=(2048, 2048), vel=dict(kind="waves2d"), vmax=None,
                      surrogate=True, nwaves=256,
                      desc="2D GALS 2048x2048 nodes on [0,1]^2, FP32, costly velocity: time-periodic "
                           "(period 1) stream function of 256 plane waves of random direction, "
                           "|k| in [pi, 4 pi] (seed 9053409; one sine and cosine per wave per "
                           "evaluation), circle SDF r=0.15 at (0.5,0.75), CFL 1; learned flow-map "
                           "trace (MLP 3-128x4-6 on the tensor cores, FP16 inference, trained on 32-sub-step RK4 "
                           "targets) with per-tile RK3 residual check, against the plain RK3 trace "
                           "at the same step and at larger steps (equal interface error)"),
    # a smaller case of the same 3D kernel, for profiler captures (state still > L2)
    "deform256": dict(dim=3, n=(256, 256, 256), vel=dict(kind="deform3d", T=3.0), vmax=2.0,
                      desc="3D GALS 256^3 nodes on [0,1]^3, FP32, LeVeque deformation T=3, "
                           "sphere SDF r=0.15 at (0.35,0.35,0.35), RK3 trace, CFL 1"),
}


def bytes_per_node(dim, layout):
    """Algorithmic bytes per node update: the stored state read once and written once."""
    planes = (4 if dim == 2 else 8) if layout == "full" else (3 if dim == 2 else 4)
    return 2 * 4 * planes


def wl_modes(wl):
    from paper_0905_3409_gb300 import inputs
    if wl.get("nwaves"):
        return inputs.wave_modes(wl["nwaves"], seed=inputs.DEFAULT_SEED)
    if not wl.get("nmodes"):
        return None
    return inputs.fourier_modes(wl["nmodes"], seed=inputs.DEFAULT_SEED, periodic=True)


def wl_dt(wl):
    """CFL 1: dt = h / max|v_i| (the Fourier field's analytic speed bound; for the plane
    waves, whose sum bound is far above the field's speed, the sampled speed times 1.1)."""
    from paper_0905_3409_gb300 import inputs
    h = 1.0 / (wl["n"][0] - 1)
    modes = wl_modes(wl)
    if wl.get("nwaves"):
        return h / inputs.wave_speed_sampled(modes)
    return h / (inputs.fourier_speed_bound(modes) if modes is not None else wl["vmax"])


def wl_oracle_velocity(wl):
    import oracle
    v = wl["vel"]
    return oracle.velocity(v["kind"], T=v.get("T", 1.0), omega=v.get("omega", 0.0),
                           center=v.get("center", (0.5, 0.5, 0.5)), modes=wl_modes(wl))


def measured_peaks(kind="hbm"):
    """(peak, source): HBM copy GB/s, or dense BF16 TFLOP/s of a burst ("bf16")."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    key, fallback = ("hbm_gbs", 6800.0) if kind == "hbm" else ("bf16_tflops", 1900.0)
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if key in d:
            return float(d[key]), "measured"
    return fallback, "fallback"


def initial_state(wl):
    from paper_0905_3409_gb300 import inputs
    n = wl["n"]
    if wl["dim"] == 2:
        if wl["vel"]["kind"] == "rotation":
            st = inputs.slotted_disk_sdf(n)
        else:
            st = inputs.circle_sdf(n)
    elif wl["vel"]["kind"] == "rotation":
        return inputs.slotted_sphere_sdf(n, dtype=np.float32)
    else:
        return inputs.sphere_sdf(n, dtype=np.float32)
    return st.astype(np.float32)


def initial_state_cached(name, wl):
    """The 512^3 signed distance takes a while in numpy; cache it per process run."""
    return initial_state(wl)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            if len(s) < 9:
                continue
            for nm, v in zip(names, s[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


SPIN_CYCLES = 200_000  # ~0.1 ms at 2 GHz: covers the host's graph submission
TIMING_S = 1.0         # timed load per measurement (--timing-s)


def time_windows(step_k, stream, R, min_s=None, min_windows=5, max_windows=4000):
    """CUDA-event times (ms) of repeated windows of K steps on `stream`.  Each window is
    bracketed by a barrier and a device synchronise on both sides; a short spin kernel
    queued on the stream ahead of the first event keeps the host's submission of the
    K-step graph out of the window.  The number of windows makes at least `min_s` of
    timed load (so that the clock samples cover a steady state); every rank runs the
    same number, from the slowest rank's first window."""
    import torch
    from paper_0905_3409_gb300 import replicas
    if min_s is None:
        min_s = TIMING_S

    def one():
        replicas.barrier(R)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            torch.cuda._sleep(SPIN_CYCLES)
        e0.record(stream)
        step_k()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    first = replicas.max_over_ranks(R, one(), device="cuda")
    n = int(min(max(math.ceil(min_s * 1e3 / max(first, 1e-3)), min_windows), max_windows))
    wins = [one() for _ in range(n)]
    replicas.barrier(R)
    return wins


def window_summary(wins):
    w = np.asarray(wins)
    return {"count": int(w.size), "median_ms": float(np.median(w)), "min_ms": float(w.min()),
            "max_ms": float(w.max()), "timed_s": float(w.sum() / 1e3)}


def gpu_numa_node(index):
    """Host NUMA node nearest to GPU `index` (its PCI device's numa_node), or None."""
    try:
        out = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True, timeout=20).stdout
        bdf = out.strip().splitlines()[0].strip().lower()
        dom, rest = bdf.split(":", 1)
        bdf = f"{int(dom, 16):04x}:{rest}"
        with open(f"/sys/bus/pci/devices/{bdf}/numa_node") as f:
            node = int(f.read().strip())
        return node if node >= 0 else None
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None


def node_cpus(node):
    """CPU ids of a NUMA node (from sysfs), or None."""
    try:
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            spec = f.read().strip()
    except OSError:
        return None
    cpus = set()
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus or None


def pinned_near_gpu(local, arrays):
    """Page-locked copies of `arrays`, allocated by this thread while it runs on the CPUs of
    the GPU's nearest NUMA node (pages are placed where they are first touched), and the
    measured host-to-device and device-to-host copy rates of the first one (GB/s, CUDA
    events, 3 copies each way)."""
    import torch
    node = gpu_numa_node(local)
    cpus = node_cpus(node) if node is not None else None
    old = os.sched_getaffinity(0)
    if cpus:
        os.sched_setaffinity(0, cpus)
    try:
        pins = [torch.from_numpy(a).pin_memory() for a in arrays]
        pins.append(torch.empty_like(pins[0]).pin_memory())
    finally:
        os.sched_setaffinity(0, old)
    dev = torch.empty(pins[0].shape, dtype=pins[0].dtype, device="cuda")
    rates = {}
    for name, dst, src in (("h2d_gbs", dev, pins[0]), ("d2h_gbs", pins[-1], dev)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        rates[name] = 3 * src.numel() * src.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev
    info = {"numa_node": node, "cpu_affinity_for_allocation": f"node {node}" if cpus else "unchanged",
            **rates}
    return pins, info


# the sources that define each benchmarked kernel: a recorded DRAM traffic figure is
# reported only while these files are unchanged
KERNEL_SOURCES = {
    2: ["step2d.cu", "step2d_tile.cuh", "gals_pair.cuh", "gals_device.cuh", "tma.cuh", "capi.cu"],
    3: ["step3d.cu", "step3d_common.cuh", "gals_pair.cuh", "gals_device.cuh", "tma.cuh"],
}


def kernel_source_hash(dim=None):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0905_3409_gb300", "csrc")
    names = KERNEL_SOURCES[dim] if dim in KERNEL_SOURCES else sorted(
        fn for fn in os.listdir(csrc) if fn.endswith((".cu", ".cuh", ".h")))
    for fn in names:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, layout):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{workload}/{layout}")
    if not e or e.get("kernel_sources") != kernel_source_hash(WORKLOADS[workload]["dim"]):
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------- CPU oracle leg

def oracle_state(wl, g, slab=None):
    """FP64 initial state for the oracle.  In 3D only the z-slices of `slab` (with a
    margin of 2 for the feet) are filled: a band update reads nothing else."""
    import oracle
    from paper_0905_3409_gb300 import inputs
    n = wl["n"]
    if wl["dim"] == 2:
        return oracle.recon_cross(g, initial_state(wl).astype(np.float64))
    st = np.zeros((8, n[2], n[1], n[0]))
    z0, z1 = max(slab[0] - 2, 0), min(slab[1] + 2, n[2])
    gen = inputs.slotted_sphere_sdf if wl["vel"]["kind"] == "rotation" else inputs.sphere_sdf
    st[:, z0:z1] = gen(n, z_range=(z0, z1))
    return st


def oracle_leg(wl, budget_s=12.0, max_bands=None, trace="rk3", cross="central"):
    """Time the FP64 oracle on row bands (2D) / z-slabs (3D) of the workload: each band
    is an exact, independent part of one step.  Returns (node-updates/s, cores, sample)."""
    import oracle
    n = wl["n"]
    g = oracle.grid(n)
    band3 = (n[-1] // 3, n[-1] // 3 + 8)
    st = oracle_state(wl, g, band3)
    ov = wl_oracle_velocity(wl)
    dt = wl_dt(wl)
    planes = oracle.state_planes(g, st)
    cores = oracle.default_threads()
    outer = n[-1]
    inner_nodes = int(np.prod(n[:-1]))
    band = 64 if wl["dim"] == 2 else 1
    done = 0
    nodes = 0
    t0 = time.perf_counter()
    b0 = outer // 3
    while True:
        oracle.step_band(g, ov, None, 0.0, dt, b0, b0 + band, planes=planes, trace_scheme=trace,
                         cross=cross)
        nodes += band * inner_nodes
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s or (max_bands and done >= max_bands):
            break
        b0 = b0 + band
        if wl["dim"] == 2:
            b0 %= outer - band
        elif b0 + band > band3[1]:
            b0 = band3[0]
    return nodes / el, cores, f"{done} bands of {band} {'rows' if wl['dim'] == 2 else 'z-slices'} " \
                              f"({nodes} node updates, one step each) of the {n} grid in {el:.1f} s"


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n = wl["n"]
    g = oracle.grid(n)
    band = 8 if wl["dim"] == 2 else 1
    slab = (n[-1] // 4, n[-1] // 4 + 16)
    st = oracle_state(wl, g, slab)
    ov = wl_oracle_velocity(wl)
    dt = wl_dt(wl)
    planes = oracle.state_planes(g, st)
    outer = n[-1]
    inner_nodes = int(np.prod(n[:-1]))
    # each reference step: one band of the grid, sized to keep the run within minutes
    def band_at(s):
        if wl["dim"] == 2:
            return (outer // 4 + s * band) % (outer - band)
        return slab[0] + (s * band) % (slab[1] - slab[0])
    trace, cross = args.trace, args.cross
    for s in range(args.warmup):
        b0 = band_at(s)
        oracle.step_band(g, ov, None, 0.0, dt, b0, b0 + band, planes=planes, trace_scheme=trace,
                         cross=cross)
    t0 = time.perf_counter()
    for s in range(args.steps):
        b0 = band_at(s)
        oracle.step_band(g, ov, None, s * dt, dt, b0, b0 + band, planes=planes, trace_scheme=trace,
                         cross=cross)
    el = time.perf_counter() - t0
    nodes = args.steps * band * inner_nodes
    value = nodes / el
    cores = oracle.default_threads()
    sample = f"each step: one band of {band} {'rows' if wl['dim'] == 2 else 'z-slices'} " \
             f"({band * inner_nodes} node updates) of the {n} grid"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "ranks_measured": 1,  # one CPU process on rank 0, whatever the launch's rank count
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"] + " (FP64 CPU oracle)", "nodes_per_step_sample": band * inner_nodes,
                   "trace": trace, "cross": cross},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------- batched mode

def _batch_state(args):
    """Initial state of one batch problem (top level: runs in a spawn pool)."""
    n, center, a, b, angle = args
    sys.path.insert(0, ROOT)
    from paper_0905_3409_gb300 import inputs
    return inputs.ellipse_sdf((n, n), center, a, b, angle, iters=50).astype(np.float32)


def batch_inputs(count):
    import multiprocessing as mp
    from paper_0905_3409_gb300 import inputs
    probs = inputs.batch_problems(count)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        states = pool.map(_batch_state, [(p.n, p.center, p.a, p.b, p.angle) for p in probs])
    return probs, states


def batch_oracle_leg(probs, states, budget_s=10.0):
    """FP64 oracle on bands of rows of the largest problems, one step each."""
    import oracle
    order = sorted(range(len(probs)), key=lambda k: -probs[k].n)[:4]
    nodes, t_used, done = 0, 0.0, 0
    for k in order:
        p = probs[k]
        g = oracle.grid((p.n, p.n))
        st = oracle.recon_cross(g, states[k].astype(np.float64))
        ov = oracle.velocity("fourier2d", modes=p.modes)
        planes = oracle.state_planes(g, st)
        t0 = time.perf_counter()
        b0 = p.n // 3
        while time.perf_counter() - t0 < budget_s / len(order):
            oracle.step_band(g, ov, None, 0.0, p.dt, b0, b0 + 16, planes=planes)
            nodes += 16 * p.n
            done += 1
            b0 = (b0 + 16) % (p.n - 16)
        t_used += time.perf_counter() - t0
    return nodes / t_used, oracle.default_threads(), \
        f"{done} bands of 16 rows of the 4 largest problems ({nodes} node updates, one step each)"


def run_batch(args, wl):
    import torch
    probs, states = batch_inputs(wl["batch"])  # before any CUDA work (spawned pool)
    from paper_0905_3409_gb300 import replicas
    R = replicas.init("nccl") if int(os.environ.get("WORLD_SIZE", "1")) > 1 else replicas.init()
    rank, world, local = R.rank, R.world, R.local
    torch.cuda.set_device(local if world > 1 else 0)
    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    replicas.barrier(R)
    from paper_0905_3409_gb300 import gals
    stream = torch.cuda.Stream()
    sizes = [(p.n, p.n) for p in probs]
    b = gals.Batch(sizes, layout=args.layout, stream=stream)
    for k, st in enumerate(states):
        b.set_state(k, st, recon=True)
    vels = [gals.Velocity("fourier2d", modes=p.modes) for p in probs]
    dts = [p.dt for p in probs]
    tuning = b.autotune(vels, dts, trial_steps=3)
    nodes = b.nodes
    b.step(vels, dts, args.warmup)
    b.step(vels, dts, args.steps)  # captures the timed graph
    b.synchronize()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    wins = time_windows(lambda: b.step(vels, dts, args.steps), stream, R)
    clocks = sampler.stop() if rank == 0 else None
    ms = replicas.max_over_ranks(R, float(np.median(wins)), device="cuda")
    value = replicas.throughput(nodes * args.steps, world, ms * 1e-3)
    bpn = bytes_per_node(2, args.layout)
    achieved = bpn * nodes / (ms * 1e-3 / args.steps) / 1e9
    peak, peak_kind = measured_peaks()
    # e2e: per step, every problem's state from pinned host memory, one batched step,
    # every state back to pinned host memory
    pins = [torch.from_numpy(st).pin_memory() for st in states]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for k, pin in enumerate(pins):
            b.set_state(k, pin.numpy(), recon=False)
        b.step(vels, dts, 1)
        for k in range(len(sizes)):
            b.read_state(k)
    el = time.perf_counter() - t0
    io_bytes = 16 * nodes
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "layout": args.layout, "problems": len(sizes),
                       "nodes": nodes, "bytes_per_node_update": bpn, "tuning": tuning,
                       "l2": f"inputs larger than L2 ({nodes * 16 / 1e6:.0f} MB state per buffer)",
                       "timing": "median of repeated K-step windows", "windows": window_summary(wins),
                       "parallelism": f"{world} independent replica(s), one per GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(args.workload, args.layout),
                         "peak_source": peak_kind, "kernel": "k_batch2d (1 launch per step)"},
            "e2e": {"value": nodes * e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "gpu_launches": args.steps + 2,
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            v, cores, sample = batch_oracle_leg(probs, states, budget_s=args.cpu_budget)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": sample}
        print(json.dumps(line))
    b.close()
    replicas.finish(R)


def run_reference_batch(args, wl):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    from paper_0905_3409_gb300 import inputs
    probs = inputs.batch_problems(wl["batch"])
    p = max(probs, key=lambda q: q.n)
    st = inputs.ellipse_sdf((p.n, p.n), p.center, p.a, p.b, p.angle, iters=50)
    g = oracle.grid((p.n, p.n))
    planes = oracle.state_planes(g, oracle.recon_cross(g, st))
    ov = oracle.velocity("fourier2d", modes=p.modes)
    band = 8
    for s in range(args.warmup):
        oracle.step_band(g, ov, None, 0.0, p.dt, 8 * s % (p.n - band), 8 * s % (p.n - band) + band, planes=planes)
    t0 = time.perf_counter()
    for s in range(args.steps):
        b0 = (p.n // 4 + s * band) % (p.n - band)
        oracle.step_band(g, ov, None, s * p.dt, p.dt, b0, b0 + band, planes=planes)
    el = time.perf_counter() - t0
    value = args.steps * band * p.n / el
    cores = oracle.default_threads()
    sample = f"each step: one band of {band} rows of the largest problem ({p.n}^2)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "ranks_measured": 1,  # one CPU process on rank 0, whatever the launch's rank count
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["desc"] + " (FP64 CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------- GPU leg

def run_ours(args, wl):
    import torch
    from paper_0905_3409_gb300 import replicas
    R = replicas.init("nccl") if int(os.environ.get("WORLD_SIZE", "1")) > 1 else replicas.init()
    rank, world, local = R.rank, R.world, R.local
    torch.cuda.set_device(local if world > 1 else 0)
    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    replicas.barrier(R)
    from paper_0905_3409_gb300 import gals

    n = wl["n"]
    dim = wl["dim"]
    nodes = int(np.prod(n))
    h = 1.0 / (n[0] - 1)
    modes = wl_modes(wl)
    dt = wl_dt(wl) if modes is not None else h / wl["vmax"]
    vel = gals.Velocity(trace=args.trace, modes=modes, **wl["vel"])
    st_host = initial_state(wl)
    stream = torch.cuda.Stream()
    g = gals.Grid(n, layout=args.layout, stream=stream, cross=args.cross)
    g.set_time_loop(args.loop)
    g.set_state(st_host, t0=0.0, recon=True)

    # warm-up (also captures the CUDA graph for K steps)
    g.step(vel, dt, args.warmup)
    g.step(vel, dt, args.steps)
    g.synchronize()

    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    wins = time_windows(lambda: g.step(vel, dt, args.steps), stream, R)
    clocks = sampler.stop() if rank == 0 else None
    ms = replicas.max_over_ranks(R, float(np.median(wins)), device="cuda")
    value = replicas.throughput(nodes * args.steps, world, ms * 1e-3)

    # roofline of the step: its kernel launches as the library counts them for one K-step
    # call (2D: one per row band of a step; 3D FULL: step + reconstruction; with --loop
    # persistent a 2D FULL approach-A call is one launch), plus coefficient and clock kernels
    cell = args.cross == "cell"
    call_launches = g.last_step_launches()
    persistent = args.loop == "persistent" and dim == 2 and args.layout == "full" and not cell
    # approach B stores no mixed derivatives: the step moves phi and psi only
    bpn = bytes_per_node(dim, "compact" if cell else args.layout)
    default_path = args.trace == "rk3" and not cell
    step_s = ms * 1e-3 / args.steps
    achieved = bpn * nodes / step_s / 1e9
    peak, peak_kind = measured_peaks()

    # e2e through the C ABI with host buffers: per step, the whole state from pinned host
    # memory, one step, the whole new state back to pinned host memory.  FULL layout: one
    # gals_step_host call (copies overlapped with the step in bands); COMPACT:
    # gals_set_state + gals_step + gals_read_state.
    nplanes = 4 if dim == 2 else 8
    (pin_in, pin_out), host_buffers = pinned_near_gpu(local, [st_host])
    e2e_steps = max(1, min(args.steps, 20))
    g2 = gals.Grid(n, layout=args.layout, stream=stream, cross=args.cross)
    banded = args.layout == "full" and not cell

    # FULL: a host-side time loop, each step's output array the next step's input, queued
    # with gals_step_host_async (a band's copy-in waits for the same band's copy-out of the
    # previous step) and one wait at the end of the timed region
    io = pin_out.numpy()
    io[:] = pin_in.numpy()

    def e2e_step(k):
        if banded:
            g2.step_host(vel, dt, k * dt, io, io, wait=False)
        else:
            g2.set_state(pin_in.numpy(), recon=False)
            g2.step(vel, dt, 1)
            g2.read_state(pin_out.numpy())

    e2e_step(0)
    g2.synchronize()
    torch.cuda.synchronize()
    replicas.barrier(R)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_step(k + 1)
    g2.synchronize()
    el = time.perf_counter() - t0
    el = replicas.max_over_ranks(R, el, device="cuda")
    e2e_value = replicas.throughput(nodes * e2e_steps, world, el)
    io_bytes = nplanes * 4 * nodes

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "layout": args.layout, "nodes": nodes,
                       "trace": args.trace, "cross": args.cross,
                       "dt": dt, "bytes_per_node_update": bpn, "time_loop": args.loop,
                       "l2": f"inputs larger than L2 ({nodes * nplanes * 4 / 1e6:.0f} MB state per buffer)",
                       "timing": "median of repeated K-step windows (CUDA events on the grid "
                                 "stream, barrier + synchronize around each)",
                       "windows": window_summary(wins),
                       "parallelism": f"{world} independent replica(s), one per GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic(args.workload, args.layout) if default_path else None,
                         "peak_source": peak_kind,
                         "kernel": ("k_step2d_run (persistent: the K steps in one launch)" if persistent
                                    else f"gals step ({call_launches} kernel launches per "
                                         f"{args.steps}-step call)")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes,
                    "api": ("gals_step_host_async, a host time loop (each step's output the next "
                            "step's input), one gals_synchronize per timed region") if banded
                           else "gals_set_state + gals_step + gals_read_state",
                    "host_buffers": host_buffers},
            # per timed window (one K-step call), coefficient-table and clock kernels included
            "gpu_launches": call_launches,
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            v, cores, sample = oracle_leg(wl, budget_s=args.cpu_budget, trace=args.trace,
                                          cross=args.cross)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": sample}
    g.close()
    g2.close()
    if args.workload == "vortex4096" and not args.no_secondary:
        sec = secondary_3d(args, R, local, stream)
        if rank == 0:
            line["secondary"] = sec
    if rank == 0:
        print(json.dumps(line))
    replicas.finish(R)


def sphere_state_device(n, center=(0.35, 0.35, 0.35), r=0.15):
    """phi = |x - c| - r and psi = (x - c)/|x - c| on the device (float32 planes), the
    sphere initial data of the 3D deformation test, built slice by slice."""
    import torch
    nx, ny, nz = n
    st = torch.empty((4, nz, ny, nx), dtype=torch.float32, device="cuda")
    ax = [torch.arange(m, device="cuda", dtype=torch.float64) / (m - 1) for m in n]
    dx = (ax[0] - center[0])[None, :]
    dy = (ax[1] - center[1])[:, None]
    for k in range(nz):
        dz = float(ax[2][k] - center[2])
        d = torch.sqrt(dx * dx + dy * dy + dz * dz)
        st[0, k] = (d - r).float()
        st[1, k] = (dx / d).float()
        st[2, k] = (dy / d).float()
        st[3, k] = (dz / d).float()
    return st


def secondary_3d(args, R, local, stream):
    """The 512^3 deformation workload timed in the same run with the same protocol
    (graph replay of K >= 50 steps, repeated windows, CUDA events on the grid stream)."""
    import torch
    from paper_0905_3409_gb300 import gals
    wl = WORKLOADS["deform512"]
    n = wl["n"]
    nodes = int(np.prod(n))
    dt = 1.0 / (n[0] - 1) / wl["vmax"]
    K = max(args.steps, 50)
    vel = gals.Velocity(**wl["vel"])
    g = gals.Grid(n, stream=stream)
    st = sphere_state_device(n)
    g.set_state(st, t0=0.0, recon=True)
    del st
    torch.cuda.empty_cache()
    g.step(vel, dt, args.warmup)
    g.step(vel, dt, K)  # captures the K-step graph
    g.synchronize()
    sampler = ClockSampler(local)
    if R.rank == 0:
        sampler.start()
    wins = time_windows(lambda: g.step(vel, dt, K), stream, R)
    clocks = sampler.stop() if R.rank == 0 else None
    ms = replicas_max(R, float(np.median(wins)))
    g.close()
    bpn = bytes_per_node(3, "full")
    achieved = bpn * nodes / (ms * 1e-3 / K) / 1e9
    peak, peak_kind = measured_peaks()
    return {"workload": wl["desc"], "nodes": nodes, "steps": K, "dt": dt,
            "value": nodes * K * R.world / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / K,
            "windows": window_summary(wins),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": recorded_traffic("deform512", "full"),
                         "kernel": "k_step3d + k_recon3d_tma (2 launches per step)"},
            "gpu_launches_per_window": 2 * K + 2, "clocks": clocks}


def replicas_max(R, v):
    from paper_0905_3409_gb300 import replicas
    return replicas.max_over_ranks(R, v, device="cuda")


# ---------------------------------------------------------------------- learned trace

MLP_FLOP_PER_POINT = 2 * (3 * 128 + 3 * 128 * 128 + 128 * 6)  # 100,608 (unpadded layers)


def run_surrogate(args, wl):
    """The learned flow-map trace against the plain RK3 trace on the same grid and field:
    train (timed apart), then K steps of each trace from the same initial state, timed
    with CUDA events on the grid stream; both end states are measured against a 4x finer
    in time RK3 run (interface symmetric difference, area, max |phi|/|psi| differences).
    The roofline is that of the tensor-core MLP evaluation over one grid's nodes."""
    import torch
    from paper_0905_3409_gb300 import replicas
    R = replicas.init("nccl") if int(os.environ.get("WORLD_SIZE", "1")) > 1 else replicas.init()
    rank, world, local = R.rank, R.world, R.local
    torch.cuda.set_device(local if world > 1 else 0)
    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    replicas.barrier(R)
    from paper_0905_3409_gb300 import gals

    n = wl["n"]
    nodes = int(np.prod(n))
    h = 1.0 / (n[0] - 1)
    dt = wl_dt(wl)
    modes = wl_modes(wl)
    kind = wl["vel"]["kind"]
    stream = torch.cuda.Stream()
    plain = gals.Velocity(kind, modes=modes, trace="rk3")
    S = gals.Surrogate(seed=7, stream=stream)
    rep = S.train(plain, dt, h, steps=args.train_steps, batch=16384, lr=2e-3, lr_min=1e-5)
    S.set_check(tol_x=args.tol, tol_J=args.tol, samples=4)
    learned = gals.Velocity(kind, modes=modes, trace="surrogate", surrogate=S)
    st_host = initial_state(wl)
    K = args.steps

    def timed(vel, g):
        g.set_state(st_host, t0=0.0, recon=True)
        g.step(vel, dt, args.warmup)
        g.step(vel, dt, K)           # captures the K-step graph
        g.set_state(st_host, t0=0.0, recon=True)
        g.synchronize()
        replicas.barrier(R)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(vel, dt, K)
        e1.record(stream)
        torch.cuda.synchronize()
        return replicas.max_over_ranks(R, e0.elapsed_time(e1), device="cuda")

    g_plain = gals.Grid(n, stream=stream)
    ms_plain = timed(plain, g_plain)
    g_sur = gals.Grid(n, stream=stream)
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    S.stats(reset=True)
    ms_sur = timed(learned, g_sur)
    clocks = sampler.stop() if rank == 0 else None
    tiles, falls = S.stats()
    # the network alone: no residual check (and so no fallback)
    S.set_check(tol_x=args.tol, tol_J=args.tol, samples=0)
    g_nc = gals.Grid(n, stream=stream)
    ms_nocheck = timed(learned, g_nc)
    e_nocheck = None
    S.set_check(tol_x=args.tol, tol_J=args.tol, samples=4)
    value = replicas.throughput(nodes * K, world, ms_sur * 1e-3)
    value_plain = replicas.throughput(nodes * K, world, ms_plain * 1e-3)

    # accuracy: both runs against RK3 with dt/4 over the same time
    g_fine = gals.Grid(n, stream=stream)
    g_fine.set_state(st_host, t0=0.0, recon=True)
    g_fine.step(plain, dt / 4, 4 * K)
    g_fine.synchronize()
    g0 = gals.Grid(n, stream=stream)
    g0.set_state(st_host, t0=0.0, recon=True)
    area0 = g0.diagnostics(q=4)["measure_negative"]
    acc = {}
    for name, g in (("plain_rk3", g_plain), ("surrogate", g_sur)):
        d = g.diagnostics(q=4, reference=g_fine)
        acc[name] = {"interface_symdiff": d["measure_symdiff"], "emax_phi": d["emax_phi"],
                     "emax_psi": d["emax_psi"],
                     "area_change": g.diagnostics(q=4)["measure_negative"] - area0}
    e_p, e_s = acc["plain_rk3"]["interface_symdiff"], acc["surrogate"]["interface_symdiff"]
    e_nocheck = g_nc.diagnostics(q=4, reference=g_fine)["measure_symdiff"]
    g_nc.close()

    # equal interface error: the plain trace with steps c times longer reaches the same end
    # time in K / c steps; each run's interface error against the same reference and its
    # time to the end time (CUDA events; graph captured by an untimed first run)
    sweep = []
    for c in (1, 2, 4, 5, 8, 10, 16, 20, 25, 32, 40, 50, 64, 100):
        if K % c or K // c < 4:
            continue
        gc = g_plain if c == 1 else gals.Grid(n, stream=stream)
        if c == 1:
            ms_c = ms_plain
        else:
            gc.set_state(st_host, t0=0.0, recon=True)
            gc.step(plain, c * dt, K // c)
            gc.set_state(st_host, t0=0.0, recon=True)
            gc.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gc.step(plain, c * dt, K // c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_c = e0.elapsed_time(e1)
        err = gc.diagnostics(q=4, reference=g_fine)["measure_symdiff"]
        sweep.append({"step_multiple": c, "steps": K // c, "ms_to_end_time": ms_c,
                      "interface_symdiff": err})
        if c != 1:
            gc.close()
    # the cheapest plain run whose error is at most 1.1 x the learned run's
    ok = [r for r in sweep if r["interface_symdiff"] <= 1.1 * e_s]
    best = min(ok, key=lambda r: r["ms_to_end_time"]) if ok else None
    equal_error = {
        "learned": {"ms_to_end_time": ms_sur, "interface_symdiff": e_s},
        "learned_without_check": {"ms_to_end_time": ms_nocheck, "interface_symdiff": e_nocheck},
        "plain_rk3_sweep": sweep,
        "plain_at_most_learned_error": best,
        "time_ratio_learned_over_plain": (ms_sur / best["ms_to_end_time"]) if best else None,
        "winner": (("plain_rk3" if best["ms_to_end_time"] < ms_sur else "learned") if best
                   else "learned (no plain run reached its error)"),
    }

    # roofline of the tensor-core MLP: one evaluation per node, device buffers > L2
    X = (torch.rand(nodes, 3, device="cuda", generator=torch.Generator("cuda").manual_seed(1)) * 2 - 1)
    Y = torch.empty(nodes, 6, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        S.forward_device(X.data_ptr(), nodes, Y.data_ptr())
    reps = 10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        S.forward_device(X.data_ptr(), nodes, Y.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    ms_mlp = e0.elapsed_time(e1) / reps
    achieved = MLP_FLOP_PER_POINT * nodes / (ms_mlp * 1e-3) / 1e12
    peak, peak_kind = measured_peaks("bf16")  # FP16 operands: the same dense rate as BF16

    # e2e through the C ABI with host buffers: per step, pinned host -> device state, one
    # learned step, device -> pinned host state
    pin_in = torch.from_numpy(st_host).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    e2e_steps = max(1, min(K, 20))
    g2 = gals.Grid(n, stream=stream)
    g2.set_state(pin_in.numpy(), recon=False)
    g2.step(learned, dt, 1)
    g2.read_state(pin_out.numpy())
    torch.cuda.synchronize()
    replicas.barrier(R)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g2.set_state(pin_in.numpy(), recon=False)
        g2.step(learned, dt, 1)
        g2.read_state(pin_out.numpy())
    el = time.perf_counter() - t0
    e2e_value = replicas.throughput(nodes * e2e_steps, world,
                                    replicas.max_over_ranks(R, el, device="cuda"))
    io_bytes = 4 * 4 * nodes

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_sur / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 mlp / f32 step",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "layout": "full", "nodes": nodes, "dt": dt,
                       "l2": "working set per step (2 state buffers 134 MB + trace planes 101 MB) "
                             "larger than L2",
                       "parallelism": f"{world} independent replica(s), one per GPU",
                       "residual_check": {"tol_x_cells": args.tol, "tol_J": args.tol, "samples": 4},
                       "training": {"steps": rep["steps"], "batch": 16384, "seconds": rep["seconds"],
                                    "initial_loss": rep["initial_loss"], "final_loss": rep["final_loss"]},
                       "plain_rk3": {"value": value_plain, "ms_per_step": ms_plain / K},
                       "speedup_vs_plain": value / value_plain,
                       "fallback_tiles": falls, "tiles": tiles,
                       "accuracy_vs_rk3_dt_over_4": acc,
                       "interface_error_ratio": (e_s / e_p) if e_p > 0 else None,
                       "equal_error": equal_error},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                         "kernel": f"k_infer_points (the MLP tile code of the learned trace) over "
                                   f"{nodes} points, {MLP_FLOP_PER_POINT} FLOP each, "
                                   f"{ms_mlp:.3f} ms per launch"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "gpu_launches": 2 * K + 2,  # MLP trace + Hermite step per step; coefficients, clock
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            v, cores, sample = oracle_leg(wl, budget_s=args.cpu_budget)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": sample + " (exact RK3 trace; the oracle has no "
                                              "learned trace)"}
        print(json.dumps(line))
    for g in (g_plain, g_sur, g_fine, g0, g2):
        g.close()
    S.close()
    replicas.finish(R)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vortex4096", choices=sorted(WORKLOADS))
    ap.add_argument("--layout", default="full", choices=["full", "compact"])
    ap.add_argument("--trace", default="rk3", choices=["rk3", "heun_psi", "euler"],
                    help="single-grid workloads: backward trace (Sec. 5.1; Heun-psi: Sec. 4)")
    ap.add_argument("--cross", default="central", choices=["central", "cell"],
                    help="single-grid workloads: mixed derivatives by approach A or B (Sec. 2.3)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--loop", default="launches", choices=["launches", "persistent"],
                    help="single-grid workloads: time loop of the K-step call")
    ap.add_argument("--timing-s", type=float, default=1.0,
                    help="seconds of timed load per measurement (repeated K-step windows, at least 5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: skip the 512^3 3D line timed in the same run")
    ap.add_argument("--train-steps", type=int, default=2000, help="learned trace: optimizer steps")
    ap.add_argument("--tol", type=float, default=0.05,
                    help="learned trace: residual-check tolerance (cells and Jacobian entries)")
    args = ap.parse_args()
    global TIMING_S
    TIMING_S = max(0.0, args.timing_s)
    if args.warmup < 3:
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        if wl.get("batch"):
            run_reference_batch(args, wl)
        else:
            run_reference(args, wl)
    elif wl.get("batch"):
        run_batch(args, wl)
    elif wl.get("surrogate"):
        run_surrogate(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
