"""Benchmark of the OSB-PD bond-force hot path on GB300: bond-updates/s and roofline fractions.

Workload (one "step" = one explicit time step over every bond: failure check + dilatation pass,
force + update pass): the 3D notched block of 200 x 100 x 50 particles (dx = 1 mm, delta = 3.015 dx,
~1.17e8 directed bonds, E = 30 GPa, nu = 0.2, clamp + twist, bond breaking at s0 from G0 = 50 J/m^2),
plain FP64 (the paper's precision).  The same line reports the FP32-bond / FP64-integration form on
the same workload, the batched form (256 uneven plates) as speed-ups over plain FP64, the nonlinear
bond model, adaptive dynamic relaxation and the paper's matrix scheme on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-forms] [--no-cpu]

N > 1 runs under torchrun: every rank runs an independent replica of the workload (one body fits one
GPU, so no data moves between ranks), timed between barriers; the slowest rank's time counts.
--sweep prints one line per configuration (FP64, mixed and oracle rates); --profile-target builds one
form of the workload and runs four eager steps (the command the ncu captures profile).
"""
from __future__ import annotations

import argparse
import hashlib
import re
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

METRIC = "bond-updates/sec and % HBM roofline; mixed/batched vs plain FP64 GPU at stated error"
UNIT = "bond-updates/s"
# The paper's own GPU figure, as context (other hardware, whole-run wall time): its 3D cantilever
# (386,984 nodes, horizon 3 dx, 1000 iterations) took 39.413 s on a GTX 1080 Ti in FP64 with its
# matrix scheme (Section 4.1, Example 1); with about 4.3e7 directed bonds from the lattice count that
# is about 1.1e9 directed bond-updates/s.
PAPER_CONTEXT = {"workload": "paper's 3D cantilever, 386,984 nodes, 1000 iterations (Section 4.1, Example 1)",
                 "hardware": "NVIDIA GTX 1080 Ti, FP64, MATLAB gpuArray matrix scheme",
                 "wall_s": 39.413, "derived_value": 1.1e9, "unit": UNIT,
                 "note": "derived from the printed wall time and an estimated bond count (about +-10%); context only"}
WORKLOAD = "3D linearized OSB-PD notched block 200x100x50 (1M particles), dx=1 mm, delta=3.015 dx, torsion + clamp, bond breaking (configuration 3)"

# Algorithmic work per directed bond and per particle and pass (3D, no body force).  Bytes: 4 B
# neighbour index per pass, status bit read each pass and written in pass 1; per particle the
# coordinates, displacements, velocities, theta, 1/m, flag and row pointer of the model.  FLOPs
# (FMA = 2): FLOPS_BOND is the sqrt-free form that recomputes the bond geometry every step;
# FLOPS_BOND_TABLED the per-step part of the tabled FP64 form, whose geometry terms (xi, V_j xi,
# s0 |xi|^2, G (1/m_i + 1/m_j) / |xi|^2) are computed once per family and whose i-end dilatation
# term is applied once per particle (pass 2: the bond coefficient and the force, 4 FMAs).
BYTES_BOND = {1: 4.25, 2: 4.125}
BYTES_PART = {1: 68.0, 2: 141.0}
FLOPS_BOND = {1: 19.0, 2: 28.0}
FLOPS_BOND_TABLED = {1: 10.0, 2: 8.0}
# ... and of the pair form, per directed bond: pass 1a forms the difference and dot product once per
# bond (8 flop per pair), pass 1b the theta FMA, pass 2 as in the tabled form.
FLOPS_BOND_PAIRS = {"k_pass1a_f64p": 4.0, "k_pass1b_f64p": 2.0, "k_pass2_f64t": 8.0}
# Geometrically nonlinear bonds (Eqs 1.10, 1.13), FP64, square root and divide counted as one flop
# each: pass 1 forms xi, eta, Y, |Y|^2 - |xi|^2, |xi|^2, |Y|^2, two roots, e and the theta term and
# the break test; pass 2 the same geometry, the Eq 1.14 coefficient and the force along Y / |Y|.
FLOPS_BOND_NL = {1: 36.0, 2: 44.0}
# ... and its per-step part when (xi, |xi|) come from the per-slot table and pass 1 leaves (e, 1/|Y|)
# for pass 2 (rsqrt counted as one flop).
FLOPS_BOND_NL_TABLED = {1: 29.0, 2: 19.0}
# ... and its pair form, per directed bond: pass 1a forms the geometry, root, divide and failure test
# once per bond, both entries' theta terms and the direction Y/|Y| (26 flop per pair without the
# theta sum, + 2 x 2 for the two terms, + 3 for the direction: 16.5 per directed bond), 1b adds the
# terms (1), pass 2 forms the coefficient from the tables and the force along the stored direction
# (12).
FLOPS_BOND_NL_PAIRS = {"k_pass1a_nlp": 16.5, "k_pass1b_nlp": 1.0, "k_pass2_nlp": 12.0}
# Algorithmic bytes per directed bond and per particle of each step kernel (the model above, 3D,
# no body force): the pair form's pass 1 is split between its two kernels (1a: index, status read and
# write, x and u; 1b: 1/m, theta and the row pointer), pass 2 is one kernel.
BYTES_KERNEL = {"k_pass1a_f64p": (4.25, 48.0), "k_pass1b_f64p": (0.0, 20.0), "k_pass2_f64t": (4.125, 141.0),
                "k_pass1_f64t": (4.25, 68.0), "k_pass2_f64": (4.125, 141.0), "k_pass1_f64": (4.25, 68.0)}
# The same per-particle model in 2D (x, u, v, b of 2 components; configuration 4 has a body force,
# the edge traction): pass 1 16 + 16 + 8 + 8 + 4, pass 2 48 + 16 + 16 + 1 + 32 + 4.
BYTES_PART_2D = {1: 52.0, 2: 117.0}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_sha(kernel):
    """First 16 hex digits of the sha256 of a step kernel's definition in pd_step.cu (from its
    __global__ line to the closing brace at column 0), so that edits elsewhere in the file do not
    invalidate a recorded capture."""
    with open(os.path.join(ROOT, "paper_2309_11273_gb300", "csrc", "pd_step.cu")) as f:
        src = f.read()
    m = re.search(r"__global__[^\n]*\b%s\(" % re.escape(kernel), src)
    if not m:
        return None
    end = src.find("\n}\n", m.start())
    return hashlib.sha256(src[m.start():end].encode()).hexdigest()[:16]


def recorded_traffic(kernel, nbonds=None):
    """DRAM bytes per launch recorded from an ncu capture (profiles/ncu_traffic.txt), or None when
    the kernel source changed since the capture.  A capture taken on a smaller case of the same
    geometry records its directed bonds (bonds=); its bytes are scaled to nbonds, as the per-slot
    streams and the per-particle state both grow in proportion."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    sha = kernel_source_sha(kernel)
    for ln in lines:
        kv = dict(p.split("=", 1) for p in ln.split() if "=" in p)
        if kv.get("kernel") == kernel and kv.get("source_sha") == sha and "dram_bytes_per_launch" in kv:
            t = float(kv["dram_bytes_per_launch"])
            if "bonds" in kv and nbonds:
                t *= nbonds / float(kv["bonds"])
            return t
    return None


def kernel_entry(kname, ms, flops, nb, n, hbm, fp64_peak):
    """One FP64 kernel of the step: its CUDA-event time, its algorithmic bytes per launch and their
    rate against the measured HBM bandwidth, its DRAM rate from the recorded ncu traffic (the tabled
    kernels stream per-slot tables, so their DRAM bytes exceed the algorithmic ones), and its FP64
    flop rate against the measured FP64 FMA rate."""
    bb, bp = BYTES_KERNEL[kname]
    alg = bb * nb + bp * n
    out = {"ms": ms, "algorithmic_bytes": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9,
           "frac": alg / (ms * 1e-3) / 1e9 / hbm,
           "flop_per_bond": flops, "achieved_tflops": flops * nb / (ms * 1e-3) / 1e12}
    if fp64_peak:
        out["alu_frac"] = out["achieved_tflops"] / fp64_peak
    t = recorded_traffic(kname, nb)
    out["traffic"] = t
    if t is not None:
        out.update({"dram_gbs": t / (ms * 1e-3) / 1e9, "dram_frac": t / (ms * 1e-3) / 1e9 / hbm})
    return out


def measure_fp64_peak(dev):
    """FP64 FMA throughput measured on this GPU (register-only probe in the library), with the SM
    clocks sampled while it runs."""
    from paper_2309_11273_gb300 import _binding as B
    B.pd_probe_fp64(dev, 2)
    with ClockSampler(dev) as clk:
        rate, ms = B.pd_probe_fp64(dev, 20)
    c = clk.summary()
    out = {"tflops": rate / 1e12, "ms_per_launch": ms, "clocks": c,
           "how": "pd_probe_fp64: 8 independent FP64 FMA chains per thread, 2048 threads per SM, 20 launches"}
    if c.get("sm_mhz") and c.get("sm_max_mhz"):
        out["tflops_at_max_clock"] = rate / 1e12 * c["sm_max_mhz"] / c["sm_mhz"]
        out["flop_per_clk_per_sm"] = rate / (c["sm_mhz"] * 1e6) / 152.0
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for ln in open(self.path):
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() in ("active", "1")})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# --------------------------------------------------------------------------------- distributed
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------------- CPU oracle
def oracle_sample_rate(target_s=12.0, max_steps=1000):
    """The oracle (plain FP64 C loops, all host cores) on a 100 x 50 x 25 sub-block of the workload
    (same dx, horizon, material, clamp / twist, notch): bond-updates/s over enough steps for about
    target_s seconds of CPU work."""
    import oracle as O
    from paper_2309_11273_gb300 import workloads as W
    w = W.notched_block(nx=100, ny=50, nz=25, dx=1e-3, notch_cells=37.5)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    sim.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0))
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(max_steps, target_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    sim.step(steps)
    el = time.perf_counter() - t0
    # the same loop on one core, a few steps (a quarter of the time budget at most)
    cores = O.get_threads()
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        sim.step(1)
        one = time.perf_counter() - t0
        s1 = int(max(1, min(20, 0.25 * target_s / max(one, 1e-6))))
        t0 = time.perf_counter()
        sim.step(s1)
        el1 = time.perf_counter() - t0
    finally:
        O.set_threads(cores)
    return {"value": sim.nbonds * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": sim.nbonds * s1 / el1,
            "sample": "%d time steps of the oracle on a 100x50x25 sub-block of the workload (%d particles, "
                      "%d directed bonds), %.1f s on %d threads; %d steps on one thread, %.1f s"
                      % (steps, sim.n, sim.nbonds, el, cores, s1, el1)}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2309_11273_gb300 import workloads as W
    w = W.notched_block(nx=100, ny=50, nz=25, dx=1e-3, notch_cells=37.5)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    sim.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0))
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    el = time.perf_counter() - t0
    value = sim.nbonds * args.steps / el
    sample = ("each step: one oracle time step on a 100x50x25 sub-block of the workload "
              "(%d particles, %d directed bonds)" % (sim.n, sim.nbonds))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "100x50x25 sub-block"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------- GPU arm
def warm(sim, n):
    """n untimed steps, then one untimed CUDA-graph chunk: the library captures a chunk's graph the
    first time a call covers a whole chunk, so a timed call of at least a chunk then replays an
    existing graph instead of capturing and instantiating it inside the timed region."""
    from paper_2309_11273_gb300 import _binding as B
    sim.step(n)
    chunk = sim.get_option(B.PD_OPT_GRAPH_CHUNK)
    if chunk > 0:
        sim.step(chunk)
    sim.sync()


def timed(sim, stream, steps, world):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1)


def profiled(sim, steps):
    """Per-kernel device time from CUDA events the library records around each launch."""
    from paper_2309_11273_gb300 import _binding as B
    sim.set_option(B.PD_OPT_PROFILE, 1)
    B.pd_get_profile(sim.h, B.PD_K_PASS1, reset=True)
    sim.step(steps)
    sim.sync()
    p1 = B.pd_get_profile(sim.h, B.PD_K_PASS1)
    p1b = B.pd_get_profile(sim.h, B.PD_K_PASS1B)
    p2 = B.pd_get_profile(sim.h, B.PD_K_PASS2, reset=True)
    sim.set_option(B.PD_OPT_PROFILE, 0)
    return {"pass1_ms": p1[0] / max(p1[1], 1), "pass1b_ms": p1b[0] / max(p1b[1], 1),
            "pass2_ms": p2[0] / max(p2[1], 1), "launches": p1[1] + p1b[1] + p2[1]}


def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, BatchSimulation, Simulation, pd_critical_stretch
    from paper_2309_11273_gb300 import _binding as B
    from paper_2309_11273_gb300 import workloads as W
    stream = torch.cuda.Stream()
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_note = "measured" if "hbm_gbs" in peaks else "fallback"
    try:
        fp64_peak = measure_fp64_peak(dev)
    except Exception as exc:  # the probe is context for the alu fraction only
        fp64_peak = None
        sys.stderr.write("FP64 probe failed: %s\n" % exc)

    w = W.config3()
    s0 = pd_critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = Simulation(w, s0=s0, precision=PD_FP64, stream=stream.cuda_stream, device=dev)
    nb = sim.nbonds
    mapping = B.pd_autotune(sim.h, 3)
    warm(sim, args.warmup)
    sim.sync()
    with ClockSampler(dev) as clk:
        ms = timed(sim, stream, args.steps, world)
    clocks = clk.summary()
    ms = max_over_ranks(ms, world)
    value = world * nb * args.steps / (ms * 1e-3)
    prof = profiled(sim, max(10, min(args.steps, 50)))
    tabled = B.pd_get_option(sim.h, B.PD_OPT_BOND_CACHE) == 1
    pairs = tabled and B.pd_get_option(sim.h, B.PD_OPT_PAIRS) == 1
    if pairs:
        kern = {"k_pass1a_f64p": prof["pass1_ms"], "k_pass1b_f64p": prof["pass1b_ms"], "k_pass2_f64t": prof["pass2_ms"]}
        fl = FLOPS_BOND_PAIRS
        form = "pair"
    else:
        sfx = "t" if tabled else ""
        kern = {"k_pass1_f64" + sfx: prof["pass1_ms"], "k_pass2_f64" + sfx: prof["pass2_ms"]}
        table = FLOPS_BOND_TABLED if tabled else FLOPS_BOND
        fl = {"k_pass1_f64" + sfx: table[1], "k_pass2_f64" + sfx: table[2]}
        form = "tabled" if tabled else "recompute"
    kname = max(kern, key=kern.get)  # the dominant kernel
    kms = kern[kname]
    step_ms = sum(kern.values())
    n_part = w.n
    peak64 = fp64_peak["tflops"] if fp64_peak else None
    kernels = {k: kernel_entry(k, v, fl[k], nb, n_part, hbm, peak64) for k, v in kern.items()}
    kd = kernels[kname]
    step_bytes = sum(BYTES_KERNEL[k][0] * nb + BYTES_KERNEL[k][1] * n_part for k in kern)
    bb, bp = BYTES_KERNEL[kname]
    roofline = {"bound": "hbm", "kernel": kname, "achieved": kd["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": kd["frac"], "traffic": kd["traffic"],
                "peak_note": "%s HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" % hbm_note,
                "algorithmic": "%.3f B per directed bond x %d bonds + %g B per particle x %d particles per launch "
                               "(neighbour index, status bits, particle state)" % (bb, nb, bp, n_part),
                "step_frac": step_bytes / (step_ms * 1e-3) / 1e9 / hbm, "step_ms": step_ms,
                "step_algorithmic_bytes": step_bytes, "kernels": kernels}
    if fp64_peak:
        ach64 = fl[kname] * nb / (kms * 1e-3) / 1e12
        roofline["alu"] = {"bound": "alu", "kernel": kname, "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                           "frac": ach64 / peak64, "peak_measured": fp64_peak,
                           "algorithmic": "%g FP64 flop per directed bond (per-step part of the %s form) x %d "
                                          "bonds per launch" % (fl[kname], form, nb),
                           "frac_recompute_model": (FLOPS_BOND[1] + FLOPS_BOND[2]) * nb / (step_ms * 1e-3) / 1e12
                           / peak64}

    # end to end through the C ABI with pinned host buffers: H2D of (u, v), one step, D2H of u
    n, dim = w.n, w.dim
    u_h = torch.empty((dim, n), dtype=torch.float64, pin_memory=True).numpy()
    v_h = torch.empty((dim, n), dtype=torch.float64, pin_memory=True).numpy()
    u_out = torch.empty((dim, n), dtype=torch.float64, pin_memory=True).numpy()
    B.pd_get_state(sim.h, dim, n, u_h, v_h, False)
    e2e_steps = max(5, min(args.steps, 20))
    for _ in range(2):  # untimed: the first calls load the transfer kernels
        B.pd_set_state(sim.h, dim, n, u_h, v_h)
        B.pd_step(sim.h, 1)
        B.pd_get_state(sim.h, dim, n, u_out, False, False)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.pd_set_state(sim.h, dim, n, u_h, v_h)
        B.pd_step(sim.h, 1)
        B.pd_get_state(sim.h, dim, n, u_out, False, False)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * nb * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(u_h.nbytes + v_h.nbytes), "d2h_bytes_per_step": int(u_out.nbytes),
           "steps": e2e_steps, "path": "pd_set_state + pd_step(1) + pd_get_state per step"}
    sim.close()

    forms = {}
    if not args.no_forms:
        forms = run_forms(args, stream, dev, world, value, nb, hbm, hbm_note,
                          fp64_peak["tflops"] if fp64_peak else None)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": w.n, "directed_bonds": nb, "precision": "fp64",
                       "graph_chunk": 100, "mapping": {"block": mapping[0], "split": mapping[1], "pairs": int(pairs)}, "l2": "inputs larger than L2 (neighbour indices %.0f MB)" % (nb * 4 / 1e6),
                       "replicas": world},
            "roofline": roofline, "e2e": e2e, "clocks": clocks,
            "gpu_launches": (3 if pairs else 2) * args.steps + 2,  # step kernels + k_set_step + k_flag_nonfinite
            "paper_context": dict(PAPER_CONTEXT, ratio=value / PAPER_CONTEXT["derived_value"])}
    line.update(forms)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = oracle_sample_rate()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def mixed_roofline(prof, a1, a2, bytes1, bytes2, hbm, hbm_note, staged, lattice=False, step_ms=None):
    kp = 1 if prof["pass1_ms"] >= prof["pass2_ms"] else 2  # the dominant kernel
    name = ("k_pass%d_lat" % kp) if lattice else "k_pass%d_mixed%s" % (kp, "_staged" if staged else "")
    ach = a1 if kp == 1 else a2
    other = 2 if kp == 1 else 1
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_note": hbm_note, "traffic": recorded_traffic(name),
            "algorithmic": "%.3f B per directed bond + %g B per particle (index, status bits, particle state)"
                           % ((BYTES_BOND[kp]), BYTES_PART[kp]),
            "other_pass": {"achieved": a2 if kp == 1 else a1, "frac": (a2 if kp == 1 else a1) / hbm,
                           "ms": prof["pass%d_ms" % other]},
            "pass1_ms": prof["pass1_ms"], "pass2_ms": prof["pass2_ms"],
            # the step's algorithmic bytes over the timed step (CUDA-graph replay, the line's
            # ms_per_step), and over the two kernels' own event times (profiled launches, with gaps)
            "step_frac": (bytes1 + bytes2) / ((step_ms if step_ms else prof["pass1_ms"] + prof["pass2_ms"]) * 1e-3)
                         / 1e9 / hbm,
            "step_frac_kernel_events": (bytes1 + bytes2) / ((prof["pass1_ms"] + prof["pass2_ms"]) * 1e-3) / 1e9 / hbm}


def mixed_error_on_workload(w, s0, stream, dev, nsteps, shadow_lo=0):
    """The mixed form against the plain FP64 GPU path on the benchmark's own workload: both run
    nsteps from the same initial state (the FP64 path is held to 1e-12 of the oracle by the parity
    tests); rel-L2(u), the largest per-particle error, and the directed bonds whose status differs,
    beside the FP64 run's broken count.  The mixed run also decides every bond in FP64 on its own
    state (validation mode) and counts the decisions that differ."""
    from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, Simulation
    from paper_2309_11273_gb300 import _binding as B
    res = {}
    for prec in (PD_FP64, PD_MIXED):
        sim = Simulation(w, s0=s0, precision=prec, stream=stream.cuda_stream, device=dev,
                         shadow_lo=shadow_lo if prec == PD_MIXED else None)
        if prec == PD_MIXED:
            sim.set_option(B.PD_OPT_VALIDATE, 1)
        sim.step(nsteps)
        u = sim.state()[0]
        intact = sim.neighbors()[2]
        res[prec] = (u, intact, sim.stats())
        sim.close()
    u64, s64, _ = res[PD_FP64]
    u32, s32, st32 = res[PD_MIXED]
    return {"workload": "this workload, first %d steps from the same state" % nsteps,
            "reference": "plain FP64 GPU path",
            "rel_l2_u": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)),
            "max_particle_err_rel": float(np.abs(u32 - u64).max() / np.abs(u64).max()),
            "status_mismatches": int((s32 != s64).sum()), "broken_fp64": int((s64 == 0).sum()),
            "validate_mismatches": int(st32["validate_mismatches"]), "band_rechecks": int(st32["band_rechecks"])}


def run_matrix_scheme(args, stream, dev, world, w):
    import torch
    from paper_2309_11273_gb300 import PD_FP64, Simulation
    from paper_2309_11273_gb300 import _binding as B
    from paper_2309_11273_gb300.matrix_scheme import MatrixScheme
    rate = w.rotation_rate(6.7381e-4)  # the twist schedule of the breaking run, bonds unbreakable here
    sim = Simulation(w, s0=0.0, rate=rate, precision=PD_FP64, stream=stream.cuda_stream, device=dev)
    rp, col, _ = sim.neighbors()
    nb = int(col.size)
    B.pd_autotune(sim.h, 3)
    warm(sim, args.warmup)
    k = max(args.steps, 50)
    ours_ms = max_over_ranks(timed(sim, stream, k, world), world) / k
    A, K, G = B.pd_material_constants(w.model, w.E, w.nu)
    sim.close()
    t0 = time.time()
    ms_obj = MatrixScheme(w, rp, col, A, K, G, rate=rate, device="cuda:%d" % dev)
    build_s = time.time() - t0
    ms_obj.set_state(w.initial_u(), w.initial_v())
    ms_obj.step(args.warmup)
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(cur)
    ms_obj.step(k)
    e1.record(cur)
    e1.synchronize()
    mat_ms = max_over_ranks(e0.elapsed_time(e1), world) / k
    res = {"value": world * nb / (mat_ms * 1e-3), "unit": UNIT, "ms_per_step": mat_ms, "steps": k, "dtype": "f64",
           "scheme": "CE, CTH, KTH, KE assembled once (Eqs 2.4-2.10), 4 cuSPARSE CSR SpMVs + update per step "
                     "(torch.sparse, 32-bit indices)",
           "workload": "configuration 3 geometry and boundary conditions without bond failure",
           "nnz": ms_obj.nnz, "matrix_bytes": ms_obj.matrix_bytes, "assembly_s": build_s,
           "matrix_gbs": ms_obj.matrix_bytes / (mat_ms * 1e-3) / 1e9,
           "fused_fp64_ms_per_step_same_workload": ours_ms, "fused_fp64_speedup": mat_ms / ours_ms}
    del ms_obj
    torch.cuda.empty_cache()
    return res


def run_forms(args, stream, dev, world, fp64_value, nb, hbm, hbm_note, fp64_tflops=None):
    """Mixed precision on the same workload and the batched form, as speed-ups over plain FP64."""
    from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, PD_NONLINEAR, BatchSimulation, Simulation, pd_critical_stretch
    from paper_2309_11273_gb300 import _binding as B
    from paper_2309_11273_gb300 import workloads as W
    out = {}
    w = W.config3()
    s0 = pd_critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = Simulation(w, s0=s0, precision=PD_MIXED, stream=stream.cuda_stream, device=dev)
    mmap = B.pd_autotune(sim.h, 5)
    steps = max(args.steps, 100)
    warm(sim, args.warmup)
    ms = max_over_ranks(timed(sim, stream, steps, world), world)
    mval = world * nb * steps / (ms * 1e-3)
    prof = profiled(sim, 50)
    st = sim.stats()
    lattice = sim.get_option(B.PD_OPT_LATTICE) == 1
    lat_stage = sim.get_option(B.PD_OPT_LAT_STAGE)
    sim.close()
    staged = mmap[1] == 1  # the staged kernels run whenever the mapping has one warp per slice
    bytes2 = BYTES_BOND[2] * nb + BYTES_PART[2] * w.n
    bytes1 = BYTES_BOND[1] * nb + BYTES_PART[1] * w.n
    a2 = bytes2 / (prof["pass2_ms"] * 1e-3) / 1e9
    a1 = bytes1 / (prof["pass1_ms"] * 1e-3) / 1e9
    out["mixed"] = {"value": mval, "unit": UNIT, "speedup_vs_fp64": mval / fp64_value,
                    "ms_per_step": ms / steps, "dtype": "f32 bond arithmetic, f64 integration",
                    "stated_error": mixed_error_on_workload(w, s0, stream, dev, 200),
                    "band_rechecks": st["band_rechecks"],
                    "mapping": {"block": mmap[0], "split": mmap[1], "lat_stage": lat_stage},
                    "layout": "lattice" if lattice else "general",
                    "roofline": mixed_roofline(prof, a1, a2, bytes1, bytes2, hbm, hbm_note, staged, lattice,
                                                step_ms=ms / steps)}
    # the same with the two-word FP32 shadow (PD_OPT_SHADOW_LO): each bond's relative displacement
    # rounded relative to itself rather than to |u|
    sim = Simulation(w, s0=s0, precision=PD_MIXED, stream=stream.cuda_stream, device=dev, shadow_lo=1)
    lmap = B.pd_autotune(sim.h, 5)
    warm(sim, args.warmup)
    ms = max_over_ranks(timed(sim, stream, steps, world), world)
    lval = world * nb * steps / (ms * 1e-3)
    prof = profiled(sim, 50)
    lo_on = sim.get_option(B.PD_OPT_SHADOW_LO) == 1
    sim.close()
    out["mixed"]["shadow_lo"] = {
        "value": lval, "unit": UNIT, "speedup_vs_fp64": lval / fp64_value, "ms_per_step": ms / steps,
        "active": lo_on, "mapping": {"block": lmap[0], "split": lmap[1]},
        "pass1_ms": prof["pass1_ms"], "pass2_ms": prof["pass2_ms"],
        "step_frac": (bytes1 + bytes2 + 48 * w.n) / ((prof["pass1_ms"] + prof["pass2_ms"]) * 1e-3) / 1e9 / hbm,
        "algorithmic": "the one-word step's bytes + 48 B per particle (the lo words read by both passes and "
                       "written by pass 2)",
        "stated_error": mixed_error_on_workload(w, s0, stream, dev, 600, shadow_lo=1)}
    # geometrically nonlinear bonds (Eqs 1.10, 1.13, 1.14) in FP64 on the same workload
    sim = Simulation(w, s0=s0, precision=PD_FP64, kinematics=PD_NONLINEAR, stream=stream.cuda_stream, device=dev)
    nmap = B.pd_autotune(sim.h, 2)
    warm(sim, args.warmup)
    k = 20
    ms = max_over_ranks(timed(sim, stream, k, world), world)
    nval = world * nb * k / (ms * 1e-3)
    prof = profiled(sim, 5)
    ntab = B.pd_get_option(sim.h, B.PD_OPT_BOND_CACHE) == 1
    npairs = ntab and B.pd_get_option(sim.h, B.PD_OPT_PAIRS) == 1
    sim.close()
    if npairs:
        nkerns = {"k_pass1a_nlp": prof["pass1_ms"], "k_pass1b_nlp": prof["pass1b_ms"], "k_pass2_nlp": prof["pass2_ms"]}
        nfls = FLOPS_BOND_NL_PAIRS
        nform = "pair"
    else:
        sfx = "t" if ntab else ""
        table = FLOPS_BOND_NL_TABLED if ntab else FLOPS_BOND_NL
        nkerns = {"k_pass1_nl" + sfx: prof["pass1_ms"], "k_pass2_nl" + sfx: prof["pass2_ms"]}
        nfls = {"k_pass1_nl" + sfx: table[1], "k_pass2_nl" + sfx: table[2]}
        nform = "tabled" if ntab else "recompute"
    nkern = max(nkerns, key=nkerns.get)
    nfl = nfls[nkern]
    ach = nfl * nb / (nkerns[nkern] * 1e-3) / 1e12
    # the same nonlinear bonds in the mixed form (FP32 bond arithmetic, FP64 state and re-decisions)
    sim = Simulation(w, s0=s0, precision=PD_MIXED, kinematics=PD_NONLINEAR, stream=stream.cuda_stream, device=dev)
    B.pd_autotune(sim.h, 3)
    warm(sim, args.warmup)
    km = max(args.steps, 100)
    msm = max_over_ranks(timed(sim, stream, km, world), world)
    nlat = sim.get_option(B.PD_OPT_LATTICE) == 1
    sim.close()
    nbytes = (BYTES_BOND[1] + BYTES_BOND[2]) * nb + (BYTES_PART[1] + BYTES_PART[2]) * w.n
    nmixed = {"value": world * nb * km / (msm * 1e-3), "ms_per_step": msm / km, "steps": km,
              "dtype": "f32 bond arithmetic, f64 integration", "speedup_vs_fp64_nonlinear": (nb * km / (msm * 1e-3)) / nval,
              "layout": "lattice" if nlat else "general",
              "step_frac_hbm": nbytes / (msm / km * 1e-3) / 1e9 / hbm,
              "step_frac_note": "the linearized step's algorithmic bytes (the same streams and state) over the "
                                "timed step, against the measured HBM copy rate"}
    out["nonlinear"] = {"value": nval, "unit": UNIT, "ms_per_step": ms / k, "steps": k, "dtype": "f64",
                        "mixed": nmixed,
                        "kinematics": "e = |Y| - |xi|, force along Y/|Y| (Eqs 1.10, 1.13, 1.14)",
                        "vs_linearized_fp64": nval / fp64_value, "mapping": {"block": nmap[0], "split": nmap[1]},
                        "roofline": {"bound": "alu", "kernel": nkern, "achieved": ach,
                                     "peak": fp64_tflops, "unit": "TFLOP/s",
                                     "frac": ach / fp64_tflops if fp64_tflops else None,
                                     "peak_note": "measured FP64 FMA rate (pd_probe_fp64)",
                                     "traffic": recorded_traffic(nkern, nb),
                                     "algorithmic": "%g FP64 flop per directed bond (%s form; root, divide = 1) x %d"
                                                    " bonds" % (nfl, nform, nb),
                                     "kernels": {kk: {"ms": v, "flop_per_bond": nfls[kk],
                                                      "traffic": recorded_traffic(kk, nb)}
                                                 for kk, v in nkerns.items()}}}
    # adaptive dynamic relaxation (the quasi-static solver) on the same block, FP64: per iteration
    # the two passes plus a damping reduction and the relaxation update
    sim = Simulation(w, s0=s0, precision=PD_FP64, stream=stream.cuda_stream, device=dev)
    sim.set_option(B.PD_OPT_SOLVER, B.PD_SOLVER_ADR)
    amap = B.pd_autotune(sim.h, 3)
    warm(sim, args.warmup)
    k = max(args.steps, 100)
    ms = max_over_ranks(timed(sim, stream, k, world), world)
    aval = world * nb * k / (ms * 1e-3)
    prof = profiled(sim, 20)
    sim.close()
    out["adr"] = {"value": aval, "unit": UNIT, "ms_per_iteration": ms / k, "iterations": k, "dtype": "f64",
                  "solver": "adaptive dynamic relaxation, clamp + prescribed twist load-stepped per iteration",
                  "vs_explicit_fp64": aval / fp64_value, "mapping": {"block": amap[0], "split": amap[1]},
                  "pass1_ms": prof["pass1_ms"] + prof["pass1b_ms"], "pass2_and_relaxation_ms": prof["pass2_ms"]}
    # the paper's matrix-based scheme (Eqs 2.4-2.10, four cuSPARSE SpMVs per step, FP64) on the same
    # block without bond failure (its failure block is not given), against the fused FP64 kernels on
    # the same no-failure workload
    out["matrix_scheme"] = run_matrix_scheme(args, stream, dev, world, w)
    # batched: 256 uneven plates (configuration 4) in one context; FP64 and mixed; 100-step graphs
    bw = W.config4()
    res = {}
    for prec, name in ((PD_FP64, "fp64"), (PD_MIXED, "mixed")):
        bs = BatchSimulation(bw, precision=prec, stream=stream.cuda_stream, device=dev)
        res["mapping_" + name] = B.pd_autotune(bs.h, 5)
        bnb = bs.nbonds
        warm(bs, args.warmup)
        k = max(args.steps, 200)
        ms = max_over_ranks(timed(bs, stream, k, world), world)
        res[name] = world * bnb * k / (ms * 1e-3)
        res["bonds"] = bnb
        bs.close()
    bms = world * res["bonds"] / res["mixed"] * 1e3  # ms per step of the mixed batch (per replica)
    bbytes = (BYTES_BOND[1] + BYTES_BOND[2]) * res["bonds"] + (BYTES_PART_2D[1] + BYTES_PART_2D[2]) * bw.n
    out["batched"] = {"value": res["mixed"], "unit": UNIT, "workload": "256 independent plane-stress plates, "
                      "sides U{20..200}, delta in {3.015, 4.015} dx, one context, 100-step CUDA graphs",
                      "particles": int(bw.n), "directed_bonds": res["bonds"], "fp64_value": res["fp64"],
                      "speedup_vs_fp64": res["mixed"] / res["fp64"], "dtype": "f32 bond arithmetic, f64 integration",
                      "mapping": {"fp64": res["mapping_fp64"], "mixed": res["mapping_mixed"]},
                      "roofline": {"bound": "hbm", "kernel": "mixed step (both passes)",
                                   "achieved": bbytes / (bms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                   "frac": bbytes / (bms * 1e-3) / 1e9 / hbm, "peak_note": hbm_note,
                                   "traffic": None,
                                   "algorithmic": "%.3f B per directed bond + %g B per particle per step (2D, with "
                                                  "the edge-traction body force)"
                                                  % (BYTES_BOND[1] + BYTES_BOND[2], BYTES_PART_2D[1] + BYTES_PART_2D[2])}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-target", choices=["fp64", "mixed", "nonlinear", "mixed-nonlinear"], default=None,
                    help="only build the workload and run 4 eager steps (the command profiled by ncu)")
    ap.add_argument("--profile-quarter", action="store_true",
                    help="with --profile-target: configuration 3's geometry at a quarter of its particles "
                         "(100x50x50, same dx and horizon), so that multi-pass ncu captures of the tabled "
                         "FP64 kernels hold a few GB")
    ap.add_argument("--profile-pairs", type=int, choices=[0, 1], default=1,
                    help="with --profile-target fp64: 0 runs the single-pass FP64 pass 1 (PD_OPT_PAIRS = 0)")
    ap.add_argument("--profile-block", type=int, default=0,
                    help="with --profile-target: threads per block of the step kernels (0: default)")
    ap.add_argument("--profile-ring", type=int, choices=[0, 1, 2, 3], default=0,
                    help="with --profile-target mixed: staging ring of the lattice kernels (PD_OPT_LAT_STAGE)")
    ap.add_argument("--sweep", action="store_true",
                    help="one JSON line per configuration (1-5): FP64 and mixed GPU rates and the oracle's "
                         "rate on all host cores and on one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.profile_target:
        return profile_target(args.profile_target, args.profile_quarter, args.profile_pairs, args.profile_block,
                              args.profile_ring)
    if args.sweep:
        return run_sweep(args)
    return run_gpu(args)


def run_sweep(args):
    """Every configuration on the GPU (FP64 and mixed, CUDA-graph chunks, events on the library's
    stream) and the oracle on the host (all cores and one core, a bounded number of steps)."""
    import torch
    import oracle as O
    from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, BatchSimulation, Simulation
    from paper_2309_11273_gb300 import _binding as B
    from paper_2309_11273_gb300 import workloads as W
    stream = torch.cuda.Stream()
    dev = torch.cuda.current_device()
    cfgs = [("config1", W.config1, 1000, 1000, 200), ("config2", W.config2, 1000, 1000, 50),
            ("config3", W.config3, 200, 10, 2), ("config4", W.config4, 200, 10, 2),
            ("config5", W.config5, 50, 2, 1), ("kalthoff", W.kalthoff, 1000, 200, 20)]
    for name, make, gpu_steps, cpu_steps, cpu1_steps in cfgs:
        w = make()
        batch = isinstance(w, W.BatchWorkload)
        line = {"sweep": name, "unit": UNIT}
        for prec, tag in ((PD_FP64, "fp64"), (PD_MIXED, "mixed")):
            if batch:
                sim = BatchSimulation(w, precision=prec, stream=stream.cuda_stream, device=dev)
            else:
                sim = Simulation(w, precision=prec, stream=stream.cuda_stream, device=dev)
            B.pd_autotune(sim.h, 3)
            warm(sim, args.warmup)
            ms = timed(sim, stream, gpu_steps, 1)
            line[tag] = {"value": sim.nbonds * gpu_steps / (ms * 1e-3), "ms_per_step": ms / gpu_steps,
                         "steps": gpu_steps, "bonds": sim.nbonds}
            sim.close()
            torch.cuda.empty_cache()
        # the oracle: configuration 4 one plate after another (it has no batched form)
        bodies = w.bodies if batch else [w]
        refs = []
        for b in bodies:
            s0 = O.critical_stretch(b.model, b.E, b.nu, b.Gc, b.delta) if b.Gc else 0.0
            r = O.OracleSim(b.model, b.E, b.nu, b.rho, b.delta, s0, b.dt, b.x, b.y, b.z, b.vol, b.cracks)
            r.set_bc(b.flag, b.b, b.axis_point, b.axis_dir, b.rotation_rate(s0))
            r.set_state(b.initial_u(), b.initial_v())
            refs.append(r)
        nb = sum(r.nbonds for r in refs)
        res = {}
        cores = O.get_threads()
        for threads, steps in ((cores, cpu_steps), (1, cpu1_steps)):
            O.set_threads(threads)
            t0 = time.perf_counter()
            for r in refs:
                r.step(steps)
            el = time.perf_counter() - t0
            res[threads] = (nb * steps / el, steps, el)
        O.set_threads(cores)
        line["oracle"] = {"value": res[cores][0], "cores": cores, "steps": res[cores][1], "seconds": res[cores][2],
                          "single_core_value": res[1][0], "single_core_steps": res[1][1],
                          "single_core_seconds": res[1][2]}
        print(json.dumps(line), flush=True)
        del refs
    return 0


def profile_target(form, quarter=False, pairs=1, block=0, ring=0):
    """Workload of the benchmark in one precision, 4 eager time steps (ncu captures this command)."""
    from paper_2309_11273_gb300 import PD_FP64, PD_LINEARIZED, PD_MIXED, PD_NONLINEAR, Simulation, pd_critical_stretch
    from paper_2309_11273_gb300 import workloads as W
    w = W.notched_block(nx=100, ny=50, nz=50) if quarter else W.config3()
    s0 = pd_critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = Simulation(w, s0=s0, precision=PD_MIXED if form.startswith("mixed") else PD_FP64, graph_chunk=0,
                     kinematics=PD_NONLINEAR if form.endswith("nonlinear") else PD_LINEARIZED,
                     pairs=None if pairs else 0)
    from paper_2309_11273_gb300 import _binding as B
    if block:
        sim.set_option(B.PD_OPT_BLOCK, block)
    if form.startswith("mixed"):
        sim.set_option(B.PD_OPT_LAT_STAGE, ring)
    sim.step(4)
    sim.sync()
    print(json.dumps({"profile_target": form, "particles": w.n, "directed_bonds": sim.nbonds, "stats": sim.stats()}))
    sim.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
