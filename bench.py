"""Benchmark of the coined quantum-walk hot path on GB300.

Workload (one "step" of the benchmark = one pass of the whole path): the 1D walk
on a cycle of N = 2^27 sites with the SU(2) coin theta = pi/4 (phases 0), a
seeded random normalised state (complex64), T = 4096 walk steps with the
temporal-blocking depth chosen by the autotuner, then the coin marginals
P(x) and the norm.  Per benchmark step: the state is re-seeded from a resident
device copy (set_state), stepped T times (fused coin + shift kernels, k steps
per HBM round trip) and reduced to P (float32) and the norm (double).

Metric: site-coin-updates/s = N * d * T / time (d = 2), whole job over all ranks.
Also reported: the roofline of the dominant kernel (live CUDA-event timing),
the FP64 / bf16-storage / compensated forms on the same input with their L1
distance to the FP64 result, an end-to-end number through the C ABI with host
buffers, the SM clocks during the timed region, and the FP64 CPU oracle timed
on the host cores on a bounded sample (``cpu_baseline``).

``--impl reference`` times that oracle alone (the reference arm).
Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the
data path ("weak" scaling); a barrier and a max-over-ranks of the time only.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-coin-updates/s and % HBM roofline, FP32 vs FP64 plain, at stated L1 err"
UNIT = "site-coin-updates/s"
N_SITES = 1 << 27
T_STEPS = 4096
THETA = math.pi / 4
SEED = 1
WORKLOAD = "1D SU(2) walk, cycle N=2^27, theta=pi/4, T=4096, random normalised complex64 state (seed 1)"

FP32_LANES = 128            # FP32 lanes per SM (Blackwell)
SMS = None                  # read from the device (cudaDevAttrMultiProcessorCount) in run_gpu


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p.get("sm_max_mhz", 2070.0), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value, device=None):
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=f"cuda:{device}" if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, max_seconds, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / max_seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.f.close()
        except Exception:
            pass

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and "Active" in r[5 + i] and "Not" not in r[5 + i]:
                    reasons.add(n)
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle (baseline)
def cpu_oracle_sample(target_s=12.0):
    """Time the FP64 oracle (OpenMP build, all host cores) on a bounded sample of
    the workload: the same coin and random-state recipe on a cycle of 2^22
    sites, as many steps as fit in ~target_s seconds."""
    import oracle
    from paper_1003_3779_gb300 import inputs
    n = 1 << 22
    psi = inputs.random_state((2, n), seed=SEED)
    C = inputs.su2(THETA)
    oracle.evolve(psi, C, 1, openmp=True)            # warm-up / page-in
    t0 = time.perf_counter()
    oracle.evolve(psi, C, 1, openmp=True)
    t1 = time.perf_counter() - t0
    steps = max(2, min(64, int(target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.evolve(psi, C, steps, openmp=True)
    dt = time.perf_counter() - t0
    # the small configuration in full on one core: the Hadamard walk on the
    # cycle of 2001 sites from |0> (x) (|0> + i|1>)/sqrt2, T = 1000
    psi_s = inputs.localized_1d(2001, 1000)
    t0 = time.perf_counter()
    oracle.evolve(psi_s, inputs.hadamard(), 1000)
    ds = time.perf_counter() - t0
    return {"value": 2.0 * n * steps / dt, "unit": UNIT, "cores": oracle.num_threads(True),
            "kind": "oracle",
            "sample": f"FP64 oracle (C, OpenMP) on a cycle of 2^22 sites, same coin and state "
                      f"recipe, {steps} steps in {dt:.2f} s",
            "single_core_small_config": {
                "workload": "Hadamard walk, cycle N=2001, T=1000, FP64 oracle, one core, in full",
                "seconds": ds, "value": 2.0 * 2001 * 1000 / ds, "unit": UNIT}}


# ------------------------------------------------------------------ GPU arm
def kernel_hash():
    """sha256 prefix of the 1D step kernels' device code and of the sweep's
    launch code (tile choice, warps per block, shared memory, segments)."""
    csrc = os.path.join(ROOT, "paper_1003_3779_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("k_step1d.cuh", "qw_internal.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    launch = open(os.path.join(csrc, "launch_step.cuh"), "rb").read()
    a = launch.find(b"// Sites per lane compiled for the sweep kernel")
    b = launch.find(b"// Can the sweep kernel run this launch?")
    h.update(launch[a:b] if 0 <= a < b else launch)
    return h.hexdigest()[:16]


def ncu_traffic(kernel="k_step1d_sweep", tile=None):
    """DRAM bytes per launch of the 1D step kernel from the committed ncu summary,
    or None when the summary is missing, was taken on different kernel sources,
    or on another tile (sites per lane) than the one the benchmark runs."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_su2_f32.md")
    try:
        s = open(p).read()
    except OSError:
        return None
    m = re.search(r"kernel_hash:\s*([0-9a-f]+)", s)
    b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", s)
    t = re.search(r"sites_per_lane:\s*(\d+)", s)
    if not m or not b or m.group(1) != kernel_hash():
        return None
    if tile is not None and (not t or int(t.group(1)) != tile):
        return None
    return float(b.group(1))


def graph_cpu_sample(target_s=4.0):
    """The FP64 graph oracle (OpenMP, all host cores) on a bounded sample of the
    random 4-regular workload: 2^20 vertices, as many steps as fit in ~target_s."""
    import oracle
    from paper_1003_3779_gb300 import inputs
    nv = 1 << 20
    off, partner = inputs.random_regular_arcs(nv, 4, seed=5)
    psi = inputs.random_state((int(off[-1]),), seed=6)
    oracle.graph_evolve(off, partner, psi, 1, openmp=True)     # warm-up / page-in
    t0 = time.perf_counter()
    oracle.graph_evolve(off, partner, psi, 1, openmp=True)
    t1 = time.perf_counter() - t0
    steps = max(1, min(32, int(target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.graph_evolve(off, partner, psi, steps, openmp=True)
    dt = time.perf_counter() - t0
    return {"value": float(off[-1]) * steps / dt, "unit": "arc-updates/s", "cores": oracle.num_threads(True),
            "kind": "oracle", "sample": f"FP64 graph oracle (C, OpenMP), random 4-regular graph with 2^20 "
                                        f"vertices, {steps} steps in {dt:.2f} s"}


def batch_oracle_sample(Nb, Tb, coins, x0b, cs):
    """CPU baseline of the batched workload: the FP64 oracle (OpenMP) run on a
    fixed sample of its walks -- every walk whose coin lies within 2e-3 of
    diagonal (theta near 0 or pi/2, where float rounding is biased), the longest
    cycle, the longest walk and four seeded others -- each on its light-cone
    window.  Returns the timing and the oracle's P of each sampled walk, against
    which the GPU forms' per-walk L1 is reported."""
    import oracle
    from paper_1003_3779_gb300 import inputs
    theta = np.array([math.atan2(abs(c[0, 1]), abs(c[0, 0])) for c in coins])
    near = [int(i) for i in np.where(np.minimum(theta, math.pi / 2 - theta) < 2e-3)[0]]
    rng = np.random.default_rng(12)
    sample = sorted(set(near + [int(np.argmax(Nb)), int(np.argmax(Tb))] +
                        [int(i) for i in rng.choice(len(Nb), 4, replace=False)]))
    ref, units = {}, 0.0
    t0 = time.perf_counter()
    for i in sample:
        n, t, x = int(Nb[i]), int(Tb[i]), int(x0b[i])
        if 2 * t + 1 < n:       # the light-cone window, placed back on the cycle
            m = 2 * t + 1
            out = oracle.evolve(inputs.localized_1d(m, t, cs), coins[i], t, openmp=True)
            P = np.zeros(n)
            P[(x - t + np.arange(m)) % n] = (np.abs(out) ** 2).sum(axis=0)
            units += 2.0 * m * t
        else:
            out = oracle.evolve(inputs.localized_1d(n, x, cs), coins[i], t, openmp=True)
            P = (np.abs(out) ** 2).sum(axis=0)
            units += 2.0 * n * t
        ref[i] = P
    dt = time.perf_counter() - t0
    return ({"value": units / dt, "unit": UNIT, "cores": oracle.num_threads(True), "kind": "oracle",
             "sample": f"FP64 oracle (C, OpenMP) on {len(sample)} of the 4096 walks (all {len(near)} "
                       f"with theta within 2e-3 of 0 or pi/2, the longest cycle, the longest walk, four "
                       f"seeded others), each on its light-cone window, in {dt:.2f} s",
             "walks": sample, "near_diagonal_walks": near}, ref)


def batch_l1(P, offsets, ref, near):
    """Per-walk L1 and max-abs of the batch's P against the oracle sample."""
    l1s, mx = {}, 0.0
    for i, Pw in ref.items():
        d = np.abs(P[offsets[i]:offsets[i + 1]].astype(np.float64) - Pw)
        l1s[i] = float(d.sum())
        mx = max(mx, float(d.max()))
    return {"max_l1": max(l1s.values()), "max_l1_near_diagonal": max((l1s[i] for i in near), default=None),
            "max_l1_others": max((v for i, v in l1s.items() if i not in near), default=None),
            "maxabs_p": mx, "walks_over_1e-4": sorted(int(i) for i, v in l1s.items() if v >= 1e-4)}


def graph_timing(qw, _in, make, stream, hbm_gbs, steps=20):
    """One graph workload: build it, autotune the kernel form, time `steps` walk
    steps with CUDA events on the launching stream, check the norm."""
    import torch
    t0 = time.perf_counter()
    off, partner = make()
    A = int(off[-1])
    gw = qw.GraphWalk(off, partner, prec="f32", stream=ctypes.c_void_p(stream.cuda_stream))
    del partner
    gw.set_state(torch.from_numpy(_in.random_state((A,), seed=6, dtype=np.complex64)).cuda())
    tune = gw.autotune()
    setup_s = time.perf_counter() - t0
    gw.step(3)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    gw.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3 / steps
    _, norm = gw.probabilities()
    gw.close()
    # algorithmic bytes of one step: read psi (8 B), write psi' (8 B), read the
    # partner index (4 B) per arc; the two-pass forms move about twice that
    alg = 20.0 * A
    return {"arc_updates_per_s": A / t, "ms_per_step": t * 1e3, "arcs": A, "vertices": len(off) - 1,
            "variant": tune["variant"], "autotune": tune, "steps": steps, "setup_s": setup_s,
            "hbm_view": {"algorithmic_bytes_per_arc_step": 20, "achieved_gbs": alg / t / 1e9,
                         "peak_gbs": hbm_gbs, "frac": alg / t / 1e9 / hbm_gbs},
            "norm_err": abs(norm - 1.0)}


# Instructions on the FP32 pipe per site-step of each coin class (2x2 coin on
# complex amplitudes): the Hadamard class adds (4 FADD), a real coin multiplies
# and accumulates (4 FMUL + 4 FFMA), a complex coin does a complex
# multiply-accumulate per entry (16 FMUL / FFMA).  Flops count an FFMA as 2.
COIN_CLASS_WORK = {"hadamard_class": (4, 4.0, "FADD"), "real": (8, 12.0, "FMUL/FFMA"),
                   "complex": (16, 28.0, "FMUL/FFMA")}


def coin_class_leg(qw, C, dev0, stream, sm_max_mhz, hbm_gbs):
    """The benchmark workload (N = 2^27, T = 4096, FP32, same state) with another
    SU(2) coin: autotuned plan, CUDA events around qw_step, and the kernel's
    roofline against the FP32 instruction issue rate of its coin class."""
    import torch
    w = qw.Walk((N_SITES,), prec="f32").set_coin(C).set_state(dev0)
    tune = json.loads(w.autotune())
    K, tile, var = w.plan_ex()
    desc = w.describe()
    qw.qw_set_state(w.h, dev0)
    qw.qw_step(w.h, 2 * K)
    qw.qw_set_state(w.h, dev0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    qw.qw_step(w.h, T_STEPS)
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    norm = w.norm()
    w.close()
    inst, flops, op = COIN_CLASS_WORK[desc["coin_kind"]]
    launches = math.ceil(T_STEPS / K)
    issue_peak = SMS * FP32_LANES * sm_max_mhz * 1e6            # FP32 instructions / s
    ach_inst = inst * N_SITES * T_STEPS / t
    return {"site_coin_updates_per_s": 2.0 * N_SITES * T_STEPS / t, "ms_per_T_steps": t * 1e3,
            "coin_kind": desc["coin_kind"], "kernel": desc["path"], "k": K, "tile": tile,
            "avg_launch_ms": t * 1e3 / launches, "norm_err": abs(norm - 1.0), "autotune": tune,
            "roofline": {"bound": "alu", "achieved": ach_inst / 1e12, "peak": issue_peak / 1e12,
                         "unit": "T FP32-instructions/s", "frac": ach_inst / issue_peak,
                         "instructions_per_site_step": inst, "op": op,
                         "achieved_tflops": flops * N_SITES * T_STEPS / t / 1e12,
                         "peak_source": f"{SMS} SMs (device attribute) x {FP32_LANES} FP32 lanes x "
                                        f"{sm_max_mhz:.0f} MHz (derived)",
                         "hbm_view": {"effective_bytes_per_site_step": 32.0 / (T_STEPS / launches),
                                      "achieved_gbs": 32.0 * N_SITES * launches / t / 1e9,
                                      "frac": 32.0 * N_SITES * launches / t / 1e9 / hbm_gbs}}}


def localized_legs(qw, stream):
    """Walks from one site: the diagonal lattice (H (x) H) on the 8192^2 torus
    from its centre for T = 500, the SU(2) theta = pi/4 walk on the cycle of 2^27
    sites from its centre for T = 4096, and the Hadamard walk on the line of 2^27
    sites (absorbing ends) from its centre for T = 1024, FP32, default plans.  Each is timed
    with light-cone clipping and with it off (the whole lattice every step);
    dense rates count every site of the lattice, active ones the light cone."""
    import torch
    from paper_1003_3779_gb300 import inputs as _in
    out = {}
    cases = (
        ("diagonal_hh_8192_from_centre_T500", (8192, 8192), 500, qw.SHIFT_DIAGONAL, _in.hadamard2(), qw.BC_PERIODIC),
        ("cycle_su2_2e27_from_centre_T4096", (N_SITES,), T_STEPS, qw.SHIFT_MOVING, _in.su2(THETA), qw.BC_PERIODIC),
        # the paper's line walk: absorbing ends, the generic tiled kernel
        ("line_hadamard_2e27_from_centre_T1024", (N_SITES,), 1024, qw.SHIFT_MOVING, _in.hadamard(), qw.BC_LINE),
    )
    for name, dims, T, shift, C, bc in cases:
        d = 2 * len(dims)
        z = torch.zeros((d,) + tuple(reversed(dims)), dtype=torch.complex64, device="cuda")
        centre = tuple(n // 2 for n in reversed(dims))
        for c in range(d):
            z[(c,) + centre] = 0.5 if d == 4 else (2 ** -0.5 if c == 0 else 1j * 2 ** -0.5)
        nsites = int(np.prod(dims))
        cone = sum(min((2 * t + 1) ** len(dims), nsites) for t in range(1, T + 1))   # light-cone site-steps
        leg = {"sites": nsites, "T": T, "active_site_steps": float(cone)}
        for clip in (True, False):
            w = qw.Walk(dims, prec="f32", shift=shift, bc=bc).set_coin(C).set_clipping(clip)
            w.set_state(z)
            w.step(16)                       # warm-up (kernels loaded, plans fixed)
            w.set_state(z)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            w.step(T)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            desc = w.describe()
            leg["clipped" if clip else "whole_lattice"] = {
                "ms": t * 1e3, "dense_site_coin_updates_per_s": d * nsites * T / t,
                "active_site_coin_updates_per_s": d * cone / t, "kernel": desc["path"], "k": desc["k"],
                "support_after": desc["support"], "norm": w.norm()}
            w.close()
        leg["clipping_speedup"] = leg["whole_lattice"]["ms"] / leg["clipped"]["ms"]
        out[name] = leg
        del z
    return out


def run_gpu(args, rank, world, local):
    import torch
    import paper_1003_3779_gb300.qw as qw
    from paper_1003_3779_gb300 import inputs

    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    hbm_gbs, sm_max_mhz, peak_src = load_peaks()
    global SMS
    SMS = torch.cuda.get_device_properties(local).multi_processor_count
    stream = torch.cuda.current_stream()

    global N_SITES
    N_SITES = args.n_sites
    psi0 = inputs.random_state((2, N_SITES), seed=SEED, dtype=np.complex64)
    dev0 = torch.from_numpy(psi0).to(f"cuda:{local}")
    C = inputs.su2(THETA)
    P_dev = torch.empty(N_SITES, dtype=torch.float32, device=f"cuda:{local}")

    w = qw.Walk((N_SITES,), prec="f32")
    w.set_coin(C)
    w.set_state(dev0)
    if args.plan:
        f = [int(x) for x in args.plan.split(",")]
        w.set_plan_ex(f[0], f[1], f[2] if len(f) > 2 else 1)
        tune = {"tuned": False, "plan": args.plan}
    else:
        tune = json.loads(w.autotune())
    K, tile, _variant = w.plan_ex()
    desc = w.describe()
    launches_step = math.ceil(T_STEPS / K)

    # one benchmark step launches the support search of qw_set_state (2 kernels:
    # a dense state returns after one wave), the step kernels (launches_step)
    # and the marginals with the norm (2 kernels)
    def one_step(ev_a=None, ev_b=None):
        qw.qw_set_state(w.h, dev0)
        if ev_a is not None:
            ev_a.record(stream)
        qw.qw_step(w.h, T_STEPS)
        if ev_b is not None:
            ev_b.record(stream)
        qw.qw_probabilities(w.h, P_dev, want_norm=False)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist, local)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            one_step(*evs[i])
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(dist, local)
    elapsed = start.elapsed_time(stop) / 1e3
    tmax = max_over_ranks(dist, elapsed, local)
    step_kernel_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    norm = qw.qw_probabilities(w.h, P_dev)
    units = 2.0 * N_SITES * T_STEPS * args.steps
    value = aggregate_throughput(units, tmax, world)

    # roofline of the dominant kernel (the temporal-blocking step kernel)
    avg_launch_s = step_kernel_s / (args.steps * launches_step)
    k_eff = T_STEPS / launches_step                       # steps per launch (average)
    if desc["coin_kind"] == "hadamard_class":
        # 4 additions per site-step (a0 +- a1, re and im); one FP32 add per lane per clock
        flops_site_step, flops_per_lane_clk, op = 4.0, 1, "FADD"
    else:
        # 8 FMAs per site-step (real 2x2 coin on complex amplitudes) = 16 flops
        flops_site_step, flops_per_lane_clk, op = 16.0, 2, "FFMA"
    flops_launch = flops_site_step * N_SITES * k_eff
    bytes_launch = 32.0 * N_SITES                         # 2 planes x 8 B read + written
    alu_peak = SMS * FP32_LANES * flops_per_lane_clk * sm_max_mhz * 1e6 / 1e12   # TFLOP/s
    ach_tflops = flops_launch / avg_launch_s / 1e12
    ach_gbs = bytes_launch / avg_launch_s / 1e9
    alu_frac, hbm_frac = ach_tflops / alu_peak, ach_gbs / hbm_gbs
    traffic = ncu_traffic(desc["path"], tile)
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": ach_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": alu_frac, "traffic": traffic,
                "peak_source": f"{SMS} SMs (device attribute) x 128 FP32 lanes x {flops_per_lane_clk} flop "
                               f"({op}) x {sm_max_mhz:.0f} MHz (derived)",
                "hbm_view": {"achieved_gbs": ach_gbs, "peak_gbs": hbm_gbs, "frac": hbm_frac,
                             "peak_source": f"{peak_src} HBM copy"}}
    else:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": hbm_frac, "traffic": traffic, "peak_source": f"{peak_src} HBM copy",
                "alu_view": {"achieved_tflops": ach_tflops, "peak_tflops": alu_peak, "frac": alu_frac}}
    roof.update({"kernel": "%s<f32,R=%d,%s coin>" % (desc["path"], tile, desc["coin_kind"]), "k": K,
                 "flops_per_site_step": flops_site_step,
                 "avg_launch_ms": avg_launch_s * 1e3,
                 "effective_bytes_per_site_step": bytes_launch / N_SITES / k_eff})

    # k = 1 (one step per HBM round trip): the plain fused step against the HBM roof
    plan_saved = w.plan_ex()
    w.set_plan(1, 0)
    qw.qw_set_state(w.h, dev0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    qw.qw_step(w.h, 8)
    e0.record(stream)
    qw.qw_step(w.h, 64)
    e1.record(stream)
    torch.cuda.synchronize()
    k1_s = e0.elapsed_time(e1) / 1e3 / 64
    roof_k1 = {"bound": "hbm", "achieved": 32.0 * N_SITES / k1_s / 1e9, "peak": hbm_gbs,
               "unit": "GB/s", "frac": 32.0 * N_SITES / k1_s / 1e9 / hbm_gbs,
               "frac_of_8000": 32.0 * N_SITES / k1_s / 1e9 / 8000.0}
    w.set_plan_ex(*plan_saved)

    # end to end through the C ABI with host buffers (pinned), rank-local; measured
    # right after the device-timed steps, before the other legs allocate and free
    # their lattices
    e2e = None
    if not args.skip_e2e:
        host_in = torch.from_numpy(psi0).pin_memory()
        host_P = torch.empty(N_SITES, dtype=torch.float32).pin_memory()
        hin, hP = host_in.numpy(), host_P.numpy()
        time.sleep(1.0)      # let the timed region's clock sampler exit first
        for _ in range(3):   # warm-up: first touches of the pinned buffers
            qw.qw_set_state(w.h, hin)
            qw.qw_step(w.h, T_STEPS)
            qw.qw_probabilities(w.h, hP)
        n_e2e = max(1, min(args.steps, 5))
        # per step, CUDA events split the copy in from the steps (the rest, up to the
        # host holding P, is the marginals and the copy out).  No clock sampler runs
        # here: host-to-device copies measured several times slower while an
        # nvidia-smi sampler started or stopped (the steps themselves did not)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_e2e)]
        barrier(dist, local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        marks = []
        for i in range(n_e2e):
            evs[i][0].record(stream)
            qw.qw_set_state(w.h, hin)
            evs[i][1].record(stream)
            qw.qw_step(w.h, T_STEPS)
            evs[i][2].record(stream)
            qw.qw_probabilities(w.h, hP)   # synchronises: the host holds the step's P
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        te = max_over_ranks(dist, time.perf_counter() - t0, local)
        phases = [[round(e[0].elapsed_time(e[1]), 2), round(e[1].elapsed_time(e[2]), 2)] for e in evs]
        per_step = [1e3 * (b - a) for a, b in zip([t0] + marks[:-1], marks)]
        sequential = {"value": aggregate_throughput(2.0 * N_SITES * T_STEPS * n_e2e, te, world),
                      "calls": "qw_set_state(host) + qw_step + qw_probabilities(host) per step",
                      "ms_per_step": [round(x, 2) for x in per_step],
                      "h2d_and_steps_ms": phases,
                      # context only: the typical step, for runs where a step met
                      # host-side interference (value above is the mean over all steps)
                      "value_at_median_step": 2.0 * N_SITES * T_STEPS * world / (statistics.median(per_step) / 1e3)}
        # the serving form of the same work, one public call: qw_run_host_batch runs
        # the n steps from the host input (each copies its 2 GiB in and its P out)
        # with every copy overlapping the neighbouring step's walk
        w.run_host_batch(hin, T_STEPS, count=2, P_out=hP)   # warm-up: allocates the third buffer
        n_pipe = 10   # ten steps (0.8 s) per call
        # five calls, the median reported: the host link is shared with the other
        # GPUs' jobs, and a slow copy episode (single copies in have taken 30 to 220
        # ms instead of 10) lands in some calls, not in the value
        tps, e2e_err = [], 0.0
        for _ in range(5):
            barrier(dist, local)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, e2e_norms = w.run_host_batch(hin, T_STEPS, count=n_pipe, P_out=hP, norms=True)
            torch.cuda.synchronize()
            tps.append(max_over_ranks(dist, time.perf_counter() - t0, local))
            e2e_err = max(e2e_err, float(np.abs(e2e_norms - 1).max()))
        tp = statistics.median(tps)
        e2e = {"value": aggregate_throughput(2.0 * N_SITES * T_STEPS * n_pipe, tp, world),
               "unit": UNIT, "h2d_bytes_per_step": int(hin.nbytes),
               "d2h_bytes_per_step": int(hP.nbytes) + 8, "steps": n_pipe,
               "calls": "qw_run_host_batch(count = steps): copies overlap the steps; median of 5 calls",
               "ms_per_step": 1e3 * tp / n_pipe, "ms_per_step_of_each_call": [round(1e3 * t / n_pipe, 2) for t in tps],
               "max_norm_err": e2e_err, "sequential": sequential}

    # the torus: the fused 2D step (k = 1) on the 8192^2 lattice, against the HBM roof
    torus = {}
    if rank == 0 and not args.skip_forms:
        from paper_1003_3779_gb300 import inputs as _in
        L = 8192
        g = torch.Generator(device=f"cuda:{local}").manual_seed(2)
        z = torch.randn((4, L, L), dtype=torch.complex64, device=f"cuda:{local}", generator=g)
        z /= z.abs().pow(2).sum().sqrt()
        for name, coin, shift in (("grover_moving", _in.grover(), 0), ("hh_moving", _in.hadamard2(), 0),
                                  ("grover_flipflop", _in.grover(), 1), ("diagonal_hh", _in.hadamard2(), 2)):
            w2 = qw.Walk((L, L), prec="f32", shift=shift).set_coin(coin).set_state(z)
            for kk in (1, 8):
                w2.set_plan(kk)
                w2.step(16)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                w2.step(128)
                b.record(stream)
                torch.cuda.synchronize()
                ts = a.elapsed_time(b) / 1e3 / 128
                gbs = 64.0 * L * L / ts / 1e9      # k = 1 algorithmic bytes per site-step (effective above k = 1)
                torus[f"{name}_k{kk}"] = {"site_coin_updates_per_s": 4.0 * L * L / ts, "ms_per_step": ts * 1e3,
                                          "kernel": w2.describe()["path"],
                                          ("hbm_gbs" if kk == 1 else "effective_gbs"): gbs,
                                          "frac_of_measured": gbs / hbm_gbs, "frac_of_8000": gbs / 8000.0}
            w2.close()
        # the rows beyond the periodic lattice walk, same lattice and state: the
        # generic kernel with a segment boundary and 5 % of the links closed
        # (fixed mask, 2 more bytes per site-step), or with links closed at
        # random afresh at every step (p = 0.05, Philox in the kernel, no mask
        # traffic); the diagonal lattice is timed above with the axis lattice
        mask = (torch.rand((2, L * L), generator=torch.Generator().manual_seed(3)) < 0.05).to(torch.uint8).cuda()
        for name, kw, setup, nbytes in (
                ("segment_fixed_links_5pct", dict(bc=qw.BC_SEGMENT),
                 lambda w_: w_.set_coin(_in.grover()).set_links(mask), 66.0),
                ("random_links_5pct_per_step", dict(),
                 lambda w_: w_.set_coin(_in.grover()).set_link_noise(0.05, 11), 64.0)):
            w2 = qw.Walk((L, L), prec="f32", **kw)
            setup(w2)
            w2.set_state(z)
            w2.step(8)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            w2.step(64)
            b.record(stream)
            torch.cuda.synchronize()
            ts = a.elapsed_time(b) / 1e3 / 64
            gbs = nbytes * L * L / ts / 1e9
            torus[name] = {"site_coin_updates_per_s": 4.0 * L * L / ts, "ms_per_step": ts * 1e3,
                           "kernel": w2.describe()["path"], "algorithmic_bytes_per_site_step": nbytes,
                           "hbm_gbs": gbs, "frac_of_measured": gbs / hbm_gbs, "norm": w2.norm()}
            w2.close()
        del z, mask
        # the paper's own timed case, the 1D segment (reflecting ends, no broken
        # links), at the benchmark's size: the cycle of 2^27 sites, Hadamard coin
        ws = qw.Walk((N_SITES,), prec="f32", bc=qw.BC_SEGMENT).set_coin(_in.hadamard()).set_state(dev0)
        ws.step(8)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ws.step(64)
        b.record(stream)
        torch.cuda.synchronize()
        ts = a.elapsed_time(b) / 1e3 / 64
        torus["cycle_2e27_segment_hadamard"] = {
            "site_coin_updates_per_s": 2.0 * N_SITES / ts, "ms_per_step": ts * 1e3, "kernel": ws.describe()["path"],
            "algorithmic_bytes_per_site_step": 32.0, "hbm_gbs": 32.0 * N_SITES / ts / 1e9,
            "frac_of_measured": 32.0 * N_SITES / ts / 1e9 / hbm_gbs, "norm": ws.norm()}
        ws.close()

    # the paper's own timed shapes: a walker started on one site (the line walk of
    # Sec. 3 and the 2D walk of Tables 2-3 on the diagonal lattice), stepped with
    # light-cone clipping (the default) and over the whole lattice
    localized = {}
    if rank == 0 and not args.skip_forms:
        localized = localized_legs(qw, stream)

    # the other SU(2) coin classes on the benchmark workload: a real rotation and a
    # complex coin (the headline's theta = pi/4 is the Hadamard class)
    coin_classes = {}
    if rank == 0 and not args.skip_forms:
        from paper_1003_3779_gb300 import inputs as _in
        for cname, Cc in (("real_theta_0.3", _in.su2(0.3)), ("complex_theta_pi4_xi_0.3_zeta_-0.2",
                                                            _in.su2(THETA, 0.3, -0.2))):
            coin_classes[cname] = coin_class_leg(qw, Cc, dev0, stream, sm_max_mhz, hbm_gbs)

    # batched walks: 4096 walks in one persistent launch (graph replay), FP32,
    # bf16 storage and double-float, with per-walk L1 against the FP64 oracle on a
    # sample of the walks (the batch's CPU baseline)
    batch = {}
    if rank == 0 and not args.skip_forms:
        from paper_1003_3779_gb300 import inputs as _in
        Nb, Tb, thb, x0b = _in.batch_1d_params()
        coins_b = np.stack([_in.su2(t) for t in thb])
        dense = float(np.sum(2.0 * Nb * Tb))
        tc = np.minimum(Tb, Nb // 2)
        active = float(np.sum(2.0 * (tc.astype(np.float64) ** 2 + (Tb - tc) * Nb.astype(np.float64))))
        batch_ref, near = None, []
        if not args.skip_cpu:
            batch["cpu_baseline"], batch_ref = batch_oracle_sample(Nb, Tb, coins_b, x0b, _in.BATCH_COIN_STATE)
            near = batch["cpu_baseline"]["near_diagonal_walks"]
        for pname in ("f32", "bf16", "comp"):
            bt = qw.Batch(Nb, Tb, coins_b, x0b, _in.BATCH_COIN_STATE, prec=pname)
            tune_b = json.loads(bt.autotune())
            bt.step()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                bt.step()
            b.record(stream)
            torch.cuda.synchronize()
            tb = a.elapsed_time(b) / 1e3 / 3
            Pb_, nb_ = bt.probabilities()
            # the real 2x2 coin is 8 FP32 instructions (4 FMUL, 4 FFMA) per site-step;
            # against the FP32 issue rate over the light-cone (active) site-steps only
            inst_rate = 8.0 * (active / 2.0) / tb / 1e12
            issue_peak = SMS * FP32_LANES * sm_max_mhz * 1e6 / 1e12
            batch[pname] = {"dense_site_coin_updates_per_s": dense / tb,
                            "active_site_coin_updates_per_s": active / tb, "ms_per_batch": tb * 1e3,
                            "k": tune_b["k"], "variant": tune_b.get("variant"), "cta_walks": tune_b.get("cta_walks"),
                            "max_norm_err": float(np.abs(nb_ - 1).max())}
            if pname != "comp":
                batch[pname]["alu_view"] = {"achieved_tinst_per_s": inst_rate, "peak_tinst_per_s": issue_peak,
                                            "frac": inst_rate / issue_peak,
                                            "note": "8 FP32 instructions per active site-step (real coin)"}
            if batch_ref is not None:
                batch[pname]["l1_vs_oracle"] = batch_l1(Pb_, bt.offsets, batch_ref, near)
            bt.close()

    # region-mass gradient on the 1024^2 torus (forward with checkpoints + adjoint sweep)
    grad_leg = {}
    if rank == 0 and not args.skip_forms:
        from paper_1003_3779_gb300 import inputs as _in
        Lg, Tg, Kg = 1024, 512, 64
        wg = qw.Walk((Lg, Lg), prec="f32")
        phi_g = torch.from_numpy(_in.region_grad_phases(Lg).reshape(-1, 4).astype(np.float32)).cuda()
        wg.set_coin_phases(_in.grover(), phi_g)
        psi_g = torch.from_numpy(_in.localized_2d(Lg).astype(np.complex64)).cuda()
        g_out = torch.empty((Lg * Lg, 4), dtype=torch.float64, device=f"cuda:{local}")
        wg.set_state(psi_g)
        qw.qw_backward(wg.h, _in.region_rect(Lg), Tg, Kg, g_out)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        reps = 3
        ev[0].record(stream)
        for _ in range(reps):
            wg.set_state(psi_g)
            lossg = qw.qw_backward(wg.h, _in.region_rect(Lg), Tg, Kg, g_out)
        ev[1].record(stream)
        # the forward phase alone (the same clipped steps, without the checkpoint copies)
        wg.set_state(psi_g)
        ev[2].record(stream)
        wg.step(Tg)
        ev[3].record(stream)
        torch.cuda.synchronize()
        tg = ev[0].elapsed_time(ev[1]) / 1e3 / reps
        tf = ev[2].elapsed_time(ev[3]) / 1e3
        tb = max(tg - tf, 1e-9)
        # the adjoint sweep per site-step (FP32): reads lambda and psi (32 B each),
        # phi (16 B) and the segment accumulator (16 B), writes lambda', psi' and
        # the accumulator (32 + 32 + 16 B)
        bwd_bytes = 176.0 * Lg * Lg * Tg
        grad_leg = {"ms": tg * 1e3, "loss": lossg, "forward_ms": tf * 1e3, "adjoint_ms": tb * 1e3,
                    "site_steps_per_s": 2.0 * Tg * Lg * Lg / tg,
                    "roofline": {"bound": "hbm", "kernel": "k_backward2d<f32, Grover>", "achieved": bwd_bytes / tb / 1e9,
                                 "peak": hbm_gbs, "unit": "GB/s", "frac": bwd_bytes / tb / 1e9 / hbm_gbs,
                                 "algorithmic_bytes_per_site_step": 176,
                                 "note": "adjoint time = the qw_backward call minus its forward phase timed alone; "
                                         "the sweep's working set (lambda and psi in and out, 4 x 32 MiB, phi and "
                                         "the accumulator, 16 MiB each) is about the L2 size, so part of it is "
                                         "served from L2 and frac can exceed 1"},
                    "note": "forward T steps (light-cone clipped from the localised start) with checkpoints + T "
                            "adjoint steps; CUDA events"}
        wg.close()

    # the walk on a general graph (Sec. 2.1), Grover coin, FP32: a random 4-regular
    # multigraph (configuration model) with 2^26 vertices and the 8192^2 torus as a
    # graph, both 2^28 arcs; the autotuner picks the kernel form
    graph_leg = {}
    if rank == 0 and not args.skip_forms:
        from paper_1003_3779_gb300 import inputs as _in
        for gname, make in (("random_4_regular_2e26", lambda: _in.random_regular_arcs(1 << 26, 4, seed=5)),
                            ("torus_8192_as_graph", lambda: _in.lattice_graph_arcs(8192, 8192))):
            graph_leg[gname] = graph_timing(qw, _in, make, stream, hbm_gbs)
        if not args.skip_cpu:
            graph_leg["random_4_regular_2e26"]["cpu_baseline"] = graph_cpu_sample()

    forms, accuracy = {}, {}
    if rank == 0 and not args.skip_forms:
        qw.qw_set_state(w.h, dev0)
        qw.qw_step(w.h, T_STEPS)
        P32 = torch.empty(N_SITES, dtype=torch.float64, device=f"cuda:{local}")
        qw.qw_probabilities(w.h, P32)
        ref = None
        for name in ("f64", "bf16", "comp"):
            wf = qw.Walk((N_SITES,), prec=name)
            wf.set_coin(C)
            wf.set_state(dev0)
            wf.autotune()
            Kf, tf, _ = wf.plan_ex()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            qw.qw_step(wf.h, T_STEPS)
            b.record(stream)
            Pf = torch.empty(N_SITES, dtype=torch.float64, device=f"cuda:{local}")
            nf = qw.qw_probabilities(wf.h, Pf)
            torch.cuda.synchronize()
            ts = a.elapsed_time(b) / 1e3
            forms[name] = {"value": 2.0 * N_SITES * T_STEPS / ts, "unit": UNIT, "k": Kf,
                           "tile": tf, "norm": nf}
            if name == "f64":
                ref = Pf
            else:
                forms[name]["l1_vs_f64"] = float((Pf - ref).abs().sum())
                forms[name]["maxabs_p_vs_f64"] = float((Pf - ref).abs().max())
            if name == "bf16":
                # one step per launch (k = 1), where 16 bytes per site-step against
                # FP32's 32 halve the HBM traffic of the memory-bound step
                wf.set_plan(1, 0)
                qw.qw_set_state(wf.h, dev0)
                qw.qw_step(wf.h, 8)
                qw.qw_set_state(wf.h, dev0)
                a.record(stream)
                qw.qw_step(wf.h, T_STEPS)
                b.record(stream)
                torch.cuda.synchronize()
                qw.qw_probabilities(wf.h, Pf)
                t1 = a.elapsed_time(b) / 1e3
                gbs = 16.0 * N_SITES * T_STEPS / t1 / 1e9
                forms["bf16_k1"] = {"value": 2.0 * N_SITES * T_STEPS / t1, "unit": UNIT, "k": 1,
                                    "kernel": wf.describe()["path"], "algorithmic_bytes_per_site_step": 16,
                                    "hbm_gbs": gbs, "frac_of_measured": gbs / hbm_gbs,
                                    "l1_vs_f64": float((Pf - ref).abs().sum()),
                                    "maxabs_p_vs_f64": float((Pf - ref).abs().max())}
            del Pf
            wf.close()
        accuracy = {"l1_vs_f64_gpu": float((P32 - ref).abs().sum()),
                    "maxabs_p_vs_f64_gpu": float((P32 - ref).abs().max()),
                    "norm_f32": norm, "reference": "FP64 GPU path, same input, T=4096"}
        forms["f32"] = {"value": value / world, "unit": UNIT, "k": K, "tile": tile,
                        "l1_vs_f64": accuracy["l1_vs_f64_gpu"]}
        del P32, ref

    if e2e is not None:
        del host_in, host_P
    w.close()
    return {
        "value": value, "elapsed": tmax, "norm": norm, "roofline": roof, "roofline_k1": roof_k1,
        "forms": forms, "accuracy": accuracy, "e2e": e2e, "clocks": clk.summary(), "tune": tune,
        "K": K, "tile": tile, "launches": args.steps * (launches_step + 4), "dist": dist,
        "torus": torus, "batch": batch, "grad": grad_leg, "graph": graph_leg,
        "coin_classes": coin_classes, "coin_kind": desc["coin_kind"], "localized": localized,
    }


def run_case(args):
    """Small named workloads for kernel captures (ncu) and quick timings; prints
    one JSON line with the case's own time.  Not the benchmark line."""
    import torch
    import paper_1003_3779_gb300.qw as qw
    from paper_1003_3779_gb300 import inputs as _in
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"case": args.case}
    if args.case == "graph":
        # random 4-regular multigraph of --n-sites vertices, Grover coin, FP32;
        # --plan: the kernel form (default: autotuned)
        nv = args.n_sites if args.n_sites != N_SITES else 1 << 23
        off, partner = _in.random_regular_arcs(nv, 4, seed=5)
        A = int(off[-1])
        gw = qw.GraphWalk(off, partner, prec="f32")
        gw.set_state(torch.from_numpy(_in.random_state((A,), seed=6, dtype=np.complex64)).cuda())
        if args.plan:
            gw.set_variant(int(args.plan))
        else:
            out["autotune"] = gw.autotune()
        gw.step(2)
        a, b = ev(), ev()
        a.record(stream)
        gw.step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        out.update(vertices=nv, arcs=A, variant=gw.variant(), ms_per_step=a.elapsed_time(b) / args.steps)
        gw.close()
        print(json.dumps(out))
        return
    if args.case == "line":
        # the paper's line walk: Hadamard coin from the centre of a line of
        # --n-sites sites (absorbing ends), --steps steps, clipped (the window CTA)
        n = args.n_sites
        z = torch.zeros((2, n), dtype=torch.complex64, device="cuda")
        z[0, n // 2] = 2 ** -0.5
        z[1, n // 2] = 1j * 2 ** -0.5
        w = qw.Walk((n,), prec="f32", bc=qw.BC_LINE).set_coin(_in.hadamard())
        w.set_state(z).step(16)
        w.set_state(z)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        w.step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        out.update(sites=n, T=args.steps, path=w.describe()["path"], ms=a.elapsed_time(b), norm=w.norm())
        w.close()
        print(json.dumps(out))
        return
    if args.case == "generic":
        # the generic kernel on an L x L torus (--n-sites L, default 4096), Grover,
        # links closed at random afresh at every step (p = 0.05)
        L = args.n_sites if args.n_sites != N_SITES else 4096
        g = torch.Generator(device="cuda").manual_seed(2)
        z = torch.randn((4, L, L), dtype=torch.complex64, device="cuda", generator=g)
        z /= z.abs().pow(2).sum().sqrt()
        w = qw.Walk((L, L), prec="f32").set_coin(_in.grover()).set_link_noise(0.05, 11).set_state(z)
        w.step(2)
        a, b = ev(), ev()
        a.record(stream)
        w.step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        out.update(L=L, path=w.describe()["path"], ms_per_step=a.elapsed_time(b) / args.steps)
        w.close()
        print(json.dumps(out))
        return
    if args.case == "cycle":
        # the 1D walk on a cycle of --n-sites sites (default 2^24), FP32, a random
        # state, --coin class, --plan "k,tile,variant" (default: autotuned);
        # 4 launches after two warm-up launches
        n = args.n_sites if args.n_sites != N_SITES else 1 << 24
        C = {"hadamard_class": _in.su2(THETA), "real": _in.su2(0.3),
             "complex": _in.su2(THETA, 0.3, -0.2)}[args.coin]
        z = torch.from_numpy(_in.random_state((2, n), seed=SEED, dtype=np.complex64)).cuda()
        w = qw.Walk((n,), prec="f32").set_coin(C).set_state(z)
        if args.plan:
            f = [int(x) for x in args.plan.split(",")]
            w.set_plan_ex(f[0], f[1], f[2] if len(f) > 2 else 1)
        else:
            out["autotune"] = json.loads(w.autotune())
        k = w.plan_ex()[0]
        w.step(2 * k)
        a, b = ev(), ev()
        a.record(stream)
        w.step(4 * k)
        b.record(stream)
        torch.cuda.synchronize()
        out.update(n=n, coin=args.coin, plan=list(w.plan_ex()), kernel=w.describe()["path"],
                   ms_per_step=a.elapsed_time(b) / (4 * k), norm=w.norm())
        w.close()
    elif args.case == "torus":
        L = args.n_sites
        g = torch.Generator(device="cuda").manual_seed(2)
        z = torch.randn((4, L, L), dtype=torch.complex64, device="cuda", generator=g)
        z /= z.abs().pow(2).sum().sqrt()
        coin2 = _in.hadamard2() if args.shift == 2 else _in.grover()
        w = qw.Walk((L, L), prec="f32", shift=args.shift).set_coin(coin2).set_state(z)
        k = int(args.plan.split(",")[0]) if args.plan else 8
        w.set_plan(k)
        w.step(2 * k)
        a, b = ev(), ev()
        a.record(stream)
        w.step(8 * k)
        b.record(stream)
        torch.cuda.synchronize()
        out.update(L=L, k=k, shift=args.shift, kernel=w.describe()["path"], ms_per_step=a.elapsed_time(b) / (8 * k))
        w.close()
    elif args.case == "batch":
        N, T, th, x0 = _in.batch_1d_params(nwalks=args.walks)
        coins = np.stack([_in.su2(t) for t in th])
        b_ = qw.Batch(N, T, coins, x0, _in.BATCH_COIN_STATE).set_plan(int(args.plan.split(",")[0]) if args.plan else 64)
        b_.step()
        a, b = ev(), ev()
        a.record(stream)
        b_.step()
        b.record(stream)
        torch.cuda.synchronize()
        out.update(walks=args.walks, ms=a.elapsed_time(b))
        b_.close()
    elif args.case == "grad":
        L, T, K = args.n_sites, 64, 64
        w = qw.Walk((L, L), prec="f32")
        w.set_coin_phases(_in.grover(), _in.region_grad_phases(L).reshape(-1, 4).astype(np.float32))
        w.set_state(_in.localized_2d(L))
        grad = torch.empty((L * L, 4), dtype=torch.float64, device="cuda")
        rect = _in.region_rect(L, centre=(L // 4, L // 4), size=max(4, L // 16))
        qw.qw_backward(w.h, rect, T, K, grad)
        t0 = time.perf_counter()
        loss = qw.qw_backward(w.h, rect, T, K, grad)
        out.update(L=L, T=T, K=K, ms=1e3 * (time.perf_counter() - t0), loss=loss)
        w.close()
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-forms", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--n-sites", type=int, default=N_SITES,
                    help="cycle length (default 2^27; smaller only for profiling captures)")
    ap.add_argument("--shift", type=int, default=0, choices=[0, 1, 2],
                    help="shift of the torus case (2: diagonal lattice, H (x) H; else Grover)")
    ap.add_argument("--coin", default="hadamard_class", choices=["hadamard_class", "real", "complex"],
                    help="coin class of the cycle case")
    ap.add_argument("--case", default="", choices=["", "cycle", "torus", "batch", "grad", "graph", "generic", "line"],
                    help="run a small named workload for kernel captures instead of the benchmark")
    ap.add_argument("--walks", type=int, default=4096, help="walks of the batch case")
    ap.add_argument("--plan", default="",
                    help="fixed 'k,tile[,variant]' instead of the autotuner (variant 1 = sweep, the default; 0 = tiles)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.case:
        run_case(args)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        samples = [cpu_oracle_sample(target_s=max(4.0, 40.0 / max(1, args.steps + args.warmup)))
                   for _ in range(args.warmup + args.steps)][args.warmup:]
        vals = [s["value"] for s in samples]
        v = statistics.median(vals)
        total = time.perf_counter() - t0
        cb = dict(samples[-1])
        cb["value"] = v
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / (args.steps + args.warmup),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}))
        return

    r = run_gpu(args, rank, world, local)
    if rank != 0:
        return
    cpu = None if args.skip_cpu else cpu_oracle_sample()
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * r["elapsed"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if N_SITES == 1 << 27 else f"{WORKLOAD} (N={N_SITES})",
                   "sites": N_SITES, "coin_dim": 2, "T": T_STEPS,
                   "k": r["K"], "tile": r["tile"], "parallelism": f"replicas{world}",
                   "coin_class": r["coin_kind"] + " (theta = pi/4 with zero phases is lambda * M, M a "
                                                  "+-1 matrix: four additions per site-step; the real and "
                                                  "complex SU(2) classes are in coin_classes)",
                   "l2": "inputs larger than L2 (2 GiB state, 129 MB L2); no flush needed",
                   "step": "set_state (device copy) + T=4096 walk steps + marginals/norm"},
        "clocks": r["clocks"], "e2e": r["e2e"], "gpu_launches": r["launches"],
        "roofline": r["roofline"], "roofline_k1": r["roofline_k1"], "cpu_baseline": cpu,
        "accuracy": r["accuracy"], "forms": r["forms"], "torus_8192": r["torus"],
        "batch_4096": r["batch"], "region_grad_1024": r["grad"], "graph": r["graph"],
        "coin_classes": r["coin_classes"], "localized_start": r["localized"],
        "norm": r["norm"], "autotune": r["tune"],
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
