#!/usr/bin/env python
"""Throughput of the short-range MD hot path on GB300.

Workload (the LJ fluid at scale): N = 2,048,000 particles on an fcc lattice
(80^3 cells x 4), reduced density 0.8442, Gaussian velocities at T* = 0.72
with zero net momentum (seeded), Lennard-Jones with eps = sigma = 1 and
r_cut = 2.5 sigma shifted to zero energy at r_cut, Verlet skin 0.3 sigma,
velocity Verlet at dt = 0.005, NVE.  One bench step is one MD step: the
device-side cell sort / Verlet-list rebuild when triggered, and the fused
pair-force + velocity-Verlet kernel, FP32 pair arithmetic with 64-bit
fixed-point force sums and FP64 positions / velocities.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs independent replicas (one 2.048M system per rank, seeds differ;
no data-path collective) under torch.distributed.run; the value is the
whole-job particle-steps/s over the slowest rank.  `--impl reference` times
the FP64 CPU oracle on bounded samples of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LJ force+integrate particle-steps/s at 2M atoms; % HBM roofline; FP32 vs FP64"
UNIT = "particle-steps/s"
NCELL = 80
RHO, T0, RC, SKIN, DT = 0.8442, 0.72, 2.5, 0.3, 0.005
# per particle and fused step, algorithmic HBM bytes of the force kernel
# besides the list: own fixed-point position 16, list length 4, x read+write 48,
# v read+write 48, new fixed-point position 16, build-time position 16
FORCE_FIXED_BYTES = 16 + 4 + 48 + 48 + 16 + 16
# FP64 path, algorithmic FP64 operations per list entry: separation 3,
# minimum image 3, r^2 5, cutoff test 1 (12 for an entry beyond r_cut); an
# interacting pair adds 1/r^2 1, (sigma/r)^2 1, ^6 2, force scalar 4, force
# accumulation 6 (26 in all)
FP64_OPS_OUT, FP64_OPS_IN = 12, 26
FP64_NOMINAL_TFLOPS = 1.25      # GB300 nominal FP64 rate, context only: the roofline uses the measured probe
# the algorithmic HBM bytes of one force + integrate step per particle, full
# Verlet list, rebuild excluded, as the scope table of the method counts them
# (a 4-byte index per list entry at 82.4 entries, twice the paper's 41.2
# neighbours per particle): own float4 16, list offset 4, list indices 329.6,
# force writes 24, integrator (F read 24, x r/w 48, v r/w 48, float4 write 16,
# x_ref read 24) 160
SCOPE_BYTES_FULL = 16 + 4 + 82.4 * 4 + 24 + 160
SCOPE_BYTES_HALF = 16 + 4 + 41.2 * 4 + 24 + 160
# the half list adds, per particle, the fixed-point force sums: 24 B written
# by the pair pass (the atomics' net result), 24 B read and 24 B cleared by
# the integrating pass
HALF_SUM_BYTES = 3 * 24
# kernels of one list rebuild: bin, 3-phase scan, scatter, reorder, tile count /
# scan / write / pieces, list build
REBUILD_KERNELS = 11


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ncell", type=int, default=NCELL)
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, FP64, CPU baseline and force error")
    ap.add_argument("--workload", default="lj", choices=["lj", "melt", "rings", "slab", "sphere", "ensemble"],
                    help="lj: the LJ fluid line (default); melt / rings / slab / sphere: one line for that workload")
    ap.add_argument("--list", default="full", choices=["full", "half"],
                    help="Verlet-list form of the timed LJ-fluid run: full (default; every pair from both ends) "
                         "or half (Newton's third law, partner shares by 64-bit atomics)")
    return ap.parse_args()


def csrc_digest():
    """Digest of the sources that define the fused force kernel."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2109_10876_gb300", "csrc")
    for f in ("k_force.cu", "md_internal.cuh"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        m = json.load(open(p))
        return float(m["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled(digest, key):
    """A per-particle figure of the fused force kernel (DRAM bytes, warp
    instructions) from the committed ncu summary, if it was taken on the
    current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "force_fp32_fused_lj_fluid.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    if vals.get("csrc_sha") != digest:
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic(digest):
    return profiled(digest, "dram_bytes_per_particle")


class Clocks:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[4 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", rank=rank, world_size=world)
        else:
            dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier_max(x, world):
    """Maximum of x over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_baseline(x, box, target_s=10.0):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: exact
    forces on S particles, each summed over all N particles.  S particle-steps
    of work; S is sized from a short calibration so the sample takes about
    target_s seconds of the host's cores."""
    import oracle
    n = len(x)
    s = oracle.System(n, box, rc=RC)
    rng = np.random.default_rng(123)
    t0 = time.perf_counter()
    oracle.forces_sample(s, x, rng.choice(n, 16, replace=False))
    per = max((time.perf_counter() - t0) / 16, 1e-6)
    S = int(min(max(16, target_s / per), n))
    idx = rng.choice(n, S, replace=False)
    t0 = time.perf_counter()
    oracle.forces_sample(s, x, idx)
    t = time.perf_counter() - t0
    return {"value": S / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"exact FP64 O(N^2) forces on {S} sampled particles of the N={n} system "
                      f"(one particle-step each), {t:.1f} s"}


def config_4000_leg(md, torch, dev, e0, e1, stream):
    """The small LJ fluid (N = 4000, fcc 10^3 x 4, T* 0.72, seed 1), 100 FP64
    velocity-Verlet steps at dt 0.005: the GPU's plain FP64 path (CUDA events)
    beside the FP64 oracle's own full run of the same steps (exact O(N^2)
    forces every step) on all host cores and on one, and the largest position
    difference between the two."""
    import oracle
    from paper_2109_10876_gb300 import inputs
    x, v, box = inputs.lj_fluid(10, rho=RHO, T=T0, seed=1)
    n = len(x)
    h = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP64)
    md.md_set_state(h, torch.tensor(x.T.copy(), device=dev), torch.tensor(v.T.copy(), device=dev))
    torch.cuda.synchronize()
    e0.record(stream)
    md.md_build_neighbors(h)
    md.md_step(h, 100)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_gpu = e0.elapsed_time(e1)
    xo = torch.zeros(3, n, dtype=torch.float64, device=dev)
    md.md_get_state(h, xo, None)
    xg = xo.cpu().numpy().T
    h.destroy()
    s = oracle.System(n, box, rc=RC, dt=DT)
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    xr, _, _ = oracle.vv_run(s, x, v, 100)
    t_all = time.perf_counter() - t0
    oracle.set_num_threads(1)
    t0 = time.perf_counter()
    oracle.vv_run(s, x, v, 100)
    t_one = time.perf_counter() - t0
    oracle.set_num_threads(cores)
    d = xg - xr
    d -= box * np.round(d / box)
    return {"steps": 100, "particles": n, "gpu_fp64_ms": ms_gpu, "gpu_fp64_value": n * 100 / (ms_gpu * 1e-3),
            "oracle_s": t_all, "oracle_cores": cores, "oracle_value": n * 100 / t_all,
            "oracle_1core_s": t_one, "oracle_1core_value": n * 100 / t_one,
            "max_abs_dx_gpu_vs_oracle": float(np.max(np.abs(d))), "unit": UNIT,
            "note": "GPU time includes the first list build; the oracle sums all pairs every step"}


def ensemble_leg(md, torch, dev, passes=3, nsteps=200, ckpt=20):
    """Batched differentiable ensemble: 64 LJ-fluid replicas, N log-uniform in
    [500, 32000], per-replica eps and sigma; one pass = set the initial state,
    build the lists, nsteps forward steps with checkpoints every ckpt, and the
    FP64 adjoint of the loss U/N + (2K + W)/(3V) per replica back to
    d(loss)/d(eps, sigma).  All replicas share one handle and one launch per
    kernel."""
    from paper_2109_10876_gb300 import inputs
    sizes, boxes, eps, sig, x, v = inputs.ensemble()
    n = int(sizes.sum())
    R = len(sizes)
    h = md.md_create(sizes, boxes, eps=eps, sigma=sig, rc_over_sigma=RC, skin=SKIN, dt=DT,
                     precision=md.MD_FP32_FIXED)
    xt = torch.tensor(x.T.copy(), device=dev)
    vt = torch.tensor(v.T.copy(), device=dev)
    vol = np.prod(boxes, axis=1)
    g = torch.tensor(np.stack([1.0 / sizes, 2.0 / (3.0 * vol), 1.0 / (3.0 * vol)], axis=1), device=dev)
    euw = torch.zeros(R, 3, dtype=torch.float64, device=dev)
    ge = torch.zeros(R, dtype=torch.float64, device=dev)
    gs = torch.zeros(R, dtype=torch.float64, device=dev)

    def one(mark=False):
        md.md_set_state(h, xt, vt)
        md.md_build_neighbors(h)
        md.md_forward(h, nsteps, ckpt, euw)
        if mark:   # a range a profiler can select
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("adjoint backward")
        md.md_backward(h, None, None, g, ge, gs)
        if mark:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()

    one()                                   # first use: allocations, untimed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(passes):
        one()
    torch.cuda.synchronize()
    dt_s = time.perf_counter() - t0
    one(mark=True)                          # untimed, inside the NVTX range "adjoint backward"
    h.destroy()
    return {"value": passes * n * nsteps / dt_s, "unit": "particle-steps/s (forward + adjoint)",
            "ms_per_pass": 1e3 * dt_s / passes, "passes": passes, "replicas": R, "particles": n,
            "n_min": int(sizes.min()), "n_max": int(sizes.max()), "steps": nsteps, "ckpt_every": ckpt,
            "loss": "U/N + (2K + W)/(3V) per replica",
            "dloss_deps_first3": [float(t) for t in ge[:3].cpu()],
            "dloss_dsigma_first3": [float(t) for t in gs[:3].cpu()],
            "workload": "64 LJ-fluid replicas (fcc sites with vacancies, rho sigma^3 = 0.8442), N log-uniform "
                        "500-32000, eps in [0.9, 1.1], sigma in [0.95, 1.05], rc = 2.5 sigma, skin 0.3, dt 0.005; "
                        "FP32 + fixed-point forward, FP64 adjoint, wall clock of whole passes"}


def timed_steps(md, torch, h, steps, stream):
    """Graph-launched md_step(steps) between CUDA events, with clocks sampled."""
    clocks = Clocks(torch.cuda.current_device())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st0 = md.md_get_stats(h)
    torch.cuda.synchronize()
    e0.record(stream)
    md.md_step(h, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    st1 = md.md_get_stats(h)
    return e0.elapsed_time(e1), st0, st1, ck


def forced_rebuilds(md, torch, h, stream, count=3):
    """Full rebuilds (cell sort + Verlet list) of the current state through
    md_build_neighbors, each timed with CUDA events, inside an NVTX range named
    "forced rebuilds" that a profiler can select."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    try:
        torch.cuda.nvtx.range_push("forced rebuilds")
        pushed = True
    except Exception:                      # no NVTX in this torch build: no range
        pushed = False
    ms = []
    for _ in range(count):
        e0.record(stream)
        md.md_build_neighbors(h)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    if pushed:
        torch.cuda.nvtx.range_pop()
    return {"mean": float(np.mean(ms)), "runs": [round(t, 4) for t in ms],
            "note": "md_build_neighbors on the state after the timed steps: the whole cell sort + "
                    "Verlet-list chain, CUDA events"}


def workload_line(md, torch, dev, args, name, n, h, prep, extra, chain_kernels=None, steps=None, emit=True):
    # systems with bonds or angle triples add one kernel to each rebuild (the
    # slots of their partners)
    chain_kernels = REBUILD_KERNELS if chain_kernels is None else chain_kernels
    steps = args.steps if steps is None else steps
    stream = torch.cuda.current_stream()
    md.md_step(h, max(args.warmup, 3))
    md.md_sync(h)
    ms, st0, st1, ck = timed_steps(md, torch, h, steps, stream)
    rb = st1["rebuilds"] - st0["rebuilds"]
    # a second pass of the same length with per-launch events: where the time goes
    md.md_set_timing(h, True)
    md.md_step(h, steps)
    sect_ms, _ = md.md_get_timing(h)
    md.md_set_timing(h, False)
    reb = forced_rebuilds(md, torch, h, stream)
    line = {"metric": f"{name} particle-steps/s", "value": n * steps / (ms * 1e-3), "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+fixed64 (f64 integration)", "data": "synthetic",
            "config": dict(extra, particles=n, tile_size=st1["tile_size"]),
            "rebuilds": rb, "steps_per_rebuild": steps / max(rb, 1),
            "gpu_launches": 2 * steps + 3 + chain_kernels * rb,
            "mean_list_len": st1["list_entries"] / n, "max_list_len": st1["max_list_len"],
            "max_cell_occupancy": st1["max_cell_occupancy"], "tiles": st1["n_tiles"],
            "max_halo": st1["max_halo"], "preparation": prep, "clocks": ck, "rebuild_ms": reb,
            "sections_ms_per_step": {"neigh": sect_ms[md.MD_SECT_NEIGH] / steps,
                                     "force_integrate": sect_ms[md.MD_SECT_FORCE] / steps,
                                     "other": sect_ms[md.MD_SECT_OTHER] / steps,
                                     "note": "second pass with per-launch events"}}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_melt(md, torch, dev, args, steps=None, emit=True):
    """Polymer melt: 2000 linear chains of 200 beads at bead density 0.85,
    WCA (r_cut = 2^(1/6)) on all pairs, FENE K = 30, R0 = 1.5, Langevin
    gamma = 0.5 at T = 1, dt = 0.01, skin 0.4.  Preparation (untimed): free
    random walks (bond 0.97), the cosine push-off with A ramped 1 -> 100
    (FP64, dt 0.005), then 300 WCA steps at dt 0.005."""
    from paper_2109_10876_gb300 import inputs
    t0 = time.perf_counter()
    x, v, box, bonds = inputs.melt(2000, 200, rho=0.85, T=1.0, seed=4)
    n = len(x)
    xt = torch.tensor(x.T.copy(), device=dev)
    vt = torch.tensor(v.T.copy(), device=dev)
    rc = 2 ** (1 / 6)
    common = dict(skin=0.4, bonds=bonds, fene_K=30.0, fene_R0=1.5, langevin_gamma=0.5, kT=1.0)
    for k, A in enumerate((1.0, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0)):
        hp = md.md_create(n, box, potential=md.MD_SOFT, rc_over_sigma=rc, eps=A, dt=0.005,
                          precision=md.MD_FP64, seed=100 + k, **common)
        md.md_set_state(hp, xt, vt)
        md.md_build_neighbors(hp)
        md.md_step(hp, 300)
        md.md_get_state(hp, xt, vt)
        hp.destroy()
    hw = md.md_create(n, box, potential=md.MD_WCA, dt=0.005, precision=md.MD_FP32_FIXED, seed=200, **common)
    md.md_set_state(hw, xt, vt)
    md.md_build_neighbors(hw)
    md.md_step(hw, 300)
    md.md_get_state(hw, xt, vt)
    hw.destroy()
    h = md.md_create(n, box, potential=md.MD_WCA, dt=0.01, precision=md.MD_FP32_FIXED, seed=4, **common)
    md.md_set_state(h, xt, vt)
    md.md_build_neighbors(h)
    md.md_autotune(h, 10)
    prep = f"free random walks, cosine push-off A = 1..100 (7 x 300 FP64 steps), 300 WCA steps at dt 0.005: " \
           f"{time.perf_counter() - t0:.1f} s"
    line = workload_line(md, torch, dev, args, "polymer melt", n, h, prep,
                         {"workload": f"Kremer-Grest melt, 2000 x 200 linear chains (N = {n}), bead density 0.85, "
                                      f"WCA + FENE (K 30, R0 1.5) + Langevin (gamma 0.5, T 1), dt 0.01, skin 0.4",
                          "l2": "working set about 60 MB (below L2); the timed steps run back to back"},
                         chain_kernels=REBUILD_KERNELS + 1, steps=steps, emit=emit)
    h.destroy()
    return line


def run_rings(md, torch, dev, args, steps=None, emit=True):
    """The paper's own polymer melt: 1600 ring polymers of 200 beads (N =
    320,000) at bead density 0.85, WCA (r_cut = 2^(1/6)) on all pairs, FENE
    (K 30, R0 1.5), the cosine angle term (K 1.5), Langevin gamma 0.5 at T 1,
    dt 0.005, skin 0.4.  Preparation (untimed): closed random walks, the
    cosine push-off with A ramped 1 -> 100 (FP64, bonds and angles on), then
    300 WCA steps."""
    from paper_2109_10876_gb300 import inputs
    t0 = time.perf_counter()
    x, v, box, bonds, angles = inputs.rings(1600, 200, rho=0.85, T=1.0, seed=7)
    n = len(x)
    xt = torch.tensor(x.T.copy(), device=dev)
    vt = torch.tensor(v.T.copy(), device=dev)
    rc = 2 ** (1 / 6)
    common = dict(skin=0.4, bonds=bonds, fene_K=30.0, fene_R0=1.5, angles=angles, angle_K=1.5,
                  langevin_gamma=0.5, kT=1.0)
    for k, A in enumerate((1.0, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0)):
        hp = md.md_create(n, box, potential=md.MD_SOFT, rc_over_sigma=rc, eps=A, dt=0.005,
                          precision=md.MD_FP64, seed=300 + k, **common)
        md.md_set_state(hp, xt, vt)
        md.md_build_neighbors(hp)
        md.md_step(hp, 300)
        md.md_get_state(hp, xt, vt)
        hp.destroy()
    hw = md.md_create(n, box, potential=md.MD_WCA, dt=0.005, precision=md.MD_FP32_FIXED, seed=400, **common)
    md.md_set_state(hw, xt, vt)
    md.md_build_neighbors(hw)
    md.md_step(hw, 300)
    md.md_get_state(hw, xt, vt)
    hw.destroy()
    h = md.md_create(n, box, potential=md.MD_WCA, dt=0.005, precision=md.MD_FP32_FIXED, seed=7, **common)
    md.md_set_state(h, xt, vt)
    md.md_build_neighbors(h)
    md.md_autotune(h, 10)
    prep = f"closed random walks, cosine push-off A = 1..100 (7 x 300 FP64 steps), 300 WCA steps: " \
           f"{time.perf_counter() - t0:.1f} s"
    line = workload_line(md, torch, dev, args, "ring polymer melt", n, h, prep,
                         {"workload": f"ring polymer melt, 1600 x 200 (N = {n}), bead density 0.85, WCA + FENE "
                                      f"(K 30, R0 1.5) + cosine angle (K 1.5) + Langevin (gamma 0.5, T 1), "
                                      f"dt 0.005, skin 0.4",
                          "l2": "working set about 50 MB (below L2); the timed steps run back to back"},
                         chain_kernels=REBUILD_KERNELS + 1, steps=steps, emit=emit)
    h.destroy()
    return line


def run_slab(md, torch, dev, args, steps=None, emit=True):
    """Liquid/vapour slab: 1,000,000 LJ particles, Lz = 4 Lx = 4 Ly, liquid at
    0.80 in the central quarter of z, vapour at 0.02 elsewhere, random
    sequential placement with minimum separation 0.8, T = 0.8, rc 2.5,
    skin 0.3, dt 0.005, NVE."""
    from paper_2109_10876_gb300 import inputs
    t0 = time.perf_counter()
    x, v, box = inputs.slab(1_000_000, rho_l=0.80, rho_v=0.02, T=0.8, seed=3, rmin=0.8)
    n = len(x)
    h = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
    md.md_set_state(h, torch.tensor(x.T.copy(), device=dev), torch.tensor(v.T.copy(), device=dev))
    md.md_build_neighbors(h)
    md.md_autotune(h, 10)
    prep = f"random sequential placement of 1e6 particles: {time.perf_counter() - t0:.1f} s"
    line = workload_line(md, torch, dev, args, "liquid/vapour slab", n, h, prep,
                         {"workload": f"LJ liquid/vapour slab, N = {n}, box {box[0]:.3f} x {box[1]:.3f} x "
                                      f"{box[2]:.3f}, liquid 0.80 / vapour 0.02, T* 0.8, rc 2.5, skin 0.3, dt 0.005, NVE",
                          "l2": "working set about 160 MB (larger than L2)"}, steps=steps, emit=emit)
    h.destroy()
    return line


def run_sphere(md, torch, dev, args, steps=None, emit=True):
    """Spherical inhomogeneous LJ system (the paper's load-imbalance case):
    2.58 million particles at density 0.8442 in a central sphere of a cubic box
    of edge 271, vacuum around it, Langevin thermostat at T = 0.1 (gamma 0.5),
    rc 2.5, skin 0.3, dt 0.005."""
    from paper_2109_10876_gb300 import inputs
    t0 = time.perf_counter()
    x, v, box = inputs.sphere()
    n = len(x)
    h = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED,
                     langevin_gamma=0.5, kT=0.1, seed=6)
    md.md_set_state(h, torch.tensor(x.T.copy(), device=dev), torch.tensor(v.T.copy(), device=dev))
    md.md_build_neighbors(h)
    md.md_autotune(h, 10)
    prep = f"fcc sites nearest the centre: {time.perf_counter() - t0:.1f} s"
    line = workload_line(md, torch, dev, args, "LJ sphere in vacuum", n, h, prep,
                         {"workload": f"LJ sphere, N = {n} at rho 0.8442 (radius 90.0) in a cubic box of edge 271, "
                                      f"Langevin T 0.1 (gamma 0.5), rc 2.5, skin 0.3, dt 0.005",
                          "l2": "working set about 800 MB (larger than L2)"}, steps=steps, emit=emit)
    h.destroy()
    return line


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_2109_10876_gb300 import inputs
    x, v, box = inputs.lj_fluid(args.ncell, rho=RHO, T=T0, seed=2)
    n = len(x)
    s = oracle.System(n, box, rc=RC)
    rng = np.random.default_rng(7)
    t0 = time.perf_counter()
    oracle.forces_sample(s, x, rng.choice(n, 8, replace=False))
    per = max((time.perf_counter() - t0) / 8, 1e-6)
    budget = 120.0                                   # whole run, seconds
    S = int(max(4, min(n, budget / per / max(args.steps + args.warmup, 1))))
    for _ in range(args.warmup):
        oracle.forces_sample(s, x, rng.choice(n, S, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forces_sample(s, x, rng.choice(n, S, replace=False))
    t = time.perf_counter() - t0
    val = S * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"LJ fluid N={n} fcc, rho={RHO}, T*={T0}, rc={RC}, skin={SKIN}, dt={DT}, NVE",
                       "sample_particles_per_step": S},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"per step: exact FP64 forces on {S} sampled particles, each over all N"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    import torch
    from paper_2109_10876_gb300 import inputs
    from paper_2109_10876_gb300 import md

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    if args.workload == "melt":
        run_melt(md, torch, dev, args)
        return
    if args.workload == "rings":
        run_rings(md, torch, dev, args)
        return
    if args.workload == "slab":
        run_slab(md, torch, dev, args)
        return
    if args.workload == "sphere":
        run_sphere(md, torch, dev, args)
        return
    if args.workload == "ensemble":
        line = ensemble_leg(md, torch, dev)
        line.update({"metric": "batched differentiable ensemble particle-steps/s (forward + adjoint)",
                     "n_gpus": 1, "higher_is_better": True, "data": "synthetic"})
        print(json.dumps(line), flush=True)
        return
    x, v, box = inputs.lj_fluid(args.ncell, rho=RHO, T=T0, seed=2 + rank)
    n = len(x)
    xt = torch.tensor(x.T.copy(), device=dev)
    vt = torch.tensor(v.T.copy(), device=dev)

    # ---- device-resident timed run (FP32 pair math + fixed-point sums)
    h = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
    half = args.list == "half"
    if half:
        md.md_set_half_list(h, True)
    md.md_set_state(h, xt, vt)
    md.md_build_neighbors(h)
    tile_size = md.md_autotune(h, 10)     # tile size by timed trial steps (state restored)
    md.md_step(h, max(args.warmup, 3))
    md.md_sync(h)
    st0 = md.md_get_stats(h)
    # timed region: md_step(K) as one CUDA graph launch (conditional rebuilds)
    clocks = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    md.md_step(h, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    st1 = md.md_get_stats(h)
    ms_max = barrier_max(ms, world)
    value = world * n * args.steps / (ms_max * 1e-3)
    # second pass of the same length with per-launch CUDA events (stream launches):
    # the fused force kernel's launch duration for the roofline
    md.md_set_timing(h, True)
    md.md_step(h, args.steps)
    sect_ms, sect_n = md.md_get_timing(h)
    md.md_set_timing(h, False)
    # full rebuilds of the steady-state system (cell sort + Verlet list), each
    # timed with CUDA events, inside an NVTX range that a profiler can select
    reb = forced_rebuilds(md, torch, h, stream)

    # ---- roofline of the dominant kernel (fused force + velocity Verlet)
    mean_nn = st1["list_entries"] / n
    pad = 4
    list_bytes = 2.0 * (mean_nn + (pad - 1) / 2.0)
    bytes_pp = FORCE_FIXED_BYTES + list_bytes + (HALF_SUM_BYTES if half else 0)
    scope_pp = SCOPE_BYTES_HALF if half else SCOPE_BYTES_FULL
    # the force section holds one fused launch per step (two with the half list)
    force_ms = sect_ms[md.MD_SECT_FORCE] / max(sect_n[md.MD_SECT_FORCE], 1)
    achieved = n * scope_pp / (force_ms * 1e-3) / 1e9
    achieved_layout = n * bytes_pp / (force_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    digest = csrc_digest()
    tpp = profiled_traffic(digest)
    # the resource that binds the kernel in practice: instruction issue (four
    # schedulers per SM, one warp instruction each per cycle), from the profiled
    # warp instructions per particle and the live launch time
    ipp = profiled(digest, "warp_instructions_per_particle")
    issue = None
    if ipp is not None and not half:
        sm_mhz = (ck or {}).get("sm_mhz") or 2070.0
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        ach = n * ipp / (force_ms * 1e-3)
        pk = 4.0 * nsm * sm_mhz * 1e6
        issue = {"bound": "issue", "achieved": round(ach / 1e9, 1), "peak": round(pk / 1e9, 1),
                 "unit": "G warp-instructions/s", "frac": round(ach / pk, 4),
                 "note": "4 schedulers x the SMs x the median SM clock under load; warp instructions "
                         "per particle from the committed ncu summary of this kernel's sources"}
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": None if (tpp is None or half) else round(tpp * n),
                "peak_source": peak_kind,
                "kernel": "k_pairs_half + k_force<FP32, fused, half>" if half else "k_force<FP32, fused>",
                "algorithmic_bytes_per_particle": round(scope_pp, 1),
                "bytes_note": "force + integrate per particle, " + ("half" if half else "full") +
                              " list with 4-byte indices at 82.4 entries (twice the paper's 41.2 neighbours), "
                              "rebuild excluded",
                "layout_bytes_per_particle": round(bytes_pp, 1),
                "layout_achieved": round(achieved_layout, 1),
                "layout_frac": round(achieved_layout / peak, 4),
                "layout_note": "the bytes this layout needs: 2-byte halo indices at the live mean list length "
                               "plus padding, 32-bit fixed-point positions",
                "launch_ms": round(force_ms, 4)}

    extras = {}
    if not args.no_extras:
        # ---- the same steps with (U, K, W) recorded every step: the energy
        # variants of the force kernels, still one graph launch
        thd = torch.zeros(args.steps, 3, dtype=torch.float64, device=dev)
        md.md_step(h, 3, 1, thd)
        torch.cuda.synchronize()
        e0.record(stream)
        md.md_step(h, args.steps, 1, thd)
        e1.record(stream)
        torch.cuda.synchronize()
        msE = e0.elapsed_time(e1)
        extras["energies_every_step"] = {"value": world * n * args.steps / (msE * 1e-3), "unit": UNIT,
                                         "ms_per_step": msE / args.steps, "steps": args.steps}
        # ---- end to end through the C ABI with pinned host buffers: upload the
        # state, build, K steps with (U, K, W) every step, download the state
        xh = torch.tensor(x.T.copy()).pin_memory()
        vh = torch.tensor(v.T.copy()).pin_memory()
        th = torch.zeros(args.steps, 3, dtype=torch.float64).pin_memory()
        xo = torch.zeros(3, n, dtype=torch.float64).pin_memory()
        vo = torch.zeros(3, n, dtype=torch.float64).pin_memory()
        h2 = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
        md.md_set_state(h2, xh, vh)          # first use: allocations and page-in, untimed
        md.md_build_neighbors(h2)
        md.md_step(h2, 3, 1, th)
        md.md_sync(h2)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        md.md_set_state(h2, xh, vh)
        md.md_build_neighbors(h2)
        md.md_step(h2, args.steps, 1, th)
        md.md_get_state(h2, xo, vo)
        t_e2e = time.perf_counter() - t0
        t_e2e = barrier_max(t_e2e, world)
        thermo = th.numpy()
        E = thermo[:, 0] + thermo[:, 1]
        extras["e2e"] = {"value": world * n * args.steps / t_e2e, "unit": UNIT,
                         "h2d_bytes_per_step": 2 * 3 * n * 8 / args.steps,
                         "d2h_bytes_per_step": (2 * 3 * n * 8 + 3 * 8 * args.steps) / args.steps,
                         "includes": "set_state from pinned host, list build, K steps with (U,K,W) "
                                     "every step, get_state to pinned host"}
        extras["nve"] = {"steps": args.steps, "E0_per_particle": float(E[0] / n),
                         "rel_drift": float((E[-1] - E[0]) / abs(E[0])),
                         "max_rel_dev": float(np.max(np.abs(E - E[0])) / abs(E[0]))}
        h2.destroy()

        # ---- the plain FP64 path on the same input
        k64 = max(5, min(args.steps, 20))
        h3 = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP64)
        md.md_set_state(h3, xt, vt)
        md.md_build_neighbors(h3)
        md.md_step(h3, 3)
        md.md_sync(h3)
        torch.cuda.synchronize()
        e0.record(stream)
        md.md_step(h3, k64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        h3.destroy()
        v64 = n * k64 / (ms64 * 1e-3)
        # algorithmic FP64 rate of the pair sums: list entries from the timed
        # run's mean length, interacting pairs from the density (4/3 pi rc^3 rho)
        n_in = 4.0 / 3.0 * math.pi * RC ** 3 * RHO
        ops = n * (n_in * FP64_OPS_IN + max(mean_nn - n_in, 0.0) * FP64_OPS_OUT)
        tf = ops / (ms64 / k64 * 1e-3) / 1e12
        # the FP64 FMA rate of this GPU, measured by the library's probe (FMA
        # chains on every SM; 2 flops per FMA)
        fp64_peak, fp64_ms = md.md_probe_fp64_fma(100000, 4)
        extras["fp64"] = {"value": world * v64, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64,
                          "speedup_fp32_fixed_over_fp64": (value / world) / v64,
                          "roofline": {"bound": "fp64", "achieved": round(tf, 4), "peak": round(fp64_peak, 4),
                                       "unit": "TFLOP/s", "frac": round(tf / fp64_peak, 4),
                                       "peak_source": "measured: md_probe_fp64_fma, FP64 FMA chains on every SM "
                                                      f"({fp64_ms:.1f} ms launch)",
                                       "nominal_peak": FP64_NOMINAL_TFLOPS},
                          "ops_per_step": ops,
                          "note": "FP64 operations of the pair sums by count per list entry (12 beyond r_cut, 26 "
                                  "within); the FP64 path also integrates in FP64"}

        # ---- the other list form on the same input (Sec. 2.1.2: the half list
        # of Newton's third law against the full list)
        kh = max(20, min(args.steps, 200))
        h5 = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
        md.md_set_tile_size(h5, tile_size)
        md.md_set_half_list(h5, not half)
        md.md_set_state(h5, xt, vt)
        md.md_build_neighbors(h5)
        md.md_step(h5, 3)
        md.md_sync(h5)
        torch.cuda.synchronize()
        e0.record(stream)
        md.md_step(h5, kh)
        e1.record(stream)
        torch.cuda.synchronize()
        msh = e0.elapsed_time(e1)
        md.md_set_timing(h5, True)
        md.md_step(h5, kh)
        sms, sn = md.md_get_timing(h5)
        h5.destroy()
        vh_ = n * kh / (msh * 1e-3)
        extras["half_list" if not half else "full_list"] = {
            "value": world * vh_, "unit": UNIT, "ms_per_step": msh / kh, "steps": kh,
            "force_ms_per_step": sms[md.MD_SECT_FORCE] / max(sn[md.MD_SECT_FORCE], 1),
            "neigh_ms_per_step": sms[md.MD_SECT_NEIGH] / kh,
            "ratio_to_timed_run": vh_ / (value / world),
            "note": "graph-launched steps on the same input; force_ms_per_step from a second pass "
                    "with per-launch events (the half list's force step is two kernels)"}

        # ---- NVE energy over the workload's own 1000 steps from the lattice
        # (records every step; the first 100 steps hold the lattice's melting)
        nE = 1000
        h6 = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
        md.md_set_tile_size(h6, tile_size)
        md.md_set_state(h6, xt, vt)
        md.md_build_neighbors(h6)
        th6 = torch.zeros(nE, 3, dtype=torch.float64, device=dev)
        md.md_step(h6, nE, 1, th6)
        md.md_sync(h6)
        h6.destroy()
        E6 = (th6[:, 0] + th6[:, 1]).cpu().numpy()
        tail = E6[100:]
        slope = float(np.polyfit(np.arange(len(tail)) * DT, tail / n, 1)[0])
        extras["nve_1000"] = {"steps": nE, "E0_per_particle": float(E6[0] / n),
                              "rel_drift": float((E6[-1] - E6[0]) / abs(E6[0])),
                              "max_rel_dev": float(np.max(np.abs(E6 - E6[0])) / abs(E6[0])),
                              "rel_drift_steps_100_to_1000": float((E6[-1] - E6[100]) / abs(E6[100])),
                              "drift_per_particle_per_tau_after_100": slope,
                              "note": "FP32 pairs + fixed-point sums, FP64 integration; (U + K) recorded every step"}

        # ---- the other workloads of the paper at full size (one GB300 each)
        kx = max(100, min(args.steps, 500))
        extras["slab"] = run_slab(md, torch, dev, args, steps=kx, emit=False)
        extras["sphere"] = run_sphere(md, torch, dev, args, steps=kx, emit=False)
        extras["melt"] = run_melt(md, torch, dev, args, steps=kx, emit=False)
        extras["rings"] = run_rings(md, torch, dev, args, steps=kx, emit=False)

        extras["ensemble"] = ensemble_leg(md, torch, dev)

        if world == 1 and rank == 0:
            import oracle
            # ---- force error of the FP32 path on a perturbed lattice of the same size
            xp, vp, _ = inputs.perturbed_lattice(args.ncell, rho=RHO, T=T0, seed=5, amp=0.1)
            h4 = md.md_create(n, box, rc_over_sigma=RC, skin=SKIN, dt=DT, precision=md.MD_FP32_FIXED)
            md.md_set_state(h4, torch.tensor(xp.T.copy(), device=dev), torch.tensor(vp.T.copy(), device=dev))
            md.md_build_neighbors(h4)
            f = torch.zeros(3, n, dtype=torch.float64, device=dev)
            md.md_compute_forces(h4, f, None)
            md.md_sync(h4)
            h4.destroy()
            idx = np.random.default_rng(9).choice(n, 256, replace=False)
            Fo, _, _ = oracle.forces_sample(oracle.System(n, box, rc=RC), xp, idx)
            Fg = f.cpu().numpy().T[idx]
            mag = np.linalg.norm(Fo, axis=1)
            rms = float(np.sqrt(np.mean(mag ** 2)))
            extras["force_error"] = {"sample": 256, "max_rel": float(np.max(np.linalg.norm(Fg - Fo, axis=1) /
                                                                           np.maximum(mag, rms))),
                                     "input": "fcc lattice with uniform +-0.1 sigma displacements"}
            extras["cpu_baseline"] = cpu_baseline(x, box)
            extras["lj_fluid_4000"] = config_4000_leg(md, torch, dev, e0, e1, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+fixed64 (f64 integration)",
                "data": "synthetic",
                "config": {"workload": f"LJ fluid N={n} per GPU (fcc {args.ncell}^3 x 4), rho={RHO}, T*={T0}, "
                                       f"rc={RC} shifted, skin={SKIN}, dt={DT}, NVE, FP32 pairs + 64-bit fixed-point "
                                       f"sums, {args.list} Verlet list", "particles_per_gpu": n,
                           "tile_size": tile_size,
                           "parallelism": "replicas only" if world > 1 else "1 GPU",
                           "l2": "working set larger than L2 (positions, velocities and the Verlet list: "
                                 f"~{(n * (FORCE_FIXED_BYTES + list_bytes)) / 1e6:.0f} MB touched per step)"},
                "roofline": roofline,
                "issue_roofline": issue,
                "gpu_launches": (3 if half else 2) * args.steps + 3 +
                                REBUILD_KERNELS * (st1["rebuilds"] - st0["rebuilds"]),
                "rebuilds": st1["rebuilds"] - st0["rebuilds"],
                "sections_ms_per_step": {"neigh": sect_ms[md.MD_SECT_NEIGH] / args.steps,
                                         "force_integrate": sect_ms[md.MD_SECT_FORCE] / args.steps,
                                         "other": sect_ms[md.MD_SECT_OTHER] / args.steps,
                                         "note": "second pass with per-launch events; the timed value "
                                                 "is the graph-launched pass"},
                "mean_list_len": mean_nn,
                "rebuild_ms": reb,
                "clocks": ck,
                "csrc_sha": digest}
        line.update(extras)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line), flush=True)
    h.destroy()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
