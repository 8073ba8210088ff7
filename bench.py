#!/usr/bin/env python
"""Benchmark of the P3T tree side on B300.

One step = one leapfrog (kick-drift-kick) step of the soft part on a Plummer
sphere of N = 2^20 equal-mass particles in N-body units (r_out = 0.0025,
r_in = 0.1 r_out, theta = 0.4, eps = 4/N, h = r_out, dt = 1/256, groups of
<= 64, leaves of <= 16):
    kick(dt/2) -> drift(dt) -> build tree -> long-range force (walk + force
    kernel, neighbour counts) -> neighbour lists -> kick(dt/2)
all through the C ABI of libp3t.  ``value`` is particles per second of whole
steps with the data resident in HBM; ``e2e`` adds the host<->device copies of
the step's inputs and outputs from/to pinned host memory.  The working set of
a step (particles, tree, lists: ~0.5 GB) is larger than L2, so no flush is
done between steps.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (tree build and walk over all particles, forces
of a random subset of groups, scaled by the subset fraction).

Multi-GPU (torchrun): every rank runs its own independent cluster (replicas,
weak scaling); ranks meet only at the timing barrier.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

N_DEFAULT = 1 << 20
THETA = 0.4
R_OUT = 0.0025
GAMMA = 0.1
DT = 1.0 / 256.0
N_LEAF = 16
N_GROUP = 64
SEED = 2

# FP32 flops per interaction (FMA = 2), fixed from the force kernel source
# Algorithmic bytes of the HBM-side steps.  Build: read x and m (32 B),
# write key and index (12 B), 8 radix passes reading and writing both (192
# B), FP64 and FP32 Morton-order copies (64 B) per particle; FP64 moments,
# box and FP32 records per cell (228 B).  Kick: read and write v (48 B),
# read a (12 B).  Drift: read and write x (48 B), read v (24 B).
B_BUILD_PER_PARTICLE = 32 + 12 + 8 * 24 + 64
B_BUILD_PER_CELL = 228
B_KICK = 60
B_DRIFT = 72
FLOPS_PC = 48
FLOPS_PP_FAR = 18
FLOPS_PP_NEAR = 31
# FP32 flops per interaction of the backward kernel (FMA = 2), fixed from its
# source: the cell term's J^T w, dL/dM and twice the quadrupole adjoint (121)
# and the three adds that sum J^T w over the sources; far and near particle
# terms likewise (35 + 3, 64 + 3).
FLOPS_BWD_PC = 124
FLOPS_BWD_PP_FAR = 38
FLOPS_BWD_PP_NEAR = 67
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-p3t", action="store_true")
    ap.add_argument("--no-king", action="store_true")
    ap.add_argument("--no-cost-model", action="store_true")
    ap.add_argument("--no-smbh", action="store_true")
    return ap.parse_args()


def workload_name(n):
    return (f"plummer_n{n}_theta{THETA}_rout{R_OUT}_kdk_dt1/256"
            f"_nleaf{N_LEAF}_ngroup{N_GROUP}")


def config(n, world):
    return {"workload": workload_name(n), "n": n, "theta": THETA,
            "r_out": R_OUT, "gamma": GAMMA, "eps": 4.0 / n, "h": R_OUT,
            "dt": DT, "n_leaf": N_LEAF, "n_group": N_GROUP,
            "model": "Plummer sphere, N-body units, equal masses",
            "parallelism": f"replicas x{world}",
            "l2": "no flush: per-step working set ~0.5 GB > 126 MB L2"}


def measured_peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def force_and_neighbours(ctx, acc, off, idx, side):
    """The force on the current stream and the neighbour lists on `side`,
    concurrently: both read the same tree (separate work counters), and the
    neighbour walk fills the SMs that the force kernel's tail leaves idle."""
    import torch
    cur = torch.cuda.current_stream()
    side.wait_stream(cur)
    ctx.long_force(acc, check=False)
    with torch.cuda.stream(side):
        ctx.neighbours_into(off, idx, sync=False)
    cur.wait_stream(side)


def fp32_peak_tflops(dev):
    """Nominal FP32 FMA peak: SMs x 128 lanes x 2 flops x the maximum SM
    clock recorded in MEASURED_PEAKS.json (2032 MHz if absent)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = float(measured_peaks().get("sm_max_mhz", 2032.0))
    return sms * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12


def profile_traffic(name="k_walk_force_plummer_1M.txt"):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary (a
    line 'dram_bytes_per_launch: <float>'), else None."""
    path = os.path.join(HERE, "profiles", name)
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_launch:"):
                return float(line.split(":", 1)[1])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms.  start()
    returns once the first sample (taken before the timed region, and
    dropped) has arrived, so the sampler is live when timing begins."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.proc.stdout.readline()  # first sample: before the timed region
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def reduce_max(value, device):
    """Max of a float over all ranks (the timing rule: the slowest rank sets
    the step time); identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, steps, ms_max, world):
    """Particles per second of the whole job: all ranks' particles over the
    slowest rank's time."""
    return world * n_per_rank * steps / (ms_max * 1e-3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------
# CPU reference arm / baseline: the FP64 oracle on the host cores
# --------------------------------------------------------------------------

SUBSAMPLE = 4096  # fixed subsample of the 16-step workload: the first 4096
                  # of a seeded permutation


def err_stats(a, ref):
    """Median, 99th percentile and maximum of the per-particle relative error
    |a - ref| / max(|ref|, 1e-3 rms|ref|) (vectors: rows; scalars: entries)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        a, ref = a[:, None], ref[:, None]
    nr = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(nr ** 2))
    e = np.linalg.norm(a - ref, axis=1) / np.maximum(nr, floor)
    return {"median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
            "max": float(e.max()), "n": int(e.size)}


def _timed(fn):
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0


def cpu_baseline_and_accuracy(gs):
    """The FP64 oracle on the host cores, on bounded samples of the GPU arm's
    workloads, and, from the same oracle results, the error of the GPU's
    outputs on those samples.  gs holds the GPU's inputs and outputs (host
    arrays, particles as rows):

    * kdk: the 16-step workload's state after the timed steps (positions,
      forces).  Timed: oracle tree build + walk over all particles, forces of
      random groups holding 1/16 of the particles, scaled (the baseline
      value, all cores); direct summation on the fixed subsample.  Accuracy:
      the subsample against the same-tree oracle and against direct sums.
    * cfg1: Plummer N = 8192, r_out 0.01, in full.  Timed: tree and direct,
      all cores and one core (the paper's one-core setup, Sect. 3.1.2).
      Accuracy: every particle; neighbour rows compared bit for bit.
    * vjp: Plummer N = 65536, r_out 0.005, loss sum w.a (seeded Gaussian
      w).  Timed: oracle forward + gradient.  Accuracy: dL/dx, dL/dm.
    * ensemble: eight clusters of the ensemble spanning its sizes (the
      largest included), forces and gradients.
    * king: the dense-core workload after its timed steps; oracle build +
      walk and forces of groups holding 1/64 of the particles (timed, scaled);
      accuracy of those particles.
    Returns (cpu_baseline, accuracy)."""
    import oracle
    cores = os.cpu_count() or 1
    base, acc_out, legs = {}, {}, {}

    # --- the 16-step workload (the bench's step) ---
    k = gs["kdk"]
    n = k["pos"].shape[0]
    tree, t_build = _timed(lambda: oracle.Tree(k["pos"], k["m"], n_leaf=N_LEAF,
                                               n_group=N_GROUP))
    _, t_walk = _timed(lambda: tree.walk(THETA, R_OUT, R_OUT))
    g = tree.groups()
    sel = np.random.default_rng(0).permutation(tree.ngroup)
    cum = np.cumsum(g["count"][sel])
    sel = sel[:int(np.searchsorted(cum, n / 16)) + 1]
    covered = int(g["count"][sel].sum())
    _, t_force = _timed(lambda: tree.force(eps=4.0 / n, r_cut=R_OUT, gamma=GAMMA,
                                           groups=sel))
    t_step = t_build + t_walk + t_force * n / covered
    base = {"value": n / t_step, "unit": "particles/s", "cores": cores,
            "kind": "oracle",
            "sample": f"oracle tree build + walk over all {n} particles, forces "
                      f"of {len(sel)} random groups ({covered} particles) scaled "
                      f"by {n / covered:.2f}; neighbour lists and kick/drift not "
                      f"included"}
    sub = k["sub"]
    a_tree = tree.force_particles(sub, eps=4.0 / n, r_cut=R_OUT, gamma=GAMMA)
    a_dir, t_dir = _timed(lambda: oracle.direct(k["pos"], k["m"], eps=4.0 / n,
                                                r_cut=R_OUT, gamma=GAMMA,
                                                rows=sub))
    legs["direct_subsample"] = {
        "value": len(sub) / t_dir, "unit": "particles/s", "cores": cores,
        "sample": f"O-direct of {len(sub)} particles against all {n}"}
    acc_out["force_16step_subsample"] = dict(
        err_stats(k["acc"][sub], a_tree), after_steps=k["steps"],
        vs_direct=err_stats(k["acc"][sub], a_dir),
        oracle_tree_vs_direct=err_stats(a_tree, a_dir))

    # --- config 1 in full, all cores and one core ---
    c = gs["cfg1"]
    n1 = c["pos"].shape[0]
    for th, name in ((None, "all_cores"), (1, "one_core")):
        def tree_full():
            t = oracle.Tree(c["pos"], c["m"], n_leaf=N_LEAF, n_group=N_GROUP)
            t.walk(THETA, 0.01, 0.01, threads=th)
            return t.force(eps=4.0 / n1, r_cut=0.01, gamma=GAMMA, threads=th)
        a1, tt = _timed(tree_full)
        d1, td = _timed(lambda: oracle.direct(c["pos"], c["m"], eps=4.0 / n1,
                                              r_cut=0.01, gamma=GAMMA,
                                              threads=th))
        legs[f"cfg1_{name}"] = {"tree": n1 / tt, "direct": n1 / td,
                                "unit": "particles/s",
                                "cores": cores if th is None else 1}
    off_o, idx_o = oracle.neighbours(c["pos"], 0.01)
    rows_eq = int(sum(np.array_equal(c["idx"][c["off"][i]:c["off"][i + 1]],
                                     idx_o[off_o[i]:off_o[i + 1]])
                      for i in range(n1)))
    acc_out["force_cfg1_full"] = dict(
        err_stats(c["acc"], a1), vs_direct=err_stats(c["acc"], d1),
        neighbour_rows_identical=f"{rows_eq}/{n1}",
        offsets_identical=bool(np.array_equal(c["off"], off_o)))

    # --- gradient workload ---
    v = gs["vjp"]
    n4 = v["pos"].shape[0]
    r4 = 0.01 * (n4 / 8192) ** (-1.0 / 3.0)

    def fwd_bwd():
        t = oracle.Tree(v["pos"], v["m"], n_leaf=N_LEAF, n_group=N_GROUP)
        t.walk(THETA, r4, r4)
        a = t.force(eps=4.0 / n4, r_cut=r4, gamma=GAMMA)
        return (a,) + t.vjp(v["w"], eps=4.0 / n4, r_cut=r4, gamma=GAMMA)
    (a4, ox, om), t4 = _timed(fwd_bwd)
    legs["vjp_fwd_bwd"] = {"value": n4 / t4, "unit": "particles/s (fwd+bwd)",
                           "cores": cores}
    acc_out["vjp_65536"] = {"force": err_stats(v["acc"], a4),
                            "dL_dx": err_stats(v["gx"], ox),
                            "dL_dm": err_stats(v["gm"], om)}

    # --- ensemble: sampled clusters ---
    e = gs.get("ensemble")
    if e:
        fa, fo, xa, xo, ma, mo = [], [], [], [], [], []
        te = 0.0
        for cl in e["clusters"]:
            def one():
                t = oracle.Tree(cl["pos"], cl["m"], n_leaf=e["n_leaf"],
                                n_group=e["n_group"])
                t.walk(THETA, cl["r_out"], cl["r_out"])
                a = t.force(eps=cl["eps"], r_cut=cl["r_out"], gamma=GAMMA)
                return (a,) + t.vjp(cl["w"], eps=cl["eps"], r_cut=cl["r_out"],
                                    gamma=GAMMA)
            (a, gx, gm), dt = _timed(one)
            te += dt
            fa.append(cl["acc"]), fo.append(a)
            xa.append(cl["gx"]), xo.append(gx)
            ma.append(cl["gm"]), mo.append(gm)
        ne = sum(len(x) for x in fo)
        legs["ensemble_sample"] = {"value": ne / te,
                                   "unit": "particles/s (fwd+bwd)",
                                   "cores": cores,
                                   "sample": f"{len(fo)} clusters, {ne} particles"}
        # errors per cluster (each cluster's own rms floor), pooled
        def pooled(xs, rs):
            errs = []
            for a, r in zip(xs, rs):
                a = a if a.ndim == 2 else a[:, None]
                r = r if r.ndim == 2 else r[:, None]
                nr = np.linalg.norm(r, axis=1)
                fl = 1e-3 * np.sqrt(np.mean(nr ** 2))
                errs.append(np.linalg.norm(a - r, axis=1) / np.maximum(nr, fl))
            q = np.concatenate(errs)
            return {"median": float(np.median(q)), "p99": float(np.quantile(q, 0.99)),
                    "max": float(q.max()), "n": int(q.size)}
        acc_out["ensemble_sampled"] = {
            "cluster_sizes": [len(x) for x in fo],
            "force": pooled(fa, fo), "dL_dx": pooled(xa, xo),
            "dL_dm": pooled(ma, mo)}

    # --- King W0 = 9 ---
    kg = gs.get("king")
    if kg:
        nk = kg["pos"].shape[0]
        tk, tb = _timed(lambda: oracle.Tree(kg["pos"], kg["m"], n_leaf=N_LEAF,
                                            n_group=N_GROUP))
        _, tw = _timed(lambda: tk.walk(kg["theta"], kg["r_out"], kg["r_out"]))
        g = tk.groups()
        sel = np.random.default_rng(1).permutation(tk.ngroup)
        sel = sel[:int(np.searchsorted(np.cumsum(g["count"][sel]), nk / 64)) + 1]
        cov = int(g["count"][sel].sum())
        ak, tf = _timed(lambda: tk.force(eps=4.0 / nk, r_cut=kg["r_out"],
                                         gamma=GAMMA, groups=sel))
        _, order = tk.particles()
        rows = np.concatenate([order[g["first"][q]:g["first"][q] + g["count"][q]]
                               for q in sel])
        legs["king"] = {"value": nk / (tb + tw + tf * nk / cov),
                        "unit": "particles/s", "cores": cores,
                        "sample": f"tree build + walk over all {nk}, forces of "
                                  f"{len(sel)} groups ({cov} particles) scaled"}
        acc_out["force_king_sampled"] = err_stats(kg["acc"][rows], ak[rows])
    base["legs"] = legs
    acc_out["measure"] = ("per-particle |x - x_ref| / max(|x_ref|, 1e-3 rms "
                          "|x_ref|) against the same-tree FP64 oracle (R12); "
                          "vs_direct: against FP64 direct summation")
    acc_out["targets"] = "forces: median <= 1e-5, max <= 1e-4"
    return base, acc_out


def run_reference(args, world, rank):
    """The oracle on the host cores.  Its tree build and walk over all
    particles are timed once; every step then times the forces of a random
    1/256 of the groups (a different sample per step) and estimates the full
    step as build + walk + those forces scaled to all particles.  This keeps
    the run to well under a minute for any --steps."""
    if rank != 0:
        return
    import oracle
    from paper_1506_04553_b300 import ics
    n = args.n
    pos, vel, mass = ics.plummer(n, SEED)
    cores = os.cpu_count() or 1
    p = np.ascontiguousarray(pos.T)
    t0 = time.perf_counter()
    tree = oracle.Tree(p, mass, n_leaf=N_LEAF, n_group=N_GROUP)
    t1 = time.perf_counter()
    tree.walk(THETA, R_OUT, R_OUT)
    t2 = time.perf_counter()
    t_build_walk = t2 - t0
    g = tree.groups()

    def forces(seed, frac=1 / 256):
        rng = np.random.default_rng(seed)
        sel = rng.permutation(tree.ngroup)
        k = int(np.searchsorted(np.cumsum(g["count"][sel]), frac * n)) + 1
        sel = sel[:k]
        ta = time.perf_counter()
        tree.force(eps=4.0 / n, r_cut=R_OUT, gamma=GAMMA, groups=sel)
        return time.perf_counter() - ta, int(g["count"][sel].sum()), k

    for w in range(args.warmup):
        forces(10_000 + w)
    ts, tfs = [], []
    for st in range(args.steps):
        tf, covered, k = forces(st)
        tfs.append(tf)
        ts.append(t_build_walk + tf * n / covered)
    t_step = float(np.mean(ts))
    value = n / t_step
    desc = (f"oracle tree build + walk over all {n} particles "
            f"({t_build_walk:.2f} s, timed once), plus per step the forces of "
            f"~1/256 of the groups (about {covered} particles, a new random "
            f"sample each step) scaled to all particles; neighbour lists and "
            f"kick/drift not included")
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(tfs)),
            "value_is_estimate": "yes: value = N / (build + walk + the sampled "
                                 "forces x N / sampled particles); ms_per_step "
                                 "is the measured time of one sampled step (the "
                                 "1/256 force sample), estimated_full_step_ms "
                                 "the extrapolated whole step",
            "estimated_full_step_ms": 1e3 * t_step,
            "build_walk_ms_once": 1e3 * t_build_walk,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config(n, world),
            "cpu_baseline": {"value": value, "unit": "particles/s",
                             "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "particles/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = ("long-range tree force particles/s & Gint/s at N=2^20 theta=0.4; "
          "fwd+bwd vs fwd ratio")


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    pos_h, vel_h, mass_h = ics.plummer(n, SEED + rank)
    params = P.Params(theta=THETA, r_out=R_OUT, gamma=GAMMA, eps=4.0 / n,
                      h=R_OUT, G=1.0, n_leaf=N_LEAF, n_group=N_GROUP)
    ctx = P.Context(params)
    stream = torch.cuda.current_stream(dev)
    pos = torch.tensor(pos_h, device=dev)
    vel = torch.tensor(vel_h, device=dev)
    mass = torch.tensor(mass_h, device=dev)
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    off = torch.empty((n + 1,), dtype=torch.int64, device=dev)

    # initial force and neighbour capacity
    ctx.build_tree(pos, mass)
    ctx.long_force(acc, check=True)
    _, idx0 = ctx.neighbours()
    cap = max(4 * int(idx0.numel()) + 1024, n)
    idx = torch.empty((cap,), dtype=torch.int32, device=dev)
    ngb_stream = torch.cuda.Stream(dev)

    def step(sequential=False):
        P.kick(vel, acc, 0.5 * DT)
        P.drift(pos, vel, DT)
        ctx.build_tree(pos, mass)
        if sequential:  # phase times: one stream
            ctx.long_force(acc, check=False)
            ctx.neighbours_into(off, idx, sync=False)
        else:
            force_and_neighbours(ctx, acc, off, idx, ngb_stream)
        P.kick(vel, acc, 0.5 * DT)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l_a = P.launch_count()
    step()
    torch.cuda.synchronize()
    launches_per_step = P.launch_count() - l_a

    # profiled steps without a graph: phase times and interaction counts
    ctx.profile(reset=True)
    ctx.profile_enable(True)
    kp = max(2, min(args.steps, 4))
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(kp):
        step(sequential=True)
    p1.record(stream)
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    prof = ctx.profile(reset=True)
    ms_nograph = p0.elapsed_time(p1) / kp

    # the timed steps: one KDK step captured in a CUDA graph (no host sync,
    # no allocation), replayed K times
    ctx.set_params(P.Params(theta=THETA, r_out=R_OUT, gamma=GAMMA, eps=4.0 / n,
                            h=R_OUT, G=1.0, n_leaf=N_LEAF, n_group=N_GROUP,
                            flags=P.FLAG_NO_SYNC))
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = P.launch_count()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()  # any error latched on the device during the timed steps
    clocks = sampler.stop()
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    gs = {}  # the GPU's inputs and outputs for the oracle leg (host arrays)
    if want_cpu:
        # the forces of the last step were evaluated at these positions
        gs["kdk"] = {"pos": pos.cpu().numpy().T.copy(), "m": mass_h,
                     "acc": acc.cpu().numpy().T.astype(np.float64),
                     "sub": np.random.default_rng(SEED).permutation(n)[:SUBSAMPLE],
                     "steps": 2 * args.warmup + 1 + kp + args.steps + 1}
    # a replay relaunches the kernels captured from one step
    launches = (P.launch_count() - l0) + args.steps * launches_per_step
    ms = reduce_max(e0.elapsed_time(e1), dev)
    ms_step = ms / args.steps
    value = whole_job_rate(n, args.steps, ms, world)
    ctx.set_params(params)

    # HBM-side steps: kick and drift alone, `reps` launches captured in a
    # CUDA graph so that host launch costs stay out (arrays exceed L2)
    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                fn()
        g.replay()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    kick_ms = timed(lambda: P.kick(vel, acc, 0.0))
    drift_ms = timed(lambda: P.drift(pos, vel, 0.0))
    st = ctx.stats()
    cells_per_particle = st["n_cells"] / n
    alu = P.alu_peaks()

    # interactions and roofline of the force kernel
    int_pc, int_pp, int_ppn = prof["int_pc"], prof["int_pp"], prof["int_pp_near"]
    nprof = max(prof["forces"], 1)
    flops = FLOPS_PC * int_pc + FLOPS_PP_NEAR * int_ppn + FLOPS_PP_FAR * (int_pp - int_ppn)
    force_s = prof["force_ms"] * 1e-3
    achieved = flops / force_s / 1e12 if force_s > 0 else None
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = float(peaks.get("sm_max_mhz", 2032.0))
    peak = fp32_peak_tflops(dev)
    traffic = profile_traffic()
    gint = world * (int_pc + int_pp) / nprof / (ms_step * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": "particles/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "precision": "FP32 group-relative interactions with compensated sums; "
                     "FP64 positions, moments, kick, drift; FP64 exact "
                     "neighbour predicate",
        "data": "synthetic", "config": config(n, world),
        "gint_per_s": gint,
        "interactions_per_particle": {"pc": int_pc / (n * nprof),
                                      "pp": int_pp / (n * nprof)},
        "phase_ms_per_step": {"build": prof["build_ms"] / nprof,
                              "walk_and_force": prof["force_ms"] / nprof,
                              "neighbours": prof["ngb_ms"] / nprof,
                              "note": "CUDA events per phase, steps without "
                                      "the graph, on one stream"},
        "no_graph": {"ms_per_step": ms_nograph,
                     "value": world * n / (ms_nograph * 1e-3),
                     "note": "the same steps, one stream"},
        "timing": "K replays of one KDK step captured in a CUDA graph; the "
                  "neighbour lists run on a second stream beside the force",
        "force_particles_per_s": world * n * nprof / force_s if force_s else None,
        "fwd_bwd_ratio": None,
        "roofline": {"kernel": "k_walk_force", "bound": "alu",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": traffic,
                     "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum "
                                       "of one ncu capture of this kernel on this "
                                       "workload, read from the committed summary "
                                       "profiles/k_walk_force_plummer_1M.txt (not "
                                       "measured in this run)",
                     "peak_note": f"FP32 FMA: {sms} SMs x 128 lanes x 2 x "
                                  f"{clk:.0f} MHz (max SM clock)"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # measured ALU ceilings beside the nominal peak (p3t_alu_peaks)
    fma_meas = max(alu["fma_flops"], alu["fma2_flops"]) / 1e12
    line["roofline"]["peak_measured"] = {
        "fp32_fma_tflops": alu["fma_flops"] / 1e12,
        "fp32x2_fma_tflops": alu["fma2_flops"] / 1e12,
        "rsqrt_tops": alu["rsqrt_ops"] / 1e12,
        "note": "register-only FMA and rsqrt loops on every SM (p3t_alu_peaks)"}
    line["roofline"]["frac_of_measured"] = achieved / fma_meas if achieved else None
    # HBM-bound steps against the measured copy bandwidth
    hbm = float(peaks.get("hbm_gbs", 6518.0))
    b_build = (B_BUILD_PER_PARTICLE + B_BUILD_PER_CELL * cells_per_particle) * n
    build_ms = prof["build_ms"] / nprof
    nb_ = max(prof["builds"], 1)
    cells = cells_per_particle * n

    def sub(name, nbytes, note):
        ms_ = prof[f"build_{name}_ms"] / nb_
        out = {"ms": ms_, "share": ms_ / build_ms if build_ms else None,
               "note": note}
        if nbytes:
            out.update(bytes=nbytes, gbs=nbytes / (ms_ * 1e-3) / 1e9,
                       frac=nbytes / (ms_ * 1e-3) / 1e9 / hbm)
        return out
    line["hbm"] = {
        "peak_gbs": hbm,
        "build": {"bytes": b_build, "ms": build_ms,
                  "gbs": b_build / (build_ms * 1e-3) / 1e9,
                  "frac": b_build / (build_ms * 1e-3) / 1e9 / hbm,
                  "note": f"{B_BUILD_PER_PARTICLE} B/particle + "
                          f"{B_BUILD_PER_CELL} B/cell algorithmic; latency and "
                          f"FP64 bound, not HBM",
                  "phases": {
                      "keys": sub("keys", 60 * n, "root box (read x) and keys "
                                  "(read x, write key and index): 60 B/particle"),
                      "sort": sub("sort", (8 * 32 + 104) * n,
                                  "8 radix passes (read the key for the "
                                  "histogram, read and write key and index: "
                                  "32 B) and the gather of the Morton-ordered "
                                  "copies (104 B) per particle"),
                      "split": sub("split", 0, "octree split, one launch per "
                                   "level (21), and the leaf order: latency "
                                   "bound, no byte count"),
                      "moments": sub("moments", 32 * n + 208 * cells,
                                     "read x and m (32 B/particle), write the "
                                     "FP64 moments, box and FP32 records "
                                     "(208 B/cell); one bottom-up launch"),
                      "groups": sub("groups", 28 * n, "groups, their boxes "
                                    "(read x and order: 28 B/particle) and "
                                    "evaluation order"),
                      "note": "CUDA events per sub-phase in the profiled steps"}},
        "kick": {"bytes_per_particle": B_KICK, "ms": kick_ms,
                 "gbs": B_KICK * n / (kick_ms * 1e-3) / 1e9,
                 "frac": B_KICK * n / (kick_ms * 1e-3) / 1e9 / hbm},
        "drift": {"bytes_per_particle": B_DRIFT, "ms": drift_ms,
                  "gbs": B_DRIFT * n / (drift_ms * 1e-3) / 1e9,
                  "frac": B_DRIFT * n / (drift_ms * 1e-3) / 1e9 / hbm},
    }
    # backward pass (gradient of sum_i w_i . a_i): fwd = build + force,
    # bwd = p3t_long_force_vjp on the same tree
    wgt = torch.randn((3, n), dtype=torch.float32, device=dev,
                      generator=torch.Generator(device=dev).manual_seed(40))
    gpos = torch.empty((3, n), dtype=torch.float64, device=dev)
    gmass = torch.empty((n,), dtype=torch.float64, device=dev)
    ctx.build_tree(pos, mass)
    ctx.long_force(acc, check=False)
    ctx.long_force_vjp(wgt, gpos, gmass)  # warm-up
    fw, bw = [], []
    ctx.profile(reset=True)
    ctx.profile_enable(True)
    for _ in range(3):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a2 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ctx.build_tree(pos, mass)
        ctx.long_force(acc, check=False)
        a1.record(stream)
        ctx.long_force_vjp(wgt, gpos, gmass, check=False)
        a2.record(stream)
        torch.cuda.synchronize()
        fw.append(a0.elapsed_time(a1))
        bw.append(a1.elapsed_time(a2))
    ctx.check()
    ctx.profile_enable(False)
    pb = ctx.profile(reset=True)
    sb = ctx.stats()  # the interaction sets of this tree, walked by both
    t_f, t_b = float(np.median(fw)), float(np.median(bw))
    line["fwd_bwd_ratio"] = (t_f + t_b) / t_f
    # roofline of the backward's walk + Jacobian kernel (k_walk_vjp)
    vjp_ms = pb["vjp_walk_ms"] / max(pb["vjp_walks"], 1)
    flops_b = (FLOPS_BWD_PC * sb["int_pc"]
               + FLOPS_BWD_PP_FAR * (sb["int_pp"] - sb["int_pp_near"])
               + FLOPS_BWD_PP_NEAR * sb["int_pp_near"])
    ach_b = flops_b / (vjp_ms * 1e-3) / 1e12
    line["roofline_bwd"] = {
        "kernel": "k_walk_vjp", "bound": "alu", "achieved": ach_b,
        "peak": peak, "unit": "TFLOP/s", "frac": ach_b / peak,
        "frac_of_measured": ach_b / fma_meas, "kernel_ms": vjp_ms,
        "flops": flops_b,
        "traffic": profile_traffic("k_walk_vjp_plummer_1M.txt"),
        "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one "
                          "ncu capture of this kernel on this workload, read "
                          "from the committed summary "
                          "profiles/k_walk_vjp_plummer_1M.txt (not measured in "
                          "this run); mostly the FP64 adjoint atomics",
        "note": f"{FLOPS_BWD_PC} / {FLOPS_BWD_PP_FAR} / {FLOPS_BWD_PP_NEAR} "
                "flops per cell / far / near interaction (FMA = 2) x the "
                "interaction counts of the same tree, over the kernel's CUDA-"
                "event time (mean of 3 calls); peak as for the forward"}
    line["fwd_bwd_ms"] = {"fwd_build_force": t_f, "bwd_vjp": t_b,
                          "note": "median of 3, same tree; bwd recomputes the "
                                  "interaction sets"}
    # end-to-end through the public API with host buffers
    if not args.no_e2e:
        pin = lambda a: torch.tensor(a).pin_memory()
        hp, hv, hm = pin(pos.cpu().numpy()), pin(vel.cpu().numpy()), pin(mass_h)
        hoff = torch.empty((n + 1,), dtype=torch.int64).pin_memory()
        hidx = torch.empty((cap,), dtype=torch.int32).pin_memory()
        nnz_last = [0]

        # the step's compute replays three captured graphs: kick + drift;
        # build + force + kick; neighbour lists.  The positions are final
        # after the drift and the velocities after the second kick (the
        # neighbour lists need only the tree), so their downloads run on a
        # side stream while the tree is built and the force evaluated, and
        # while the neighbour lists are made
        ctx.set_params(P.Params(theta=THETA, r_out=R_OUT, gamma=GAMMA,
                                eps=4.0 / n, h=R_OUT, G=1.0, n_leaf=N_LEAF,
                                n_group=N_GROUP, flags=P.FLAG_NO_SYNC))
        side = torch.cuda.Stream(dev)
        copy_s = torch.cuda.Stream(dev)

        def part1():
            P.kick(vel, acc, 0.5 * DT)
            P.drift(pos, vel, DT)

        def part2():
            ctx.build_tree(pos, mass)
            ctx.long_force(acc, check=False)
            P.kick(vel, acc, 0.5 * DT)

        def part3():
            ctx.neighbours_into(off, idx, sync=False)

        side.wait_stream(stream)
        with torch.cuda.stream(side):
            part1()
            part2()
            part3()
        stream.wait_stream(side)
        g1, g2, g3 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1):
            part1()
        with torch.cuda.graph(g2):
            part2()
        with torch.cuda.graph(g3):
            part3()
        drifted, kicked = torch.cuda.Event(), torch.cuda.Event()
        uploaded = torch.cuda.Event()
        # device staging of the inputs: each step's copies from pinned host
        # memory run on the copy stream during the previous step, right after
        # that step's results came down (the positions and velocities a step
        # uploads are the ones the step before returned): the positions and
        # masses during the build and force, the velocities during the
        # neighbour lists; the step starts with device-to-device copies
        pos_in, vel_in = torch.empty_like(pos), torch.empty_like(vel)
        mass_in = torch.empty_like(mass)
        vel_up = torch.cuda.Event()
        with torch.cuda.stream(copy_s):
            pos_in.copy_(hp, non_blocking=True)
            mass_in.copy_(hm, non_blocking=True)
            uploaded.record(copy_s)
            vel_in.copy_(hv, non_blocking=True)
            vel_up.record(copy_s)

        def e2e_step():
            stream.wait_event(uploaded)
            pos.copy_(pos_in)
            mass.copy_(mass_in)
            stream.wait_event(vel_up)
            vel.copy_(vel_in)
            g1.replay()
            drifted.record(stream)
            copy_s.wait_event(drifted)
            with torch.cuda.stream(copy_s):
                hp.copy_(pos, non_blocking=True)
                # the next step's inputs, from pinned host memory
                pos_in.copy_(hp, non_blocking=True)
                mass_in.copy_(hm, non_blocking=True)
                uploaded.record(copy_s)
            g2.replay()
            kicked.record(stream)
            copy_s.wait_event(kicked)
            with torch.cuda.stream(copy_s):
                hv.copy_(vel, non_blocking=True)
                vel_in.copy_(hv, non_blocking=True)  # the next step's input
                vel_up.record(copy_s)
            g3.replay()
            hoff.copy_(off, non_blocking=True)
            stream.synchronize()
            nnz = int(hoff[n])
            hidx[:nnz].copy_(idx[:nnz], non_blocking=True)
            nnz_last[0] = nnz

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ke = max(2, min(args.steps, 8))
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        ctx.check()
        ctx.set_params(params)
        te = reduce_max((time.perf_counter() - t0) / ke, dev)
        line["e2e"] = {"value": world * n / te, "unit": "particles/s",
                       "h2d_bytes_per_step": 7 * 8 * n,
                       "d2h_bytes_per_step": 6 * 8 * n + 8 * (n + 1) + 4 * nnz_last[0],
                       "ms_per_step": te * 1e3}
    if not args.no_ensemble:
        line["ensemble"], gs["ensemble"] = run_ensemble(args, dev, want_cpu)
    if not args.no_p3t:
        line["p3t_step"] = run_p3t_step(args, dev)
    if not args.no_king:
        line["king"], gs["king"] = run_king(args, dev, want_cpu)
    if not args.no_cost_model:
        line["cost_model"] = run_cost_model(args, dev)
    if not args.no_smbh:
        line["smbh"] = run_smbh(args, dev)
    line["vjp_65536"], gs["vjp"] = run_vjp_small(args, dev)
    if want_cpu:
        gs["cfg1"] = run_cfg1(dev)
        line["cpu_baseline"], line["accuracy"] = cpu_baseline_and_accuracy(gs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_p3t_step(args, dev):
    """Whole P3T steps (Sect. 2.2) at the paper's standard parameters
    (Table 1) for N = 2^20: half-kick by F_soft, the hard step (isolated
    drift + Hermite block steps of the non-isolated particles on the
    neighbour lists), new tree, F_soft and neighbour lists within
    h = r_cut + 3 sigma dt_soft, half-kick.  One step captured in a CUDA
    graph and replayed; the hard step is also timed alone (same graph
    replays, events around it in an uncaptured step)."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    n = 1 << 20
    dt = (1 / 256) * (n / 16384) ** (-1 / 3)
    r_cut = 4 * dt
    h = r_cut + 3 * dt / np.sqrt(2)
    eps = 4.0 / n
    pos_h, vel_h, mass_h = ics.plummer(n, SEED)
    params = P.Params(theta=THETA, r_out=r_cut, gamma=GAMMA, eps=eps, h=h,
                      G=1.0, n_leaf=N_LEAF, n_group=N_GROUP)
    ctx = P.Context(params)
    pos = torch.tensor(pos_h, device=dev)
    vel = torch.tensor(vel_h, device=dev)
    mass = torch.tensor(mass_h, device=dev)
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    off = torch.empty((n + 1,), dtype=torch.int64, device=dev)
    hp = P.HermiteParams(dt_soft=dt)
    ctx.build_tree(pos, mass)
    ctx.long_force(acc)
    _, idx0 = ctx.neighbours()
    idx = torch.empty((max(4 * int(idx0.numel()) + 1024, n),), dtype=torch.int32,
                      device=dev)
    ctx.neighbours_into(off, idx)
    ctx.hard_step(pos.clone(), vel.clone(), mass, off, idx, hp)  # scratch

    ngb_stream = torch.cuda.Stream(dev)

    def step(ev=None):
        # with events (phase times): one stream; without: the neighbour
        # lists beside the force
        rec = (lambda k: ev[k].record(torch.cuda.current_stream(dev))) if ev else (lambda k: None)
        rec(0)
        P.kick(vel, acc, 0.5 * dt)
        rec(1)
        ctx.hard_step(pos, vel, mass, off, idx, hp, check=False)
        rec(2)
        ctx.build_tree(pos, mass)
        rec(3)
        if ev:
            ctx.long_force(acc, check=False)
            rec(4)
            ctx.neighbours_into(off, idx, sync=False)
            rec(5)
        else:
            force_and_neighbours(ctx, acc, off, idx, ngb_stream)
        P.kick(vel, acc, 0.5 * dt)
        rec(6)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    # phases, in uncaptured steps
    phases = []
    for _ in range(3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        step(ev)
        torch.cuda.synchronize()
        phases.append([ev[k].elapsed_time(ev[k + 1]) for k in range(6)])
    ph = np.median(np.array(phases), axis=0)
    hard = [ph[1]]
    st = ctx.stats()
    nonis = int((off[1:] > off[:-1]).sum().item())
    ctx.set_params(P.Params(theta=THETA, r_out=r_cut, gamma=GAMMA, eps=eps, h=h,
                            G=1.0, n_leaf=N_LEAF, n_group=N_GROUP,
                            flags=P.FLAG_NO_SYNC))
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(args.steps // 4, 8)
    e0.record(stream)
    for _ in range(k):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = e0.elapsed_time(e1) / k
    return {"workload": "Plummer N=2^20, P3T standard parameters (Table 1): "
                        f"dt_soft {dt:.6g}, r_cut 4 dt_soft, h = r_cut + "
                        "3 sigma dt_soft (sigma 1/sqrt 2), dt_max dt_soft/4, "
                        "eps 4/N, eta 0.1, alpha 0.1, theta 0.4",
            "step": "half-kick, hard step (isolated drift + Hermite), build, "
                    "F_soft, neighbour lists, half-kick; one CUDA graph",
            "n": n, "value": n / (ms * 1e-3), "unit": "particles/s",
            "ms_per_step": ms, "hard_ms": float(np.median(hard)),
            "phase_ms_per_step": {"kicks": float(ph[0] + ph[5]), "hard": float(ph[1]),
                                  "build": float(ph[2]), "force": float(ph[3]),
                                  "neighbours": float(ph[4]),
                                  "note": "CUDA events, steps without the graph"},
            "non_isolated": nonis, "components": st["herm_components"],
            "largest_component": st["herm_max_component"],
            "hard_particle_steps": st["herm_particle_steps"],
            "hard_pairs": st["herm_pairs"], "steps_at_kmax": st["herm_capped"],
            "max_block_steps": st["herm_max_block_steps"],
            "fp64_measured": dict(P.fp64_peaks(),
                                  note="p3t_fp64_peaks: FP64 FMA/s over all SMs; "
                                       "latency (SM cycles) of one dependent add, "
                                       "division, square root in one warp")}


def run_smbh(args, dev):
    """Whole P3T steps of the black hole binary run of Sect. 3.2.2: a
    Plummer model of 2^17 stars (N-body units) with two black holes of 1% of
    its mass at (+-0.5, 0, 0) moving at (0, +-0.5, 0); cut-offs 1/256
    between stars and 1/32 between a black hole and a star, none between the
    black holes (not split, unsoftened); eps 1e-4; eta 0.1 for stars, 0.03
    for black holes; dr_buff = 3 sigma dt_soft (sigma 1/sqrt 2), dt_max =
    dt_soft / 4, theta 0.4, dt_soft 1/1024.  Each step: half-kick, hard step,
    build, F_soft, neighbour lists, half-kick; one step captured in a CUDA
    graph and replayed."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    nfs, n_bh = 1 << 17, 2
    n = nfs + n_bh
    dt = 1.0 / 1024
    buf = 3 * dt / np.sqrt(2)
    r_fs, r_bh = 1 / 256, 1 / 32
    ps, vs, ms = ics.plummer(nfs, 7000)
    pos_h = np.concatenate([ps, [[0.5, -0.5], [0.0, 0.0], [0.0, 0.0]]], axis=1)
    vel_h = np.concatenate([vs, [[0.0, 0.0], [0.5, -0.5], [0.0, 0.0]]], axis=1)
    mass_h = np.concatenate([ms, [0.01, 0.01]])

    def mk(flags=0):
        return P.Params(theta=THETA, r_out=r_fs, gamma=GAMMA, eps=1e-4,
                        h=r_fs + buf, G=1.0, n_leaf=N_LEAF, n_group=N_GROUP,
                        flags=flags)
    ctx = P.Context(mk())
    ctx.set_species(n, n_bh, r_cut_bh=r_bh, eps_bh=1e-4, h_bh=r_bh + buf,
                    eta_bh=0.03)
    pos = torch.tensor(np.ascontiguousarray(pos_h), device=dev)
    vel = torch.tensor(np.ascontiguousarray(vel_h), device=dev)
    mass = torch.tensor(mass_h, device=dev)
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    off = torch.empty((n + 1,), dtype=torch.int64, device=dev)
    hp = P.HermiteParams(dt_soft=dt, eta=0.1, alpha=0.1)
    ctx.build_tree(pos, mass)
    ctx.long_force(acc)
    _, idx0 = ctx.neighbours()
    idx = torch.empty((max(4 * int(idx0.numel()) + 1024, n),), dtype=torch.int32,
                      device=dev)
    ctx.neighbours_into(off, idx)
    ngb_stream = torch.cuda.Stream(dev)

    def step():
        P.kick(vel, acc, 0.5 * dt)
        ctx.hard_step(pos, vel, mass, off, idx, hp, check=False)
        ctx.build_tree(pos, mass)
        force_and_neighbours(ctx, acc, off, idx, ngb_stream)
        P.kick(vel, acc, 0.5 * dt)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    st = ctx.stats()
    ctx.set_params(mk(P.FLAG_NO_SYNC))
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(args.steps // 4, 8)
    e0.record(stream)
    for _ in range(k):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms_step = e0.elapsed_time(e1) / k
    bh = pos[:, nfs:].cpu().numpy()
    return {"workload": "black hole binary in a Plummer model (Sect. 3.2.2): "
                        "2^17 stars + 2 black holes of 0.01 at (+-0.5, 0, 0), "
                        "(0, +-0.5, 0); r_cut 1/256 star-star, 1/32 black "
                        "hole-star, none black hole-black hole; eps 1e-4 "
                        "(0 between black holes); eta 0.1 / 0.03; dt_soft "
                        "1/1024; theta 0.4",
            "step": "half-kick, hard step, build, F_soft, neighbour lists, "
                    "half-kick; one CUDA graph",
            "n": n, "value": n / (ms_step * 1e-3), "unit": "particles/s",
            "ms_per_step": ms_step,
            "black_hole_rows": int((off[nfs + 1:] - off[nfs:-1]).sum().item()),
            "hard_particle_steps": st["herm_particle_steps"],
            "largest_component": st["herm_max_component"],
            "binary_separation": float(np.linalg.norm(bh[:, 0] - bh[:, 1])),
            "steps_done": max(args.warmup, 3) + 4 + k}


def run_king(args, dev, sample=False):
    """KDK steps on the dense-core workload: King (1966) W0 = 9, N = 2^21,
    Salpeter masses on [0.1, 10] normalised to M = 1, r_out = 0.002, theta
    0.5, eps = 4/N, neighbour lists within h = r_out; dt = 1/256.  One step
    captured in a CUDA graph and replayed; phases from uncaptured steps."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    n = 1 << 21
    masses = ics.salpeter_masses(n, seed=3 + 7919)
    pos_h, vel_h, mass_h = ics.king(n, 3, W0=9.0, masses=masses)
    r_out, theta = 0.002, 0.5
    mk = lambda flags=0: P.Params(theta=theta, r_out=r_out, gamma=GAMMA,
                                  eps=4.0 / n, h=r_out, G=1.0, n_leaf=N_LEAF,
                                  n_group=N_GROUP, flags=flags)
    ctx = P.Context(mk())
    pos = torch.tensor(pos_h, device=dev)
    vel = torch.tensor(vel_h, device=dev)
    mass = torch.tensor(mass_h, device=dev)
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    off = torch.empty((n + 1,), dtype=torch.int64, device=dev)
    ctx.build_tree(pos, mass)
    ctx.long_force(acc)
    _, idx0 = ctx.neighbours()
    idx = torch.empty((max(4 * int(idx0.numel()) + 1024, n),), dtype=torch.int32,
                      device=dev)

    ngb_stream = torch.cuda.Stream(dev)

    def step(sequential=False):
        P.kick(vel, acc, 0.5 * DT)
        P.drift(pos, vel, DT)
        ctx.build_tree(pos, mass)
        if sequential:  # phase times: one stream
            ctx.long_force(acc, check=False)
            ctx.neighbours_into(off, idx, sync=False)
        else:
            force_and_neighbours(ctx, acc, off, idx, ngb_stream)
        P.kick(vel, acc, 0.5 * DT)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ctx.profile(reset=True)
    ctx.profile_enable(True)
    for _ in range(3):
        step(sequential=True)
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    prof = ctx.profile(reset=True)
    nnz = int(off[-1].item())
    ctx.set_params(mk(P.FLAG_NO_SYNC))
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(args.steps // 4, 8)
    e0.record(stream)
    for _ in range(k):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = e0.elapsed_time(e1) / k
    nprof = max(prof["forces"], 1)
    state = None
    if sample:  # the forces of the last step were evaluated at these positions
        state = {"pos": pos.cpu().numpy().T.copy(), "m": mass_h,
                 "acc": acc.cpu().numpy().T.astype(np.float64),
                 "theta": theta, "r_out": r_out}
    return {"workload": "King W0=9, N=2^21, Salpeter masses 0.1-10 (M=1), "
                        "r_out 0.002, theta 0.5, eps 4/N, h = r_out, dt 1/256",
            "step": "KDK (kick, drift, build, force, neighbour lists, kick); "
                    "one CUDA graph",
            "n": n, "value": n / (ms * 1e-3), "unit": "particles/s",
            "ms_per_step": ms,
            "phase_ms_per_step": {"build": prof["build_ms"] / nprof,
                                  "walk_and_force": prof["force_ms"] / nprof,
                                  "neighbours": prof["ngb_ms"] / nprof},
            "interactions_per_particle": {"pc": prof["int_pc"] / (n * nprof),
                                          "pp": prof["int_pp"] / (n * nprof)},
            "neighbour_pairs": nnz}, state


def run_cfg1(dev):
    """Plummer N = 8192 (seed 1), r_out 0.01, theta 0.4, eps 4/N, h = r_out:
    one tree build, force and neighbour lists, for the accuracy record."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    n = 8192
    pos_h, _, m_h = ics.plummer(n, 1)
    ctx = P.Context(P.Params(theta=THETA, r_out=0.01, gamma=GAMMA, eps=4.0 / n,
                             h=0.01, n_leaf=N_LEAF, n_group=N_GROUP))
    ctx.build_tree(torch.tensor(pos_h, device=dev), torch.tensor(m_h, device=dev))
    acc = ctx.long_force()
    off, idx = ctx.neighbours()
    return {"pos": pos_h.T.copy(), "m": m_h,
            "acc": acc.cpu().numpy().T.astype(np.float64),
            "off": off.cpu().numpy(), "idx": idx.cpu().numpy()}


def run_vjp_small(args, dev):
    """The gradient workload: Plummer N = 65536 (seed 4), theta 0.4, r_out =
    0.01 (N/8192)^(-1/3) = 0.005, eps 4/N, loss L = sum_i w_i . a_i with
    w_i ~ N(0, I) (seed 40).  Times the forward (build + force) and the
    backward (p3t_long_force_vjp) with CUDA events, median of 5; returns
    (result, host arrays for the accuracy record)."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    n = 65536
    r_out = 0.01 * (n / 8192) ** (-1.0 / 3.0)
    pos_h, _, m_h = ics.plummer(n, 4)
    w_h = np.random.default_rng(40).normal(size=(n, 3))
    ctx = P.Context(P.Params(theta=THETA, r_out=r_out, gamma=GAMMA, eps=4.0 / n,
                             h=r_out, n_leaf=N_LEAF, n_group=N_GROUP))
    pos = torch.tensor(pos_h, device=dev)
    mass = torch.tensor(m_h, device=dev)
    w = torch.tensor(w_h.T.copy(), dtype=torch.float32, device=dev)
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    gx = torch.empty((3, n), dtype=torch.float64, device=dev)
    gm = torch.empty((n,), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    fw, bw = [], []
    for it in range(6):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        ctx.build_tree(pos, mass)
        ctx.long_force(acc, check=False)
        ev[1].record(stream)
        ctx.long_force_vjp(w, gx, gm, check=False)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if it:
            fw.append(ev[0].elapsed_time(ev[1]))
            bw.append(ev[1].elapsed_time(ev[2]))
    ctx.check()
    t_f, t_b = float(np.median(fw)), float(np.median(bw))
    res = {"workload": "Plummer N=65536, theta 0.4, r_out 0.005, eps 4/N, "
                       "L = sum w.a, w ~ N(0, I) seed 40",
           "fwd_ms": t_f, "bwd_ms": t_b, "fwd_bwd_ratio": (t_f + t_b) / t_f,
           "value": n / ((t_f + t_b) * 1e-3), "unit": "particles/s (fwd+bwd)"}
    return res, {"pos": pos_h.T.copy(), "m": m_h, "w": w.cpu().numpy().T.astype(np.float64),
                 "acc": acc.cpu().numpy().T.astype(np.float64),
                 "gx": gx.cpu().numpy().T.copy(), "gm": gm.cpu().numpy()}


def run_cost_model(args, dev):
    """Soft-interaction counts against theta and N, for the cost model of
    Sect. 3.1.2 (the tree part costs O(theta^-3 N log N) per soft step):
    Plummer spheres of 2^16, 2^18 and 2^20 particles, theta in {0.3, 0.4,
    0.5, 0.6, 0.8}, r_out = 0.01 (N/8192)^(-1/3), eps = 4/N, h = r_out.  Per
    point one build and force evaluation; the force kernel counts its
    interactions itself.  Reported per point: interactions per particle
    (cells, particles) and the force time; per N the least-squares exponent
    of N_int in theta; and N_int / (theta^-3 N ln N) over the grid."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    thetas = (0.3, 0.4, 0.5, 0.6, 0.8)
    points, fits = [], {}
    for lg in (16, 18, 20):
        n = 1 << lg
        pos_h, _, mass_h = ics.plummer(n, 4000 + lg)
        r_out = 0.01 * (n / 8192) ** (-1.0 / 3.0)
        pos = torch.tensor(pos_h, device=dev)
        mass = torch.tensor(mass_h, device=dev)
        acc = torch.empty((3, n), dtype=torch.float32, device=dev)
        tot = []
        for th in thetas:
            ctx = P.Context(P.Params(theta=th, r_out=r_out, gamma=GAMMA,
                                     eps=4.0 / n, h=r_out, G=1.0,
                                     n_leaf=N_LEAF, n_group=N_GROUP))
            ctx.build_tree(pos, mass)
            ctx.long_force(acc)
            ts = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.long_force(acc, check=False)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ctx.check()
            st = ctx.stats()
            pc, pp = st["int_pc"] / n, st["int_pp"] / n
            tot.append(pc + pp)
            points.append({"n": n, "theta": th, "pc_per_particle": pc,
                           "pp_per_particle": pp,
                           "force_ms": float(np.median(ts)),
                           "ns_per_interaction": float(np.median(ts)) * 1e6
                           / ((pc + pp) * n),
                           "n_int_over_model": (pc + pp) * n
                           / (th ** -3 * n * np.log(n))})
            del ctx
        fits[n] = float(np.polyfit(np.log(thetas), np.log(tot), 1)[0])
    return {"workload": "Plummer N = 2^16, 2^18, 2^20; theta 0.3-0.8; r_out "
                        "0.01 (N/8192)^(-1/3); eps 4/N; h = r_out; one force "
                        "evaluation per point",
            "model": "N_int,soft ~ theta^-3 N ln N per soft step (Sect. 3.1.2)",
            "theta_exponent": {str(k): v for k, v in fits.items()},
            "points": points}


def run_ensemble(args, dev, sample=False):
    """256 independent Plummer clusters, N_c log-uniform in [1024, 65536],
    r_out = 0.01 (N_c / 8192)^(-1/3), eps = 4 / N_c, theta 0.4.  One step =
    tree build + force + backward (gradient of sum w.a) for all clusters,
    group/leaf sizes from the autotuner, the step captured once in a CUDA
    graph and replayed."""
    import torch
    import paper_1506_04553_b300 as P
    from paper_1506_04553_b300 import ics
    pos_h, _, m_h, off = ics.plummer_ensemble(256, seed=5000)
    n = int(off[-1])
    sizes = np.diff(off)
    r_out = 0.01 * (sizes / 8192.0) ** (-1.0 / 3.0)
    eps = 4.0 / sizes
    ctx = P.Context(P.Params(theta=THETA, gamma=GAMMA))
    ctx.set_ensemble(off, r_out=r_out, eps=eps)
    pos = torch.tensor(pos_h, device=dev)
    mass = torch.tensor(m_h, device=dev)
    w = torch.randn((3, n), dtype=torch.float32, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(41))
    tune = ctx.autotune(pos, mass, w=w, reps=2)
    ng, nl = tune["n_group"], tune["n_leaf"]
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    gx = torch.empty((3, n), dtype=torch.float64, device=dev)
    gm = torch.empty((n,), dtype=torch.float64, device=dev)
    ctx.build_tree(pos, mass)
    ctx.long_force(acc)
    ctx.long_force_vjp(w, gx, gm)
    p = ctx.params
    ctx.set_params(P.Params(theta=THETA, gamma=GAMMA, n_group=p.n_group,
                            n_leaf=p.n_leaf, flags=P.FLAG_NO_SYNC))
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        ctx.build_tree(pos, mass)
        ctx.long_force(acc, check=False)
        ctx.long_force_vjp(w, gx, gm, check=False)
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.build_tree(pos, mass)
        ctx.long_force(acc, check=False)
        ctx.long_force_vjp(w, gx, gm, check=False)
    for _ in range(max(args.warmup, 3)):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(args.steps // 2, 4)
    e0.record(stream)
    for _ in range(k):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = e0.elapsed_time(e1) / k
    # phases, in uncaptured steps: the library's event profile for the build
    # and the walk + force kernel, events around the whole backward
    ctx.profile(reset=True)
    ctx.profile_enable(True)
    tb = []
    for _ in range(3):
        ctx.build_tree(pos, mass)
        ctx.long_force(acc, check=False)
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        ctx.long_force_vjp(w, gx, gm, check=False)
        b1.record(stream)
        torch.cuda.synchronize()
        tb.append(b0.elapsed_time(b1))
    ctx.profile_enable(False)
    pr = ctx.profile(reset=True)
    ctx.check()
    f_ms = pr["force_ms"] / max(pr["forces"], 1)
    b_ms = pr["vjp_walk_ms"] / max(pr["vjp_walks"], 1)
    nf = max(pr["forces"], 1)
    ipc, ipp, ippn = pr["int_pc"] / nf, pr["int_pp"] / nf, pr["int_pp_near"] / nf
    fl_f = FLOPS_PC * ipc + FLOPS_PP_NEAR * ippn + FLOPS_PP_FAR * (ipp - ippn)
    fl_b = (FLOPS_BWD_PC * ipc + FLOPS_BWD_PP_NEAR * ippn
            + FLOPS_BWD_PP_FAR * (ipp - ippn))
    peak = fp32_peak_tflops(dev)
    phases = {"build": pr["build_ms"] / max(pr["builds"], 1),
              "walk_and_force": f_ms,
              "backward": float(np.median(tb)),
              "backward_walk_kernel": b_ms,
              "force_frac_of_fp32_peak": fl_f / (f_ms * 1e-3) / 1e12 / peak,
              "backward_frac_of_fp32_peak": fl_b / (b_ms * 1e-3) / 1e12 / peak,
              "note": "CUDA events, three uncaptured steps (medians / means); "
                      "fractions: the forward's and backward's flops per "
                      "interaction (as in roofline and roofline_bwd) times "
                      "the kernel's own interaction counts, over its time, "
                      "of the nominal FP32 peak"}
    res = {"workload": "256 Plummer clusters, N_c log-uniform in [1024, 65536], "
                       "theta 0.4, r_out 0.01 (N_c/8192)^(-1/3), eps 4/N_c",
           "n": n, "clusters": 256, "step": "build + force + backward, "
           "one CUDA graph, one walk+force launch for all clusters",
           "value": n / (ms * 1e-3), "unit": "particles/s (fwd+bwd)",
           "ms_per_step": ms,
           "phase_ms_per_step": phases,
           "autotuned": {"n_group": ng, "n_leaf": nl,
                         "force_warps": tune["force_warps"],
                         "vjp_warps": tune["vjp_warps"],
                         "objective": "build + force + backward (ms, best of 2)",
                         "ms": tune["ms"],
                         "err_median": tune["err_median"],
                         "err_max": tune["err_max"],
                         "start_err_median": tune["base_err_median"],
                         "start_err_max": tune["base_err_max"],
                         "evaluated": tune["evaluated"],
                         "rejected_by_accuracy": tune["rejected"],
                         "note": "error: |a - a_ref| / max(|a_ref|, 1e-3 rms) "
                                 "against the starting configuration at "
                                 "theta / 2; kept if median <= 1.25x and "
                                 "max <= 2x the starting configuration's"}}
    if not sample:
        return res, None
    # eight clusters spanning the sizes (smallest and largest included)
    order = np.argsort(sizes, kind="stable")
    pick = order[np.round(np.linspace(0, len(sizes) - 1, 8)).astype(int)]
    a_h = acc.cpu().numpy().T.astype(np.float64)
    w_h = w.cpu().numpy().T.astype(np.float64)
    gx_h, gm_h = gx.cpu().numpy().T, gm.cpu().numpy()
    cl = []
    for c in pick:
        lo, hi = int(off[c]), int(off[c + 1])
        cl.append({"pos": pos_h[:, lo:hi].T.copy(), "m": m_h[lo:hi],
                   "acc": a_h[lo:hi], "w": w_h[lo:hi], "gx": gx_h[lo:hi],
                   "gm": gm_h[lo:hi], "r_out": float(r_out[c]),
                   "eps": float(eps[c])})
    return res, {"clusters": cl, "n_group": ng, "n_leaf": nl}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
