#!/usr/bin/env python
"""Benchmark of the MSTAR hot path on GB300: FP64 pair-forces/s and GBS steps/s.

Workload: Plummer sphere of 10^4 equal-mass stars (total mass 1, virial radius 1, seed 5)
plus two SMBHs of mass 0.005 at +/-0.1 on half-circular orbits (N = 10002), FP64,
eta_GBS = 1e-12, k_fix = 8 (Deuflhard), N_d = 2. One benchmark step is one accepted GBS
step (MST, edge coordinates, 73 pair-loop evaluations over 8 concurrent divisions,
extrapolation, convergence test; rejected attempts are counted and included).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mstar|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank integrates its own
replica of the system: the path has no data-path exchange, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "plummer10k_two_smbh"
WORKLOAD_DESC = ("Plummer N=10000 (m=1e-4, r_vir=1, seed 5) + 2 SMBHs of 0.005 at +/-0.1 (N=10002); "
                 "eta_GBS=1e-12, k_fix=8 Deuflhard, N_d=2, G=1")
# Algorithmic FP64 flops of one unordered far-pair interaction. The loop evaluates each
# unordered pair once and applies it to both bodies: separation 3, r^2 5, reciprocal square
# root 7 (one DMUL, three DFMA), r^-3 2, two mass scalings 2, force function 2, two 3-vector
# accumulations 12; 16.5 flops per ordered pair-force.
FLOPS_PER_UNORDERED_PAIR = 33
# Flops of one ordered pair-force evaluated on its own, without the i<->j symmetry (3 DADD,
# r^2 and a Newton-refined reciprocal square root, the mass scaling, 3 DFMA accumulations, U);
# reported beside the symmetric count.
FLOPS_PER_ORDERED_PAIR_NONSYM = 28
# FP64-pipe instructions the tiled kernel issues per unordered pair: 3 DADD for the separation
# and 6 DFMA for the two force accumulations (ncu counts 3.0 DADD and 5.95 DFMA per pair).
# r^2, 1/r, 1/r^3, the mass products and the force-function sum run on the integer pipe.
FP64_INSTR_PER_PAIR = 9
NOMINAL_FP64_TFLOPS = 1.25
# FP64 FMA units: 2 DFMA per clock per SM (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained = 2 inst/cycle/SM), 152 SMs; the roofline peak is that rate at the SM clock
# sampled during the timed region, 2 flops per DFMA.
DFMA_PER_CLK_PER_SM = 2
NUM_SMS = 152
L2_FLUSH_BYTES = 256 << 20
# Figures from ncu captures of k_pair_tiles<4> (128-body tiles) at N = 10002, each valid for the
# kernel built from the sources whose SHA-256 (csrc/pair.cu then csrc/device.cuh) starts with
# the given prefix; for other sources or another tile the bench reports them as null.
#  - DRAM bytes (read + write) of one launch by the number of division slots it evaluates;
#    an attempt launches the kernel for 1 (step start), 8, 8, 7, 7, ..., 1, 1 slots;
#  - the FP64 pipe's active fraction (sm__inst_executed_pipe_fp64 over its peak).
PAIR_TILE_SRC_SHA = "54214f1fde9b5cd9"
PAIR_TILE_PIPE_SRC_SHA = "54214f1fde9b5cd9"
PAIR_TILE_DRAM_BYTES_BY_SLOTS = {1: 0.166e6, 2: 0.510e6, 3: 1.295e6, 4: 2.572e6, 5: 3.626e6, 6: 4.615e6, 7: 6.120e6, 8: 11.925e6}
PAIR_TILE_FP64_PIPE_NCU = 0.870
ATTEMPT_SLOT_PATTERN = [1] + [k for k in range(8, 0, -1) for _ in range(2)]
# Algorithmic DRAM bytes of one force evaluation per body: positions 24 and mass 8 read,
# accelerations 24 written (parent and grandparent indices are another 8 read).
ALGO_BYTES_PER_BODY_EVAL = 64


def tuned_pair_loop(M, m, r, v, repeats):
    """The pair loop for this system: the tuner's fastest, when it beats the size rule's (the
    library's default) by more than 2 %, the spread of single attempts; else the size rule's."""
    best, ms = M.mstar_tune_pair_tile(m, r, v, repeats=repeats)
    n = len(m)
    rule = (32, 4) if n <= 512 else ((32, 1) if n <= 4096 else ((64, 1) if n <= 8192 else (128, 1)))
    pick = best if ms[best] < 0.98 * ms[rule] else rule
    return pick, {f"{k[0]}x{k[1]}": x for k, x in ms.items()}


def pair_source_sha():
    import hashlib

    h = hashlib.sha256()
    for f in ("pair.cu", "device.cuh"):
        with open(os.path.join(ROOT, "paper_2001_03180_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mstar", choices=["mstar", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched-subsystems measurement and print its object")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint measurement and print its object (profiling)")
    ap.add_argument("--no-rebuild-test", action="store_true")
    ap.add_argument("--batched-schedule", default=None,
                    help="comma-separated schedule per size class instead of the autotuner's (profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the single-system extras (small configurations, tree builders, rebuild test, adjoint)")
    ap.add_argument("--no-single-context", action="store_true",
                    help="skip timing the one-context-per-system path beside the batch")
    ap.add_argument("--pair-tile", default=None,
                    help="TILExSPLIT (e.g. 128x1) for the headline steps instead of the tuner's pick (profiling: "
                         "under a profiler the tuner's serialised timings can pick another tiling)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    from paper_2001_03180_gb300 import replicas as R

    return R.env_ranks()


def reduce_max(x, world, dev):
    from paper_2001_03180_gb300 import replicas as R

    return R.reduce_max(x, world, dev)


def reduce_sum(x, world, dev):
    from paper_2001_03180_gb300 import replicas as R

    return R.reduce_sum(x, world, dev)


def barrier(world):
    from paper_2001_03180_gb300 import replicas as R

    R.barrier(world)


def host_cpu():
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm implementer/part codes)."""
    import platform

    desc = {"machine": platform.machine(), "nproc": os.cpu_count()}
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return desc
    for key in ("model name", "CPU implementer", "CPU part"):
        for line in info:
            if line.split(":")[0].strip() == key:
                desc[key.replace(" ", "_").lower()] = line.split(":", 1)[1].strip()
                break
    return desc


def cpu_baseline_sample(n_threads):
    """The oracle, as it stands, on the host cores: one GBS step attempt of the workload."""
    import oracle
    from paper_2001_03180_gb300 import workloads as W

    oracle.build()
    oracle.set_threads(n_threads)
    m, r, v = W.workload(WORKLOAD)
    s = oracle.System(m, r, v)
    H = 3e-4
    t0 = time.perf_counter()
    s.attempt(H)
    dt = time.perf_counter() - t0
    n = len(m)
    pairs = 73 * n * (n - 1)
    # the same oracle on one core: one pair-loop evaluation of the same state
    oracle.set_threads(1)
    st = s.state()
    root, parent, level, order = oracle.prim(st["r"])
    X = oracle.to_mst(parent, st["r"])
    t1 = time.perf_counter()
    oracle.forces(m, st["r"], parent, level, X)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(n_threads)
    return {"value": pairs / dt, "unit": "pair-forces/s", "cores": n_threads, "kind": "oracle",
            "sample": f"one GBS step attempt (73 pair-loop evaluations, Prim, rebuilds, extrapolation) of "
                      f"the N={n} workload at H={H}, {dt:.2f} s wall on {n_threads} threads",
            "single_core": {"value": n * (n - 1) / dt1, "unit": "pair-forces/s", "cores": 1,
                            "sample": f"one oracle pair-loop evaluation of the N={n} state, {dt1:.2f} s"},
            "host": host_cpu()}


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only)."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2001_03180_gb300 import workloads as W

    oracle.build()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    m, r, v = W.workload(WORKLOAD)
    n = len(m)
    sysd = oracle.System(m, r, v)
    st = sysd.state()
    root, parent, level, order = oracle.prim(st["r"])
    X = oracle.to_mst(parent, st["r"])
    for _ in range(args.warmup):
        oracle.forces(m, st["r"], parent, level, X)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forces(m, st["r"], parent, level, X)
    dt = time.perf_counter() - t0
    pairs = n * (n - 1) * args.steps
    value = pairs / dt
    sample = (f"each step: one oracle pair-loop evaluation (Eq. 2, near rule N_d=2) of the N={n} state, "
              f"1/73 of a GBS step's pair work; {threads} threads")
    out = {"impl": "reference", "metric": "FP64 pair-forces/s", "value": value, "unit": "pair-forces/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_DESC, "n": n},
           "cpu_baseline": {"value": value, "unit": "pair-forces/s", "cores": threads, "kind": "oracle",
                            "sample": sample, "host": host_cpu()},
           "e2e": {"value": value, "unit": "pair-forces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


BATCH_DESC = ("4096 independent systems (seed 3): even indices hierarchical triples (masses 1, 1, 0.1; inner a=1, "
              "e~U[0,0.9]; outer a~U[10,50]; inclination~U[40,140] deg), odd indices Plummer clusters of "
              "N~round(exp U[ln 3, ln 200]) bodies with a central mass of 0.1 of the cluster; eta_GBS=1e-12, k_fix=8")


def run_batched(args, dev, M, W, torch, world=1, rank=0):
    """Batched subsystems: each launch gives every system one GBS step attempt (one CTA per
    system). Throughput = accepted system steps per second over the timed launches; the
    plain one-context-per-system path is timed beside it on a sample of the same systems.
    With several ranks the systems are split by the greedy longest-first rule on N^2 (no
    collective on the data path); the rate is the sum of accepted steps over the max time."""
    import numpy as np

    from paper_2001_03180_gb300 import replicas as R

    all_systems = W.batched_systems(4096, 3)
    mine = R.shard_greedy([len(s.m) ** 2 for s in all_systems], world)[rank]
    systems = [all_systems[i] for i in mine]
    t_end = 1000.0  # no system gets there within the launches below: each launch is an attempt for all
    b = M.Batch([(s.m, s.r, s.v) for s in systems], device=dev)
    b.step(t_end, 40)  # step-size controllers settle from the first-step rule (halvings)
    if args.batched_schedule:
        sched = np.array([int(x) for x in args.batched_schedule.split(",")], np.int32)
        b.set_schedule(sched)
        tune_ms = None
    else:
        sched, tune_ms = b.autotune(t_end, repeats=2)  # setup, state unchanged
    launches = 5 * max(args.steps, 1)
    st0 = b.step(t_end, 0)
    l0 = M.mstar_batch_launch_count(b.b)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    R.barrier(world)
    torch.cuda.synchronize(dev)
    e0.record(b.stream)
    st1 = b.step(t_end, launches)
    e1.record(b.stream)
    torch.cuda.synchronize(dev)
    R.barrier(world)
    ms = R.reduce_max(e0.elapsed_time(e1), world, dev)
    nl = M.mstar_batch_launch_count(b.b) - l0
    b.close()
    acc = R.reduce_sum(st1["accepted"] - st0["accepted"], world, dev)
    att = acc + R.reduce_sum(st1["rejected"] - st0["rejected"], world, dev)
    out = {"workload": BATCH_DESC, "systems": len(all_systems), "bodies": sum(len(s.m) for s in all_systems),
           "ranks": world,
           "launches": nl, "ms_per_launch": ms / launches, "system_steps_per_s": acc / (ms * 1e-3),
           "system_attempts_per_s": att / (ms * 1e-3), "failed": st1["failed"],
           "schedule": {"warps_per_division_group_by_size_class": sched.tolist(),
                        "size_classes": "[2,8] [9,16] [17,32] [33,64] [65,128] [129,256] [257,512]",
                        "values": "G > 0: one CTA per system, four division groups of G warps; -G: the same "
                                  "groups as one CTA each (start, divisions, finish nodes); 0: 4-, 8- or 16-lane "
                                  "groups, one body per lane",
                        "autotune_launch_ms": tune_ms},
           "launch": "one CUDA graph launch per attempt (independent kernel nodes per schedule kind; a chain "
                     "of three for a split schedule)"}
    if args.no_single_context or rank != 0:
        return out
    # the single-system path, one context per system, on every 128th system
    secs = 0.0
    steps = 0
    for s in systems[::128]:
        g = M.Integrator(s.m, s.r, s.v, device=dev)
        g.step(t_end, 3)
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        _, st = g.step(t_end, 5)
        secs += time.perf_counter() - w0
        steps += st["accepted"]
        g.close()
    out["single_context_system_steps_per_s"] = steps / secs
    out["single_context_sample"] = "every 128th system (%d), 5 steps each, sequential" % len(systems[::128])
    return out


ADJOINT_DESC = ("Plummer N=256 (seed 4), fixed fictitious step H = the first accepted step of the step control "
                "(ds = q U dt with t_end = 1, halved until eps <= 1e-12), k_fix=8, 100 steps, checkpoints every 10; "
                "loss w_r.r_f + w_v.v_f + w_E E_f with seeded weights")


def first_accepted_H(M, m, r, v, dev):
    g = M.Integrator(m, r, v, device=dev)
    _, U = g.accelerations()
    H = 0.1 * U
    for _ in range(60):
        if g.attempt(H)["eps"] <= 1e-12:
            break
        H *= 0.5
    g.close()
    return H


def run_adjoint(args, dev, M, W, torch):
    """Adjoint of the fixed-step run: wall time of the checkpointed forward and of the
    reverse sweep (which recomputes each segment once), and their ratio."""
    m, r, v = W.workload("plummer256")
    n = len(m)
    H = first_accepted_H(M, m, r, v, dev)
    st = W.Stream(4, 5)
    w_r = (st.uniform(3 * n) - 0.5).reshape(n, 3)
    w_v = (st.uniform(3 * n) - 0.5).reshape(n, 3)
    steps, every = 100, 10
    fw, bw = [], []
    for rep in range(3):  # the first repetition warms up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        run = M.FixedRun(m, r, v, H, steps, checkpoint_every=every, device=dev)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        run.backward(w_r, w_v, 0.7)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        run.close()
        if rep:
            fw.append(t1 - t0)
            bw.append(t2 - t1)
    f, b = min(fw), min(bw)
    return {"workload": ADJOINT_DESC, "n": n, "steps": steps, "checkpoint_every": every, "H": H,
            "forward_ms": f * 1e3, "adjoint_ms": b * 1e3, "adjoint_to_forward": b / f,
            "note": "wall time with the stream synchronised; the forward includes context set-up and checkpoints, "
                    "the adjoint recomputes each segment once (a second forward) and runs one VJP pair loop "
                    "per kick"}


def run_mst_builders(args, dev, M, m, r, v, torch):
    """Spanning-tree build time on the benchmark workload: the step's exact MST builder
    (Boruvka rounds, Prim on ties), the divide-and-conquer tree of Sec. 3.3, and Prim's
    algorithm (one CTA).
    Each repetition re-sets the state from device copies so that the tree is rebuilt; the
    time covers the build and the copy of parent and level to the host."""
    import numpy as np

    out = {}
    for name, meth in (("exact_mst", 0), ("divide_and_conquer", 1)):
        g = M.Integrator(m, r, v, device=dev, mst_method=meth)
        rd = torch.empty((len(m), 3), dtype=torch.float64, device=dev)
        vd = torch.empty((len(m), 3), dtype=torch.float64, device=dev)
        t = M.mstar_get_state(g.ctx, rd, vd)
        times = []
        for rep in range(6):
            M.mstar_set_state(g.ctx, t, rd, vd)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            root, parent, level, _ = g.mst(with_order=False)
            times.append(time.perf_counter() - t0)
        g.close()
        out[name + "_ms"] = 1e3 * statistics.median(times[1:])
        out[name + "_mean_level"] = float(np.mean(level))
        d = np.linalg.norm(np.asarray(r)[np.flatnonzero(parent >= 0)] - np.asarray(r)[parent[parent >= 0]], axis=1)
        out[name + "_length"] = float(d.sum())
    # Prim's algorithm itself (the one-CTA kernel that also records the insertion order)
    g = M.Integrator(m, r, v, device=dev)
    times = []
    for rep in range(4):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g.mst(with_order=True)
        times.append(time.perf_counter() - t0)
    g.close()
    out["prim_one_cta_ms"] = 1e3 * statistics.median(times[1:])
    out["length_ratio"] = out["divide_and_conquer_length"] / out["exact_mst_length"]
    return out


REBUILD_DESC = ("rebuild test of Sec. 3.5: Hernquist N=379 (r_half=1, G=M=1; seeds 1..10, clusters with a hard "
                "binary redrawn), 1e5 build/deconstruct cycles per system, MST and chain coordinates; "
                "deconstruction by per-vertex path sums with the centre-of-mass shift (the integrator's) or the "
                "root position kept, or from the root outwards (w_v = w_parent + X_v) with the root kept or "
                "followed by the shift; topology rebuilt every 1000 cycles; energies with compensated sums")


def run_rebuild_test(args, dev, M, W, O_unused=None):
    """The paper's rebuild experiment: mean |dE/E| over 10 seeds after n build/deconstruct
    cycles, for the MST and the chain under both deconstruction rules."""
    import numpy as np

    systems = [W.hernquist(379, s)[:3] for s in range(1, 11)]
    samples = [0, 1, 3, 10, 30, 100, 300, 1000, 3000, 10000, 30000, 100000]
    rules = ((0, "com_shift"), (1, "root_kept"), (2, "root_outwards"), (3, "root_outwards_com_shift"))
    jobs = [(s, c, d) for d, _ in rules for c in (0, 1) for s in range(10)]
    t0 = time.perf_counter()
    g = M.mstar_rebuild_test([systems[s] for s, _, _ in jobs], [c for _, c, _ in jobs], [d for _, _, d in jobs],
                             samples[-1], 1000, samples)
    wall = time.perf_counter() - t0
    out = {"workload": REBUILD_DESC, "samples": samples, "wall_s": wall, "jobs": len(jobs)}
    for d, dname in rules:
        for c, cname in ((0, "mst"), (1, "chain")):
            idx = [k for k, (s, cc, dd) in enumerate(jobs) if cc == c and dd == d]
            E = g["E"][idx]
            rel = np.abs(E / E[:, :1] - 1.0)
            out[f"{cname}_{dname}_mean_dE"] = rel.mean(axis=0).tolist()
            out[f"{cname}_{dname}_mean_level"] = float(np.mean(g["mean_level"][idx]))
            out[f"{cname}_{dname}_topo_changes"] = int(np.sum(g["topo_changes"][idx]))
        mst_e = out[f"mst_{dname}_mean_dE"][-1]
        out[f"chain_over_mst_{dname}_at_1e5"] = out[f"chain_{dname}_mean_dE"][-1] / mst_e if mst_e > 0 else None
    return out


def run_small_configs(args, dev, M, W, torch):
    """The two smaller configurations: Plummer 64 integrated to t = 1, and Plummer 2048 with a
    central SMBH binary for 200 accepted GBS steps (wall time through mstar_step, energy error)."""
    out = {}
    for key, name, t_end, steps in (("plummer64_to_t1", "plummer64", 1.0, 1 << 30),
                                    ("plummer2048_smbh_binary_200_steps", "plummer2048_smbh_binary", 10.0, 200)):
        m, r, v = W.workload(name)
        if len(m) <= 160:  # a CTA cluster per division (the library's size rule): no pair tiles to tune
            (tile, split), tile_ms = (0, 0), None
        else:
            (tile, split), tile_ms = tuned_pair_loop(M, m, r, v, repeats=3)
        g = M.Integrator(m, r, v, device=dev, pair_tile=tile, pair_split=split)
        e0 = g.energy()["E"]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, st = g.step(t_end, steps)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        e1 = g.energy()["E"]
        n = len(m)
        out[key] = {"n": n, "wall_s": wall, "accepted": st["accepted"], "rejected": st["rejected"],
                    "t_reached": st["t"], "gbs_steps_per_s": st["accepted"] / wall,
                    "pair_forces_per_s": st["force_evals"] * n * (n - 1) / wall, "abs_dE_over_E": abs((e1 - e0) / e0),
                    "division_schedule": ("a CTA cluster per division" if len(m) <= 160 else
                                          ("a stream per division" if len(m) >= 1000 else "level by level")),
                    "pair_tile": tile, "pair_split": split, "pair_tile_tuner_ms_per_attempt": tile_ms}
        g.close()
    out["plummer64_to_t1_batch_of_one"] = run_batch_of_one(dev, M, W, torch)
    return out


def run_batch_of_one(dev, M, W, torch):
    """Plummer 64 to t = 1 as a batch of one system: each attempt is one graph launch of the
    batched kernels (the system in one CTA, or over four with a split schedule). The schedule
    comes from the autotuner, run
    beforehand on a snapshot and not timed. The energy error is taken by mstar_energy on a
    context made from the end state."""
    m, r, v = W.workload("plummer64")
    g = M.Integrator(m, r, v, device=dev)
    e0 = g.energy()["E"]
    g.close()
    b = M.Batch([(m, r, v)], device=dev)
    sched, tune_ms = b.autotune(1.0)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    launches = 0
    for _ in range(4096):
        st = b.step(1.0, launches=8)
        launches += 8
        if st["finished"] == 1:
            break
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    S = b.state()
    b.close()
    g = M.Integrator(m, S["r"][0], S["v"][0], device=dev)
    e1 = g.energy()["E"]
    g.close()
    n = len(m)
    return {"n": n, "wall_s": wall, "accepted": st["accepted"], "rejected": st["rejected"],
            "status": int(S["status"][0]), "t_reached": float(S["t"][0]), "graph_launches": launches,
            "schedule": [int(x) for x in sched], "gbs_steps_per_s": st["accepted"] / wall,
            "pair_forces_per_s": st["force_evals"] * n * (n - 1) / wall, "abs_dE_over_E": abs((e1 - e0) / e0)}


def run_mstar(args):
    import numpy as np
    import torch

    from paper_2001_03180_gb300 import build as B
    from paper_2001_03180_gb300 import workloads as W

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    B.build()
    from paper_2001_03180_gb300 import mstar as M

    M.load()
    if args.batched_only:
        print(json.dumps(run_batched(args, dev, M, W, torch)), flush=True)
        return
    if args.adjoint_only:
        print(json.dumps(run_adjoint(args, dev, M, W, torch)), flush=True)
        return
    m, r, v = W.workload(WORKLOAD)
    n = len(m)
    # the pair loop's tiling, timed on this system before anything is measured (setup)
    (tile, split), tile_ms = tuned_pair_loop(M, m, r, v, repeats=2)
    if args.pair_tile:
        tile, split = (int(x) for x in args.pair_tile.lower().split("x"))
    g = M.Integrator(m, r, v, device=dev, pair_tile=tile, pair_split=split)
    stream = g.stream
    e_init = g.energy()["E"]
    t_end = 1.0
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # warm-up: the first steps also let the controller find the step size from the
    # first-step rule ds = q U dt (several rejections); the flush runs here once too, so
    # that its one-time kernel load is not timed
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            g.step(t_end, 1)
    torch.cuda.synchronize(dev)

    # the FP64 FMA probe on the warm GPU (best of three), with the clock it ran at
    probe_clk = ClockSampler(local)
    probe_clk.start()
    fma_rate = max(M.mstar_fp64_fma_rate(stream.cuda_stream) for _ in range(3))
    probe_clocks = probe_clk.stop()

    def run_steps(profile):
        """args.steps steps bracketed by a barrier and a device synchronisation, timed with CUDA
        events on the context's stream, the SM clock sampled meanwhile."""
        if profile:
            M.mstar_profile_enable(g.ctx, True)
        launches0 = M.mstar_launch_count(g.ctx)
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize(dev)
        acc = rej = fev = 0
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                flush.zero_()
                rc, st = g.step(t_end, 1)
                acc += st["accepted"]
                rej += st["rejected"]
                fev += st["force_evals"]
            e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        clk = sampler.stop()
        prof = None
        if profile:
            prof = M.mstar_profile_read(g.ctx)
            M.mstar_profile_enable(g.ctx, False)
        return e0.elapsed_time(e1), acc, rej, fev, M.mstar_launch_count(g.ctx) - launches0, clk, prof

    # ---- device-resident timed region: the steps as the library runs them (each attempt one
    # graph launch; from 1000 bodies each division on its own stream)
    ms, acc, rej, fev, launches, clocks, _ = run_steps(False)
    # ---- the same number of steps again with CUDA events around every pair-loop launch (the
    # attempts issued kernel by kernel, level by level, so that each event pair times one
    # launch alone): the pair kernel's mean launch time for the roofline
    ms_prof, acc_p, rej_p, fev_p, _, clocks_prof, prof = run_steps(True)
    ms_max = reduce_max(ms, world, dev)
    pair_forces = float(fev) * n * (n - 1)
    # energy error of the run so far (warm-up and both timed runs from the initial state)
    dE_c5 = abs((g.energy()["E"] - e_init) / e_init)
    steps_c5 = args.warmup + acc + acc_p
    total_pf = reduce_sum(pair_forces, world, dev)
    total_steps = reduce_sum(float(acc), world, dev)
    value = total_pf / (ms_max * 1e-3)

    # ---- end to end: host buffers in, host buffers out, every step
    e2e = None
    if args.steps > 0:
        rh = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        vh = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        S = g.state()
        rh[:] = S["r"]
        vh[:] = S["v"]
        t_now = S["t"]
        barrier(world)
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        fev2 = 0
        for _ in range(args.steps):
            M.mstar_set_state(g.ctx, t_now, rh, vh)
            rc, st = g.step(t_end, 1)
            fev2 += st["force_evals"]
            t_now = M.mstar_get_state(g.ctx, rh, vh)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
        wall = reduce_max(wall, world, dev)
        e2e_pf = reduce_sum(float(fev2) * n * (n - 1), world, dev)
        e2e = {"value": e2e_pf / wall, "unit": "pair-forces/s", "h2d_bytes_per_step": 2 * 3 * n * 8,
               "d2h_bytes_per_step": 2 * 3 * n * 8}

    # ---- roofline of the dominant kernel (tiled pair loop), CUDA events on its stream
    avg_ms = prof.pair_ms / max(prof.pair_launches, 1)
    pairs_per_launch = prof.pair_interactions / max(prof.pair_launches, 1)
    achieved = FLOPS_PER_UNORDERED_PAIR * pairs_per_launch / (avg_ms * 1e-3) / 1e12
    clk_mhz = clocks_prof.get("sm_mhz") or 2070.0
    fp64_peak = 2.0 * DFMA_PER_CLK_PER_SM * NUM_SMS * clk_mhz * 1e6 / 1e12
    fp64_issue = DFMA_PER_CLK_PER_SM * NUM_SMS * clk_mhz * 1e6  # FP64 instructions/s the pipe takes
    sha_ok = pair_source_sha() == PAIR_TILE_SRC_SHA and (tile, split) == (128, 1)
    slots_per_launch = prof.force_evals / max(prof.pair_launches, 1)
    # per launch, averaged over an attempt's launches (the pattern of slot counts is fixed)
    traffic = (sum(PAIR_TILE_DRAM_BYTES_BY_SLOTS[k] for k in ATTEMPT_SLOT_PATTERN) / len(ATTEMPT_SLOT_PATTERN)
               if sha_ok else None)
    algo_bytes = ALGO_BYTES_PER_BODY_EVAL * n * slots_per_launch
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": traffic,
                "kernel": "k_pair_tiles (symmetric pair loop: FP64 separations and force accumulations; "
                          "integer-pipe r^2, 1/r, m/r^3 and the exact fixed-point sum of m/r)",
                "achieved_source": ("33 algorithmic FP64 flops per unordered far pair (each evaluated once and "
                                    "applied to both bodies) x N(N-1)/2 pairs x evaluations per launch / mean "
                                    "CUDA-event launch time on the context stream, over a second run of the "
                                    "timed steps with events around every pair launch (profiled_steps)"),
                "peak_source": ("FP64 unit peak from unit counts and clocks (no FP64 entry among the measured "
                                "peaks): 2 DFMA/clk/SM x 152 SMs x the SM clock sampled in the timed region x "
                                "2 flops"),
                "frac_above_1_because": ("r^2, 1/r, r^-3, m r^-3 and the sum of m/r run on the integer pipe: the "
                                         "FP64 pipe issues 9 instructions (3 DADD + 6 DFMA) of the 33 flops"),
                "fp64_pipe_util": pairs_per_launch * FP64_INSTR_PER_PAIR / (avg_ms * 1e-3) / fp64_issue,
                "fp64_pipe_util_source": ("pair rate x 9 FP64 instructions per pair / (2 per clk per SM x 152 "
                                          "SMs x sampled clock)"),
                "fp64_pipe_util_ncu": (PAIR_TILE_FP64_PIPE_NCU
                                       if pair_source_sha() == PAIR_TILE_PIPE_SRC_SHA and (tile, split) == (128, 1)
                                       else None),
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch by slot count, "
                                   "averaged over an attempt's 17 launches; null when the kernel's sources "
                                   "differ from the captured ones" + ("" if sha_ok else " (they differ)")),
                "algorithmic_bytes": algo_bytes,
                "traffic_over_algorithmic": traffic / algo_bytes if traffic else None,
                "survey_unit_tflops": FLOPS_PER_ORDERED_PAIR_NONSYM * 2 * pairs_per_launch / (avg_ms * 1e-3) / 1e12,
                "survey_unit_frac": (FLOPS_PER_ORDERED_PAIR_NONSYM * 2 * pairs_per_launch / (avg_ms * 1e-3) / 1e12
                                     / fp64_peak),
                "survey_unit_note": "28 flops per ordered pair-force as if each ordered pair were evaluated alone",
                "probe_tflops": 2.0 * fma_rate / 1e12,
                "probe_sm_mhz": probe_clocks.get("sm_mhz"),
                "probe_frac_of_unit_peak": (2.0 * fma_rate / 1e12) / (
                    2.0 * DFMA_PER_CLK_PER_SM * NUM_SMS * (probe_clocks.get("sm_mhz") or clk_mhz) * 1e6 / 1e12),
                "peak_nominal_tflops": NOMINAL_FP64_TFLOPS,
                "pair_kernel_share_of_step": prof.pair_ms / ms_prof if ms_prof > 0 else None,
                "profiled_steps": {"ms": ms_prof, "accepted": acc_p, "rejected": rej_p,
                                   "pair_forces_per_s": float(fev_p) * n * (n - 1) / (ms_prof * 1e-3),
                                   "sm_mhz": clocks_prof.get("sm_mhz")},
                # the whole timed step (every kernel of the hot path, rejected attempts and the
                # L2 flush included) against the same peak
                "whole_step_tflops": FLOPS_PER_UNORDERED_PAIR * 0.5 * pair_forces / (ms * 1e-3) / 1e12,
                "whole_step_frac": FLOPS_PER_UNORDERED_PAIR * 0.5 * pair_forces / (ms * 1e-3) / 1e12 / fp64_peak}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(os.cpu_count() or 1)
    batched = None
    if not args.no_batched:
        with torch.cuda.stream(stream):
            batched = run_batched(args, dev, M, W, torch, world, rank)
    # the single-system extras (no data-path collective) run in single-GPU runs only, so that
    # a multi-GPU run holds its GPUs for the timed work and the sharded batch alone
    extras = world == 1 and not args.no_extras
    small = None
    if extras:
        with torch.cuda.stream(stream):
            small = run_small_configs(args, dev, M, W, torch)
    mst = None
    if extras:
        with torch.cuda.stream(stream):
            mst = run_mst_builders(args, dev, M, m, r, v, torch)
    rebuild = None
    if extras and not args.no_rebuild_test:
        rebuild = run_rebuild_test(args, dev, M, W)
    adjoint = None
    if extras and not args.no_adjoint:
        with torch.cuda.stream(stream):
            adjoint = run_adjoint(args, dev, M, W, torch)

    if rank == 0:
        out = {"metric": "FP64 pair-forces/s", "value": value, "unit": "pair-forces/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / max(args.steps, 1),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD_DESC, "n": n, "gbs_steps_per_bench_step": 1,
                          "l2": "flushed between steps (256 MiB write)",
                          "parallelism": "replicas" if world > 1 else "single",
                          "division_schedule": ("one CTA per division" if len(m) <= 96 else
                                          ("a stream per division" if len(m) >= 1000 else "level by level")),
                    "pair_tile": tile, "pair_split": split, "pair_tile_tuner_ms_per_attempt": tile_ms},
               "gbs_steps_per_s": total_steps / (ms_max * 1e-3), "attempts": acc + rej, "rejected": rej,
               "force_evals": fev, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clocks, "batched": batched,
               "adjoint": adjoint, "mst_builders": mst,
               "rebuild_test": rebuild, "small_configs": small}
        sc = small or {}
        # the figures of every section in a few keys at the end of the line
        out["summary"] = {
            "abs_dE_over_E": dE_c5, "abs_dE_over_E_steps": steps_c5,
            "roofline_frac": roofline["frac"], "fp64_pipe_util": roofline["fp64_pipe_util"],
            "c1_plummer64_abs_dE_over_E": sc.get("plummer64_to_t1", {}).get("abs_dE_over_E"),
            "c1_plummer64_gbs_steps_per_s": sc.get("plummer64_to_t1", {}).get("gbs_steps_per_s"),
            "c2_smbh2050_abs_dE_over_E": sc.get("plummer2048_smbh_binary_200_steps", {}).get("abs_dE_over_E"),
            "c2_smbh2050_gbs_steps_per_s": sc.get("plummer2048_smbh_binary_200_steps", {}).get("gbs_steps_per_s"),
            "batched_system_steps_per_s": (batched or {}).get("system_steps_per_s"),
            "batched_ms_per_launch": (batched or {}).get("ms_per_launch"),
            "adjoint_to_forward": (adjoint or {}).get("adjoint_to_forward")}
        print(json.dumps(out), flush=True)
    g.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mstar(args)


if __name__ == "__main__":
    main()
