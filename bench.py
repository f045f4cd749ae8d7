"""Throughput of the vdW-DF nonlocal hot path on GB300: ordered pair interactions
per second for E_c^nl + v_nl (one step = gradient, q0, trimming, fused pair pass
for A and U, potential assembly, energy) on the periodic rare-gas monolayer
workload (48 x 84 x 120 grid, 16.4 x 28.4 x 40 bohr, 20 bohr pair cutoff,
density cutoff 1e-6, seeded synthetic density), FP32 pair arithmetic with FP64
accumulation.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on bounded samples of
the same workload (each step: A_i, U_i of a random sample of active points).
Multi-GPU (torchrun): every rank runs its own replica (weak scaling); rank 0
reports the sum of pairs over ranks divided by the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vdW-DF pair interactions/s (E_nl+v_nl), FP32 vs FP64 path at ≤1e-6 rel err"
UNIT = "pair interactions/s"
WORKLOAD = "xe_monolayer 48x84x120 periodic-xy r_cut=20 n_cut=1e-6 (E_nl + v_nl)"
# FP32-pipe operations per ordered pair interaction of the fused E + v pass, table
# branch, counted from the formulation: one evaluation serves the pair in both
# orders (123 operations per unordered pair: geometry, r, D, delta, cell split,
# B-spline weights and their derivatives, 4x4 combine for phi, phi_D, phi_delta,
# chain rule for both d1 and d2, accumulation on both sides); shared-memory loads
# and MUFU operations are not in this count.
OPS_PER_PAIR_EV = 62
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [s for s in sm if s >= 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def combine_ranks(ms, e2e, pairs, device):
    """Replicas, one per rank with no data exchange (the path does not shard): the
    slowest rank's step and end-to-end times, and the pair interactions summed over
    the ranks (weak scaling).  At one rank, or without a process group, the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(e2e), float(pairs)
    t = torch.tensor([ms, e2e, float(pairs)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(tot[2])


def build_table(V):
    """The standard 400 x 200 table (0 <= D <= 30), cached under .cache/."""
    path = os.path.join(ROOT, ".cache", "vdwdf_table_400x200_D30_q1.npz")
    if os.path.exists(path):
        return V.Table.load(path)
    T = V.Table.build(400, 30.0, 200, 1)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    T.save(path)
    return T


def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda:%d" % local)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    import paper_0810_2273_gb300 as V
    from paper_0810_2273_gb300 import inputs

    T = build_table(V)
    w = inputs.xe_monolayer()
    n_host = torch.from_numpy(w["density"]).pin_memory()
    n = n_host.to(dev)
    a = (w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], T)
    v = torch.empty_like(n)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        V.potential(n, *a, precision="fp32", out=v)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = V.launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    pair_ms = []
    results = []
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                      # L2 flush between steps, outside the timed events
        starts[k].record()
        E, _, res = V.potential(n, *a, precision="fp32", out=v)
        ends[k].record()
        pair_ms.append(res["ms_pairs"])
        results.append((E, res))
    barrier()
    wall = time.perf_counter() - t_wall
    launches = V.launch_count() - l0
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = float(np.mean(step_ms))
    pairs = results[-1][1]["pairs"]

    # end to end: pinned host density in, potential out to pinned host memory
    v_host = torch.empty(n.shape, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(2, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_dev = n_host.to(dev, non_blocking=True)
        E2, v2, _ = V.potential(n_dev, *a, precision="fp32")
        v_host.copy_(v2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e = float(np.mean(e2e_ms))

    # FP64 path on the same workload, energy + potential once (outside the timed steps)
    t0 = time.perf_counter()
    E64, _, r64 = V.potential(n, *a, precision="fp64")
    fp64_s = time.perf_counter() - t0

    # the semilocal terms of eq. 3 on the same density (outside the timed steps; the
    # call's own CUDA events, L2 flushed before each call)
    semi_ms = []
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        semi = V.semilocal(n, w["lengths"], w["periodic"])
        semi_ms.append(semi["ms"])
    semi_t = float(np.median(semi_ms[1:]))

    ms, e2e, total_pairs = combine_ranks(ms, e2e, pairs, dev)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    value = total_pairs / (ms * 1e-3)
    sm_mhz = clocks["sm_mhz"] if clocks else None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = 2070.0
    peak = sms * FP32_LANES_PER_SM * clk * 1e6 / 1e12
    pms = float(np.mean(pair_ms))
    achieved = OPS_PER_PAIR_EV * pairs / (pms * 1e-3) / 1e12
    prof_traffic = None
    tr_path = os.path.join(ROOT, "profiles", "pair_traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            if tr.get("kernel_hash") == kernel_hash():
                prof_traffic = tr.get("bytes_per_launch_full")
        except (OSError, ValueError):
            pass
    cpu = oracle_sample(w, T, seconds=args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(n.shape), "n_active": results[-1][1]["n_active"],
                   "pairs_per_step": pairs, "precision": "fp32 pairs, fp64 accumulation",
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "E_hartree": results[-1][0],
        "fp64_path": {"value": pairs / fp64_s, "unit": UNIT, "E_hartree": E64,
                      "rel_err_fp32_vs_fp64": abs(results[-1][0] - E64) / abs(E64),
                      "seconds": fp64_s},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T fp32-lane-ops/s",
                     "frac": achieved / peak, "traffic": prof_traffic,
                     "kernel": "k_pair<float, potential, %d>" % results[-1][1]["pair_threads"],
                     "ms_per_launch": pms,
                     "ops_per_pair": OPS_PER_PAIR_EV,
                     "peak_basis": "%d SMs x %d FP32 lanes x %.0f MHz (max SM clock)" % (sms, FP32_LANES_PER_SM, clk)},
        "semilocal": {"ms_per_call": semi_t, "points": int(n.numel()),
                      "points_per_s": n.numel() / (semi_t * 1e-3),
                      "hbm_gbs": 8.0 * n.numel() / (semi_t * 1e-3) / 1e9,
                      "bound": "fp64 (per-point cbrt, log, expm1 at GB300's FP64 rate)",
                      "E_hartree": {k: semi[k] for k in ("Ex_lda", "Ec_lda", "Ex_pbe", "Ec_pbe", "Ex_revpbe")},
                      "eq3_needed_number": semi["Ec_lda"] - semi["Ec_pbe"] + results[-1][0]},
        "cpu_baseline": cpu,
        "e2e": {"value": total_pairs / (e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(n.numel() * 8),
                "d2h_bytes_per_step": int(n.numel() * 8 + 8), "ms_per_step": e2e},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def kernel_hash():
    """Hash of the pair kernel's code (pair.cu and common.cuh without comments or
    layout): the recorded DRAM traffic belongs to the code with this hash."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("pair.cu", "common.cuh"):
        src = open(os.path.join(ROOT, "paper_0810_2273_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def oracle_sample(w, T, seconds=15.0, max_points=4096, seed=0):
    """The FP64 CPU oracle on the host cores: A_i, U_i for random active points of the
    workload (pairs within the cutoff counted by the oracle), grown until ~seconds."""
    import oracle
    nodes = T.nodes
    P = oracle.Problem(w["density"], w["lengths"], w["periodic"], w["n_cut"], w["r_cut"],
                       oracle.Spline(nodes, 30.0))
    rng = np.random.default_rng(seed)
    k = 16
    done_pairs, done_t, done_pts = 0, 0.0, 0
    while done_t < seconds and done_pts < max_points:
        q = rng.choice(P.n_active, k, replace=False)
        t0 = time.perf_counter()
        _, _, npairs, _ = P.AU(q)
        dt = time.perf_counter() - t0
        done_pairs += int(npairs.sum())
        done_t += dt
        done_pts += k
        if dt < seconds / 4:
            k *= 2
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done_pairs / done_t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "A_i and U_i (FP64) of %d random active points of the same workload, %d pairs, %.1f s"
                      % (done_pts, done_pairs, done_t)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import __graft_entry__
    from oracle import build as obuild
    obuild.build()
    import oracle
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer()
    nodes = oracle.cached_table(400, 30.0, 200, oracle.QUAD_TABLE)
    P = oracle.Problem(w["density"], w["lengths"], w["periodic"], w["n_cut"], w["r_cut"],
                       oracle.Spline(nodes, 30.0))
    rng = np.random.default_rng(1)
    per_step = args.ref_points
    for _ in range(args.warmup):
        P.AU(rng.choice(P.n_active, max(1, per_step // 4), replace=False))
    t_pairs, t_time = 0, 0.0
    for _ in range(args.steps):
        q = rng.choice(P.n_active, per_step, replace=False)
        t0 = time.perf_counter()
        _, _, npairs, _ = P.AU(q)
        t_time += time.perf_counter() - t0
        t_pairs += int(npairs.sum())
    value = t_pairs / t_time
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = ("each step: FP64 A_i, U_i of %d random active points of the same workload "
              "(%d pairs in total)" % (per_step, t_pairs))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_time / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    del __graft_entry__


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-points", type=int, default=48)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
