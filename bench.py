"""Throughput of the vdW-DF nonlocal hot path on GB300: ordered pair interactions
per second for E_c^nl + v_nl (one step = gradient, q0, trimming, fused pair pass
for A and U, potential assembly, energy) on the periodic rare-gas monolayer
workload (48 x 84 x 120 grid, 16.4 x 28.4 x 40 bohr, 20 bohr pair cutoff,
density cutoff 1e-6, seeded synthetic density), FP32 pair arithmetic with FP64
accumulation.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Besides the headline step, the line carries one entry per standard workload
under "workloads" (pairs/s, fraction of the FP32 lane peak, the FP64 path's
rate and the FP32/FP64 ratio), timed after the headline steps: the Kr dimer
(FP64 E), the open 24-atom molecule (FP32 E + v), the 18-cell binding curve
(batched CUDA graph, default and autotuned launch shapes) and the metal slab
with a flake (FP32 E + v).  --no-workloads skips them.

SM clocks and throttle reasons are sampled during the timed steps; a timed
region that saw a thermal or hardware slowdown, or SM clocks under 80 % of
their maximum with no reason given, is measured once more, and the line keeps
the first region's clocks under clocks.remeasured_after.

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
# The same count for the energy-only pass: 71 operations per unordered pair
# (no derivative weights, no chain rule, one accumulation side), 35.5 per ordered pair.
OPS_PER_PAIR_E = 35.5
SM_COUNT_NOMINAL = 152
SLOWDOWNS = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
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

    def timed_steps():
        sampler = ClockSampler(local)
        sampler.start()
        l0 = V.launch_count()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        pair_ms, results = [], []
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
        return step_ms, pair_ms, results, launches, clocks, wall

    step_ms, pair_ms, results, launches, clocks, wall = timed_steps()
    # a timed region that saw a thermal or hardware slowdown, or SM clocks well below
    # their maximum with no reason given, is measured once more (every rank agrees)
    bad = float(bool(clocks) and (bool(set(clocks["reasons"]) & SLOWDOWNS) or
                                  (not clocks["reasons"] and clocks["sm_mhz"] < 0.8 * clocks["sm_max_mhz"])))
    if ws > 1:
        flag = torch.tensor([bad], device=dev)
        torch.distributed.all_reduce(flag, op=torch.distributed.ReduceOp.MAX)
        bad = float(flag.item())
    first_clocks = None
    if bad:
        first_clocks = clocks
        step_ms, pair_ms, results, launches, clocks, wall = timed_steps()
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

    # FP64 path on the same workload, energy + potential once (outside the timed
    # steps), after a warm-up call of the FP64 kernels on a small grid of the same cell
    ws_small = inputs.xe_monolayer((12, 21, 30))
    V.potential(torch.from_numpy(ws_small["density"]).to(dev), *a, precision="fp64")
    torch.cuda.synchronize()
    e64a, e64b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e64a.record()
    E64, _, r64 = V.potential(n, *a, precision="fp64")
    e64b.record()
    torch.cuda.synchronize()
    fp64_s = 1e-3 * e64a.elapsed_time(e64b)

    # the GPU's own arithmetic rates (FMA microbenchmarks, outside the timed steps),
    # with the SM clock sampled meanwhile: the measured denominators of the ALU rooflines
    rsamp = ClockSampler(local)
    rsamp.start()
    lane = {}
    for kind in ("fp32", "fp32x2", "fp64"):
        V.lane_rate(kind, 20.0, dev)
        lane[kind] = V.lane_rate(kind, 200.0, dev)
    rclocks = rsamp.stop()

    # the semilocal terms of eq. 3 on the same density (outside the timed steps; the
    # call's own CUDA events, L2 flushed before each call)
    semi_ms = []
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        semi = V.semilocal(n, w["lengths"], w["periodic"])
        semi_ms.append(semi["ms"])
    semi_t = float(np.median(semi_ms[1:]))

    # the far field past the cutoff (eq. 17 and the lattice continuum) on the same
    # density, outside the timed steps: T, E + T and the call's own device time
    tails = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        tails.append(V.far_tail(n, w["lengths"], w["periodic"], w["n_cut"], w["r_cut"]))
    tail = {"T_hartree": tails[-1]["T"], "E_plus_T_hartree": results[-1][0] + tails[-1]["T"],
            "ms_per_call": float(np.median([t["ms"] for t in tails[1:]])), "nodes": tails[-1]["nodes"],
            "planes": tails[-1]["planes"], "bound": "fp64 (one exp per active point and quadrature node)"}
    # the same at a 30 bohr cutoff (FP32 energy): E + T should hardly move
    E30, _ = V.energy(n, w["lengths"], w["periodic"], w["n_cut"], 30.0, T, precision="fp32")
    T30 = V.far_tail(n, w["lengths"], w["periodic"], w["n_cut"], 30.0)["T"]
    tail["r_cut_30"] = {"E_hartree": E30, "T_hartree": T30, "E_plus_T_hartree": E30 + T30,
                        "E_change_from_r_cut_20": E30 - results[-1][0],
                        "E_plus_T_change_from_r_cut_20": E30 + T30 - tail["E_plus_T_hartree"]}

    ms, e2e, total_pairs = combine_ranks(ms, e2e, pairs, dev)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    value = total_pairs / (ms * 1e-3)
    sm_mhz = clocks["sm_mhz"] if clocks else None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    r_mhz = (rclocks or {}).get("sm_mhz") or 2070.0
    lane_rates = {k: {"T_lane_ops_per_s": r / 1e12, "ms": t, "per_sm_per_clock": r / (sms * r_mhz * 1e6)}
                  for k, (r, t) in lane.items()}
    lane_rates["clocks"] = rclocks
    lane_rates["note"] = ("vdwdf_lane_rate: every SM full of 512-thread blocks, 8 independent FMA chains "
                          "per thread; one FMA of one lane = 1 lane operation (2 per packed FP32x2 FMA)")
    fp64_peak = lane["fp64"][0] / 1e12
    clk, clk_basis = (sm_mhz, "median SM clock sampled during the timed steps") if sm_mhz else \
        (2070.0, "maximum SM clock (no clock samples)")
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
    wl = None if args.no_workloads else run_workloads(V, inputs, T, dev, flush, sms, fp64_peak)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_keys(ws),
        "workload_stats": {"n_active": results[-1][1]["n_active"], "pairs_per_step": pairs,
                           "precision": "fp32 pairs, fp64 accumulation"},
        "E_hartree": results[-1][0],
        "fp64_path": {"value": pairs / fp64_s, "unit": UNIT, "E_hartree": E64,
                      "rel_err_fp32_vs_fp64": abs(results[-1][0] - E64) / abs(E64),
                      "seconds": fp64_s, "fp32_over_fp64": value / (pairs / fp64_s),
                      "timing": "CUDA events around one call, after an FP64 warm-up call on a 12x21x30 grid",
                      "roofline": {"bound": "alu", "achieved": OPS_PER_PAIR_EV * pairs / fp64_s / 1e12,
                                   "peak": fp64_peak, "unit": "T fp64-lane-ops/s",
                                   "frac": OPS_PER_PAIR_EV * pairs / fp64_s / 1e12 / fp64_peak,
                                   "ops_per_pair": OPS_PER_PAIR_EV,
                                   "peak_basis": "measured FP64 FMA rate (lane_rates.fp64)"}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T fp32-lane-ops/s",
                     "frac": achieved / peak, "traffic": prof_traffic,
                     "kernel": "k_pair<float, potential, %d>" % results[-1][1]["pair_threads"],
                     "ms_per_launch": pms,
                     "ops_per_pair": OPS_PER_PAIR_EV,
                     "peak_basis": "%d SMs x %d FP32 lanes x %.0f MHz (%s)" % (sms, FP32_LANES_PER_SM, clk,
                                                                                clk_basis),
                     "peak_measured_fp32_fma": lane["fp32"][0] / 1e12,
                     "frac_of_measured_fp32_fma": achieved / (lane["fp32"][0] / 1e12)},
        "lane_rates": lane_rates,
        "semilocal": {"ms_per_call": semi_t, "points": int(n.numel()),
                      "points_per_s": n.numel() / (semi_t * 1e-3),
                      "hbm_gbs": 8.0 * n.numel() / (semi_t * 1e-3) / 1e9,
                      "bound": "fp64 (per-point cbrt, log, expm1 at GB300's FP64 rate)",
                      "E_hartree": {k: semi[k] for k in ("Ex_lda", "Ec_lda", "Ex_pbe", "Ec_pbe", "Ex_revpbe")},
                      "eq3_needed_number": semi["Ec_lda"] - semi["Ec_pbe"] + results[-1][0]},
        "far_tail": tail,
        "cpu_baseline": cpu,
        "e2e": {"value": total_pairs / (e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(n.numel() * 8),
                "d2h_bytes_per_step": int(n.numel() * 8 + 8), "ms_per_step": e2e},
        "gpu_launches": int(launches),
        "clocks": clocks if first_clocks is None else dict(clocks, remeasured_after=first_clocks),
        "wall_s_timed": wall,
        "workloads": wl,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_workloads(V, inputs, T, dev, flush, sms, fp64_peak):
    """Every standard workload in the launch configuration the library uses by
    default: pair interactions/s from the pair kernel's CUDA-event time (the
    call's ms_pairs; for the batched graph the replay's whole time), L2 flushed
    before each timed call, the fraction of the FP32 lane peak at the SM clock
    sampled during these runs, and the FP64 path on the same input with its
    fraction of the measured FP64 FMA rate (fp64_peak, T lane operations/s)."""
    import torch

    def to_dev(wk):
        return torch.from_numpy(wk["density"]).to(dev)

    def args_of(wk):
        return (wk.get("cell", wk["lengths"]), wk["periodic"], wk["n_cut"], wk["r_cut"], T)

    def timed(fn, reps, warm=True):
        if warm:
            fn()                            # warm-up (and, for batches, the graph recording)
        out = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            out.append(fn())
        ms = float(np.mean([r[1]["ms_pairs"] for r in out]))
        return ms, out[-1][1]["pairs"], out[-1][0], out[-1][1]

    def energy(n, a, prec):
        return lambda: V.energy(n, *a, precision=prec)

    def potential(n, a, prec):
        def f():
            E, _, r = V.potential(n, *a, precision=prec)
            return E, r
        return f

    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    raw = {}
    # kr_dimer: FP64 E (and FP32 E for the ratio)
    w0 = inputs.kr_dimer()
    n0, a0 = to_dev(w0), args_of(w0)
    raw["kr_dimer"] = dict(workload="kr_dimer 24x18x18 open, E_nl", mode="energy",
                           f32=timed(energy(n0, a0, "fp32"), 5), f64=timed(energy(n0, a0, "fp64"), 5))
    # molecule24: FP32 E + v, FP64 E + v once
    w2 = inputs.molecule24()
    n2, a2 = to_dev(w2), args_of(w2)
    raw["molecule24"] = dict(workload="molecule24 64^3 open, E_nl + v_nl", mode="potential",
                             f32=timed(potential(n2, a2, "fp32"), 3), f64=timed(potential(n2, a2, "fp64"), 1, warm=False))
    # binding curve: 18 cells in one recorded graph (FP32 E), default and autotuned shapes
    ws3 = inputs.binding_curve()
    ns3 = [to_dev(x) for x in ws3]
    L3, P3 = [x["lengths"] for x in ws3], [x["periodic"] for x in ws3]

    def batched(prec, tu):
        def f():
            E, r = V.energy_batched(ns3, L3, P3, 1e-6, 0.0, T, prec, tuning=tu)
            return float(np.sum(E)), r
        return f
    big = int(np.argmax([x["density"].size for x in ws3]))
    t_tune = time.perf_counter()
    tuned = V.autotune(ns3[big], L3[big], P3[big], 1e-6, 0.0, T, "fp32")
    t_tune = time.perf_counter() - t_tune
    raw["binding_curve"] = dict(workload="binding_curve 18 open cells (32x24x24 .. 64x32x32) in one graph, E_nl",
                                mode="energy", f32=timed(batched("fp32", None), 5),
                                f32_auto=timed(batched("fp32", {"threads": -1}), 5),
                                f64=timed(batched("fp64", None), 2))
    # slab_adsorbate: FP32 E + v at full size; the FP64 ratio on its 64x56x100 regrid
    w4 = inputs.slab_adsorbate()
    n4, a4 = to_dev(w4), args_of(w4)
    f32_full = timed(potential(n4, a4, "fp32"), 2)
    del n4
    w4c = inputs.slab_adsorbate((64, 56, 100))
    n4c, a4c = to_dev(w4c), args_of(w4c)
    raw["slab_adsorbate"] = dict(workload="slab_adsorbate 128x112x200 periodic-xy r_cut=20, E_nl + v_nl",
                                 mode="potential", f32=f32_full, f32_regrid=timed(potential(n4c, a4c, "fp32"), 2),
                                 f64_regrid=timed(potential(n4c, a4c, "fp64"), 1, warm=False))
    clocks = sampler.stop()
    clk = clocks["sm_mhz"] if clocks else 2070.0
    peak = sms * FP32_LANES_PER_SM * clk * 1e6 / 1e12

    def rate(t, ops, ops64=None):
        ms, pairs, E, r = t
        d = {"pairs_per_s": pairs / (ms * 1e-3), "ms_pairs": ms, "pairs": int(pairs), "E_hartree": E,
             "pair_threads": r.get("pair_threads")}
        if ops:
            d["frac"] = ops * pairs / (ms * 1e-3) / 1e12 / peak
        if ops64:
            d["frac_of_measured_fp64"] = ops64 * pairs / (ms * 1e-3) / 1e12 / fp64_peak
        return d

    out = {"clocks": clocks, "peak_T_lane_ops": peak,
           "note": "frac: FP32 lane operations (62 per ordered pair for E + v, 35.5 for E) over "
                   "%d SMs x %d lanes x the sampled SM clock" % (sms, FP32_LANES_PER_SM)}
    for key, d in raw.items():
        ops = OPS_PER_PAIR_EV if d["mode"] == "potential" else OPS_PER_PAIR_E
        e = {"workload": d["workload"], "fp32": rate(d["f32"], ops)}
        if "f64" in d:
            e["fp64"] = rate(d["f64"], None, ops)
            e["fp32_over_fp64"] = e["fp32"]["pairs_per_s"] / e["fp64"]["pairs_per_s"]
            e["rel_err_fp32_vs_fp64"] = abs(d["f32"][2] - d["f64"][2]) / abs(d["f64"][2])
        if "f32_auto" in d:
            e["fp32_autotuned"] = rate(d["f32_auto"], ops)
            e["autotune"] = {"largest_cell_choice": tuned, "seconds": t_tune,
                             "batched_auto_over_default": d["f32_auto"][0] and d["f32"][0] / d["f32_auto"][0]}
        if "f64_regrid" in d:
            e["fp32_64x56x100"] = rate(d["f32_regrid"], ops)
            e["fp64_64x56x100"] = rate(d["f64_regrid"], None, ops)
            e["fp32_over_fp64"] = e["fp32_64x56x100"]["pairs_per_s"] / e["fp64_64x56x100"]["pairs_per_s"]
            e["rel_err_fp32_vs_fp64"] = abs(d["f32_regrid"][2] - d["f64_regrid"][2]) / abs(d["f64_regrid"][2])
            e["fp64_note"] = "the FP64 E + v pass at full size takes about 11 min; ratio on the 64x56x100 regrid"
        out[key] = e
    return out


def config_keys(ws):
    """The workload the line is quoted on, the same in both arms."""
    return {"workload": WORKLOAD, "grid": [48, 84, 120],
            "l2": "flushed (256 MB write) between timed GPU steps",
            "parallelism": "replicas" if ws > 1 else "single"}


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
        "data": "synthetic", "config": config_keys(ws),
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
    ap.add_argument("--no-workloads", action="store_true", help="skip the per-workload entries")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
