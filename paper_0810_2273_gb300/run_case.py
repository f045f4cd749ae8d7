"""Run one standard workload through the library and print per-call timings.

    python -m paper_0810_2273_gb300.run_case --workload xe_monolayer \
        [--dims 24 42 60] [--mode potential|energy|semilocal|diag|gradient|tail|compare]
        [--precision fp32|fp64] [--gradient fd|spectral] [--repeat 3]

Workloads are the seeded densities of ``paper_0810_2273_gb300.inputs``
(kr_dimer, xe_monolayer, xe_monolayer_hex, rare_gas_chain, molecule24,
slab_adsorbate); --dims regrids the
same cell.  The kernel table is built on the host (quadrature level 1) or
loaded from --table (an .npz written by Table.save).
"""
import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="xe_monolayer",
                    choices=["kr_dimer", "xe_monolayer", "xe_monolayer_hex", "rare_gas_chain", "molecule24",
                             "slab_adsorbate"])
    ap.add_argument("--dims", type=int, nargs=3, default=None)
    ap.add_argument("--mode", default="potential",
                    choices=["potential", "energy", "semilocal", "diag", "gradient", "tail", "compare"])
    ap.add_argument("--gradient", default="fd", choices=["fd", "spectral"], help="the library's density gradient")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--table", default=None)
    ap.add_argument("--quad-level", type=int, default=1)
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: library default)")
    ap.add_argument("--items-per-sm", type=int, default=0, help="work items per warp slot (0: default)")
    a = ap.parse_args(argv)

    import torch

    import paper_0810_2273_gb300 as V
    from paper_0810_2273_gb300 import build, inputs

    build.build()
    T = V.Table.load(a.table) if a.table else V.Table.build(400, 30.0, 200, a.quad_level)
    maker = getattr(inputs, a.workload)
    w = maker(tuple(a.dims)) if a.dims else maker()
    dev = torch.device("cuda:0")
    n = torch.from_numpy(w["density"]).to(dev)
    cell = w.get("cell", w["lengths"])  # general cells carry their lattice vectors
    args = (cell, w["periodic"], w["n_cut"], w["r_cut"], T)
    tu = {"threads": a.threads, "items_per_sm": a.items_per_sm} if (a.threads or a.items_per_sm) else None
    for k in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if a.mode == "gradient":
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g = V.gradient(n, cell, a.gradient)
            e1.record()
            torch.cuda.synchronize()
            print(json.dumps(dict(call=k, ms=e0.elapsed_time(e1), wall_ms=1e3 * (time.perf_counter() - t0),
                                  workload=a.workload, dims=list(n.shape), mode=a.mode, gradient=a.gradient,
                                  max_abs=float(g.abs().max()))), flush=True)
            continue
        if a.mode == "compare":
            # the FP32 and FP64 paths on the same density: E relative and v max-norm
            # relative differences, pair counts, and each path's pair-kernel time
            E32, v32, r32 = V.potential(n, *args, precision="fp32", gradient=a.gradient)
            E64, v64, r64 = V.potential(n, *args, precision="fp64", gradient=a.gradient)
            torch.cuda.synchronize()
            vmax = float(v64.abs().max())
            print(json.dumps(dict(call=k, workload=a.workload, dims=list(n.shape), mode=a.mode,
                                  E32=E32, E64=E64, E_rel=abs(E32 - E64) / abs(E64),
                                  v_maxnorm_rel=float((v32 - v64).abs().max()) / vmax,
                                  pairs32=r32["pairs"], pairs64=r64["pairs"],
                                  ms_pairs32=r32["ms_pairs"], ms_pairs64=r64["ms_pairs"],
                                  wall_ms=1e3 * (time.perf_counter() - t0))), flush=True)
            continue
        if a.mode == "tail":
            res = V.far_tail(n, cell, w["periodic"], w["n_cut"], w["r_cut"], gradient=a.gradient)
            torch.cuda.synchronize()
            res.update(call=k, wall_ms=1e3 * (time.perf_counter() - t0), workload=a.workload,
                       dims=list(n.shape), mode=a.mode)
            print(json.dumps(res), flush=True)
            continue
        if a.mode == "diag":
            res = V.diag_voxel(n, cell, w["periodic"], w["n_cut"], T, gradient=a.gradient)
            torch.cuda.synchronize()
            res.update(call=k, wall_ms=1e3 * (time.perf_counter() - t0), workload=a.workload,
                       dims=list(n.shape), mode=a.mode)
            print(json.dumps(res), flush=True)
            continue
        if a.mode == "semilocal":
            res = V.semilocal(n, cell, w["periodic"], gradient=a.gradient)
            torch.cuda.synchronize()
            res.update(call=k, wall_ms=1e3 * (time.perf_counter() - t0), workload=a.workload,
                       dims=list(n.shape), mode=a.mode, points_per_s=n.numel() / max(res["ms"] * 1e-3, 1e-12))
            print(json.dumps(res), flush=True)
            continue
        if a.mode == "potential":
            E, _, res = V.potential(n, *args, precision=a.precision, tuning=tu, gradient=a.gradient)
        else:
            E, res = V.energy(n, *args, precision=a.precision, tuning=tu, gradient=a.gradient)
        torch.cuda.synchronize()
        res = dict(res)
        res.update(call=k, E=E, wall_ms=1e3 * (time.perf_counter() - t0), workload=a.workload,
                   dims=list(n.shape), mode=a.mode, precision=a.precision, tuning=tu, gradient=a.gradient,
                   pairs_per_s=res["pairs"] / max(res["ms_pairs"] * 1e-3, 1e-12))
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
