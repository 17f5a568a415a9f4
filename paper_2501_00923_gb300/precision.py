"""Precision of the storage options against FP64 storage on one workload (a measurement CLI).

For each Kn: the steady primal solve, the drag adjoint and the full-discrete sensitivity in FP64
storage (the reference; moment-space mixing shortens the FP64 solve without changing its solution),
in FP32 storage stopped at its rounding floor, in FP32 storage with mixed-precision refinement
(dvm_solve_opts.refine_tol) and in BF16 storage.  Reported: drag and sensitivity errors against the
FP64 results, sweeps, wall time, and the FP64 residual each FP32 state reaches.  The FP64 sweeps are
the ones the oracle parity tests check.  Without --fp64 the reference is skipped (for workloads where
an FP64 solve would take hours) and the refined FP32 solve is reported with its FP64 residual.

    python -m paper_2501_00923_gb300.precision --workload 4 --kn 0.01,0.1 --out report.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, dvm
from . import workloads as W


def _run(ctx, m, g, mesh, Kn, Ma, storage, args, refine=0.0, accel=None):
    sw = 0 if storage == "fp64" else args.stall
    tol = args.tol64 if storage == "fp64" else args.tol
    t0 = time.time()
    st, pr = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=tol, max_iter=args.max_sweeps, storage=storage, stall_window=sw,
                              accel=accel, refine_tol=refine)
    t1 = time.time()
    ad, ar = dvm.adjoint_solve(ctx, st, tol=tol, max_iter=args.max_sweeps, stall_window=sw)
    t2 = time.time()
    grad = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    out = {"J": pr.J, "Cd": pr.Cd, "primal_sweeps": pr.iters, "primal_status": dvm.status_string(pr.status),
           "primal_residual": pr.residual, "adjoint_sweeps": ar.iters, "adjoint_residual": ar.residual,
           "adjoint_status": dvm.status_string(ar.status), "primal_s": t1 - t0, "adjoint_s": t2 - t1,
           "grad_full": grad.tolist()}
    if refine > 0:
        out.update({"refine_steps": pr.refine_steps, "refine_sweeps": pr.refine_sweeps,
                    "residual_fp32_floor": pr.residual_fp32, "residual_fp64_entering": pr.residual_fp64})
    ad.close()
    st.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2501_00923_gb300.precision")
    ap.add_argument("--workload", type=int, default=4, help="recipe index: 4 (256x128, GL48) or 2 (384x192, 64^2)")
    ap.add_argument("--kn", default="0.01")
    ap.add_argument("--alpha-seed", type=int, default=2024, help="seed of the 24 bump amplitudes U(-0.005, 0.005)")
    ap.add_argument("--max-sweeps", type=int, default=400000)
    ap.add_argument("--tol", type=float, default=1e-7, help="FP32/BF16 sweeps (they stop at their floor)")
    ap.add_argument("--tol64", type=float, default=1e-11)
    ap.add_argument("--refine-tol", type=float, default=1e-10)
    ap.add_argument("--stall", type=int, default=3000)
    ap.add_argument("--fp64", type=int, default=1, help="1: solve the FP64 reference")
    ap.add_argument("--bf16", type=int, default=1)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    build.build()
    ctx = dvm.Context(0)
    wl = W.config(args.workload)
    rng = np.random.default_rng(args.alpha_seed)
    raw = rng.uniform(-0.005, 0.005, 24)
    alpha = raw * min(1.0, W.valid_amplitude_scale(wl.mesh.ni, raw))
    mesh = W.omesh(wl.mesh.ni, wl.mesh.nj, alpha)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, wl.grid.vx, wl.grid.vy, wl.grid.w)
    Ma = wl.flow.Ma
    report = {"workload": f"omesh{mesh.ni}x{mesh.nj}-v{wl.grid.nv}-24bumps-Ma{Ma}", "alpha_seed": args.alpha_seed,
              "runs": []}
    for Kn in [float(x) for x in args.kn.split(",")]:
        res = {}
        if args.fp64:
            res["fp64"] = _run(ctx, m, g, mesh, Kn, Ma, "fp64", args, accel=(5, 10, "moments"))
        res["fp32"] = _run(ctx, m, g, mesh, Kn, Ma, "fp32", args)
        res["fp32_refined"] = _run(ctx, m, g, mesh, Kn, Ma, "fp32", args, refine=args.refine_tol)
        if args.bf16:
            res["bf16"] = _run(ctx, m, g, mesh, Kn, Ma, "bf16", args)
        cmp = {}
        ref = res.get("fp64")
        for k, v in res.items():
            if k == "fp64":
                continue
            gs = np.array(v["grad_full"])
            if ref is not None:
                gref = np.array(ref["grad_full"])
                cmp[k] = {"drag_rel": abs(v["J"] - ref["J"]) / abs(ref["J"]),
                          "sens_max_rel_to_max": float(np.abs(gs - gref).max() / np.abs(gref).max()),
                          "sens_max_componentwise_rel": float(np.max(np.abs(gs - gref) / np.abs(gref)))}
            elif k != "fp32_refined":
                gr = np.array(res["fp32_refined"]["grad_full"])
                cmp[k] = {"drag_rel_to_refined": abs(v["J"] - res["fp32_refined"]["J"]) / abs(res["fp32_refined"]["J"]),
                          "sens_max_componentwise_rel_to_refined": float(np.max(np.abs(gs - gr) / np.abs(gr)))}
        run = {"Kn": Kn, "results": {k: {kk: vv for kk, vv in v.items() if kk != "grad_full"} for k, v in res.items()},
               "errors": cmp}
        print(json.dumps(run), flush=True)
        report["runs"].append({"Kn": Kn, "results": res, "errors": cmp})
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(report, fh, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
