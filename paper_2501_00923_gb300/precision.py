"""Precision of the storage options against FP64 storage on one workload (a measurement CLI).

For each Kn: the steady primal solve, the drag adjoint and the full-discrete sensitivity in FP64
storage (the reference; the macroscopic prediction, or moment-space mixing without --predict,
shortens the FP64 solve without changing its solution), and in the arms of --arms:
  fp32            FP32 storage stopped at its rounding floor (plain sweeps);
  fp32_refined    the same, then mixed-precision refinement (dvm_solve_opts.refine_tol);
  fp32_predicted  predicted FP32 sweeps to --tol-predicted (stall window 1000), then refinement with
                  predicted correction sweeps; the adjoint predicted too, to --tol (needs --predict);
  bf16            BF16 storage (plain sweeps).
Reported: drag and sensitivity errors against the FP64 results, sweeps, wall time, and the FP64
residual each FP32 state reaches.  The FP64 sweeps are the ones the oracle parity tests check.
Without --fp64 the reference is skipped and the errors are taken against the last refined arm.

    python -m paper_2501_00923_gb300.precision --workload 4 --kn 0.01,0.1 --predict 40 --out report.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, dvm
from . import workloads as W


def _run(ctx, m, g, mesh, Kn, Ma, storage, args, refine=0.0, accel=None, predict=0, tol=None, stall=None,
         precond=0):
    asw = 0 if storage == "fp64" else args.stall
    sw = asw if stall is None else stall
    if tol is None:
        tol = args.tol64 if storage == "fp64" else args.tol
    atol = args.tol64 if storage == "fp64" else args.tol
    t0 = time.time()
    st, pr = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=tol, max_iter=args.max_sweeps, storage=storage, stall_window=sw,
                              accel=accel, refine_tol=refine, predict=predict, predict_precond=precond)
    t1 = time.time()
    ad, ar = dvm.adjoint_solve(ctx, st, tol=atol, max_iter=args.max_sweeps, stall_window=asw, predict=predict,
                               predict_precond=precond)
    t2 = time.time()
    grad = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
    out = {"J": pr.J, "Cd": pr.Cd, "primal_sweeps": pr.iters, "primal_status": dvm.status_string(pr.status),
           "primal_residual": pr.residual, "adjoint_sweeps": ar.iters, "adjoint_residual": ar.residual,
           "adjoint_status": dvm.status_string(ar.status), "primal_s": t1 - t0, "adjoint_s": t2 - t1,
           "predictions": [pr.predictions, ar.predictions], "grad_full": grad.tolist()}
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
    ap.add_argument("--arms", default="fp32,fp32_refined,bf16", help="comma list of arms (module docstring)")
    ap.add_argument("--predict", type=int, default=0, help="> 0: block-Jacobi iterations of the prediction")
    ap.add_argument("--tol-predicted", type=float, default=1e-5, help="FP32 sweeps of the predicted arm")
    ap.add_argument("--predict-precond", type=int, default=0, choices=[0, 1],
                    help="preconditioner of the prediction's GMRES: 0 diagonal blocks, 1 multigrid")
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
        arms = args.arms.split(",")
        if args.fp64:
            res["fp64"] = (_run(ctx, m, g, mesh, Kn, Ma, "fp64", args, predict=args.predict,
                                precond=args.predict_precond) if args.predict else
                           _run(ctx, m, g, mesh, Kn, Ma, "fp64", args, accel=(5, 10, "moments")))
        if "fp32" in arms:
            res["fp32"] = _run(ctx, m, g, mesh, Kn, Ma, "fp32", args)
        if "fp32_refined" in arms:
            res["fp32_refined"] = _run(ctx, m, g, mesh, Kn, Ma, "fp32", args, refine=args.refine_tol)
        if "fp32_predicted" in arms:
            if args.predict <= 0:
                raise SystemExit("the fp32_predicted arm needs --predict > 0")
            res["fp32_predicted"] = _run(ctx, m, g, mesh, Kn, Ma, "fp32", args, refine=args.refine_tol,
                                         predict=args.predict, tol=args.tol_predicted, stall=1000,
                                         precond=args.predict_precond)
        if "bf16" in arms:
            res["bf16"] = _run(ctx, m, g, mesh, Kn, Ma, "bf16", args)
        cmp = {}
        ref = res.get("fp64")
        refined = "fp32_predicted" if "fp32_predicted" in res else "fp32_refined"
        for k, v in res.items():
            if k == "fp64":
                continue
            gs = np.array(v["grad_full"])
            if ref is not None:
                gref = np.array(ref["grad_full"])
                cmp[k] = {"drag_rel": abs(v["J"] - ref["J"]) / abs(ref["J"]),
                          "sens_max_rel_to_max": float(np.abs(gs - gref).max() / np.abs(gref).max()),
                          "sens_max_componentwise_rel": float(np.max(np.abs(gs - gref) / np.abs(gref)))}
            elif k != refined and refined in res:
                gr = np.array(res[refined]["grad_full"])
                cmp[k] = {"drag_rel_to_refined": abs(v["J"] - res[refined]["J"]) / abs(res[refined]["J"]),
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
