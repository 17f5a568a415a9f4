"""Precision study on the design-loop workload (O-mesh 256x128, 48x48 Gauss-Legendre grid on
[-6, 6]^2, 24 bumps, Ma 0.8): the steady primal, the drag adjoint and the full-discrete and paper
sensitivities in FP64, FP32 and BF16 storage on the GPU, each compared with the FP64 result; the
FP64 state and adjoint are then checked against the oracle (its residual, drag, adjoint residual
and four sensitivity components on that state).

    python tests/precision_study.py --kn 1,0.1,0.01 --max-sweeps 60000 --out report.json
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2501_00923_gb300 import build, dvm  # noqa: E402
from paper_2501_00923_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kn", default="1,0.1,0.01")
    ap.add_argument("--max-sweeps", type=int, default=60000)
    ap.add_argument("--tol", type=float, default=1e-11)
    ap.add_argument("--stall", type=int, default=3000, help="stagnation window of the FP32/BF16 solves")
    ap.add_argument("--storages", default="fp64,fp32,bf16", help="fp64 first: it is the reference")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    build.build()
    from oracle import oracle as O
    ctx = dvm.Context(0)
    wl = W.config(4)
    rng = np.random.default_rng(2024)
    raw = rng.uniform(-0.005, 0.005, 24)
    alpha = raw * min(1.0, W.valid_amplitude_scale(256, raw))
    mesh = W.omesh(256, 128, alpha)
    grid = wl.grid
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    Ma = wl.flow.Ma
    report = {"workload": "omesh256x128-gl48x48-24bumps-Ma0.8", "alpha_seed": 2024, "runs": []}
    for Kn in [float(x) for x in args.kn.split(",")]:
        res = {}
        storages = args.storages.split(",")
        assert storages[0] == "fp64", "the FP64 solve is the reference"
        for storage in storages:
            sw = 0 if storage == "fp64" else args.stall
            t0 = time.time()
            st, pr_ = dvm.primal_solve(ctx, m, g, Kn, Ma, tol=args.tol, max_iter=args.max_sweeps, storage=storage,
                                       stall_window=sw)
            t1 = time.time()
            ad, ar = dvm.adjoint_solve(ctx, st, tol=args.tol, max_iter=args.max_sweeps, stall_window=sw)
            t2 = time.time()
            gf = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
            gp = dvm.sensitivity(ctx, st, ad, mesh.dwall, mode="paper")
            res[storage] = {"J": pr_.J, "Cd": pr_.Cd, "primal_iters": pr_.iters, "primal_residual": pr_.residual,
                            "primal_status": dvm.status_string(pr_.status), "adjoint_iters": ar.iters,
                            "adjoint_residual": ar.residual, "adjoint_status": dvm.status_string(ar.status),
                            "primal_s": t1 - t0, "adjoint_s": t2 - t1, "grad_full": gf.tolist(),
                            "grad_paper": gp.tolist()}
            if storage == "fp64":
                f, phi = st.get(), ad.get()
            ad.close()
            st.close()
            print(Kn, storage, {k: v for k, v in res[storage].items() if not k.startswith("grad")}, flush=True)
        ref = res["fp64"]
        gref = np.array(ref["grad_full"])
        cmp = {}
        for s in storages[1:]:
            gs = np.array(res[s]["grad_full"])
            cmp[s] = {"drag_rel": abs(res[s]["J"] - ref["J"]) / abs(ref["J"]),
                      "sens_max_rel_to_max": float(np.abs(gs - gref).max() / np.abs(gref).max()),
                      "sens_max_componentwise_rel": float(np.max(np.abs(gs - gref) / np.abs(gref)))}
        t0 = time.time()
        pr = O.Problem(mesh.nodes, grid.vx, grid.vy, grid.w, Kn, Ma)
        _, rn = pr.residual(f)
        _, rn0 = pr.residual(pr.freestream())
        Jo = pr.functional(f)
        dJ = pr.functional_grad(f)
        Ra = pr.apply_RT(f, phi * grid.w[None, :, None]) + dJ
        sel = [0, 7, 12, 23]
        go = pr.sens_full(f, phi, mesh.dnodes()[sel])
        orc = {"oracle_residual_rel": rn / rn0, "oracle_drag_rel": abs(Jo - ref["J"]) / abs(Jo),
               "oracle_adjoint_residual_rel": float(np.sqrt(np.sum(Ra ** 2)) / np.sqrt(np.sum(dJ ** 2))),
               "oracle_sens_params": sel,
               "oracle_sens_max_rel": float(np.abs(go - gref[sel]).max() / np.abs(gref).max()),
               "oracle_seconds": time.time() - t0, "oracle_threads": O.threads()}
        print(Kn, "vs fp64", cmp, "oracle", orc, flush=True)
        report["runs"].append({"Kn": Kn, "results": res, "vs_fp64": cmp, "oracle_on_fp64_state": orc})
        del f, phi, dJ, Ra
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(report, fh, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
