"""Sweeps and time to a steady solution with and without Anderson mixing, on the design workload
(O-mesh 256x128, 48x48 Gauss-Legendre grid on [-6, 6]^2, Ma 0.8, 24 seeded bumps): primal to tol,
adjoint to tol, then the full-discrete sensitivity; one JSON line per (Kn, mixing) pair.

    python -m paper_2501_00923_gb300.convergence --kn 0.1,0.01 --accel none,5x10,5x20
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, dvm
from . import workloads as W


def _accel(tok: str):
    if tok == "none":
        return None
    m, k = tok.lower().split("x")
    return int(m), int(k)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2501_00923_gb300.convergence")
    ap.add_argument("--kn", default="0.1,0.01")
    ap.add_argument("--accel", default="none,5x10,5x20", help="comma list of none or MxK (depth x period)")
    ap.add_argument("--mesh", default="256x128")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--stall", type=int, default=3000)
    ap.add_argument("--max-sweeps", type=int, default=200000)
    args = ap.parse_args(argv)
    build.build()
    ni, nj = (int(x) for x in args.mesh.lower().split("x"))
    wl = W.config(4)
    rng = np.random.default_rng(2024)
    raw = rng.uniform(-0.005, 0.005, 24)
    mesh = W.omesh(ni, nj, raw * min(1.0, W.valid_amplitude_scale(ni, raw)))
    ctx = dvm.Context(0)
    m = dvm.Mesh(ctx, mesh.nodes)
    g = dvm.VGrid(ctx, wl.grid.vx, wl.grid.vy, wl.grid.w)
    for kn in (float(x) for x in args.kn.split(",")):
        for tok in args.accel.split(","):
            accel = _accel(tok)
            t0 = time.perf_counter()
            st, pr = dvm.primal_solve(ctx, m, g, kn, wl.flow.Ma, tol=args.tol, max_iter=args.max_sweeps,
                                      storage=args.storage, accel=accel, stall_window=args.stall)
            t1 = time.perf_counter()
            ad, ar = dvm.adjoint_solve(ctx, st, tol=args.tol, max_iter=args.max_sweeps, accel=accel,
                                       stall_window=args.stall)
            t2 = time.perf_counter()
            grad = dvm.sensitivity(ctx, st, ad, mesh.dwall, mesh.s, mode="full")
            t3 = time.perf_counter()
            print(json.dumps({"Kn": kn, "accel": tok, "mesh": args.mesh, "nv": wl.grid.nv, "storage": args.storage,
                              "tol": args.tol, "J": pr.J, "primal_sweeps": pr.iters,
                              "primal_status": dvm.status_string(pr.status), "primal_residual": pr.residual,
                              "adjoint_sweeps": ar.iters, "adjoint_status": dvm.status_string(ar.status),
                              "adjoint_residual": ar.residual, "primal_s": t1 - t0, "adjoint_s": t2 - t1,
                              "sensitivity_s": t3 - t2, "grad_max": float(np.abs(grad).max())}), flush=True)
            ad.close()
            st.close()
    ctx.close()


if __name__ == "__main__":
    main()
