"""Sweeps and time to a steady solution with and without Anderson mixing, on the design workload
(O-mesh 256x128, 48x48 Gauss-Legendre grid on [-6, 6]^2, Ma 0.8, 24 seeded bumps): primal to tol,
adjoint to tol, then the full-discrete sensitivity; one JSON line per (Kn, mixing) pair.

    python -m paper_2501_00923_gb300.convergence --kn 0.1,0.01 --accel none,5x10,5x20

With --refine the tool measures mixed-precision refinement instead: an FP32 solve to its rounding
floor, then FP64 sweeps with mixing (--accel, one value) started from the FP32 state and adjoint,
against a cold FP64 solve with the same mixing; both to --tol.

    python -m paper_2501_00923_gb300.convergence --refine --kn 0.01 --accel 5x10 --tol 1e-11
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
    ap.add_argument("--refine", action="store_true", help="FP32 solve, then FP64 sweeps from it (see above)")
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
    if args.refine:
        for kn in (float(x) for x in args.kn.split(",")):
            _refine(ctx, m, g, mesh, kn, wl.flow.Ma, _accel(args.accel.split(",")[0]), args)
        ctx.close()
        return
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


def _refine(ctx, m, g, mesh, kn, Ma, accel, args):
    """FP32 to its floor, FP64 with mixing from there, against a cold FP64 solve with mixing."""
    t = [time.perf_counter()]
    s32, p32 = dvm.primal_solve(ctx, m, g, kn, Ma, tol=args.tol, max_iter=args.max_sweeps, storage="fp32",
                                stall_window=args.stall)
    a32, q32 = dvm.adjoint_solve(ctx, s32, tol=args.tol, max_iter=args.max_sweeps, stall_window=args.stall)
    t.append(time.perf_counter())
    s64 = dvm.State(ctx, m, g, kn, Ma, storage="fp64")
    s64.set(s32.get())
    s64, p64 = dvm.primal_solve(ctx, m, g, kn, Ma, tol=args.tol, max_iter=args.max_sweeps, storage="fp64",
                                state=s64, accel=accel)
    a64 = dvm.Adjoint(s64)
    a64.set(a32.get())
    a64, q64 = dvm.adjoint_solve(ctx, s64, tol=args.tol, max_iter=args.max_sweeps, adjoint=a64, accel=accel)
    t.append(time.perf_counter())
    g_ref = dvm.sensitivity(ctx, s64, a64, mesh.dwall, mesh.s, mode="full")
    g32 = dvm.sensitivity(ctx, s32, a32, mesh.dwall, mesh.s, mode="full")
    for h in (a32, s32, a64, s64):
        h.close()
    t.append(time.perf_counter())
    c64, cp = dvm.primal_solve(ctx, m, g, kn, Ma, tol=args.tol, max_iter=args.max_sweeps, storage="fp64", accel=accel)
    ca, cq = dvm.adjoint_solve(ctx, c64, tol=args.tol, max_iter=args.max_sweeps, accel=accel)
    t.append(time.perf_counter())
    g_cold = dvm.sensitivity(ctx, c64, ca, mesh.dwall, mesh.s, mode="full")
    ca.close()
    c64.close()
    scale = float(np.abs(g_cold).max())
    print(json.dumps({
        "Kn": kn, "accel": accel, "tol": args.tol,
        "fp32": {"s": t[1] - t[0], "primal_sweeps": p32.iters, "adjoint_sweeps": q32.iters,
                 "drag_rel_to_fp64": abs(p32.J - cp.J) / abs(cp.J),
                 "sens_rel_to_fp64": float(np.abs(g32 - g_cold).max()) / scale},
        "fp64_from_fp32": {"s": t[2] - t[1], "primal_sweeps": p64.iters, "primal_status": dvm.status_string(p64.status),
                           "adjoint_sweeps": q64.iters, "adjoint_status": dvm.status_string(q64.status),
                           "drag_rel_to_cold": abs(p64.J - cp.J) / abs(cp.J),
                           "sens_rel_to_cold": float(np.abs(g_ref - g_cold).max()) / scale},
        "fp64_cold": {"s": t[4] - t[3], "primal_sweeps": cp.iters, "primal_status": dvm.status_string(cp.status),
                      "adjoint_sweeps": cq.iters, "adjoint_status": dvm.status_string(cq.status), "J": cp.J}}),
          flush=True)


if __name__ == "__main__":
    main()
