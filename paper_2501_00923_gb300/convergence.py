"""Sweeps and time to a steady solution with and without Anderson mixing, on the design workload
(O-mesh 256x128, 48x48 Gauss-Legendre grid on [-6, 6]^2, Ma 0.8, 24 seeded bumps): primal to tol,
adjoint to tol, then the full-discrete sensitivity; one JSON line per (Kn, mixing) pair.

    python -m paper_2501_00923_gb300.convergence --kn 0.1,0.01 --accel none,5x10,5x20

With --mesh-study the tool measures the spatial order of accuracy instead: the drag of the NACA 0012
section at the first --kn on a nested family of O-meshes (--mesh-study 64x32,128x64,...: the angular
count and the radial count double, and the radial stretching ratio goes to its square root, so every
coarse node is a fine node), at spatial order 1 and 2 (linear reconstruction, Eq. gaussgrad) with
the same velocity grid (--nv points per axis), the second-order solve started from the converged
first-order state of the same mesh; the observed order from the last three levels and the
Richardson-extrapolated drag.

    python -m paper_2501_00923_gb300.convergence --mesh-study 64x32,128x64,256x128,512x256 --kn 0.1
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
    ap.add_argument("--mesh-study", default="", help="comma list of nested O-mesh sizes (see above)")
    ap.add_argument("--nv", type=int, default=24, help="velocity points per axis of the mesh study")
    ap.add_argument("--ma", type=float, default=0.8)
    args = ap.parse_args(argv)
    build.build()
    if args.mesh_study:
        _mesh_study(args)
        return
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


def _nested_meshes(sizes, radius=10.0, first=1e-3):
    """O-meshes whose radial ratio q_L = q_0^(1/2^L) with the radial count doubling: nested families."""
    ni0, nj0 = sizes[0]
    s0 = W.radial_blend(nj0, first, radius)
    q0 = s0[2] / s0[1] - 1.0                  # s_2 / s_1 = q + 1 for s_j = (q^j - 1)/(q^nj - 1)
    out = []
    for L, (ni, nj) in enumerate(sizes):
        if ni != ni0 << L or nj != nj0 << L:
            raise ValueError("mesh-study sizes must double in both directions")
        q = q0 ** (1.0 / (1 << L))
        first_L = radius * (q - 1.0) / (q ** nj - 1.0)
        out.append(W.omesh(ni, nj, np.zeros(0), first=first_L, radius=radius))
    return out


def _observed(J):
    """Observed order and Richardson estimate from the last three values of a nested sequence."""
    if len(J) < 3:
        return None, None
    d1, d2 = J[-3] - J[-2], J[-2] - J[-1]
    if d1 == 0.0 or d2 == 0.0 or d1 / d2 <= 0.0:
        return None, None
    p = float(np.log2(d1 / d2))
    # J_h = J* + c h^p: J[-2] - J[-1] = (2^p - 1) (J[-1] - J*)
    return p, float(J[-1] - d2 / (2.0 ** p - 1.0))


def _mesh_study(args):
    sizes = [tuple(int(x) for x in t.lower().split("x")) for t in args.mesh_study.split(",")]
    kn = float(args.kn.split(",")[0])
    grid = W.velocity_grid(args.nv, 4.0)
    meshes = _nested_meshes(sizes)
    ctx = dvm.Context(0)
    g = dvm.VGrid(ctx, grid.vx, grid.vy, grid.w)
    J = {1: [], 2: []}
    for (ni, nj), mesh in zip(sizes, meshes):
        m = dvm.Mesh(ctx, mesh.nodes)
        st = dvm.State(ctx, m, g, kn, args.ma, storage=args.storage)
        for order in (1, 2):        # second order starts from the converged first-order state
            st.order = order
            t0 = time.perf_counter()
            try:
                _, pr = dvm.primal_solve(ctx, m, g, kn, args.ma, tol=args.tol, max_iter=args.max_sweeps,
                                         storage=args.storage, state=st, stall_window=args.stall)
            except dvm.DVMError as e:          # a diverged solve: reported, and the level left out
                print(json.dumps({"mesh": f"{ni}x{nj}", "order": order, "Kn": kn, "status": str(e)}), flush=True)
                J[order].append(float("nan"))
                break
            dt = time.perf_counter() - t0
            J[order].append(pr.Cd)
            print(json.dumps({"mesh": f"{ni}x{nj}", "order": order, "Kn": kn, "Ma": args.ma, "nv": grid.nv,
                              "storage": args.storage, "Cd": pr.Cd, "sweeps": pr.iters,
                              "status": dvm.status_string(pr.status), "residual": pr.residual, "s": dt}),
                  flush=True)
        st.close()
        m.close()
    for order in (1, 2):
        ok = [x for x in J[order] if np.isfinite(x)]
        p, Jinf = _observed(ok)
        print(json.dumps({"order": order, "Cd": J[order], "observed_order": p, "richardson_Cd": Jinf,
                          "differences": [ok[k] - ok[k + 1] for k in range(len(ok) - 1)]}),
              flush=True)
    g.close()
    ctx.close()


if __name__ == "__main__":
    main()
