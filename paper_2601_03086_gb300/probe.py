"""Small drivers of the library's kernels for profilers (ncu) and quick timing.

    python -m paper_2601_03086_gb300.probe apply --n 160 --reps 3 [--vec f64] [--kind nh]
            [--op residual]
        tangent apply (or residual) on the n^3 x 6 Kuhn cube (FP32 element arithmetic;
        f64 = FP64 vectors with FP32 arithmetic, the PCG configuration)
    python -m paper_2601_03086_gb300.probe solve --n 40 --max-iter 40 [--mode plain]
        Jacobi-PCG on the n^3 cube (the benchmark workload at n = 40); --mode persistent
        (default), graph, or plain (one kernel at a time, so a profiler can attribute time
        per kernel); --reps solves after one warm-up solve
Prints one JSON line with the timings (CUDA events, after warm-up).
"""

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["apply", "solve"])
    ap.add_argument("--n", type=int, default=40)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--vec", choices=["f32", "f64"], default="f32")
    ap.add_argument("--kind", choices=["linear", "nh"], default="linear")
    ap.add_argument("--max-iter", type=int, default=100000)
    ap.add_argument("--mode", choices=["persistent", "plain", "graph"], default="persistent")
    ap.add_argument("--op", choices=["tangent", "residual"], default="tangent")
    a = ap.parse_args(argv)

    import torch

    import pfem_inputs as pi
    import paper_2601_03086_gb300 as P
    from paper_2601_03086_gb300 import build

    build.build()
    if a.kind == "linear":
        p = pi.cube_problem(a.n, seed=2)
    else:
        p = pi.bar_problem(4 * a.n, a.n, a.n, seed=3)
    mesh = P.Mesh(p)
    out = {"mode": a.mode, "n": a.n, "stats": mesh.stats()}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    if a.mode == "apply":
        dt = torch.float32 if a.vec == "f32" else torch.float64
        v = torch.randn(mesh.n_dofs, device="cuda", dtype=dt)
        u = 0.01 * torch.randn_like(v) if a.kind == "nh" else None
        y = torch.empty_like(v)
        arith = "f32" if a.vec == "f64" else None
        if a.op == "residual":
            u = 0.01 * torch.randn_like(v)

        def op():
            if a.op == "tangent":
                P.pfem_tangent_apply(mesh, u, v, y, arith=arith)
            else:
                P.pfem_residual(mesh, u, y, arith=arith)

        op()
        ev[0].record()
        for _ in range(a.reps):
            op()
        ev[1].record()
        ev[1].synchronize()
        out["apply_us"] = ev[0].elapsed_time(ev[1]) * 1e3 / a.reps
        out["op"] = a.op
    else:
        P.pfem_set_solver_mode({"persistent": 0, "plain": 1, "graph": 2}[a.mode])
        P.pfem_solve_linear(mesh, tol=1e-8, max_iter=a.max_iter, raise_on_error=False)
        ev[0].record()
        for _ in range(a.reps):
            _, info = P.pfem_solve_linear(mesh, tol=1e-8, max_iter=a.max_iter, raise_on_error=False)
        ev[1].record()
        ev[1].synchronize()
        out["solve_ms"] = ev[0].elapsed_time(ev[1]) / a.reps
        out["iterations"] = info["iterations"]
        out["us_per_iteration"] = 1e3 * out["solve_ms"] / max(info["iterations"], 1)
        out["mode"] = a.mode
    print(json.dumps(out))
    mesh.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
