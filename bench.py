"""Benchmark: warm-started solves of the GB300 P1 finite-element operator (PFEM warm start).

One step = one warm-started Jacobi-PCG solve of the 3-D linear-elastic unit cube
(40^3 hexes x 6 = 384,000 P1 tets, 68,921 nodes; per-element E = exp(0.5 N(0,1)) and
nu ~ U[0.25, 0.35] from seed 2; z=0 clamped; z=1 traction (0, 0, -0.1)) to relative
residual 1e-8, FP32 element kernels with FP64 vectors, dots and residual replacement.
The warm start of step i is the converged solution plus a seeded smooth perturbation of
1% relative L2 (a fresh seed per step), resident in HBM before the timed region. L2 is
flushed (256 MB write) between steps, outside the per-step CUDA events.

value  = solves/s over all ranks (each rank solves its own stream of requests: replicas,
         no data-path collective; time = max over ranks).
e2e    = the same solves through the public API from pinned host buffers (H2D of u0 and
         D2H of the solution inside the timed region).
Extra keys: per-solve latency p50/p99, the plain one-iteration-at-a-time GPU loop on the
same inputs, zero-start solves, the FP32-vs-FP64 solution difference, the roofline of the
dominant kernel (element tangent apply), the same kernel on the 160^3 cube (24.6 M tets,
beyond L2), the Neo-Hookean Newton solves of the 64x16x16 bar, and the FP64 CPU oracle
timed on this host.

--probe apply|solve runs one kernel-level driver instead (for ncu captures and quick timing):
    --probe apply --n 160 --reps 3 [--vec f64] [--kind nh] [--op residual]
        tangent apply (or residual) on the n^3 x 6 Kuhn cube (FP32 element arithmetic;
        f64 = FP64 vectors with FP32 arithmetic, the PCG configuration)
    --probe solve --n 40 --max-iter 40 [--solver-mode plain]
        Jacobi-PCG solves of the n^3 cube (the benchmark workload at n = 40); plain runs one
        kernel at a time, so that a profiler attributes time per kernel
    --probe attn --n 1048576 --reps 3
        physics-attention forwards on n points (128 channels, 128 tokens, 8 heads)
  and prints one JSON line with CUDA-event timings after warm-up.

--impl reference times the FP64 CPU oracle (global sparse assembly + Jacobi-PCG) on the
same workload: each step is one full warm-started solve of the cube (its own seeded warm
start, as in the GPU arm) with the oracle's assembled K; assembly happens once, untimed.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("element-op GB/s vs HBM peak; warm-start solves/s + p50/p99 latency vs plain GPU loop")
MODES = {"persistent": 0, "plain": 1, "graph": 2}  # pfem_set_solver_mode values
TOL = 1e-8
WORKLOAD = {
    "workload": "cube40_lognormal_linear_warm_pcg",
    "mesh": "40^3 hexes x 6 = 384000 P1 tets, 68921 nodes, 201720 free DOFs",
    "material": "E lognormal(0,0.5), nu U[0.25,0.35], seed 2",
    "bc": "z=0 clamped, z=1 traction (0,0,-0.1)",
    "solver": "Jacobi-PCG, rel residual 1e-8 (FP64 true residual)",
    "warm_start": "exact + smooth 1% rel L2 perturbation, new seed per step",
    "precision": "FP32 element kernels, FP64 vectors/dots/residual replacement",
    "l2": "flushed between steps (256 MB write)",
    "parallelism": "replicas (independent solves per GPU)",
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic FP32 flops per 3-D simplex (FMA = 2 flops), counted from the element formulas
# the kernels evaluate: geometry (edges, adjugate rows, det, 1/det) 43; gradient of a field
# from corner values 54 (63 with the 1/det scale of the Neo-Hookean path); linear stress 18;
# contraction T c_a with f_0 = -sum 51; linear energy 40; Neo-Hookean kinematic state (J - 1,
# cof, H - I, ln J) 96; first Piola stress 55; its derivative along grad v 159; Psi 10.
FLOPS_PER_ELEM = {
    ("linear", "tangent"): 43 + 54 + 18 + 51,                       # 166
    ("nh", "tangent"): 43 + 63 + 96 + 63 + 159 + 51,                # 475
    ("linear", "energy+grad+hvp"): 43 + 54 + 40 + 18 + 51 + 54 + 18 + 51,   # 329
    ("nh", "energy+grad+hvp"): 43 + 63 + 96 + 10 + 55 + 51 + 63 + 159 + 51,  # 591
}


def _fp32_peak_tflops():
    """FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x the maximum SM clock
    (MEASURED_PEAKS.json sm_max_mhz, else 2070 MHz)."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12, mhz


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(round(q * (len(v) - 1)))))
    return v[k]


def step_seeds(rank, n_steps):
    """Warm-start seeds of one rank's steps: every rank solves its own requests (replicas,
    no exchange), so the seeds of different ranks never coincide."""
    return [20 + 1000 * rank + i for i in range(n_steps)]


def whole_job_rate(dist, world, units_per_rank, seconds_local, device):
    """Whole-job throughput of independent replicas: every rank processed units_per_rank in
    seconds_local; the job took the slowest rank's time (max over ranks). Returns (rate,
    max seconds)."""
    import torch

    t = torch.tensor([float(seconds_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return world * units_per_rank / t_max, t_max


def cpu_oracle_warm_solve(n_sample=None):
    """Oracle timing worker (runs in a single-threaded child process). Returns a dict."""
    import numpy as np

    import pfem_inputs as pi
    from oracle import fem, solve

    p = pi.cfg2_cube()
    t0 = time.perf_counter()
    m = fem.Mesh(p)
    K = fem.assemble_linear_K(m)
    t_asm = time.perf_counter() - t0
    u_star, _, _ = solve.solve_linear(m, tol=1e-10, K=K)
    warm = pi.make_warm_start(p, u_star, seed=20)
    t0 = time.perf_counter()
    _, it_full, _ = solve.solve_linear(m, u0=warm, tol=TOL, K=K)
    t_full = time.perf_counter() - t0
    out = {"assembly_s": t_asm, "solve_s": t_full, "iterations": it_full}
    if n_sample:  # (untimed warm-up solves, timed full solves), each with its own warm start
        n_warm, n_timed = n_sample
        solves, iters = [], []
        for i in range(n_warm + n_timed):
            w = pi.make_warm_start(p, u_star, seed=21 + i)
            t0 = time.perf_counter()
            _, it, _ = solve.solve_linear(m, u0=w, tol=TOL, K=K)
            if i >= n_warm:
                solves.append(time.perf_counter() - t0)
                iters.append(it)
        out["solve_samples_s"] = solves
        out["solve_samples_it"] = iters
    del np
    return out


def _run_oracle_child(args_list):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    res = subprocess.run([sys.executable, os.path.abspath(__file__)] + args_list, env=env, capture_output=True,
                         text=True, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    k, w = args.steps, args.warmup
    # warm-up: one full warm solve in the setup plus (w - 1) more; timed: k full warm solves
    r = _run_oracle_child(["--oracle-worker", str(max(w - 1, 0)), str(k)])
    total = sum(r["solve_samples_s"])
    solve_s = total / k
    value = k / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": k,
        "warmup": w, "ms_per_step": solve_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "per step one full warm-started Jacobi-PCG solve to 1e-8 (%d-%d iterations) on "
                                   "the oracle's assembled K (assembly %.1f s, once, untimed), single-threaded"
                                   % (min(r["solve_samples_it"]), max(r["solve_samples_it"]), r["assembly_s"])},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_full_warm_solve_s": r["solve_s"],
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the 160^3 cube, Newton and CPU-oracle extras")
    ap.add_argument("--solver-mode", default="graph", choices=list(MODES),
                    help="graph (device while loop, default), persistent (one cooperative launch per "
                         "replacement interval) or plain (one launch per kernel, for profiler launch lists)")
    ap.add_argument("--oracle-worker", nargs=2, type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--probe", choices=["apply", "solve", "attn"], default=None,
                    help="run one kernel-level driver (see the module docstring) instead of the benchmark")
    ap.add_argument("--n", type=int, default=40, help="probe: cube of n^3 hexes x 6 tets")
    ap.add_argument("--reps", type=int, default=3, help="probe: timed repetitions after one warm-up")
    ap.add_argument("--vec", choices=["f32", "f64"], default="f32", help="probe apply: vector type")
    ap.add_argument("--kind", choices=["linear", "nh"], default="linear", help="probe apply: material")
    ap.add_argument("--op", choices=["tangent", "residual"], default="tangent", help="probe apply: operator")
    ap.add_argument("--max-iter", type=int, default=100000, help="probe solve: PCG iteration cap")
    ap.add_argument("--k", type=int, default=0, help="probe apply: k > 0 applies to k vectors at once")
    ap.add_argument("--serving", default=None, metavar="N,HI,EVERY[,NLAT]",
                    help="run only the serving workload on N requests of up to HI tets with the plain loop "
                         "on every EVERY-th request (config 5: 1000,2000000,20,200): served with all arrivals "
                         "at t=0 and at 2x the plain-loop rate, and the first NLAT requests at 0.5x; prints "
                         "one JSON line")
    args = ap.parse_args()
    if args.oracle_worker is not None:
        print(json.dumps(cpu_oracle_warm_solve(tuple(args.oracle_worker))))
        return 0
    if args.probe is not None:
        return probe(args)
    if args.serving is not None:
        return serving_only(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import pfem_inputs as pi
    from paper_2601_03086_gb300 import build

    if rank == 0:
        build.build()
    barrier()
    if rank != 0:
        build.build()
    import paper_2601_03086_gb300 as P

    # ---- workload -------------------------------------------------------------------------
    p = pi.cfg2_cube()
    mesh = P.Mesh(p)
    st = mesh.stats()
    n = mesh.n_dofs
    u_star, _ = P.pfem_solve_linear(mesh, tol=1e-12, precision="f64")
    u_star_h = u_star.cpu().numpy()
    n_steps = args.warmup + args.steps
    seeds = step_seeds(rank, n_steps)
    warm_h = [pi.make_warm_start(p, u_star_h, seed=s) for s in seeds]
    warm_d = [torch.tensor(w, device="cuda") for w in warm_h]
    u_out = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def flush_l2():
        flush.fill_(1.0)

    P.pfem_set_solver_mode(MODES[args.solver_mode])
    for i in range(args.warmup):
        P.pfem_solve_linear(mesh, warm_d[i], tol=TOL, u_out=u_out)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev = [_events(torch) for _ in range(args.steps)]
    infos = []
    for i in range(args.steps):
        flush_l2()
        ev[i][0].record()
        _, info = P.pfem_solve_linear(mesh, warm_d[args.warmup + i], tol=TOL, u_out=u_out)
        ev[i][1].record()
        infos.append(info)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    value, total_max = whole_job_rate(dist, world, args.steps, total_s, "cuda")
    ok = all(i["status"] == 0 and i["rel_residual_true_f64"] < TOL for i in infos)

    # ---- end to end through the public API from pinned host buffers ------------------------
    host_in = [torch.tensor(w).pin_memory() for w in warm_h[args.warmup:]]
    host_out = torch.empty(n, dtype=torch.float64).pin_memory()
    u0_dev = torch.empty(n, dtype=torch.float64, device="cuda")
    barrier()
    torch.cuda.synchronize()
    e2e_ms = []
    for i in range(args.steps):
        flush_l2()
        a, b = _events(torch)
        a.record()
        u0_dev.copy_(host_in[i], non_blocking=True)
        P.pfem_solve_linear(mesh, u0_dev, tol=TOL, u_out=u_out)
        host_out.copy_(u_out, non_blocking=True)
        b.record()
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_value, _ = whole_job_rate(dist, world, args.steps, sum(e2e_ms) / 1e3, "cuda")

    extras = {}
    if rank == 0:
        # plain one-iteration-at-a-time loop (host-synchronised check every iteration)
        P.pfem_set_solver_mode(1)
        plain_ms = []
        for i in range(min(args.steps, 5)):
            flush_l2()
            a, b = _events(torch)
            a.record()
            P.pfem_solve_linear(mesh, warm_d[args.warmup + i], tol=TOL, u_out=u_out)
            b.record()
            b.synchronize()
            plain_ms.append(a.elapsed_time(b))
        graph_ms = []
        P.pfem_set_solver_mode(MODES["persistent"])
        for i in range(min(args.steps, 5)):
            flush_l2()
            a, b = _events(torch)
            a.record()
            P.pfem_solve_linear(mesh, warm_d[args.warmup + i], tol=TOL, u_out=u_out)
            b.record()
            b.synchronize()
            graph_ms.append(a.elapsed_time(b))
        extras["persistent_loop"] = {"solves_per_s": 1e3 / statistics.mean(graph_ms),
                                     "ms_mean": statistics.mean(graph_ms)}
        P.pfem_set_solver_mode(MODES[args.solver_mode])
        zero_ms, zero_it = [], []
        for i in range(2):
            flush_l2()
            a, b = _events(torch)
            a.record()
            _, zi = P.pfem_solve_linear(mesh, None, tol=TOL, u_out=u_out)
            b.record()
            b.synchronize()
            zero_ms.append(a.elapsed_time(b))
            zero_it.append(zi["iterations"])
        u32, _ = P.pfem_solve_linear(mesh, warm_d[args.warmup], tol=TOL)
        u64, i64 = P.pfem_solve_linear(mesh, warm_d[args.warmup], tol=TOL, precision="f64")
        fp_err = float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64))
        extras.update({
            "latency_ms_p50": _pct(step_ms, 0.5), "latency_ms_p99": _pct(step_ms, 0.99),
            "plain_loop": {"solves_per_s": 1e3 / statistics.mean(plain_ms), "ms_mean": statistics.mean(plain_ms)},
            "speedup_vs_plain_loop": statistics.mean(plain_ms) / statistics.mean(step_ms),
            "zero_start": {"solves_per_s": 1e3 / statistics.mean(zero_ms), "iterations": zero_it},
            "warm_iterations": [i["iterations"] for i in infos][:5],
            "fp32_vs_fp64_rel_l2": fp_err, "fp64_iterations": i64["iterations"],
            "fp64_true_rel_residual_max": max(i["rel_residual_true_f64"] for i in infos),
        })

        # ---- roofline of the dominant kernel: the PCG-fused apply ----------------------------
        # One more warm solve of the same mesh in the plain loop with kernel timing on: CUDA
        # events on the mesh's stream around each iteration's fused apply and update (the graph
        # loop runs the same two kernels back to back but cannot be bracketed per kernel).
        peak, peak_kind = _peaks()
        P.pfem_set_solver_mode(MODES["plain"])
        P.pfem_set_kernel_timing(1)
        _, ti = P.pfem_solve_linear(mesh, warm_d[0], tol=TOL)
        P.pfem_set_kernel_timing(0)
        P.pfem_set_solver_mode(MODES[args.solver_mode])
        nt = max(ti["timed_iterations"], 1)
        us_pcg = 1e3 * ti["apply_ms"] / nt
        # bytes: connectivity + materials 24 B/elem; per node X 12 B, mask 1 B and five FP64
        # 3-vectors (r, dinv, p_old read; p_new, q written)
        alg_pcg = st["n_elems"] * 24 + st["n_nodes"] * (12 + 1 + 5 * 24)
        ach_pcg = alg_pcg / (us_pcg * 1e-6) / 1e9
        # the plain tangent apply of the same mesh (FP64 vectors, FP32 elements), for reference
        alg = st["n_elems"] * 24 + st["n_nodes"] * 37
        v64 = torch.randn(n, dtype=torch.float64, device="cuda")
        y64 = torch.empty_like(v64)
        for _ in range(5):
            P.pfem_tangent_apply(mesh, None, v64, y64, arith="f32")
        a, b = _events(torch)
        reps = 200
        a.record()
        for _ in range(reps):
            P.pfem_tangent_apply(mesh, None, v64, y64, arith="f32")
        b.record()
        b.synchronize()
        us = a.elapsed_time(b) * 1e3 / reps
        ach = alg / (us * 1e-6) / 1e9
        extras["roofline"] = {
            "bound": "hbm", "achieved": ach_pcg, "peak": peak, "unit": "GB/s", "frac": ach_pcg / peak,
            "traffic": _committed_traffic("cube40_pcg"),
            "kernel": "tile_kernel<3,linear,tangent+PCG,f64 vectors,f32> (PCG-fused apply)",
            "launch_us": us_pcg, "launches_timed": ti["timed_iterations"], "algorithmic_bytes": alg_pcg,
            "update_kernel_us": 1e3 * ti["update_ms"] / nt, "peak_kind": peak_kind + " hbm_gbs",
            "timing": "CUDA events on the mesh stream around every fused apply of one warm plain-loop solve",
            "note": "384k-tet operator and FP64 vectors are L2-resident; latency bound",
        }
        extras["apply_only"] = {"kernel": "tile_kernel<3,linear,tangent,f64 vectors,f32> + halo", "launch_us": us,
                                "achieved_gbs": ach, "algorithmic_bytes": alg, "frac": ach / peak}
        if not args.quick:
            extras["roofline_large"] = _large_cube(P, pi, torch, peak, peak_kind)
            extras["newton"] = _newton(P, pi, torch, peak)
            extras["batch_loss"] = _batch_loss(P, pi, torch, np, peak)
            extras["serving"] = _serving(P, pi, torch, np)
            extras["attention"] = _attention(P, torch, np, peak)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": WORKLOAD,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
        "clocks": clocks, "all_converged": ok, "solver_mode": args.solver_mode,
    }
    if rank == 0:
        line["roofline"] = extras.pop("roofline")
        line.update(extras)
        if world == 1 and not args.quick:
            line["cpu_baseline"] = _cpu_baseline()
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    mesh.close()
    barrier()
    if world > 1:
        dist.destroy_process_group()
    return 0


TILE_SOURCES = ("kernels_tile.cu", "tile.cuh", "element.cuh", "pfem_internal.h")


def tile_source_sha():
    """Digest of the element-tile kernel sources (a committed ncu traffic figure is used only
    while it still describes the compiled kernel)."""
    import hashlib

    h = hashlib.sha256()
    for name in TILE_SOURCES:
        with open(os.path.join(ROOT, "paper_2601_03086_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _committed_traffic(key):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(key)
        if e and e.get("tile_sources_sha") == tile_source_sha():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def _large_cube(P, pi, torch, peak, peak_kind):
    p = pi.roofline_cube()
    mesh = P.Mesh(p)
    st = mesh.stats()
    alg = st["n_elems"] * 24 + st["n_nodes"] * 37
    v = torch.randn(mesh.n_dofs, dtype=torch.float32, device="cuda")
    y = torch.empty_like(v)
    for _ in range(3):
        P.pfem_tangent_apply(mesh, None, v, y)
    reps = 20
    a, b = _events(torch)
    a.record()
    for _ in range(reps):
        P.pfem_tangent_apply(mesh, None, v, y)
    b.record()
    b.synchronize()
    us = a.elapsed_time(b) * 1e3 / reps
    ach = alg / (us * 1e-6) / 1e9
    # several right-hand sides per pass over the element data (pfem_tangent_apply_multi):
    # algorithmic bytes per launch = 24 B/elem + (X 12 + mask 1) B/node once + (v 12 + y 12)
    # B/node per vector
    multi = []
    for k in (1, 2, 4, 6):
        V = torch.randn((k, mesh.n_dofs), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(V)
        for _ in range(2):
            P.pfem_tangent_apply_multi(mesh, V, Y)
        reps_k = 10
        a, b = _events(torch)
        a.record()
        for _ in range(reps_k):
            P.pfem_tangent_apply_multi(mesh, V, Y)
        b.record()
        b.synchronize()
        us_k = a.elapsed_time(b) * 1e3 / reps_k
        alg_k = st["n_elems"] * 24 + st["n_nodes"] * (13 + 24 * k)
        multi.append({"k": k, "launch_us": us_k, "us_per_rhs": us_k / k, "algorithmic_bytes": alg_k,
                      "bytes_per_rhs": alg_k / k, "achieved_gbs": alg_k / (us_k * 1e-6) / 1e9,
                      "frac": alg_k / (us_k * 1e-6) / 1e9 / peak, "rhs_applies_per_s": k / (us_k * 1e-6)})
        del V, Y
    mesh.close()
    fp32_peak, mhz = _fp32_peak_tflops()
    tflops = FLOPS_PER_ELEM[("linear", "tangent")] * st["n_elems"] / (us * 1e-6) / 1e12
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": _committed_traffic("cube160_f32v"), "launch_us": us, "algorithmic_bytes": alg,
            "elements_per_s": st["n_elems"] / (us * 1e-6), "multi_rhs": multi,
            "fp32": {"achieved_tflops": tflops, "peak_tflops": fp32_peak, "frac": tflops / fp32_peak,
                     "flops_per_elem": FLOPS_PER_ELEM[("linear", "tangent")], "clock_mhz": mhz},
            "workload": "160^3 x 6 = 24,576,000 tets, 4,173,281 nodes, f32 vectors", "peak_kind": peak_kind}


def _batch_loss(P, pi, torch, np, peak=None):
    """64-mesh ragged batch (cube / L-shape / holed plate, 5k-200k tets, mixed materials):
    energy + gradient + Hessian-vector product of every mesh in one element launch. Also:
    algorithmic bytes (per mesh 24 B/elem + per node X 12, mask 1, u, v, grad, hvp 12 each) and
    flops (FLOPS_PER_ELEM) per evaluation against the HBM and FP32 peaks, and the FP32 results
    against the same gradients and Hessian products evaluated per mesh in FP64."""
    items = pi.cfg4_batch()
    meshes = [P.Mesh(p) for p, _ in items]
    batch = P.Batch(meshes)
    u = torch.tensor(np.concatenate([uu.reshape(-1) for _, uu in items]), device="cuda")
    v = torch.randn_like(u)
    for _ in range(3):
        batch.eval(u, v, energy=True, grad=True, hvp=True)
    reps = 20
    a, b = _events(torch)
    a.record()
    for _ in range(reps):
        batch.eval(u, v, energy=True, grad=True, hvp=True)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    n_tets = int(sum(p["conn"].shape[0] for p, _ in items))
    n_nodes = int(sum(p["coords"].shape[0] for p, _ in items))
    alg = n_tets * 24 + n_nodes * (12 + 1 + 4 * 12)
    flops = sum(p["conn"].shape[0] * FLOPS_PER_ELEM[("linear" if p["kind"] == "linear" else "nh",
                                                      "energy+grad+hvp")] for p, _ in items)
    _, g32, h32 = batch.eval(u, v, energy=False, grad=True, hvp=True)
    g64, h64 = [], []
    off = batch.offsets
    for k, m in enumerate(meshes):
        uk = u[off[k]:off[k + 1]].double().contiguous()
        vk = v[off[k]:off[k + 1]].double().contiguous()
        g64.append(P.pfem_energy_gradient(m, uk))
        h64.append(P.pfem_energy_hvp(m, uk, vk))
    g64, h64 = torch.cat(g64), torch.cat(h64)
    err_g = float(torch.linalg.norm(g32.double() - g64) / torch.linalg.norm(g64))
    err_h = float(torch.linalg.norm(h32.double() - h64) / torch.linalg.norm(h64))
    batch.close()
    for m in meshes:
        m.close()
    fp32_peak, mhz = _fp32_peak_tflops()
    tflops = flops / (ms * 1e-3) / 1e12
    gbs = alg / (ms * 1e-3) / 1e9
    return {"meshes": len(items), "tets": n_tets, "ms_per_eval": ms, "evals_per_s": 1e3 / ms,
            "tets_per_s": n_tets * 1e3 / ms, "ops": "energy + gradient + Hessian-vector, FP32 elements",
            "hbm": {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak if peak else None,
                    "algorithmic_bytes": alg},
            "fp32": {"achieved_tflops": tflops, "peak_tflops": fp32_peak, "frac": tflops / fp32_peak,
                     "flops_per_eval": flops, "clock_mhz": mhz},
            "fp32_vs_fp64_rel_l2": {"gradient": err_g, "hvp": err_h}}


def _serving(P, pi, torch, np, n_req=400, rate_factors=(20.0,), hi=50_000, plain_every=1, ref_tol=1e-12,
             ref_precision="f64", budget=120 << 30, timeout_s=900.0):
    """The serving workload: the first n_req records of the seeded request stream (Poisson
    arrivals, 70% linear cubes / 30% Neo-Hookean bars at 10% stretch, 50% warm started), mesh
    sizes log-uniform in [2k, hi] tets (config 5 is 1,000 requests up to 2M), tol 1e-8;
    zero-start Neo-Hookean requests take 5 load steps, warm-started ones 1.
    Plain loop (and graph loop): the requests one at a time, each creating its mesh (host
    planning + upload, timed separately) and solving with the host-synchronised
    one-iteration-at-a-time loop (graph loop: the device while-loop); with plain_every = k only
    every k-th request runs and the loop's time is that sample's sum times k (an unbiased
    estimate: the loop's time is the sum of independent per-request times).
    Served: every request submitted at its arrival time to one server (`budget` bytes of
    admission budget), arrivals at rate_factor x the plain loop's solves/s for each factor
    (inf = all at t = 0, the server's capacity; 2; 0.5 = latency run), an entry (factor, n)
    serving only the first n requests; solves/s = requests / makespan, latency = completion
    - arrival. Warm starts perturb a solve of the request to ref_tol (input preparation,
    untimed); the served solutions are compared with those references (FP32-vs-FP64 line)."""
    reqs = pi.cfg5_requests(n_requests=n_req, seed=5, hi=hi)
    probs = [pi.request_problem(r) for r in reqs]
    u0s, urefs = [], []
    t_prep = time.perf_counter()
    for r, p in zip(reqs, probs):
        urefs.append(None)
        if not r["warm"]:
            u0s.append(None)
            continue
        m = P.Mesh(p)
        if r["kind"] == "linear":
            u, info = P.pfem_solve_linear(m, tol=ref_tol, precision=ref_precision, raise_on_error=False)
        else:
            for ls in (5, 20):
                u, info = P.pfem_solve_newton(m, tol=ref_tol, n_load_steps=ls, precision=ref_precision,
                                              raise_on_error=False)
                if info["status"] == 0:
                    break
        m.close()
        if info["status"] != 0:  # no reference solution to perturb: served as a zero start
            u0s.append(None)
            continue
        urefs[-1] = u.cpu().numpy()
        u0s.append(pi.make_warm_start(p, urefs[-1], seed=1 + r["seed"] % 100000))
    t_prep = time.perf_counter() - t_prep

    def steps(r, u0):
        return 1 if (r["kind"] == "linear" or u0 is not None) else 5

    def solve_one(m, r, u0):
        u0d = None if u0 is None else torch.tensor(u0, device="cuda")
        if r["kind"] == "linear":
            u, info = P.pfem_solve_linear(m, u0d, tol=TOL, raise_on_error=False)
        else:
            u, info = P.pfem_solve_newton(m, u0d, tol=TOL, n_load_steps=steps(r, u0), raise_on_error=False)
        return u.cpu(), info

    sample = list(range(0, n_req, plain_every))
    out = {"requests": n_req, "tets_range": [2000, hi], "budget_bytes": budget,
           "tets_total": int(sum(r["n_tets"] for r in reqs)), "warm_start_prep_s": t_prep,
           "linear": sum(r["kind"] == "linear" for r in reqs), "warm": sum(u is not None for u in u0s),
           "plain_loop_sample": {"every": plain_every, "requests": len(sample)}}
    loop_info = {}
    for mode_name, mode in (("plain_loop", MODES["plain"]), ("graph_loop", MODES["graph"])):
        P.pfem_set_solver_mode(mode)
        torch.cuda.synchronize()
        lat, ok, plan_s, total = [], 0, 0.0, 0.0
        for k in sample:
            r, p, u0 = reqs[k], probs[k], u0s[k]
            a = time.perf_counter()
            m = P.Mesh(p)  # host planning + upload (the server does this on planner threads)
            b = time.perf_counter()
            _, info = solve_one(m, r, u0)
            m.close()
            loop_info.setdefault(k, {})[mode_name] = (info["iterations"], info["newton_iterations"],
                                                     time.perf_counter() - b)
            lat.append(time.perf_counter() - a)
            plan_s += b - a
            total += time.perf_counter() - a
            ok += info["status"] == 0
        wall = total * plain_every  # the loop's time for all n_req requests (estimate if sampled)
        plan_all = plan_s * plain_every
        out[mode_name] = {"solves_per_s": n_req / wall, "wall_s": wall, "converged_in_sample": ok,
                          "plan_upload_s": plan_all, "solves_per_s_excluding_planning": n_req / (wall - plan_all),
                          "solve_ms_p50": 1e3 * _pct(lat, 0.5), "solve_ms_p99": 1e3 * _pct(lat, 0.99)}
    P.pfem_set_solver_mode(MODES["graph"])

    served_iters = []

    def served_run(rate_factor, n_run=None):
        n_run = n_req if n_run is None else min(n_run, n_req)
        rate = rate_factor * out["plain_loop"]["solves_per_s"]
        arrive = np.cumsum([r["gap"] for r in reqs[:n_run]]) / rate  # rate_factor inf: all at t = 0
        server = P.Server(budget, max_slots=128)
        tickets, t_sub, done = [], [], {}
        t0 = time.perf_counter()
        i = 0
        while len(done) < n_run:
            now = time.perf_counter() - t0
            while i < n_run and arrive[i] <= now:
                r = reqs[i]
                tickets.append(server.submit(probs[i], u0s[i], TOL, r["kind"] if r["kind"] == "linear" else "newton",
                                             steps(r, u0s[i])))
                t_sub.append(time.perf_counter() - t0)
                i += 1
            for k, t in enumerate(tickets):
                if k not in done:
                    res = server.poll(t)
                    if res is not None:
                        done[k] = (time.perf_counter() - t0, res[0], res[2], res[1])
            if time.perf_counter() - t0 > timeout_s:
                raise RuntimeError("served requests did not finish in %.0f s" % timeout_s)
            time.sleep(0.0005)
        makespan = max(v[0] for v in done.values()) - arrive[0]
        worker = server.stats()
        server.close()
        served_iters.append({k: (done[k][2]["iterations"], done[k][2]["newton_iterations"]) for k in range(n_run)})
        lat = [done[k][0] - t_sub[k] for k in range(n_run)]
        errs = [float(np.linalg.norm(done[k][3] - urefs[k]) / np.linalg.norm(urefs[k]))
                for k in range(n_run) if urefs[k] is not None and done[k][1] == 0]
        return {"rate_factor": rate_factor if np.isfinite(rate_factor) else "all at t=0", "requests": n_run,
                "arrival_rate_per_s": rate if np.isfinite(rate) else None, "solves_per_s": n_run / makespan,
                "makespan_s": makespan, "converged": sum(done[k][1] == 0 for k in range(n_run)),
                "latency_ms_p50": 1e3 * _pct(lat, 0.5), "latency_ms_p99": 1e3 * _pct(lat, 0.99),
                "pcg_iterations_total": int(sum(done[k][2]["iterations"] for k in range(n_run))),
                "worker": worker,
                "vs_reference_rel_l2": {"requests": len(errs), "max": max(errs) if errs else None,
                                        "median": _pct(errs, 0.5) if errs else None,
                                        "reference": "%s solve of each warm request to %g" % (ref_precision, ref_tol)}}

    runs = [served_run(*(f if isinstance(f, tuple) else (f,))) for f in rate_factors]
    # per sampled request: size, kind, start, PCG / Newton iterations and solve seconds of the
    # graph loop against the PCG / Newton iterations of the first served run
    out["sampled_requests"] = [
        {"request": k, "tets": int(reqs[k]["n_tets"]), "kind": reqs[k]["kind"], "warm": u0s[k] is not None,
         "graph_loop": loop_info[k].get("graph_loop"), "served": served_iters[0].get(k)} for k in sample]
    out["served"] = runs[0]
    if len(runs) > 1:
        out["served_runs"] = runs
    out["served"]["fp32_vs_fp64_rel_l2"] = runs[0]["vs_reference_rel_l2"]
    out["speedup_vs_plain_loop"] = out["served"]["solves_per_s"] / out["plain_loop"]["solves_per_s"]
    out["speedup_vs_plain_loop_excluding_planning"] = (out["served"]["solves_per_s"] /
                                                       out["plain_loop"]["solves_per_s_excluding_planning"])
    out["speedup_vs_graph_loop"] = out["served"]["solves_per_s"] / out["graph_loop"]["solves_per_s"]
    return out


def _attention(P, torch, np, peak, n=1 << 20, S=128, H=8, reps=20):
    """Physics-attention forward (Method, subsection "Transolver"): C = 128 channels, S = 128
    tokens, 8 heads, bf16 activations, on the 131,072 material points of a 64^3 gyroid cell
    (the homogenisation backbone's input) and on 2^20 points (inputs beyond L2: X, M and X^t
    are 256 MB each), random weights.  CUDA events around each forward on the module's stream
    and around each of its kernels (timing on).  Algorithmic HBM bytes per point: X 2C,
    M written and read 2 x 2 S_pad, X^t 2C; tensor flops per point: 2C(C+S) + 2S(C+1) + 2SC."""
    import pfem_inputs.attention as ai

    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            tc_peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        tc_peak = 1900.0
    C, SP = 128, (64 if S <= 64 else 128)
    params = ai.layer_params(C, S, seed=5, slice_gain=4.0)
    attn = P.Attention(params, H, 1.0)
    out = {"channels": C, "tokens": S, "heads": H, "dtype": "bf16 activations, FP32 accumulate",
           "weights": "random (no trained weights)"}

    def run(x, label):
        xt = torch.empty_like(x)
        for _ in range(3):
            attn.forward(x, xt)
        a, b = _events(torch)
        a.record()
        for _ in range(reps):
            attn.forward(x, xt)
        b.record()
        b.synchronize()
        attn.sync()
        ms = a.elapsed_time(b) / reps
        attn.set_timing(True)
        attn.forward(x, xt)
        k = attn.kernel_ms()
        attn.set_timing(False)
        npts = x.shape[0]
        alg = npts * (2 * C + 4 * SP + 2 * C)
        flops = npts * (2 * C * (C + S) + 2 * S * (C + 1) + 2 * S * C)
        tot_k = sum(k.values())
        dom = max(("slice", "deslice"), key=lambda q: k[q])
        dom_bytes = npts * ((2 * C + 2 * SP) if dom == "slice" else (2 * SP + 2 * C))
        dom_flops = npts * ((2 * C * (C + S) + 2 * S * (C + 1)) if dom == "slice" else 2 * S * C)
        return {"workload": label, "points": int(npts), "ms_per_forward": ms, "points_per_s": npts / (ms * 1e-3),
                "kernel_ms": k, "algorithmic_bytes": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9,
                "hbm_frac": alg / (ms * 1e-3) / 1e9 / peak, "tensor_tflops": flops / (ms * 1e-3) / 1e12,
                "tensor_frac": flops / (ms * 1e-3) / 1e12 / tc_peak,
                "dominant_kernel": {"kernel": "attn_%s_kernel<%d>" % (dom, SP), "ms": k[dom],
                                    "share_of_kernels": k[dom] / tot_k, "algorithmic_bytes": dom_bytes,
                                    "achieved_gbs": dom_bytes / (k[dom] * 1e-3) / 1e9,
                                    "hbm_frac": dom_bytes / (k[dom] * 1e-3) / 1e9 / peak,
                                    "tensor_frac": dom_flops / (k[dom] * 1e-3) / 1e12 / tc_peak}}

    pts = ai.tpms_points(64)
    x64 = torch.tensor(ai.point_features(pts, C, seed=3).astype(np.float32), device="cuda").to(torch.bfloat16)
    out["gyroid64"] = run(x64, "64^3 gyroid cell, %d material points" % pts.shape[0])
    xl = torch.randn((n, C), device="cuda").to(torch.bfloat16)
    out["large"] = run(xl, "%d points, N(0,1) features" % n)
    out["peaks"] = {"hbm_gbs": peak, "bf16_tflops": tc_peak, "kind": "measured burst (kernels timed alone)"}
    attn.close()
    return out


def _newton(P, pi, torch, peak=None):
    """Neo-Hookean bar (config 3): zero start with 5 load steps, warm start with 1; the warm
    solve again in FP64 element arithmetic (FP32-vs-FP64 solution difference) and once in the
    plain loop with kernel timing (the inner PCG-fused Neo-Hookean apply against the HBM and
    FP32 peaks: algorithmic bytes 24 B/elem + per node X 12, mask 1, u 24 and five FP64
    vectors 120; flops FLOPS_PER_ELEM[nh, tangent])."""
    p = pi.cfg3_bar()
    mesh = P.Mesh(p)
    out = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u5, i5 = P.pfem_solve_newton(mesh, tol=1e-8, n_load_steps=5, inner_tol=1e-8)
    torch.cuda.synchronize()
    out["zero_5steps"] = {"s": time.perf_counter() - t0, "newton": i5["newton_iterations"], "pcg": i5["iterations"]}
    warm = pi.make_warm_start(p, u5.cpu().numpy(), seed=30)
    wd = torch.tensor(warm, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    uw, iw = P.pfem_solve_newton(mesh, wd, tol=1e-8, n_load_steps=1, inner_tol=1e-8)
    torch.cuda.synchronize()
    out["warm_1step"] = {"s": time.perf_counter() - t0, "newton": iw["newton_iterations"], "pcg": iw["iterations"]}
    u64, i64 = P.pfem_solve_newton(mesh, wd, tol=1e-8, n_load_steps=1, inner_tol=1e-8, precision="f64")
    out["fp32_vs_fp64_rel_l2"] = float(torch.linalg.norm(uw - u64) / torch.linalg.norm(u64))
    out["fp64_newton"] = i64["newton_iterations"]
    st = mesh.stats()
    mode = MODES["plain"]
    P.pfem_set_solver_mode(mode)
    P.pfem_set_kernel_timing(1)
    _, ti = P.pfem_solve_newton(mesh, wd, tol=1e-8, n_load_steps=1, inner_tol=1e-8)
    P.pfem_set_kernel_timing(0)
    P.pfem_set_solver_mode(MODES["graph"])
    nt = max(ti["timed_iterations"], 1)
    us = 1e3 * ti["apply_ms"] / nt
    alg = st["n_elems"] * 24 + st["n_nodes"] * (12 + 1 + 24 + 5 * 24)
    fp32_peak, mhz = _fp32_peak_tflops()
    tflops = FLOPS_PER_ELEM[("nh", "tangent")] * st["n_elems"] / (us * 1e-6) / 1e12
    out["inner_apply"] = {"kernel": "tile_kernel<3,neohookean,tangent+PCG,f64 vectors,f32>", "launch_us": us,
                          "launches_timed": ti["timed_iterations"], "algorithmic_bytes": alg,
                          "hbm_frac": alg / (us * 1e-6) / 1e9 / peak if peak else None,
                          "fp32_tflops": tflops, "fp32_frac": tflops / fp32_peak, "clock_mhz": mhz,
                          "update_kernel_us": 1e3 * ti["update_ms"] / nt,
                          "note": "98k-tet working set is L2-resident; events around each fused apply"}
    out["workload"] = "NH bar 64x16x16 hexes x 6 = 98,304 tets, 20% stretch, tol 1e-8, inner PCG 1e-8"
    mesh.close()
    return out


def probe(a):
    """Kernel-level driver for profilers: one warm-up call, then a.reps timed calls."""
    import torch

    import pfem_inputs as pi
    import paper_2601_03086_gb300 as P
    from paper_2601_03086_gb300 import build

    build.build()
    if a.probe == "attn":  # physics attention on a.n points, 128 channels, 128 tokens, 8 heads
        import pfem_inputs.attention as ai

        attn = P.Attention(ai.layer_params(128, 128, seed=5, slice_gain=4.0), 8, 1.0)
        x = torch.randn((a.n, 128), device="cuda").to(torch.bfloat16)
        xt = torch.empty_like(x)
        attn.forward(x, xt)
        ev = _events(torch)
        ev[0].record()
        for _ in range(a.reps):
            attn.forward(x, xt)
        ev[1].record()
        ev[1].synchronize()
        attn.sync()
        attn.set_timing(True)
        attn.forward(x, xt)
        k = {q: 1e3 * v for q, v in attn.kernel_ms().items()}
        print(json.dumps({"probe": "attn", "n": a.n, "forward_us": ev[0].elapsed_time(ev[1]) * 1e3 / a.reps,
                          "kernel_us": k}))
        attn.close()
        return 0
    p = pi.cube_problem(a.n, seed=2) if a.kind == "linear" else pi.bar_problem(4 * a.n, a.n, a.n, seed=3)
    mesh = P.Mesh(p)
    out = {"probe": a.probe, "n": a.n, "stats": mesh.stats()}
    ev = _events(torch)
    if a.probe == "apply":
        dt = torch.float32 if a.vec == "f32" else torch.float64
        v = torch.randn(mesh.n_dofs, device="cuda", dtype=dt)
        u = 0.01 * torch.randn_like(v) if (a.kind == "nh" or a.op == "residual") else None
        y = torch.empty_like(v)
        arith = "f32" if a.vec == "f64" else None

        if a.k > 0:
            v = torch.randn((a.k, mesh.n_dofs), device="cuda", dtype=dt)
            y = torch.empty_like(v)

        def op():
            if a.k > 0:
                P.pfem_tangent_apply_multi(mesh, v, y)
            elif a.op == "tangent":
                P.pfem_tangent_apply(mesh, u, v, y, arith=arith)
            else:
                P.pfem_residual(mesh, u, y, arith=arith)

        op()
        ev[0].record()
        for _ in range(a.reps):
            op()
        ev[1].record()
        ev[1].synchronize()
        out.update({"apply_us": ev[0].elapsed_time(ev[1]) * 1e3 / a.reps, "op": a.op, "k": a.k})
    else:
        P.pfem_set_solver_mode(MODES[a.solver_mode])
        P.pfem_solve_linear(mesh, tol=TOL, max_iter=a.max_iter, raise_on_error=False)
        ev[0].record()
        for _ in range(a.reps):
            _, info = P.pfem_solve_linear(mesh, tol=TOL, max_iter=a.max_iter, raise_on_error=False)
        ev[1].record()
        ev[1].synchronize()
        ms = ev[0].elapsed_time(ev[1]) / a.reps
        out.update({"solve_ms": ms, "iterations": info["iterations"], "solver_mode": a.solver_mode,
                    "us_per_iteration": 1e3 * ms / max(info["iterations"], 1)})
    print(json.dumps(out))
    mesh.close()
    return 0


def serving_only(a):
    """The serving measurement alone (config 5 at full size takes tens of minutes)."""
    import numpy as np
    import torch

    import pfem_inputs as pi
    import paper_2601_03086_gb300 as P
    from paper_2601_03086_gb300 import build

    build.build()
    f = [int(x) for x in a.serving.split(",")]
    n, hi, every = f[:3]
    n_lat = f[3] if len(f) > 3 else n
    out = _serving(P, pi, torch, np, n_req=n, rate_factors=((float("inf"), n), (2.0, n), (0.5, n_lat)), hi=hi,
                   plain_every=every, ref_tol=1e-10, ref_precision="f32", timeout_s=3600.0)
    out["workload"] = ("serving stream: %d requests, %d..%d tets; served with every request submitted at t=0 "
                       "(capacity) and at 2x the plain-loop rate, and the first %d requests at 0.5x (latency)"
                       % (n, 2000, hi, n_lat))
    print(json.dumps(out))
    return 0


def _cpu_baseline():
    try:
        r = _run_oracle_child(["--oracle-worker", "0", "0"])
    except Exception as e:  # reported, never fatal
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "error": str(e)[-300:]}
    return {"value": 1.0 / r["solve_s"], "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "one full warm-started Jacobi-PCG solve (%d iterations, %.1f s) of the same cube with the "
                      "oracle's assembled K (assembly %.1f s not counted), single-threaded child process"
                      % (r["iterations"], r["solve_s"], r["assembly_s"]),
            "host_cores_available": len(os.sched_getaffinity(0))}


if __name__ == "__main__":
    sys.exit(main())
