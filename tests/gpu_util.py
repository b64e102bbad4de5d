"""Helpers shared by the GPU parity tests (no oracle arithmetic here)."""

import numpy as np
import torch

_BUILT = []


def pfem():
    """Build (once per process) and import the CUDA package."""
    import paper_2601_03086_gb300 as pkg
    from paper_2601_03086_gb300 import build

    if not _BUILT:
        build.build()
        _BUILT.append(True)
    return pkg


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(np.asarray(x).reshape(-1)), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def sub_problem(problem, nodes):
    """Elements incident to `nodes` and the nodes they touch, renumbered.

    Rows of the assembled operator at `nodes` only involve these elements, so a small
    oracle mesh built from them reproduces those rows exactly. Returns (sub_problem,
    old ids of the sub-problem's nodes, positions of `nodes` in the sub numbering).
    """
    conn = np.asarray(problem["conn"])
    n = problem["coords"].shape[0]
    want = np.zeros(n, dtype=bool)
    want[nodes] = True
    sel = np.any(want[conn], axis=1)
    sc = conn[sel]
    used = np.unique(sc)
    new = -np.ones(n, dtype=np.int64)
    new[used] = np.arange(used.size)
    sub = dict(problem)
    sub["coords"] = problem["coords"][used]
    sub["conn"] = new[sc].astype(np.int32)
    sub["mat_a"] = problem["mat_a"][sel]
    sub["mat_b"] = problem["mat_b"][sel]
    sub["dirichlet_mask"] = problem["dirichlet_mask"][used]
    sub["dirichlet_values"] = problem["dirichlet_values"][used]
    sub["facets"] = np.zeros((0, problem["dim"]), np.int32)
    sub["traction"] = np.zeros((0, problem["dim"]))
    sub["f_ext_extra"] = None
    return sub, used, new[nodes]
