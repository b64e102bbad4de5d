"""pfem_tangent_apply_noalloc: the tangent action for callers that cannot allocate.

Callers running with a frozen or exhausted device memory pool, inside allocator callbacks,
or in runtimes that only own memory handed to them up front cannot let a call allocate. The
no-alloc entry point keeps its per-call scratch (the halo partial sums) in a fixed 16 MiB
device array instead; the array is created when a mesh is created on the device.

These tests call it through the C ABI (ctypes), two calls in a row with different inputs
(so stale contents of the shared array would show), and require the result to be bit for
bit that of pfem_tangent_apply (the same kernels on the same plan) and to match the FP64
oracle. Two meshes cover both halo completion modes: a small one whose halo nodes are
finished inside the tiles (integer tickets) and a 1 M-tet cube with 2^18 <= n_partials <=
2^20, whose halo nodes are finished by the separate halo pass reading the fixed array. The
FP32, FP64-vector/FP32-arithmetic and FP64 operators are covered. Oversized meshes are
refused. This file is collected last on purpose.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from oracle import fem
from tests.gpu_util import dev, host, pfem, rel_l2, sub_problem

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64f32": 1e-5, "f64": 1e-12}
SCRATCH_BYTES = 16 << 20
DEFER_PARTIALS = 1 << 18  # from this many halo partials on, the halo pass runs as its own launch


def _codes():
    from paper_2601_03086_gb300._lib import PFEM_F32, PFEM_F64, PFEM_F64_F32

    return {"f32": (PFEM_F32, torch.float32, 4), "f64f32": (PFEM_F64_F32, torch.float64, 4),
            "f64": (PFEM_F64, torch.float64, 8)}


def _noalloc(mesh, code, u, v, y):
    from paper_2601_03086_gb300._lib import lib

    up = C.c_void_p(u.data_ptr()) if u is not None else None
    return lib().pfem_tangent_apply_noalloc(mesh.handle, code, up, C.c_void_p(v.data_ptr()),
                                            C.c_void_p(y.data_ptr()))


def _regular(mesh, code, u, v):
    from paper_2601_03086_gb300._lib import check, lib

    y = torch.empty_like(v)
    up = C.c_void_p(u.data_ptr()) if u is not None else None
    check(lib().pfem_tangent_apply(mesh.handle, code, up, C.c_void_p(v.data_ptr()), C.c_void_p(y.data_ptr())))
    return y


def _check_twice(P, p, mesh, prec, kind, rows=None):
    code, dt, csize = _codes()[prec]
    st = mesh.stats()
    assert st["n_partials"] * 4 * csize <= SCRATCH_BYTES
    x = p["coords"][p["conn"]]
    h = float(np.mean(np.linalg.norm(x[:, 1] - x[:, 0], axis=1)))
    u_h = np.random.default_rng(1).normal(0.0, 0.03 * h, p["coords"].size) if kind == "neohookean" else None
    u = dev(u_h, dt) if u_h is not None else None
    for call in range(2):
        v_h = np.random.default_rng(10 + call).standard_normal(p["coords"].size)
        v = dev(v_h, dt)
        y_ref = _regular(mesh, code, u, v)
        y = torch.full_like(v, float("nan"))
        assert _noalloc(mesh, code, u, v, y) == 0
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref), (prec, call)
        # the oracle (exact rows of the sampled nodes, or every row)
        uo = None if u_h is None else u_h.astype(np.float64)
        vo = v_h.astype(np.float32).astype(np.float64) if dt == torch.float32 else v_h
        if uo is not None and dt == torch.float32:
            uo = uo.astype(np.float32).astype(np.float64)
        yh = host(y).reshape(-1, 3)
        if rows is None:
            yo = fem.tangent_apply(fem.Mesh(p), uo, vo).reshape(-1, 3)
            assert rel_l2(yh, yo) <= TOL[prec], prec
        else:
            sub, used, pos = sub_problem(p, rows)
            us = None if uo is None else uo.reshape(-1, 3)[used]
            ys = fem.tangent_apply(fem.Mesh(sub), us, vo.reshape(-1, 3)[used]).reshape(-1, 3)
            assert rel_l2(yh[rows], ys[pos]) <= TOL[prec], prec


@pytest.mark.parametrize("kind", ["linear", "neohookean"])
@pytest.mark.parametrize("prec", ["f32", "f64f32", "f64"])
def test_noalloc_in_tile_halo_path(kind, prec):
    P = pfem()
    p = pi.small_problem(3, kind, shape=(16, 8, 8), seed=41)  # several tiles, halo partials
    mesh = P.Mesh(p)
    assert 0 < mesh.stats()["n_partials"] < DEFER_PARTIALS
    _check_twice(P, p, mesh, prec, kind)
    mesh.close()


@pytest.fixture(scope="module")
def mid_cube():
    P = pfem()
    p = pi.cube_problem(56, seed=2)  # 1,053,696 tets, 347,746 halo partials
    mesh = P.Mesh(p)
    yield p, mesh
    mesh.close()


@pytest.mark.parametrize("prec", ["f32", "f64f32", "f64"])
def test_noalloc_deferred_halo_path(mid_cube, prec):
    P = pfem()
    p, mesh = mid_cube
    n_part = mesh.stats()["n_partials"]
    assert DEFER_PARTIALS <= n_part <= 1 << 20
    rows = np.random.default_rng(5).choice(p["coords"].shape[0], size=2000, replace=False)
    _check_twice(P, p, mesh, prec, "linear", rows=rows)


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    P = pfem()
    code, _, csize = _codes()["f64"]
    p = pi.cube_problem(100, seed=2)  # 6 M tets: more halo partials than 16 MiB of FP64
    mesh = P.Mesh(p)
    need = mesh.stats()["n_partials"] * 4 * csize
    assert need > SCRATCH_BYTES
    v = torch.zeros(mesh.n_dofs, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(v)
    assert _noalloc(mesh, code, None, v, y) == 1  # PFEM_ERR_INVALID_ARG
    mesh.close()
