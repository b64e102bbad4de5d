"""Failure detection on the GPU without a GPU fault: bounded waits that run out, non-finite
inputs and error returns come back as statuses, and the mesh and the context stay usable.

  * the persistent PCG kernel's grid-barrier waits are bounded: with a short limit and one
    CTA made to leave without arriving (host-side injection), the other CTAs' waits run out,
    the solve returns PFEM_ERR_TIMEOUT within milliseconds, and the next solve on the same
    mesh is bitwise the one a fresh mesh gives;
  * a NaN in the warm start makes the linear and the Newton solve return PFEM_ERR_NONFINITE;
  * a Newton solve that fails leaves the mesh's load scale as the caller set it.
"""

import time

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from tests.gpu_util import dev, host, pfem

pytestmark = pytest.mark.gpu

PFEM_ERR_NONFINITE = 4
PFEM_ERR_TIMEOUT = 9


def test_persistent_barrier_wait_runs_out_with_timeout_status():
    P = pfem()
    p = pi.cube_problem(8, seed=3)
    mesh = P.Mesh(p)
    try:
        P.pfem_set_solver_mode(0)
        P.pfem_set_barrier_test(spin_limit=1 << 14, absent_cta=0)  # >= 0.5 ms of polling
        t0 = time.perf_counter()
        _, info = P.pfem_solve_linear(mesh, tol=1e-8, raise_on_error=False)
        elapsed = time.perf_counter() - t0
        assert info["status"] == PFEM_ERR_TIMEOUT, info
        assert elapsed < 10.0
    finally:
        P.pfem_set_barrier_test()  # defaults: long limit, no absent CTA
    try:
        u1, i1 = P.pfem_solve_linear(mesh, tol=1e-8)
        fresh = P.Mesh(p)
        u2, i2 = P.pfem_solve_linear(fresh, tol=1e-8)
        fresh.close()
    finally:
        P.pfem_set_solver_mode(2)
    assert i1["status"] == 0 and i1["iterations"] == i2["iterations"]
    assert np.array_equal(host(u1), host(u2))
    mesh.close()


def test_barrier_test_hook_rejects_bad_cta():
    P = pfem()
    with pytest.raises(RuntimeError):
        P.pfem_set_barrier_test(absent_cta=-2)


def _nan_start(p):
    u0 = np.zeros(p["coords"].size)
    free = np.flatnonzero(np.asarray(p["dirichlet_mask"]).reshape(-1) == 0)
    u0[free[len(free) // 2]] = np.nan
    return u0


def test_nan_warm_start_linear_is_nonfinite():
    P = pfem()
    p = pi.cube_problem(6, seed=4)
    mesh = P.Mesh(p)
    for mode in (2, 1, 0):
        P.pfem_set_solver_mode(mode)
        _, info = P.pfem_solve_linear(mesh, dev(_nan_start(p)), tol=1e-8, raise_on_error=False)
        assert info["status"] == PFEM_ERR_NONFINITE, (mode, info)
        assert info["iterations"] == 0
    P.pfem_set_solver_mode(2)
    _, info = P.pfem_solve_linear(mesh, tol=1e-8)  # the mesh is still usable
    assert info["status"] == 0
    mesh.close()


def test_nan_warm_start_newton_is_nonfinite_and_keeps_load_scale():
    P = pfem()
    p = pi.cube_problem(6, seed=5)  # traction load: the residual depends on the load scale
    mesh = P.Mesh(p)
    u = dev(0.01 * np.random.default_rng(2).standard_normal(p["coords"].size))
    P.pfem_mesh_set_load_scale(mesh, 0.7)
    r_before = host(P.pfem_residual(mesh, u))
    _, info = P.pfem_solve_newton(mesh, dev(_nan_start(p)), tol=1e-8, n_load_steps=1, max_newton=1,
                                  raise_on_error=False)
    assert info["status"] == PFEM_ERR_NONFINITE, info
    r_after = host(P.pfem_residual(mesh, u))
    assert np.array_equal(r_before, r_after)  # the scale 0.7 is back after the error return
    P.pfem_mesh_set_load_scale(mesh, 1.0)
    assert not np.array_equal(host(P.pfem_residual(mesh, u)), r_before)
    mesh.close()
