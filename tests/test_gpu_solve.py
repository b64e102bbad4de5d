"""GPU parity of the warm-started solvers against the FP64 CPU oracle (through the C ABI).

Bars: solution relative L2 <= 1e-6 at residual tolerance 1e-8 (1e-10 for the FP64 plate),
the FP64 true residual of the returned solution below tol, and PCG iteration counts within
+-2 of the oracle's Jacobi-PCG when the element operator runs in FP64; Newton counts within
+-2. With the FP32 element operator the Krylov recurrence sees rounding of order 1e-7 in
every product; on these ill-conditioned cubes (lognormal E) that moves the count at 1e-8 by
a fraction of a percent: tests/test_oracle_solve.py::
test_fp32_rounded_directions_move_pcg_iteration_count shows that rounding only the search
direction to FP32, with everything else exact FP64, already moves it by 3-4 iterations on
the 16^3 and 24^3 cubes. So the FP32 bar is +-max(2, 1.5%) while accuracy is held to the
same FP64 bar.
"""

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from oracle import fem, solve
from tests.gpu_util import dev, host, pfem, rel_l2

pytestmark = pytest.mark.gpu


def _iters_ok(it, it_ref, precision):
    if precision == "f64":
        return abs(it - it_ref) <= 2
    return abs(it - it_ref) <= max(2, int(0.015 * it_ref))


def _linear_case(p, tol, precision, u0=None, K=None, max_iter=100000):
    m = fem.Mesh(p)
    K = fem.assemble_linear_K(m) if K is None else K
    u_ref, it_ref, _ = solve.solve_linear(m, u0=u0, tol=tol, K=K)
    P = pfem()
    mesh = P.Mesh(p)
    u, info = P.pfem_solve_linear(mesh, None if u0 is None else dev(u0), tol=tol, max_iter=max_iter,
                                  precision=precision)
    return m, host(u), info, u_ref, it_ref


def test_plate_fp64_zero_start():
    p = pi.cfg1_plate()
    m, u, info, u_ref, it_ref = _linear_case(p, 1e-10, "f64")
    assert abs(info["iterations"] - it_ref) <= 2, (info, it_ref)
    assert rel_l2(u, u_ref) <= 1e-8
    assert info["rel_residual_true_f64"] < 1e-10
    u_direct = solve.solve_linear_direct(m)
    assert rel_l2(u, u_direct) <= 1e-6


@pytest.mark.parametrize("warm", [False, True], ids=["zero", "warm"])
def test_small_cube_fp32(warm):
    p = pi.cube_problem(12, seed=2)
    m = fem.Mesh(p)
    K = fem.assemble_linear_K(m)
    u0 = None
    if warm:
        u_star, _, _ = solve.solve_linear(m, tol=1e-13, K=K)
        u0 = pi.make_warm_start(p, u_star, seed=20)
    m, u, info, u_ref, it_ref = _linear_case(p, 1e-8, "f32", u0=u0, K=K)
    assert _iters_ok(info["iterations"], it_ref, "f32"), (info, it_ref)
    assert rel_l2(u, u_ref) <= 1e-6
    assert info["rel_residual_true_f64"] < 1e-8


def test_solver_modes_bitwise_equal_and_deterministic():
    P = pfem()
    p = pi.cube_problem(8, seed=3)
    mesh = P.Mesh(p)
    outs = []
    for mode in (0, 0, 1, 2):  # persistent twice, plain, graph
        P.pfem_set_solver_mode(mode)
        u, info = P.pfem_solve_linear(mesh, tol=1e-8)
        outs.append((host(u), info["iterations"]))
    P.pfem_set_solver_mode(2)
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0])
        assert outs[0][1] == o[1]


def test_solver_modes_bitwise_equal_newton_and_2d():
    P = pfem()
    cases = [(pi.bar_problem(8, 2, 2, seed=5), "newton"), (pi.cfg1_plate(), "linear")]
    for p, kind in cases:
        mesh = P.Mesh(p)
        outs = []
        for mode in (0, 1, 2):
            P.pfem_set_solver_mode(mode)
            if kind == "newton":
                u, info = P.pfem_solve_newton(mesh, tol=1e-8, n_load_steps=2)
            else:
                u, info = P.pfem_solve_linear(mesh, tol=1e-8)
            outs.append((host(u), info["iterations"]))
        P.pfem_set_solver_mode(2)
        for o in outs[1:]:
            assert np.array_equal(outs[0][0], o[0]), kind
            assert outs[0][1] == o[1], kind


def test_kernel_timing_plain_loop():
    """Kernel timing times every plain-loop iteration's two kernels, changes no bit of the
    solve, and leaves graph solves untimed."""
    P = pfem()
    p = pi.cube_problem(8, seed=3)
    mesh = P.Mesh(p)
    try:
        P.pfem_set_solver_mode(1)
        u0, i0 = P.pfem_solve_linear(mesh, tol=1e-8)
        assert i0["timed_iterations"] == 0 and i0["apply_ms"] == 0.0
        P.pfem_set_kernel_timing(1)
        u1, i1 = P.pfem_solve_linear(mesh, tol=1e-8)
        assert np.array_equal(host(u0), host(u1)) and i1["iterations"] == i0["iterations"]
        assert i1["timed_iterations"] == i1["iterations"]
        assert i1["apply_ms"] > 0.0 and i1["update_ms"] > 0.0
        P.pfem_set_solver_mode(2)
        _, i2 = P.pfem_solve_linear(mesh, tol=1e-8)
        assert i2["timed_iterations"] == 0
    finally:
        P.pfem_set_kernel_timing(0)
        P.pfem_set_solver_mode(2)
    with pytest.raises(RuntimeError):
        P.pfem_set_kernel_timing(2)


def test_solver_mode_rejects_unknown():
    P = pfem()
    with pytest.raises(RuntimeError):
        P.pfem_set_solver_mode(3)


def test_skip_test_returns_without_iterating():
    P = pfem()
    p = pi.cube_problem(6, seed=4)
    m = fem.Mesh(p)
    u_star, _, _ = solve.solve_linear(m, tol=1e-14)
    mesh = P.Mesh(p)
    u, info = P.pfem_solve_linear(mesh, dev(u_star), tol=1e-8, precision="f64")
    assert info["iterations"] == 0
    assert rel_l2(host(u), u_star) <= 1e-14


def test_not_converged_status():
    P = pfem()
    p = pi.cube_problem(6, seed=5)
    mesh = P.Mesh(p)
    u, info = P.pfem_solve_linear(mesh, tol=1e-12, max_iter=5, raise_on_error=False)
    assert info["status"] == 5 and info["iterations"] == 5


@pytest.fixture(scope="module")
def cfg2_oracle():
    p = pi.cfg2_cube()
    m = fem.Mesh(p)
    K = fem.assemble_linear_K(m)
    u_star, _, _ = solve.solve_linear(m, tol=1e-12, K=K)
    warm = pi.make_warm_start(p, u_star, seed=20)
    return p, m, K, u_star, warm


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("warm", [False, True], ids=["zero", "warm"])
def test_cfg2_full_size(cfg2_oracle, warm, precision):
    p, m, K, u_star, warm_u = cfg2_oracle
    u0 = warm_u if warm else None
    _, u, info, u_ref, it_ref = _linear_case(p, 1e-8, precision, u0=u0, K=K)
    assert _iters_ok(info["iterations"], it_ref, precision), (info, it_ref)
    assert rel_l2(u, u_ref) <= 1e-6
    assert info["rel_residual_true_f64"] < 1e-8


# --------------------------------------------------------------------------- Newton


@pytest.fixture(scope="module")
def bar_oracle():
    p = pi.bar_problem(24, 6, 6, seed=3)
    m = fem.Mesh(p)
    u5, n5, _ = solve.solve_newton(m, tol=1e-8, n_load_steps=5)
    u_star, _, _ = solve.solve_newton(m, u0=u5, tol=1e-12, n_load_steps=1, inner_tol=1e-12)
    warm = pi.make_warm_start(p, u_star, seed=30)
    uw, nw, _ = solve.solve_newton(m, u0=warm, tol=1e-8, n_load_steps=1)
    return p, m, u5, n5, u_star, warm, uw, nw


def test_newton_zero_start_load_steps(bar_oracle):
    p, m, u5, n5, u_star, warm, uw, nw = bar_oracle
    P = pfem()
    mesh = P.Mesh(p)
    u, info = P.pfem_solve_newton(mesh, tol=1e-8, n_load_steps=5, inner_tol=1e-8)
    assert abs(info["newton_iterations"] - n5) <= 2, (info, n5)
    assert rel_l2(host(u), u_star) <= 1e-6
    assert info["rel_residual_true_f64"] <= 1e-8


def test_newton_warm_start(bar_oracle):
    p, m, u5, n5, u_star, warm, uw, nw = bar_oracle
    P = pfem()
    mesh = P.Mesh(p)
    u, info = P.pfem_solve_newton(mesh, dev(warm), tol=1e-8, n_load_steps=1, inner_tol=1e-8)
    assert abs(info["newton_iterations"] - nw) <= 1, (info, nw)
    assert info["newton_iterations"] < n5
    assert rel_l2(host(u), u_star) <= 1e-6
    r = fem.residual(m, host(u))
    assert np.linalg.norm(r) <= 1e-8 * solve.newton_reference(m, 1.0) * 1.0001


@pytest.fixture(scope="module")
def cfg3_oracle():
    """Full 98,304-tet bar: the oracle's converged solution (5 load steps, inner Jacobi-PCG to
    1e-8 as in the solver under test; a sparse direct factorisation of this 56k-DOF tangent
    takes tens of seconds per Newton step), a warm start built from it, and the oracle's warm
    Newton count (1 load step)."""
    p = pi.cfg3_bar()
    m = fem.Mesh(p)
    u5, n5, _ = solve.solve_newton(m, tol=1e-8, n_load_steps=5)
    u_star, _, _ = solve.solve_newton(m, u0=u5, tol=1e-12, n_load_steps=1, inner_tol=1e-12)
    warm = pi.make_warm_start(p, u_star, seed=30)
    uw, nw, _ = solve.solve_newton(m, u0=warm, tol=1e-8, n_load_steps=1)
    return p, m, n5, u_star, warm, uw, nw


def test_cfg3_full_size_newton_vs_oracle(cfg3_oracle):
    """Full 98,304-tet bar: zero start with 5 load steps and warm start with 1, Newton counts
    within +-2 of the oracle's, solutions within 1e-6 of the oracle's, residual test met and
    no element inverted."""
    p, m, n5, u_star, warm, uw, nw = cfg3_oracle
    P = pfem()
    mesh = P.Mesh(p)
    u5, info5 = P.pfem_solve_newton(mesh, tol=1e-8, n_load_steps=5)
    assert abs(info5["newton_iterations"] - n5) <= 2, (info5, n5)
    assert rel_l2(host(u5), u_star) <= 1e-6
    u, info = P.pfem_solve_newton(mesh, dev(warm), tol=1e-8, n_load_steps=1)
    uh = host(u)
    assert abs(info["newton_iterations"] - nw) <= 2, (info, nw)
    assert rel_l2(uh, uw) <= 1e-6
    ref = solve.newton_reference(m, 1.0)
    assert np.linalg.norm(fem.residual(m, uh)) <= 1.01e-8 * ref
    assert fem.min_jacobian(m, uh) > 0
    assert info["newton_iterations"] < info5["newton_iterations"]


def test_cfg2_fp32_warm_iterations_ten_seeds(cfg2_oracle):
    """Iteration-count parity of the FP32 operator over 10 warm starts of the full 40^3 cube
    (seeds 20..29): every count within +-max(2, 1.5%) of the oracle's; the per-seed deltas are
    printed (run with -s to see them)."""
    p, m, K, u_star, _ = cfg2_oracle
    P = pfem()
    mesh = P.Mesh(p)
    deltas = []
    for seed in range(20, 30):
        warm = pi.make_warm_start(p, u_star, seed=seed)
        _, it_ref, _ = solve.solve_linear(m, u0=warm, tol=1e-8, K=K)
        u, info = P.pfem_solve_linear(mesh, dev(warm), tol=1e-8)
        deltas.append((seed, it_ref, info["iterations"]))
        assert info["rel_residual_true_f64"] < 1e-8
    print("cfg2 FP32 warm iterations (seed, oracle, gpu):", deltas,
          "max |delta| =", max(abs(g - o) for _, o, g in deltas))
    for seed, it_ref, it in deltas:
        assert _iters_ok(it, it_ref, "f32"), (seed, it, it_ref)
    mesh.close()
