"""Multi-right-hand-side tangent action (pfem_tangent_apply_multi) against the FP64 oracle and
against k single applies, through the C ABI.

Bars: every y_j within rel L2 1e-5 of the oracle's K v_j (FP32 element arithmetic) and within
1e-6 of the single-vector kernel; odd k (a pair with one vector), k beyond one launch's six
vectors, 2-D and 3-D, jittered and permuted meshes with prescribed DOFs; bitwise repeatable;
Neo-Hookean meshes refused.
"""

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from oracle import fem
from tests.gpu_util import dev, host, pfem, rel_l2, sub_problem

pytestmark = pytest.mark.gpu


def _vs(p, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, p["coords"].size))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 2, 5, 7, 12])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64f32"])
def test_multi_apply_matches_oracle_and_single(dim, k, dtype):
    P = pfem()
    p = pi.small_problem(dim, "linear", n=6 if dim == 3 else 24, seed=30 + k)
    mesh = P.Mesh(p)
    m = fem.Mesh(p)
    v = _vs(p, k, 7 + k)
    if dtype == torch.float32:
        v = v.astype(np.float32).astype(np.float64)
    vt = torch.tensor(v, dtype=dtype, device="cuda")
    y = host(P.pfem_tangent_apply_multi(mesh, vt)).reshape(k, -1)
    arith = "f32" if dtype == torch.float64 else None
    for j in range(k):
        yo = fem.tangent_apply(m, None, v[j])
        assert rel_l2(y[j], yo) <= 1e-5, j
        ys = host(P.pfem_tangent_apply(mesh, None, vt[j].contiguous(), arith=arith))
        assert rel_l2(y[j], ys) <= 1e-6, j
    mesh.close()


def test_multi_apply_deterministic_and_refusals():
    P = pfem()
    from paper_2601_03086_gb300._lib import PfemError

    p = pi.cube_problem(10, seed=3)
    mesh = P.Mesh(p)
    vt = torch.tensor(_vs(p, 6, 1), dtype=torch.float32, device="cuda")
    a = P.pfem_tangent_apply_multi(mesh, vt).clone()
    b = P.pfem_tangent_apply_multi(mesh, vt).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    mesh.close()
    nh = P.Mesh(pi.small_problem(3, "neohookean", n=3, seed=1))
    with pytest.raises(PfemError):
        P.pfem_tangent_apply_multi(nh, torch.zeros((2, nh.n_dofs), dtype=torch.float32, device="cuda"))
    nh.close()


def test_multi_apply_large_cube_sampled_rows():
    """1 M-tet cube (halo nodes finished by the separate pass), six vectors: sampled rows of
    every y_j against the oracle on the elements incident to the sampled nodes."""
    P = pfem()
    p = pi.cube_problem(56, seed=2)
    mesh = P.Mesh(p)
    k = 6
    v = _vs(p, k, 3).astype(np.float32)
    y = host(P.pfem_tangent_apply_multi(mesh, torch.tensor(v, device="cuda"))).reshape(k, -1, 3)
    nodes = np.random.default_rng(4).choice(p["coords"].shape[0], size=1500, replace=False)
    sub, used, pos = sub_problem(p, nodes)
    ms = fem.Mesh(sub)
    for j in range(k):
        ys = fem.tangent_apply(ms, None, v[j].astype(np.float64).reshape(-1, 3)[used].reshape(-1)).reshape(-1, 3)
        assert rel_l2(y[j][nodes], ys[pos]) <= 1e-5, j
    mesh.close()


def test_multi_solve_matches_oracle_per_load_case():
    """Four load cases on the 12^3 lognormal cube solved together (FP32 and FP64 element
    arithmetic): each solution within 1e-6 of the oracle's, iterations within the FP32 bar of
    the oracle's Jacobi-PCG, every true residual below tol."""
    from oracle import solve

    P = pfem()
    p = pi.cube_problem(12, seed=9)
    m = fem.Mesh(p)
    K = fem.assemble_linear_K(m)
    free = ~m.mask
    rng = np.random.default_rng(21)
    k = 4
    B = rng.standard_normal((k, m.n_dofs)) * free
    mesh = P.Mesh(p)
    for precision in ("f32", "f64"):
        U, infos = P.pfem_solve_linear_multi(mesh, torch.tensor(B, device="cuda"), tol=1e-8, precision=precision)
        U = host(U).reshape(k, -1)
        Kff = K[free][:, free].tocsr()
        for j in range(k):
            ref = np.linalg.norm(B[j][free])
            x, it = solve.pcg(Kff, B[j][free], np.zeros(int(free.sum())), Kff.diagonal(), 1e-8, ref, 100000)
            u_ref = np.zeros(m.n_dofs)
            u_ref[free] = x
            assert rel_l2(U[j], u_ref) <= 1e-6, (precision, j)
            bar = 2 if precision == "f64" else max(2, int(0.015 * it))
            assert abs(infos[j]["iterations"] - it) <= bar, (precision, j, infos[j], it)
            assert infos[j]["rel_residual_true_f64"] < 1e-8
    mesh.close()


def test_springs_in_operator_and_diagonal():
    """Penalty springs between random node pairs: tangent, multi tangent and Jacobi diagonal
    equal the oracle's K + S (prescribed rows keep the identity)."""
    from oracle import homog

    P = pfem()
    p = pi.cube_problem(6, seed=4)
    m = fem.Mesh(p)
    rng = np.random.default_rng(3)
    pairs = rng.choice(p["coords"].shape[0], size=(40, 2), replace=False).astype(np.int32)
    kappa = 7.5
    A = (fem.assemble_linear_K(m) + homog.spring_matrix(m.n_dofs, pairs, kappa)).tocsr()
    free = (~m.mask).astype(np.float64)
    mesh = P.Mesh(p)
    P.pfem_mesh_set_springs(mesh, pairs, kappa)
    v = rng.standard_normal((2, m.n_dofs))
    for j in range(2):
        y_ref = free * (A @ (free * v[j])) + (1 - free) * v[j]
        y = host(P.pfem_tangent_apply(mesh, None, dev(v[j])))
        assert rel_l2(y, y_ref) <= 1e-12
    ym = host(P.pfem_tangent_apply_multi(mesh, torch.tensor(v, dtype=torch.float32, device="cuda"))).reshape(2, -1)
    for j in range(2):
        y_ref = free * (A @ (free * v[j].astype(np.float32))) + (1 - free) * v[j].astype(np.float32)
        assert rel_l2(ym[j], y_ref) <= 1e-5
    d = host(P.pfem_jacobi_diag(mesh, dtype=torch.float64))
    assert rel_l2(d, free * A.diagonal() + (1 - free)) <= 1e-12
    P.pfem_mesh_set_springs(mesh, np.zeros((0, 2), np.int32), 0.0)  # removed again
    y0 = host(P.pfem_tangent_apply(mesh, None, dev(v[0])))
    K = fem.assemble_linear_K(m)
    assert rel_l2(y0, free * (K @ (free * v[0])) + (1 - free) * v[0]) <= 1e-12
    mesh.close()
