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
