"""GPU parity of the element operator (energy, residual, tangent action, Jacobi diagonal)
against the FP64 CPU oracle, through the C ABI.

Tolerances: FP32 element arithmetic -> relative L2 <= 1e-5 (the element-residual target);
FP64 element arithmetic -> relative L2 <= 1e-12 (summation order only). Inputs are random
fields on jittered, permuted meshes so cancellation does not hide errors.
"""

import math

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from oracle import fem
from tests.gpu_util import dev, host, pfem, rel_l2, sub_problem

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def _fields(p, seed):
    # Neo-Hookean: nodal noise of 3% of the mean edge length keeps every J > 0
    x = p["coords"][p["conn"]]
    h = float(np.mean(np.linalg.norm(x[:, 1] - x[:, 0], axis=1)))
    std = 0.1 if p["kind"] == "linear" else 0.03 * h
    u = pi.random_field(p, seed, std=std, zero_masked=False)
    u = np.where(p["dirichlet_mask"].astype(bool), p["dirichlet_values"], u)
    v = np.random.default_rng(seed + 1).standard_normal(p["coords"].shape)
    return u, v


CASES = [
    ("2d-lin", lambda: pi.small_problem(2, "linear", n=24, seed=1)),
    ("2d-nh", lambda: pi.small_problem(2, "neohookean", n=24, seed=2)),
    ("3d-lin", lambda: pi.small_problem(3, "linear", n=7, seed=3)),
    ("3d-nh", lambda: pi.small_problem(3, "neohookean", n=7, seed=4)),
    ("3d-lin-tiles", lambda: pi.small_problem(3, "linear", shape=(18, 9, 7), seed=5)),
    ("3d-nh-tiles", lambda: pi.small_problem(3, "neohookean", shape=(17, 8, 9), seed=6)),
    ("3d-nh-prescribed", lambda: pi.small_problem(3, "neohookean", n=6, seed=7, prescribed=0.05)),
    ("plate-cfg1", lambda: pi.cfg1_plate()),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    p = request.param[1]()
    m = fem.Mesh(p)
    u, v = _fields(p, 11)
    K = fem.stiffness(m, u)
    ref = dict(
        y=fem.masked_operator(m, K) @ v.reshape(-1),
        r=fem.residual(m, u),
        d=fem.masked_operator(m, K).diagonal(),
        es=fem.strain_energy(m, u),
        e=fem.total_energy(m, u),
    )
    mesh = pfem().Mesh(p)
    return p, mesh, u, v, ref


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_tangent_apply(case, dtype):
    p, mesh, u, v, ref = case
    P = pfem()
    y = P.pfem_tangent_apply(mesh, dev(u, dtype), dev(v, dtype))
    assert rel_l2(host(y), ref["y"]) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_residual(case, dtype):
    p, mesh, u, v, ref = case
    r = pfem().pfem_residual(mesh, dev(u, dtype))
    assert rel_l2(host(r), ref["r"]) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_jacobi_diag(case, dtype):
    p, mesh, u, v, ref = case
    d = pfem().pfem_jacobi_diag(mesh, dev(u, dtype) if p["kind"] != "linear" else None, dtype=dtype)
    assert rel_l2(host(d), ref["d"]) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_energy(case, dtype):
    p, mesh, u, v, ref = case
    e, es = pfem().pfem_energy(mesh, dev(u, dtype))
    assert abs(es - ref["es"]) <= TOL[dtype] * abs(ref["es"])
    scale = abs(ref["es"]) + abs(ref["es"] - ref["e"])
    assert abs(e - ref["e"]) <= TOL[dtype] * scale


def test_bitwise_deterministic(case):
    p, mesh, u, v, ref = case
    P = pfem()
    for dtype in (torch.float32, torch.float64):
        uu, vv = dev(u, dtype), dev(v, dtype)
        a = P.pfem_tangent_apply(mesh, uu, vv).clone()
        b = P.pfem_tangent_apply(mesh, uu, vv).clone()
        r1 = P.pfem_residual(mesh, uu).clone()
        r2 = P.pfem_residual(mesh, uu).clone()
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(r1, r2)
        assert P.pfem_energy(mesh, uu) == P.pfem_energy(mesh, uu)


def test_load_scale_scales_external_force():
    P = pfem()
    p = pi.small_problem(3, "linear", n=4, seed=9)
    m = fem.Mesh(p)
    mesh = P.Mesh(p)
    u = np.zeros(p["coords"].shape)
    P.pfem_mesh_set_load_scale(mesh, 0.25)
    r = host(P.pfem_residual(mesh, dev(u)))
    assert rel_l2(r, fem.residual(m, u, scale=0.25)) <= 1e-12


def test_empty_mesh_and_orphan_nodes():
    """No elements: K = 0, so A = I - P (+ nothing) and r = -P f; orphan nodes behave alike."""
    P = pfem()
    p = pi.small_problem(3, "linear", n=2, seed=1, permute=False)
    q = dict(p)
    q["conn"] = np.zeros((0, 4), np.int32)
    q["mat_a"] = np.zeros(0)
    q["mat_b"] = np.zeros(0)
    f = np.random.default_rng(0).standard_normal(p["coords"].shape)
    q["f_ext_extra"] = f
    q["facets"] = np.zeros((0, 3), np.int32)
    q["traction"] = np.zeros((0, 3))
    mesh = P.Mesh(q)
    v = np.random.default_rng(1).standard_normal(p["coords"].shape)
    mask = q["dirichlet_mask"].astype(bool)
    y = host(P.pfem_tangent_apply(mesh, None, dev(v)))
    assert np.array_equal(y.reshape(v.shape), np.where(mask, v, 0.0))
    r = host(P.pfem_residual(mesh, dev(np.zeros_like(v))))
    assert np.array_equal(r.reshape(v.shape), np.where(mask, 0.0, -f))
    e, es = P.pfem_energy(mesh, dev(v))
    assert es == 0.0 and math.isclose(e, -float(f.reshape(-1) @ v.reshape(-1)), rel_tol=1e-12)
    # orphans next to a real mesh
    o = dict(p)
    o["coords"] = np.vstack([p["coords"], [[7.0, 7.0, 7.0]]])
    o["dirichlet_mask"] = np.vstack([p["dirichlet_mask"], [[0, 1, 0]]]).astype(np.uint8)
    o["dirichlet_values"] = np.vstack([p["dirichlet_values"], [[0.0, 0.0, 0.0]]])
    mo = fem.Mesh(o)
    mesh_o = P.Mesh(o)
    vo = np.random.default_rng(2).standard_normal(o["coords"].shape)
    yo = host(P.pfem_tangent_apply(mesh_o, None, dev(vo)))
    assert rel_l2(yo, fem.tangent_apply(mo, None, vo)) <= 1e-12


def test_inverted_element_reports_status():
    P = pfem()
    from paper_2601_03086_gb300._lib import PfemError

    p = pi.small_problem(3, "neohookean", n=3, seed=2, permute=False)
    mesh = P.Mesh(p)
    u = np.zeros(p["coords"].shape)
    u[:, 0] = -1.7 * p["coords"][:, 0]  # F11 = -0.7 everywhere: J < 0
    with pytest.raises(PfemError) as ei:
        P.pfem_energy(mesh, dev(u))
    assert ei.value.status == 3


def test_cfg2_full_size_parity():
    """Full 384,000-tet cube (the benchmarked operator) against the assembled oracle."""
    P = pfem()
    p = pi.cfg2_cube()
    m = fem.Mesh(p)
    K = fem.assemble_linear_K(m)
    v = np.random.default_rng(3).standard_normal(m.n_dofs)
    ref = fem.masked_operator(m, K) @ v
    mesh = P.Mesh(p)
    for dtype in (torch.float32, torch.float64):
        y = host(P.pfem_tangent_apply(mesh, None, dev(v, dtype)))
        assert rel_l2(y, ref) <= TOL[dtype]
    u = pi.random_field(p, 4, std=0.1)
    r = host(P.pfem_residual(mesh, dev(u, torch.float32)))
    assert rel_l2(r, fem.residual(m, u)) <= TOL[torch.float32]


def test_roofline_cube_sampled_rows():
    """24.6 M-tet cube (160^3 x 6): sampled output rows against the oracle on the elements
    incident to the sampled nodes (which determine those rows exactly)."""
    P = pfem()
    p = pi.roofline_cube()
    mesh = P.Mesh(p)
    rng = np.random.default_rng(8)
    v = rng.standard_normal(p["coords"].shape).astype(np.float32)
    y = host(P.pfem_tangent_apply(mesh, None, dev(v, torch.float32))).reshape(-1, 3)
    nodes = rng.choice(p["coords"].shape[0], size=3000, replace=False)
    sub, used, pos = sub_problem(p, nodes)
    ms = fem.Mesh(sub)
    ys = fem.tangent_apply(ms, None, v.astype(np.float64)[used]).reshape(-1, 3)
    assert rel_l2(y[nodes], ys[pos]) <= 1e-5
