"""Pins of the FP64 oracle's element operator against closed forms, invariants and FD.

None of these compare the oracle with itself: each check comes from the mathematics
(patch test, rigid motions, symmetry, energy identities, finite differences, the small-
strain limit of Neo-Hookean, library volumes) or from hand-derived values in
tests/golden/single_elements.json.
"""

import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import ConvexHull

import pfem_inputs as pi
from oracle import fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "single_elements.json")


def _gold():
    with open(GOLDEN) as f:
        return json.load(f)


def _single(coords, kind, a, b):
    coords = np.asarray(coords, dtype=np.float64)
    d = coords.shape[1]
    return dict(dim=d, coords=coords, conn=np.arange(d + 1, dtype=np.int32)[None, :], kind=kind,
                mat_a=np.array([a]), mat_b=np.array([b]), dirichlet_mask=np.zeros(coords.shape, np.uint8),
                dirichlet_values=np.zeros(coords.shape), facets=np.zeros((0, d), np.int32),
                traction=np.zeros((0, d)), f_ext_extra=None, name="single", seed=0)


# --------------------------------------------------------------------------- geometry


@pytest.mark.parametrize("dim", [2, 3])
def test_shape_gradients_reproduce_affine_fields(dim):
    p = pi.small_problem(dim, "linear", n=3, seed=7)
    m = fem.Mesh(p)
    Xe = m.coords[m.conn]
    # sum_a X_a (x) grad N_a = I and sum_a grad N_a = 0 (P1 completeness)
    eye = np.einsum("eai,eaj->eij", Xe, m.grads)
    assert np.allclose(eye, np.eye(dim), atol=1e-12)
    assert np.allclose(m.grads.sum(axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_measure_matches_convex_hull(dim):
    p = pi.small_problem(dim, "linear", n=2, seed=3)
    m = fem.Mesh(p)
    for e in range(m.n_elems):
        hull = ConvexHull(m.coords[m.conn[e]])
        assert math.isclose(hull.volume, m.vol[e], rel_tol=1e-12)


# --------------------------------------------------------------------------- closed forms


def test_linear_tet_uniaxial_closed_form():
    g = _gold()["linear_tet_uniaxial_strain"]
    p = _single(g["coords"], "linear", g["E"], g["nu"])
    m = fem.Mesh(p)
    u = np.zeros((4, 3))
    u[:, 0] = g["strain"] * m.coords[:, 0]
    f = fem.internal_force(m, u).reshape(4, 3)
    assert np.allclose(f, np.array(g["f"]), rtol=0, atol=1e-15)
    assert math.isclose(fem.strain_energy(m, u), g["energy"], rel_tol=1e-12)


def test_nh_tet_uniaxial_closed_form():
    g = _gold()["nh_tet_uniaxial_stretch"]
    p = _single(g["coords"], "neohookean", g["mu"], g["lambda"])
    m = fem.Mesh(p)
    u = np.zeros((4, 3))
    u[:, 0] = g["stretch"] * m.coords[:, 0]
    f = fem.internal_force(m, u).reshape(4, 3)
    assert np.allclose(f, np.array(g["f"]), rtol=0, atol=1e-14)
    assert math.isclose(fem.strain_energy(m, u), g["energy"], rel_tol=1e-12)


def test_linear_triangle_stiffness_closed_form():
    g = _gold()["linear_tri_plane_strain_stiffness"]
    m = fem.Mesh(_single(g["coords"], "linear", g["E"], g["nu"]))
    K = fem.assemble_linear_K(m).toarray()
    assert np.allclose(K, np.array(g["K"]), rtol=0, atol=1e-14)


def test_plate_edge_load_closed_form():
    g = _gold()["plate_edge_load"]
    p = pi.cfg1_plate(g["n"])
    m = fem.Mesh(p)
    f = fem.external_force(m).reshape(-1, 2)
    right = np.isclose(m.coords[:, 0], 1.0)
    corner = right & (np.isclose(m.coords[:, 1], 0.0) | np.isclose(m.coords[:, 1], 1.0))
    assert np.allclose(f[right & ~corner, 0], g["interior"], rtol=1e-14)
    assert np.allclose(f[corner, 0], g["corner"], rtol=1e-14)
    assert np.allclose(f[~right], 0.0)
    assert math.isclose(f[:, 0].sum(), g["resultant"], rel_tol=1e-13)


def test_traction_resultant_3d():
    p = pi.cube_problem(5, seed=1)
    m = fem.Mesh(p)
    f = fem.external_force(m).reshape(-1, 3)
    # resultant = traction x face area (unit square face)
    assert np.allclose(f.sum(axis=0), [0.0, 0.0, -0.1], atol=1e-14)


def test_traction_per_node_3d_kuhn_face():
    """Per-node consistent load on the z = 1 face of the Kuhn-split cube (App. B: each facet
    node gets t |facet| / 3). The face is a square grid of spacing h with every square cut
    along the same diagonal, so a node inside the face touches 6 triangles of area h^2 / 2
    (share 6 (h^2/2) / 3 = h^2), a node on a face edge (not a corner) touches 3 (share
    h^2 / 2); the 4 corners touch 1 or 2 (shares h^2 / 6 or h^2 / 3, two of each)."""
    n = 5
    h = 1.0 / n
    t = -0.1
    p = pi.cube_problem(n, seed=1)
    m = fem.Mesh(p)
    f = fem.external_force(m).reshape(-1, 3)
    x = m.coords
    top = np.isclose(x[:, 2], 1.0)
    on_x = np.isclose(x[:, 0], 0.0) | np.isclose(x[:, 0], 1.0)
    on_y = np.isclose(x[:, 1], 0.0) | np.isclose(x[:, 1], 1.0)
    interior = top & ~on_x & ~on_y
    edge = top & (on_x ^ on_y)
    corner = top & on_x & on_y
    assert interior.sum() == (n - 1) ** 2 and edge.sum() == 4 * (n - 1) and corner.sum() == 4
    assert np.allclose(f[interior, 2], t * h * h, rtol=1e-13)
    assert np.allclose(f[edge, 2], t * h * h / 2, rtol=1e-13)
    assert np.allclose(np.sort(f[corner, 2] / (t * h * h)), [1 / 6, 1 / 6, 1 / 3, 1 / 3], rtol=1e-12)
    assert np.allclose(f[~top], 0.0) and np.allclose(f[:, :2], 0.0)


# --------------------------------------------------------------------------- patch test


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["linear", "neohookean"])
def test_patch_test_affine_field(dim, kind):
    """Classical FE patch test (Sec. "Patch tests for PFEM" cites it): affine u gives constant strain / F and
    zero internal force at every node not on the patch boundary."""
    p = pi.small_problem(dim, kind, n=4, seed=11, permute=True)
    # the patch test needs one material over the patch (constant stress)
    p["mat_a"] = np.full_like(p["mat_a"], 1.3)
    p["mat_b"] = np.full_like(p["mat_b"], 0.3 if kind == "linear" else 2.5)
    m = fem.Mesh(p)
    rng = np.random.default_rng(5)
    A = 0.05 * rng.standard_normal((dim, dim))
    b = rng.standard_normal(dim)
    u = m.coords @ A.T + b
    gu = fem.displacement_gradient(m.grads, m.gather(u))
    assert np.allclose(gu, A, atol=1e-13)
    f = fem.internal_force(m, u).reshape(-1, dim)
    lo, hi = m.coords.min(0), m.coords.max(0)
    interior = np.all((m.coords > lo + 1e-9) & (m.coords < hi - 1e-9), axis=1)
    assert interior.sum() > 0
    scale = np.abs(f).max()
    assert scale > 1e-6
    assert np.abs(f[interior]).max() <= 1e-12 * max(1.0, scale)
    # and the boundary forces balance (sum of all nodal forces vanishes)
    assert np.allclose(f.sum(axis=0), 0.0, atol=1e-12 * scale * m.n_nodes)


# --------------------------------------------------------------------------- rigid motion


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_infinitesimal_rotation_is_force_free(dim):
    p = pi.small_problem(dim, "linear", n=3, seed=2)
    m = fem.Mesh(p)
    rng = np.random.default_rng(1)
    W = rng.standard_normal((dim, dim))
    W = W - W.T
    u = m.coords @ W.T + rng.standard_normal(dim)
    f = fem.internal_force(m, u)
    assert np.abs(f).max() < 1e-12
    assert abs(fem.strain_energy(m, u)) < 1e-24 + 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_nh_finite_rotation_is_stress_free(dim):
    p = pi.small_problem(dim, "neohookean", n=3, seed=4)
    m = fem.Mesh(p)
    th = 0.6
    if dim == 2:
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    else:
        ax = np.array([1.0, 2.0, -1.0]) / math.sqrt(6.0)
        Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
    u = m.coords @ (R - np.eye(dim)).T + 0.3
    f = fem.internal_force(m, u)
    assert np.abs(f).max() < 1e-12
    assert abs(fem.strain_energy(m, u)) < 1e-13


# --------------------------------------------------------------------------- stiffness


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["linear", "neohookean"])
def test_stiffness_symmetric_and_masked_spd(dim, kind):
    p = pi.small_problem(dim, kind, n=3, seed=8)
    m = fem.Mesh(p)
    u = pi.random_field(p, 3, std=0.02)
    K = fem.stiffness(m, u)
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-12 * np.abs(Kd).max()
    A = fem.masked_operator(m, K).toarray()
    np.linalg.cholesky(A)  # raises if not SPD


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_energy_equals_half_uKu(dim):
    p = pi.small_problem(dim, "linear", n=4, seed=9)
    m = fem.Mesh(p)
    u = pi.random_field(p, 1, std=0.1, zero_masked=False)
    K = fem.assemble_linear_K(m)
    e1 = fem.strain_energy(m, u)
    e2 = 0.5 * float(u.reshape(-1) @ (K @ u.reshape(-1)))
    assert math.isclose(e1, e2, rel_tol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_nh_small_strain_limit_is_linear(dim):
    """At u = 0 the Neo-Hookean tangent equals the linear stiffness with the same Lame
    parameters (C = I, S = 0, C^SE = lam I(x)I + 2 mu I_sym)."""
    p = pi.small_problem(dim, "neohookean", n=3, seed=12)
    m_nh = fem.Mesh(p)
    mu, lam = p["mat_a"], p["mat_b"]
    # invert Lame -> (E, nu): nu = lam / (2 (lam + mu)), E = mu (3 lam + 2 mu) / (lam + mu)
    q = dict(p)
    q["kind"] = "linear"
    q["mat_a"] = mu * (3 * lam + 2 * mu) / (lam + mu)
    q["mat_b"] = lam / (2 * (lam + mu))
    m_lin = fem.Mesh(q)
    K_nh = fem.stiffness(m_nh, np.zeros(m_nh.n_dofs)).toarray()
    K_lin = fem.assemble_linear_K(m_lin).toarray()
    assert np.abs(K_nh - K_lin).max() <= 1e-12 * np.abs(K_lin).max()


# --------------------------------------------------------------------------- finite differences


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["linear", "neohookean"])
def test_energy_gradient_is_internal_force_fd(dim, kind):
    p = pi.small_problem(dim, kind, n=3, seed=21)
    m = fem.Mesh(p)
    u = pi.random_field(p, 4, std=0.03, zero_masked=False).reshape(-1)
    w = np.random.default_rng(6).standard_normal(m.n_dofs)
    h = 1e-6
    fd = (fem.total_energy(m, u + h * w) - fem.total_energy(m, u - h * w)) / (2 * h)
    an = float((fem.internal_force(m, u) - fem.external_force(m)) @ w)
    assert abs(fd - an) <= 1e-6 * abs(an)


@pytest.mark.parametrize("dim", [2, 3])
def test_nh_tangent_is_force_jacobian_fd(dim):
    p = pi.small_problem(dim, "neohookean", n=3, seed=22)
    m = fem.Mesh(p)
    u = pi.random_field(p, 5, std=0.03, zero_masked=False).reshape(-1)
    v = np.random.default_rng(7).standard_normal(m.n_dofs)
    h = 1e-6
    fd = (fem.internal_force(m, u + h * v) - fem.internal_force(m, u - h * v)) / (2 * h)
    an = fem.stiffness(m, u) @ v
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)


def test_masked_operator_and_residual_conventions():
    p = pi.small_problem(3, "linear", n=3, seed=30)
    m = fem.Mesh(p)
    v = np.random.default_rng(1).standard_normal(m.n_dofs)
    y = fem.tangent_apply(m, None, v)
    assert np.allclose(y[m.mask], v[m.mask])  # identity block on Dirichlet DOFs
    vf = v.copy()
    vf[m.mask] = 0.0
    K = fem.assemble_linear_K(m)
    yf = K @ vf
    assert np.allclose(y[~m.mask], yf[~m.mask], rtol=1e-13, atol=1e-13)
    r = fem.residual(m, v)
    assert np.all(r[m.mask] == 0.0)
    d = fem.jacobi_diagonal(m)
    assert np.allclose(d[m.mask], 1.0)
    assert np.allclose(d[~m.mask], K.diagonal()[~m.mask])


def test_nh_inverted_element_energy_is_inf():
    g = _gold()["nh_tet_uniaxial_stretch"]
    m = fem.Mesh(_single(g["coords"], "neohookean", 1.0, 4.0))
    u = np.zeros((4, 3))
    u[:, 0] = -1.5 * m.coords[:, 0]  # F11 = -0.5 -> J < 0
    assert math.isinf(fem.strain_energy(m, u))
