"""Pins of the Q4 / Q8 oracle (oracle/quad.py): shape-function completeness (Q8 reproduces
quadratics), exact areas, the patch test on distorted meshes, rigid rotations, symmetry,
E = 1/2 u.Ku, central finite differences energy -> force -> tangent and the small-strain
limit of the Neo-Hookean tangent."""

import numpy as np
import pytest

import pfem_inputs as pi
from oracle import quad

CORNERS = [(0.0, 0.0), (2.0, 0.3), (2.3, 1.7), (-0.2, 1.2)]  # a general quadrilateral


@pytest.mark.parametrize("npe", [4, 8])
def test_shape_functions_complete(npe):
    rng = np.random.default_rng(1)
    nodes = quad._Q4 if npe == 4 else quad._Q8
    for xi, eta in rng.uniform(-1, 1, (20, 2)):
        N, dN = quad.shape(npe, xi, eta)
        assert abs(N.sum() - 1) < 1e-14 and np.abs(dN.sum(axis=0)).max() < 1e-14
        assert np.allclose(N @ nodes, [xi, eta], atol=1e-14)
        if npe == 8:  # quadratic completeness of the serendipity element
            for f in (lambda x, y: x * x, lambda x, y: x * y, lambda x, y: y * y):
                assert abs(N @ np.array([f(*q) for q in nodes]) - f(xi, eta)) < 1e-14
        h = 1e-6  # derivatives by central differences
        Np, _ = quad.shape(npe, xi + h, eta)
        Nm, _ = quad.shape(npe, xi - h, eta)
        assert np.allclose((Np - Nm) / (2 * h), dN[:, 0], atol=1e-8)


@pytest.mark.parametrize("npe", [4, 8])
def test_area_and_patch_test(npe):
    p = pi.quad_problem(4, 3, CORNERS, npe, "linear", 1.0, 0.3, jitter=0.2, seed=3)
    m = quad.QuadMesh(p)
    c = np.asarray(CORNERS)
    d1, d2 = c[2] - c[0], c[3] - c[1]
    area = 0.5 * abs(d1[0] * d2[1] - d1[1] * d2[0])
    assert abs(sum(dv.sum() for dv in m.dv) - area) < 1e-12 * area
    A = np.array([[0.01, -0.02], [0.015, 0.005]])
    for kind, mats in (("linear", (1.0, 0.3)), ("neohookean", (1.0, 4.0))):
        p["kind"] = kind
        p["mat_a"][:], p["mat_b"][:] = mats
        m = quad.QuadMesh(p)
        u = (m.coords @ A.T).reshape(-1)
        f = quad.internal_force(m, u).reshape(-1, 2)
        # interior: nodes not on the domain boundary (no element edge on the boundary)
        counts = np.bincount(m.conn[:, :4].reshape(-1), minlength=m.n_nodes)
        interior = counts == 4
        if npe == 8:
            mids = np.bincount(m.conn[:, 4:].reshape(-1), minlength=m.n_nodes)
            interior = (counts == 4) | (mids == 2)
        assert interior.sum() > 0
        assert np.abs(f[interior]).max() < 1e-12 * np.abs(f).max()


def test_rigid_rotation_and_symmetry():
    p = pi.quad_problem(3, 3, CORNERS, 8, "neohookean", 1.0, 4.0, jitter=0.2, seed=4)
    m = quad.QuadMesh(p)
    th = 0.4
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    u = (m.coords @ R.T - m.coords).reshape(-1)
    assert np.abs(quad.internal_force(m, u)).max() < 1e-12
    assert abs(quad.strain_energy(m, u)) < 1e-12
    K = quad.stiffness(m, 0.01 * np.random.default_rng(0).standard_normal(m.n_dofs)).toarray()
    assert np.allclose(K, K.T, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("npe", [4, 8])
def test_energy_identity_fd_and_small_strain_limit(npe):
    p = pi.quad_problem(3, 2, CORNERS, npe, "linear", 1.3, 0.3, jitter=0.2, seed=5)
    m = quad.QuadMesh(p)
    rng = np.random.default_rng(6)
    u = 0.01 * rng.standard_normal(m.n_dofs)
    K = quad.stiffness(m)
    assert abs(quad.strain_energy(m, u) - 0.5 * u @ (K @ u)) < 1e-13
    pn = dict(p, kind="neohookean")
    mu, lam = quad.QuadMesh(p).mu, quad.QuadMesh(p).lam
    pn["mat_a"], pn["mat_b"] = mu.copy(), lam.copy()
    mn = quad.QuadMesh(pn)
    assert np.allclose(quad.stiffness(mn).toarray(), K.toarray(), atol=1e-12 * abs(K).max())
    v = rng.standard_normal(m.n_dofs)
    h = 1e-6
    fd = (quad.strain_energy(mn, u + h * v) - quad.strain_energy(mn, u - h * v)) / (2 * h)
    assert abs(fd - quad.internal_force(mn, u) @ v) < 1e-7 * abs(fd)
    fdk = (quad.internal_force(mn, u + h * v) - quad.internal_force(mn, u - h * v)) / (2 * h)
    kv = quad.stiffness(mn, u) @ v
    assert np.linalg.norm(fdk - kv) < 1e-6 * np.linalg.norm(kv)
