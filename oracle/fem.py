"""FP64 CPU oracle: P1 finite-element energy, internal force and stiffness by global assembly.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
reference arm may import this module. The CUDA product path never calls it, and it shares
no code with that path (the only shared module is pfem_inputs, which generates inputs).

Every routine is vectorised over elements with numpy but keeps the paper's formulation:
  * explicit shape-function differentiation of P1 simplices (App. A; App. B interpolation
    X_i = N_I X_iI, u_i = N_I u_iI);
  * linear elasticity: eps = sym grad u, sigma = E/(1+nu) eps + E nu/((1+nu)(1-2nu)) tr(eps) I,
    Psi = 1/2 sigma:eps (Sec. "Linear elastic plate with arbitrary holes" energy loss); element stiffness assembled in Voigt form
    K_e = V B^T D B (App. B, f_int = K u in linear FEM);
  * compressible Neo-Hookean (Sec. "Nonlinear hyperelasticity" energy loss): Psi = 1/2 lam (ln J)^2 - mu ln J +
    1/2 mu (I1 - d), with I1 = tr C, C = F^T F, F = I + grad u; Lame parameters from (E, nu)
    by the Sec. "Nonlinear hyperelasticity" formula. Total-Lagrangian internal force f_iI = int dN_I/dX_l F_ik S_kl
    (App. B) with S = 2 dPsi/dC = mu (I - C^-1) + lam ln J C^-1, and tangent
    K = K_geo + K_mat, K_geo = int G0^T S G0, K_mat = int B0^T C^SE B0 (App. B) with
    C^SE = 2 dS/dC = lam C^-1 (x) C^-1 + (mu - lam ln J)(C^-1_ik C^-1_jl + C^-1_il C^-1_jk);
  * external force f_ext = int N_I f + int_Gamma_t N_I t (App. B, principle of virtual power).

Readings where the paper is silent (listed with the design notes): the Neo-Hookean offset
is (I1 - d) (the paper prints the 2-D form I1 - 2); 2-D is plane strain with unit
thickness; Dirichlet DOFs are eliminated, i.e. the operator acting on full-length vectors
is A = P K P + (I - P) with P the projector on free DOFs; a load scale s multiplies both
f_ext and the prescribed values (load stepping, App. B).
"""

import math

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------------------
# Geometry: explicit shape-function differentiation (App. A)
# ---------------------------------------------------------------------------------------


def shape_gradients(Xe):
    """Gradients of the P1 shape functions and element measure.

    Xe: (E, d+1, d) corner coordinates. With D = [X_1 - X_0, ..., X_d - X_0] (columns),
    X(xi) = X_0 + D xi, N_a = xi_a for a >= 1 and N_0 = 1 - sum xi, so dN_a/dX = row a-1
    of D^-1 and dN_0/dX = -sum of those rows. Measure V = |det D| / d!.
    Returns grads (E, d+1, d) and vol (E,).
    """
    d = Xe.shape[2]
    D = np.transpose(Xe[:, 1:, :] - Xe[:, :1, :], (0, 2, 1))
    det = np.linalg.det(D)
    if np.any(np.abs(det) == 0.0):
        raise ValueError("degenerate element")
    Dinv = np.linalg.inv(D)
    g = np.empty((Xe.shape[0], d + 1, d))
    g[:, 1:, :] = Dinv
    g[:, 0, :] = -Dinv.sum(axis=1)
    return g, np.abs(det) / math.factorial(d)


def lame(E, nu):
    """Lame parameters from Young's modulus and Poisson's ratio (Sec. "Linear elastic plate with arbitrary holes")."""
    lam = nu * E / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return mu, lam


def displacement_gradient(grads, ue):
    """grad u_ij = sum_a u_a,i dN_a/dX_j (explicit differentiation). ue: (E, d+1, d)."""
    return np.einsum("eai,eaj->eij", ue, grads)


# ---------------------------------------------------------------------------------------
# Mesh-level helpers
# ---------------------------------------------------------------------------------------


class Mesh:
    """Problem dictionary plus cached element geometry (FP64)."""

    def __init__(self, problem):
        self.p = problem
        self.dim = int(problem["dim"])
        self.coords = np.asarray(problem["coords"], dtype=np.float64)
        self.conn = np.asarray(problem["conn"], dtype=np.int64)
        self.n_nodes = self.coords.shape[0]
        self.n_elems = self.conn.shape[0]
        self.n_dofs = self.n_nodes * self.dim
        self.kind = problem["kind"]
        self.mat_a = np.asarray(problem["mat_a"], dtype=np.float64)
        self.mat_b = np.asarray(problem["mat_b"], dtype=np.float64)
        self.mask = np.asarray(problem["dirichlet_mask"], dtype=bool).reshape(-1)
        self.values = np.asarray(problem["dirichlet_values"], dtype=np.float64).reshape(-1)
        self.grads, self.vol = shape_gradients(self.coords[self.conn])
        d = self.dim
        self.edofs = (self.conn[:, :, None] * d + np.arange(d)[None, None, :]).reshape(self.n_elems, -1)
        if self.kind == "linear":
            self.mu, self.lam = lame(self.mat_a, self.mat_b)
        else:
            self.mu, self.lam = self.mat_a, self.mat_b

    def gather(self, u):
        return np.asarray(u, dtype=np.float64).reshape(self.n_nodes, self.dim)[self.conn]


def external_force(mesh, scale=1.0):
    """Consistent nodal external force (App. B): f_I = int_Gamma_t N_I t dGamma (+ extra).

    For a P1 facet with constant traction t, int N_I dGamma = |facet| / d for each of its d
    nodes (|facet| = edge length in 2-D, triangle area in 3-D).
    """
    p = mesh.p
    d = mesh.dim
    f = np.zeros((mesh.n_nodes, d))
    facets = np.asarray(p["facets"], dtype=np.int64).reshape(-1, d)
    if facets.shape[0]:
        t = np.asarray(p["traction"], dtype=np.float64).reshape(-1, d)
        x = mesh.coords[facets]
        if d == 2:
            meas = np.linalg.norm(x[:, 1] - x[:, 0], axis=1)
        else:
            meas = 0.5 * np.linalg.norm(np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), axis=1)
        share = (meas / d)[:, None] * t
        for a in range(d):
            np.add.at(f, facets[:, a], share)
    if p.get("f_ext_extra") is not None:
        f += np.asarray(p["f_ext_extra"], dtype=np.float64).reshape(mesh.n_nodes, d)
    return scale * f.reshape(-1)


def _scatter(mesh, fe):
    out = np.zeros(mesh.n_dofs)
    np.add.at(out, mesh.edofs.reshape(-1), fe.reshape(-1))
    return out


def _assemble(mesh, Ke):
    ne, m, _ = Ke.shape
    rows = np.repeat(mesh.edofs, m, axis=1).reshape(-1)
    cols = np.tile(mesh.edofs, (1, m)).reshape(-1)
    K = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(mesh.n_dofs, mesh.n_dofs)).tocsr()
    K.sum_duplicates()
    return K


# ---------------------------------------------------------------------------------------
# Linear elasticity (Sec. "Linear elastic plate with arbitrary holes" energy loss; App. B with f_int = K u)
# ---------------------------------------------------------------------------------------


def linear_stress(eps, E, nu):
    """sigma = E/(1+nu) eps + E nu/((1+nu)(1-2nu)) tr(eps) I (Sec. "Linear elastic plate with arbitrary holes")."""
    d = eps.shape[-1]
    tr = np.trace(eps, axis1=-2, axis2=-1)
    return (E / (1.0 + nu))[:, None, None] * eps + (E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) * tr)[:, None, None] * np.eye(d)


def linear_energy_density(mesh, u):
    """Psi_e = 1/2 sigma:eps per element, eps = sym grad u."""
    gu = displacement_gradient(mesh.grads, mesh.gather(u))
    eps = 0.5 * (gu + np.transpose(gu, (0, 2, 1)))
    sig = linear_stress(eps, mesh.mat_a, mesh.mat_b)
    return 0.5 * np.einsum("eij,eij->e", sig, eps)


def _voigt_B_linear(g):
    """Small-strain B matrix (engineering shear). g: (E, n, d) -> (E, nv, n*d)."""
    ne, n, d = g.shape
    if d == 2:
        B = np.zeros((ne, 3, n * 2))
        B[:, 0, 0::2] = g[:, :, 0]
        B[:, 1, 1::2] = g[:, :, 1]
        B[:, 2, 0::2] = g[:, :, 1]
        B[:, 2, 1::2] = g[:, :, 0]
        return B
    B = np.zeros((ne, 6, n * 3))
    B[:, 0, 0::3] = g[:, :, 0]
    B[:, 1, 1::3] = g[:, :, 1]
    B[:, 2, 2::3] = g[:, :, 2]
    B[:, 3, 1::3] = g[:, :, 2]  # gamma_23
    B[:, 3, 2::3] = g[:, :, 1]
    B[:, 4, 0::3] = g[:, :, 2]  # gamma_13
    B[:, 4, 2::3] = g[:, :, 0]
    B[:, 5, 0::3] = g[:, :, 1]  # gamma_12
    B[:, 5, 1::3] = g[:, :, 0]
    return B


def _voigt_D_linear(mu, lam, d):
    ne = mu.shape[0]
    if d == 2:
        D = np.zeros((ne, 3, 3))
        D[:, 0, 0] = D[:, 1, 1] = lam + 2 * mu
        D[:, 0, 1] = D[:, 1, 0] = lam
        D[:, 2, 2] = mu
        return D
    D = np.zeros((ne, 6, 6))
    for i in range(3):
        for j in range(3):
            D[:, i, j] = lam
        D[:, i, i] = lam + 2 * mu
        D[:, 3 + i, 3 + i] = mu
    return D


def linear_element_stiffness(mesh, sel=slice(None)):
    """K_e = V B^T D B, (E, (d+1)d, (d+1)d)."""
    B = _voigt_B_linear(mesh.grads[sel])
    D = _voigt_D_linear(mesh.mu[sel], mesh.lam[sel], mesh.dim)
    return mesh.vol[sel][:, None, None] * np.einsum("evi,evw,ewj->eij", B, D, B)


def assemble_linear_K(mesh):
    """Global stiffness K (CSR, unconstrained)."""
    return _assemble(mesh, linear_element_stiffness(mesh))


# ---------------------------------------------------------------------------------------
# Compressible Neo-Hookean (Sec. "Nonlinear hyperelasticity" energy loss; App. B total Lagrangian)
# ---------------------------------------------------------------------------------------


def deformation_gradient(mesh, u, sel=slice(None)):
    ue = np.asarray(u, dtype=np.float64).reshape(mesh.n_nodes, mesh.dim)[mesh.conn[sel]]
    return np.eye(mesh.dim) + displacement_gradient(mesh.grads[sel], ue)


def nh_energy_density(F, mu, lam):
    """Psi = 1/2 lam (ln J)^2 - mu ln J + 1/2 mu (I1 - d); +inf where J <= 0."""
    d = F.shape[-1]
    J = np.linalg.det(F)
    C = np.einsum("eki,ekj->eij", F, F)
    I1 = np.trace(C, axis1=1, axis2=2)
    out = np.full(F.shape[0], np.inf)
    ok = J > 0
    lnJ = np.log(J[ok])
    out[ok] = 0.5 * lam[ok] * lnJ**2 - mu[ok] * lnJ + 0.5 * mu[ok] * (I1[ok] - d)
    return out


def nh_pk2(F, mu, lam):
    """Second Piola-Kirchhoff stress S = mu (I - C^-1) + lam ln J C^-1."""
    d = F.shape[-1]
    C = np.einsum("eki,ekj->eij", F, F)
    Ci = np.linalg.inv(C)
    lnJ = np.log(np.linalg.det(F))
    return mu[:, None, None] * (np.eye(d) - Ci) + (lam * lnJ)[:, None, None] * Ci, Ci, lnJ


_VOIGT = {2: [(0, 0), (1, 1), (0, 1)], 3: [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]}


def nh_material_tangent_voigt(Ci, lnJ, mu, lam):
    """C^SE in Voigt form: lam C^-1 (x) C^-1 + (mu - lam ln J)(Ci_ik Ci_jl + Ci_il Ci_jk)."""
    d = Ci.shape[-1]
    idx = _VOIGT[d]
    nv = len(idx)
    c2 = mu - lam * lnJ
    D = np.zeros((Ci.shape[0], nv, nv))
    for I, (i, j) in enumerate(idx):
        for Jv, (k, l) in enumerate(idx):
            D[:, I, Jv] = lam * Ci[:, i, j] * Ci[:, k, l] + c2 * (Ci[:, i, k] * Ci[:, j, l] + Ci[:, i, l] * Ci[:, j, k])
    return D


def _voigt_B0(F, g):
    """Nonlinear strain-displacement matrix: delta E (Voigt, engineering shear) per delta u_a."""
    ne, n, d = g.shape
    idx = _VOIGT[d]
    B = np.zeros((ne, len(idx), n * d))
    for I, (k, l) in enumerate(idx):
        for a in range(n):
            for i in range(d):
                if k == l:
                    B[:, I, a * d + i] = F[:, i, k] * g[:, a, k]
                else:
                    B[:, I, a * d + i] = F[:, i, k] * g[:, a, l] + F[:, i, l] * g[:, a, k]
    return B


def nh_element_force(mesh, u, sel=slice(None)):
    """f_a = V F S dN_a/dX (App. B total-Lagrangian internal force). (E, d+1, d)."""
    F = deformation_gradient(mesh, u, sel)
    if np.any(np.linalg.det(F) <= 0):
        raise FloatingPointError("inverted element (J <= 0)")
    S, _, _ = nh_pk2(F, mesh.mu[sel], mesh.lam[sel])
    return mesh.vol[sel][:, None, None] * np.einsum("eik,ekl,eal->eai", F, S, mesh.grads[sel])


def nh_element_stiffness(mesh, u, sel=slice(None)):
    """K_e = V (B0^T C^SE B0 + G0^T S G0) (App. B)."""
    F = deformation_gradient(mesh, u, sel)
    if np.any(np.linalg.det(F) <= 0):
        raise FloatingPointError("inverted element (J <= 0)")
    g = mesh.grads[sel]
    S, Ci, lnJ = nh_pk2(F, mesh.mu[sel], mesh.lam[sel])
    D = nh_material_tangent_voigt(Ci, lnJ, mesh.mu[sel], mesh.lam[sel])
    B0 = _voigt_B0(F, g)
    Kmat = np.einsum("evi,evw,ewj->eij", B0, D, B0)
    d = mesh.dim
    gSg = np.einsum("eak,ekl,ebl->eab", g, S, g)
    Kgeo = np.einsum("eab,ij->eaibj", gSg, np.eye(d)).reshape(g.shape[0], (d + 1) * d, (d + 1) * d)
    return mesh.vol[sel][:, None, None] * (Kmat + Kgeo)


# ---------------------------------------------------------------------------------------
# Operator-level functions used by tests and solvers
# ---------------------------------------------------------------------------------------


def strain_energy(mesh, u):
    """sum_e V_e Psi_e(u)."""
    if mesh.kind == "linear":
        return float(np.sum(mesh.vol * linear_energy_density(mesh, u)))
    F = deformation_gradient(mesh, u)
    return float(np.sum(mesh.vol * nh_energy_density(F, mesh.mu, mesh.lam)))


def total_energy(mesh, u, scale=1.0):
    """Pi(u) = sum_e V_e Psi_e - f_ext . u (energy losses of the plate and
    hyperelasticity results on the FE space)."""
    return strain_energy(mesh, u) - float(external_force(mesh, scale) @ np.asarray(u).reshape(-1))


def internal_force(mesh, u):
    """f_int(u), full length (no Dirichlet masking)."""
    if mesh.kind == "linear":
        return assemble_linear_K(mesh) @ np.asarray(u, dtype=np.float64).reshape(-1)
    return _scatter(mesh, nh_element_force(mesh, u))


def stiffness(mesh, u=None):
    """Unconstrained tangent K(u) (linear: K)."""
    if mesh.kind == "linear":
        return assemble_linear_K(mesh)
    if u is None:
        u = np.zeros(mesh.n_dofs)
    return _assemble(mesh, nh_element_stiffness(mesh, u))


def masked_operator(mesh, K):
    """A = P K P + (I - P): identity on Dirichlet DOFs, K_ff on free DOFs."""
    free = (~mesh.mask).astype(np.float64)
    P = sp.diags(free)
    return (P @ K @ P + sp.diags(1.0 - free)).tocsr()


def residual(mesh, u, scale=1.0):
    """r = P (f_int(u) - s f_ext): zero on Dirichlet DOFs."""
    r = internal_force(mesh, u) - external_force(mesh, scale)
    r[mesh.mask] = 0.0
    return r


def tangent_apply(mesh, u, v):
    """y = A(u) v with A = P K(u) P + (I - P)."""
    return masked_operator(mesh, stiffness(mesh, u)) @ np.asarray(v, dtype=np.float64).reshape(-1)


def jacobi_diagonal(mesh, u=None):
    """Diagonal of A(u): diag K(u) on free DOFs, 1 on Dirichlet DOFs."""
    return masked_operator(mesh, stiffness(mesh, u)).diagonal()


def lifted(mesh, u, scale=1.0):
    """Copy of u with the prescribed values (times the load scale) on Dirichlet DOFs."""
    out = np.array(u, dtype=np.float64).reshape(-1).copy()
    out[mesh.mask] = scale * mesh.values[mesh.mask]
    return out


def min_jacobian(mesh, u):
    F = deformation_gradient(mesh, u)
    return float(np.min(np.linalg.det(F)))
