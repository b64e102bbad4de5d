"""FP64 CPU oracle of bilinear (Q4) and serendipity (Q8) quadrilaterals in plane strain with
Gauss quadrature (the element families of the hyperelastic beam and Cook-membrane results,
Sec. "Nonlinear hyperelasticity"; App. B isoparametric interpolation, total-Lagrangian
internal force and tangent K = K_geo + K_mat).

TEST INFRASTRUCTURE (see oracle/fem.py): only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import it; it shares no code with the CUDA path.

Element definitions (reference square [-1, 1]^2):
  * Q4: corners (-1,-1), (1,-1), (1,1), (-1,1); N_a = (1 + xi xi_a)(1 + eta eta_a) / 4;
    2 x 2 Gauss points (+-1/sqrt 3, weights 1).
  * Q8: corners as Q4, then mid-edge nodes (0,-1), (1,0), (0,1), (-1,0) (edges 0-1, 1-2, 2-3,
    3-0); corner N_a = (1 + xi xi_a)(1 + eta eta_a)(xi xi_a + eta eta_a - 1) / 4, mid-edge
    N_a = (1 - xi^2)(1 + eta eta_a) / 2 or (1 + xi xi_a)(1 - eta^2) / 2; 3 x 3 Gauss points
    (0, +-sqrt(3/5); weights 8/9, 5/9).
Per Gauss point: J = dX/dxi, grad N = J^-T dN/dxi, dV = w det J (unit thickness). Materials
and the Dirichlet elimination are those of oracle/fem.py (linear: sigma(eps) of the plate law;
Neo-Hookean: Psi = 1/2 lam ln^2 J - mu ln J + 1/2 mu (I1 - 2), S = mu (I - C^-1) +
lam ln J C^-1, C^SE = lam C^-1 (x) C^-1 + (mu - lam ln J)(C^-1 (x) C^-1 sym)); everything
is assembled globally (COO -> CSR).
"""

import math

import numpy as np
import scipy.sparse as sp

from . import fem

_Q4 = np.array([(-1, -1), (1, -1), (1, 1), (-1, 1)], dtype=np.float64)
_Q8 = np.array([(-1, -1), (1, -1), (1, 1), (-1, 1), (0, -1), (1, 0), (0, 1), (-1, 0)], dtype=np.float64)


def gauss(npe):
    """Tensor-product Gauss points and weights of the element family."""
    if npe == 4:
        g = np.array([-1.0, 1.0]) / math.sqrt(3.0)
        w = np.array([1.0, 1.0])
    else:
        g = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
        w = np.array([5.0, 8.0, 5.0]) / 9.0
    pts = np.array([(a, b) for b in g for a in g])
    wts = np.array([wa * wb for wb in w for wa in w])
    return pts, wts


def shape(npe, xi, eta):
    """N (npe,) and dN/dxi (npe, 2) at one reference point."""
    if npe == 4:
        xa, ya = _Q4[:, 0], _Q4[:, 1]
        N = 0.25 * (1 + xi * xa) * (1 + eta * ya)
        dN = np.stack([0.25 * xa * (1 + eta * ya), 0.25 * ya * (1 + xi * xa)], axis=1)
        return N, dN
    N = np.zeros(8)
    dN = np.zeros((8, 2))
    for a in range(4):
        xa, ya = _Q8[a]
        N[a] = 0.25 * (1 + xi * xa) * (1 + eta * ya) * (xi * xa + eta * ya - 1)
        dN[a, 0] = 0.25 * xa * (1 + eta * ya) * (2 * xi * xa + eta * ya)
        dN[a, 1] = 0.25 * ya * (1 + xi * xa) * (xi * xa + 2 * eta * ya)
    for a in range(4, 8):
        xa, ya = _Q8[a]
        if xa == 0:
            N[a] = 0.5 * (1 - xi * xi) * (1 + eta * ya)
            dN[a] = (-xi * (1 + eta * ya), 0.5 * ya * (1 - xi * xi))
        else:
            N[a] = 0.5 * (1 + xi * xa) * (1 - eta * eta)
            dN[a] = (0.5 * xa * (1 - eta * eta), -eta * (1 + xi * xa))
    return N, dN


class QuadMesh:
    """Problem dict (conn with npe node ids per element) plus Gauss-point geometry."""

    def __init__(self, problem):
        self.p = problem
        self.coords = np.asarray(problem["coords"], dtype=np.float64)
        self.conn = np.asarray(problem["conn"], dtype=np.int64)
        self.npe = self.conn.shape[1]
        self.n_nodes = self.coords.shape[0]
        self.n_elems = self.conn.shape[0]
        self.n_dofs = 2 * self.n_nodes
        self.kind = problem["kind"]
        a, b = np.asarray(problem["mat_a"], float), np.asarray(problem["mat_b"], float)
        self.mu, self.lam = fem.lame(a, b) if self.kind == "linear" else (a, b)
        self.mask = np.asarray(problem["dirichlet_mask"], dtype=bool).reshape(-1)
        self.values = np.asarray(problem["dirichlet_values"], dtype=np.float64).reshape(-1)
        pts, wts = gauss(self.npe)
        Xe = self.coords[self.conn]  # (E, npe, 2)
        self.grads, self.dv = [], []
        for (xi, eta), w in zip(pts, wts):
            _, dN = shape(self.npe, xi, eta)
            J = np.einsum("eai,aj->eij", Xe, dN)  # dX_i/dxi_j
            det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
            if np.any(det <= 0):
                raise ValueError("element with det J <= 0 at a Gauss point")
            Jinv = np.linalg.inv(J)
            self.grads.append(np.einsum("aj,eji->eai", dN, Jinv))  # dN_a/dX_i
            self.dv.append(w * det)
        self.edofs = (self.conn[:, :, None] * 2 + np.arange(2)[None, None, :]).reshape(self.n_elems, -1)

    def gather(self, u):
        return np.asarray(u, dtype=np.float64).reshape(self.n_nodes, 2)[self.conn]


def _assemble(m, Ke):
    ne, k, _ = Ke.shape
    rows = np.repeat(m.edofs, k, axis=1).reshape(-1)
    cols = np.tile(m.edofs, (1, k)).reshape(-1)
    K = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(m.n_dofs, m.n_dofs)).tocsr()
    K.sum_duplicates()
    return K


def _B_small(g):
    """Voigt B of small strain (eps_xx, eps_yy, gamma_xy) for per-element gradients (E, npe, 2)."""
    E, n, _ = g.shape
    B = np.zeros((E, 3, 2 * n))
    B[:, 0, 0::2] = g[:, :, 0]
    B[:, 1, 1::2] = g[:, :, 1]
    B[:, 2, 0::2] = g[:, :, 1]
    B[:, 2, 1::2] = g[:, :, 0]
    return B


def _D_linear(mu, lam):
    D = np.zeros((mu.size, 3, 3))
    D[:, 0, 0] = D[:, 1, 1] = lam + 2 * mu
    D[:, 0, 1] = D[:, 1, 0] = lam
    D[:, 2, 2] = mu
    return D


def deformation_gradients(m, u):
    ue = m.gather(u)
    return [np.eye(2)[None] + np.einsum("eai,eaj->eij", ue, g) for g in m.grads]


def element_stiffness(m, u=None):
    """(E, 2 npe, 2 npe) element matrices: linear V B^T D B, Neo-Hookean K_geo + K_mat."""
    Ke = np.zeros((m.n_elems, 2 * m.npe, 2 * m.npe))
    if m.kind == "linear":
        D = _D_linear(m.mu, m.lam)
        for g, dv in zip(m.grads, m.dv):
            B = _B_small(g)
            Ke += dv[:, None, None] * np.einsum("eki,ekl,elj->eij", B, D, B)
        return Ke
    Fs = deformation_gradients(m, np.zeros(m.n_dofs) if u is None else u)
    for g, dv, F in zip(m.grads, m.dv, Fs):
        C = np.einsum("eki,ekj->eij", F, F)
        Ci = np.linalg.inv(C)
        J = np.linalg.det(F)
        lnJ = np.log(J)
        S = m.mu[:, None, None] * (np.eye(2)[None] - Ci) + (m.lam * lnJ)[:, None, None] * Ci
        # K_geo: (grad N_a . S grad N_b) I
        Kg = np.einsum("eai,eij,ebj->eab", g, S, g)
        Kgeo = np.zeros_like(Ke)
        Kgeo[:, 0::2, 0::2] = Kg
        Kgeo[:, 1::2, 1::2] = Kg
        # K_mat: B0^T C^SE B0 with B0 the Green-Lagrange variation (Voigt, engineering shear)
        E_, n, _ = g.shape
        B0 = np.zeros((E_, 3, 2 * n))
        for a in range(n):
            for i in range(2):
                col = 2 * a + i
                B0[:, 0, col] = F[:, i, 0] * g[:, a, 0]
                B0[:, 1, col] = F[:, i, 1] * g[:, a, 1]
                B0[:, 2, col] = F[:, i, 0] * g[:, a, 1] + F[:, i, 1] * g[:, a, 0]
        v = [(0, 0), (1, 1), (0, 1)]
        Cse = np.zeros((E_, 3, 3))
        for I, (i, j) in enumerate(v):
            for K_, (k, l) in enumerate(v):
                Cse[:, I, K_] = (m.lam * Ci[:, i, j] * Ci[:, k, l] + (m.mu - m.lam * lnJ) *
                                 (Ci[:, i, k] * Ci[:, j, l] + Ci[:, i, l] * Ci[:, j, k]))
        Kmat = np.einsum("eki,ekl,elj->eij", B0, Cse, B0)
        Ke += dv[:, None, None] * (Kgeo + Kmat)
    return Ke


def stiffness(m, u=None):
    return _assemble(m, element_stiffness(m, u))


def internal_force(m, u):
    """f_a = sum_gp dV P grad N_a (linear: sigma(eps) grad N_a)."""
    f = np.zeros(m.n_dofs)
    ue = m.gather(u)
    for g, dv, F in zip(m.grads, m.dv, deformation_gradients(m, u)):
        if m.kind == "linear":
            G = np.einsum("eai,eaj->eij", ue, g)
            eps = 0.5 * (G + np.transpose(G, (0, 2, 1)))
            T = 2 * m.mu[:, None, None] * eps + (m.lam * np.trace(eps, axis1=1, axis2=2))[:, None, None] * np.eye(2)
        else:
            C = np.einsum("eki,ekj->eij", F, F)
            Ci = np.linalg.inv(C)
            lnJ = np.log(np.linalg.det(F))
            S = m.mu[:, None, None] * (np.eye(2)[None] - Ci) + (m.lam * lnJ)[:, None, None] * Ci
            T = np.einsum("eik,ekj->eij", F, S)
        fe = dv[:, None, None] * np.einsum("eij,eaj->eai", T, g)
        np.add.at(f, m.edofs.reshape(-1), fe.reshape(-1))
    return f


def strain_energy(m, u):
    """sum_gp dV Psi."""
    e = 0.0
    ue = m.gather(u)
    for g, dv, F in zip(m.grads, m.dv, deformation_gradients(m, u)):
        if m.kind == "linear":
            G = np.einsum("eai,eaj->eij", ue, g)
            eps = 0.5 * (G + np.transpose(G, (0, 2, 1)))
            tr = np.trace(eps, axis1=1, axis2=2)
            psi = m.mu * np.einsum("eij,eij->e", eps, eps) + 0.5 * m.lam * tr * tr
        else:
            J = np.linalg.det(F)
            lnJ = np.log(J)
            I1 = np.einsum("eij,eij->e", F, F)
            psi = 0.5 * m.lam * lnJ ** 2 - m.mu * lnJ + 0.5 * m.mu * (I1 - 2.0)
        e += float(np.sum(dv * psi))
    return e


def external_force(m, scale=1.0):
    """Consistent edge loads of constant traction: Q4 edges (a, b) get |edge|/2 t at each end;
    Q8 edges (a, b, mid) get |edge| t (1/6, 1/6, 2/3) (Simpson weights of the quadratic edge)."""
    p = m.p
    f = np.zeros((m.n_nodes, 2))
    fac = np.asarray(p["facets"], dtype=np.int64)
    if fac.size:
        t = np.asarray(p["traction"], dtype=np.float64).reshape(-1, 2)
        L = np.linalg.norm(m.coords[fac[:, 1]] - m.coords[fac[:, 0]], axis=1)[:, None]
        if fac.shape[1] == 2:
            np.add.at(f, fac[:, 0], 0.5 * L * t)
            np.add.at(f, fac[:, 1], 0.5 * L * t)
        else:
            np.add.at(f, fac[:, 0], L * t / 6.0)
            np.add.at(f, fac[:, 1], L * t / 6.0)
            np.add.at(f, fac[:, 2], 2.0 * L * t / 3.0)
    return scale * f.reshape(-1)


def residual(m, u, scale=1.0):
    r = internal_force(m, u) - external_force(m, scale)
    r[m.mask] = 0.0
    return r


def tangent_apply(m, u, v):
    """A v = P K(u) P v + (I - P) v."""
    free = (~m.mask).astype(np.float64)
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    return free * (stiffness(m, u) @ (free * v)) + (1 - free) * v


# ---------------------------------------------------------------------------------------
# Solvers (the algorithms of oracle/solve.py on quadrilateral meshes)
# ---------------------------------------------------------------------------------------


def min_jacobian(m, u):
    return min(float(np.linalg.det(F).min()) for F in deformation_gradients(m, u))


def lifted(m, u, scale=1.0):
    out = np.array(u, dtype=np.float64).reshape(-1).copy()
    out[m.mask] = scale * m.values[m.mask]
    return out


def solve_linear(m, u0=None, tol=1e-8, max_iter=100000):
    """Jacobi-PCG on K_ff u_f = f_f - K_fc u_c (oracle/solve.py's stopping rule)."""
    from . import solve

    K = stiffness(m)
    u = lifted(m, np.zeros(m.n_dofs) if u0 is None else u0)
    free = ~m.mask
    Kff = K[free][:, free].tocsr()
    b = external_force(m)[free] - K[free][:, m.mask] @ u[m.mask]
    ref = float(np.linalg.norm(b)) or 1.0
    x, it = solve.pcg(Kff, b, u[free], Kff.diagonal(), tol, ref, max_iter)
    u[free] = x
    return u, it


def solve_newton(m, u0=None, tol=1e-8, n_load_steps=1, max_newton=50, inner_tol=1e-8):
    """Newton-Raphson with load steps and halving on J <= 0 (oracle/solve.py's algorithm),
    inner Jacobi-PCG to inner_tol. Returns (u, newton_iterations)."""
    from . import solve

    u = np.zeros(m.n_dofs) if u0 is None else np.array(u0, dtype=np.float64).reshape(-1).copy()
    free = ~m.mask
    n_newton = 0
    for s in range(1, n_load_steps + 1):
        scale = s / n_load_steps
        u = lifted(m, u, scale)
        r0 = residual(m, lifted(m, np.zeros(m.n_dofs), scale), scale)
        ref = float(np.linalg.norm(r0)) or 1.0
        for _ in range(max_newton + 1):
            r = residual(m, u, scale)
            if float(np.linalg.norm(r)) / ref <= tol:
                break
            K = stiffness(m, u)
            Kff = K[free][:, free].tocsr()
            rf = r[free]
            d, _ = solve.pcg(Kff, -rf, np.zeros_like(rf), Kff.diagonal(), inner_tol, float(np.linalg.norm(rf)), 100000)
            t = 1.0
            for _ in range(11):
                trial = u.copy()
                trial[free] += t * d
                if min_jacobian(m, trial) > 0.0:
                    break
                t *= 0.5
            else:
                raise FloatingPointError("inverted element in every trial step")
            u = trial
            n_newton += 1
        else:
            raise RuntimeError("Newton did not converge")
    return u, n_newton
