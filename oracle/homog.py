"""FP64 CPU oracle of the numerical homogenisation (appendix "Numerical homogenization
theory"; TPMS cells from appendix "Generation of TPMS geometries").

TEST INFRASTRUCTURE (see oracle/fem.py): only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import it; it shares no code with the CUDA path.

Steps, in the appendix's order:
  * six macroscopic unit strain tensors eps0^(IJ), IJ in (11, 22, 33, 12, 13, 23), with both
    off-diagonal entries 1 for the shear cases (the matrices as printed);
  * the fluctuation field X^v of each case from the weak form int E eps(X*) : eps(X^v) =
    int E eps(X*) : eps0, i.e. K X^v = F with F_a = sum_e V_e sigma0_e grad N_a (sigma0_e = E_e
    : eps0, the stress of the uniform strain in element e);
  * periodicity of X^v through penalty "virtual elements" between corresponding nodes of
    opposite faces (energy 1/2 kappa |X_a - X_b|^2 per pair), one node fixed (the periodic
    coupling leaves the rigid translations free);
  * E^H_(IJ)(KL) = 1/|Omega| int (eps0^(IJ) - eps(X^v(IJ))) : E : (eps0^(KL) - eps(X^v(KL)))
    summed element by element (P1: the strains are constant per element).
Solves are sparse direct (scipy spsolve) on the free DOFs.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem

CASES = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def unit_strains():
    """The six unit strain tensors eps0^(IJ) (3 x 3 each), in the appendix's order."""
    out = []
    for i, j in CASES:
        e = np.zeros((3, 3))
        e[i, j] = 1.0
        e[j, i] = 1.0
        out.append(e)
    return np.array(out)


def _stress(eps, mu, lam):
    """sigma = 2 mu eps + lam tr(eps) I for per-element (E, 3, 3) strains."""
    tr = np.trace(eps, axis1=1, axis2=2)
    return 2.0 * mu[:, None, None] * eps + lam[:, None, None] * tr[:, None, None] * np.eye(3)[None]


def spring_matrix(n_dofs, pairs, kappa, dim=3):
    """Penalty springs between node pairs: S = kappa sum_pairs (e_a - e_b)(e_a - e_b)^T per DOF."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    rows, cols, vals = [], [], []
    for c in range(dim):
        a = pairs[:, 0] * dim + c
        b = pairs[:, 1] * dim + c
        rows += [a, b, a, b]
        cols += [a, b, b, a]
        vals += [np.full(a.size, kappa), np.full(a.size, kappa), np.full(a.size, -kappa), np.full(a.size, -kappa)]
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n_dofs, n_dofs)).tocsr()


def load_vectors(mesh):
    """F^(IJ)_a = sum_e V_e sigma0_e grad N_a for the six unit strains, (6, n_dofs)."""
    F = np.zeros((6, mesh.n_dofs))
    for c, e0 in enumerate(unit_strains()):
        sig = _stress(np.broadcast_to(e0, (mesh.n_elems, 3, 3)), mesh.mu, mesh.lam)
        fe = mesh.vol[:, None, None] * np.einsum("eij,eaj->eai", sig, mesh.grads)
        np.add.at(F[c], mesh.edofs.reshape(-1), fe.reshape(-1))
    return F


def fluctuations(problem, kappa, mesh=None):
    """X^v of the six cases: (K + S) X^v = F on the free DOFs, fixed DOFs 0. (6, n_dofs)."""
    m = mesh if mesh is not None else fem.Mesh(problem)
    A = (fem.assemble_linear_K(m) + spring_matrix(m.n_dofs, problem["pairs"], kappa)).tocsr()
    free = ~m.mask
    Aff = A[free][:, free].tocsc()
    F = load_vectors(m)
    lu = spla.splu(Aff)
    X = np.zeros((6, m.n_dofs))
    for c in range(6):
        X[c, free] = lu.solve(F[c, free])
    return X, F


def homogenized_tensor(problem, kappa, mesh=None):
    """E^H (6 x 6) of the appendix's formula, the fluctuations X^v and the load vectors F."""
    m = mesh if mesh is not None else fem.Mesh(problem)
    X, F = fluctuations(problem, kappa, m)
    e0 = unit_strains()
    eps = []
    for c in range(6):
        g = fem.displacement_gradient(m.grads, m.gather(X[c]))
        ev = 0.5 * (g + np.transpose(g, (0, 2, 1)))
        eps.append(e0[c][None] - ev)
    omega = float(np.prod(m.coords.max(axis=0) - m.coords.min(axis=0)))
    EH = np.zeros((6, 6))
    for a in range(6):
        sa = _stress(eps[a], m.mu, m.lam)
        for b in range(6):
            EH[a, b] = float(np.sum(m.vol * np.einsum("eij,eij->e", sa, eps[b]))) / omega
    return EH, X, F


def isotropic_tensor(E, nu):
    """E^H of a homogeneous isotropic solid in the appendix's normalisation (shear cases with
    both off-diagonal entries 1: the shear block is 4 mu)."""
    mu, lam = fem.lame(np.array([E]), np.array([nu]))
    mu, lam = float(mu[0]), float(lam[0])
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[[0, 1, 2], [0, 1, 2]] = lam + 2 * mu
    C[[3, 4, 5], [3, 4, 5]] = 4 * mu
    return C


def laminate_tensor(Es, nus, fractions, axis=0):
    """Exact effective tensor of a periodic laminate of isotropic layers normal to `axis`
    (layer-wise constant strains; continuity of traction and in-plane strain), in the
    appendix's normalisation. Voigt order (11, 22, 33, 12, 13, 23)."""
    Es, nus, f = (np.asarray(x, dtype=np.float64) for x in (Es, nus, fractions))
    mu, lam = fem.lame(Es, nus)
    M = lam + 2 * mu
    inv = lambda x: 1.0 / np.sum(f * x)  # noqa: E731
    avg = lambda x: float(np.sum(f * x))  # noqa: E731
    c_nn = inv(1.0 / M)                        # normal-normal along the stacking axis
    c_nt = avg(lam / M) * c_nn                 # normal along the axis, in-plane normal
    c_tt = avg(M - lam * lam / M) + avg(lam / M) ** 2 * c_nn   # in-plane normal, same direction
    c_tu = avg(lam - lam * lam / M) + avg(lam / M) ** 2 * c_nn  # in-plane normal, other direction
    g_n = inv(1.0 / mu)                        # shear in a plane containing the axis
    g_t = avg(mu)                              # shear in the layer plane
    C = np.zeros((6, 6))
    t = [d for d in range(3) if d != axis]
    C[axis, axis] = c_nn
    for d in t:
        C[axis, d] = C[d, axis] = c_nt
        C[d, d] = c_tt
    C[t[0], t[1]] = C[t[1], t[0]] = c_tu
    for s, (i, j) in enumerate(CASES[3:]):
        C[3 + s, 3 + s] = 4 * (g_n if axis in (i, j) else g_t)
    return C
