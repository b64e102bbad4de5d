"""FP64 CPU oracle solvers: Jacobi-PCG for K U = F and Newton-Raphson with load steps.

TEST INFRASTRUCTURE (see oracle/fem.py): never imported by the product path.

  * Linear system and stopping rule: K U = F with ||K U - F|| / ||F|| < tol (App. B).
    Dirichlet DOFs are eliminated (K_ff u_f = f_f - K_fc u_c); the reference norm is the
    residual of the lifted start (zero free DOFs, prescribed values on Dirichlet DOFs),
    which equals ||f_f|| when the prescribed values are zero and does not depend on u0.
  * Warm start: the iteration starts from U^(0) = U^NO instead of zero (Sec. "Warm-start", the
    iteration U^(k+1) = phi(U^(k); K, F, U^(0) = U^NO)); the skip test of Sec. "Warm-start" is the
    k = 0 check of the same criterion.
  * Jacobi-PCG: the preconditioned conjugate gradient method with M = diag(K_ff) (the
    paper uses "PCG" without naming the preconditioner; Jacobi is this build's reading).
  * Newton-Raphson (App. B): r = f_int(U) - f_ext, Delta U = -K(U)^-1 r, U += Delta U,
    stop when ||r|| <= tol * ref; load steps scale prescribed values and f_ext by s/n_s;
    the warm start bypasses the first n_s - 1 steps (U_0^(N_f) = U^NO).
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


def pcg(A, b, x0, diag, tol, ref, max_iter, history=None):
    """Jacobi-preconditioned CG on A x = b, stopping when ||b - A x|| / ref < tol.

    The recursive residual is used for the test; the check happens before every
    iteration (so a start that already satisfies it costs zero iterations).
    Returns (x, iterations).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    dinv = 1.0 / diag
    z = dinv * r
    p = z.copy()
    rho = float(r @ z)
    k = 0
    while True:
        rel = float(np.sqrt(r @ r)) / ref
        if history is not None:
            history.append(rel)
        if rel < tol or k >= max_iter:
            break
        q = A @ p
        alpha = rho / float(p @ q)
        x += alpha * p
        r -= alpha * q
        k += 1
        z = dinv * r
        rho_new = float(r @ z)
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    return x, k


def _reduced(mesh, K, u_full, scale):
    free = ~mesh.mask
    f = fem.external_force(mesh, scale)
    Kff = K[free][:, free].tocsr()
    Kfc = K[free][:, mesh.mask]
    b = f[free] - Kfc @ u_full[mesh.mask]
    return Kff, b, free


def solve_linear(problem_or_mesh, u0=None, tol=1e-8, max_iter=100000, history=None, K=None):
    """Warm-started Jacobi-PCG for the linear problem. Returns (u, iterations, rel_true).

    rel_true is the true relative residual ||f_f - K_ff u_f|| / ref of the returned u.
    """
    mesh = problem_or_mesh if isinstance(problem_or_mesh, fem.Mesh) else fem.Mesh(problem_or_mesh)
    if K is None:
        K = fem.assemble_linear_K(mesh)
    u = fem.lifted(mesh, np.zeros(mesh.n_dofs) if u0 is None else u0)
    Kff, b, free = _reduced(mesh, K, u, 1.0)
    ref = float(np.linalg.norm(b))
    if ref == 0.0:
        ref = 1.0
    x, it = pcg(Kff, b, u[free], Kff.diagonal(), tol, ref, max_iter, history)
    u[free] = x
    rel_true = float(np.linalg.norm(b - Kff @ x)) / ref
    return u, it, rel_true


def solve_linear_direct(problem_or_mesh, K=None):
    """Exact (sparse direct) solution of the constrained linear problem."""
    mesh = problem_or_mesh if isinstance(problem_or_mesh, fem.Mesh) else fem.Mesh(problem_or_mesh)
    if K is None:
        K = fem.assemble_linear_K(mesh)
    u = fem.lifted(mesh, np.zeros(mesh.n_dofs))
    Kff, b, free = _reduced(mesh, K, u, 1.0)
    u[free] = spla.spsolve(Kff.tocsc(), b)
    return u


def newton_reference(mesh, scale):
    """||r(u_lift)||: residual of zero free DOFs with the step's prescribed values."""
    r = fem.residual(mesh, fem.lifted(mesh, np.zeros(mesh.n_dofs), scale), scale)
    ref = float(np.linalg.norm(r))
    return ref if ref > 0.0 else 1.0


def solve_newton(problem_or_mesh, u0=None, tol=1e-8, n_load_steps=1, max_newton=50, inner_tol=1e-8,
                 inner_max=100000, direct=False, log=None):
    """Newton-Raphson with load stepping (App. B). Returns (u, newton_iters, inner_iters).

    Per load step s = 1..n_s (scale = s/n_s): set the prescribed DOFs to scale * values,
    then iterate r = P(f_int(u) - scale f_ext); stop if ||r|| <= tol * ||r(u_lift)||;
    solve K_ff(u) Delta = -r_f (Jacobi-PCG to inner_tol relative to ||r_f|| from zero, or a
    direct solve); if the trial u + t Delta inverts an element, halve t (at most 10 times).
    newton_iters counts tangent solves over all steps.
    """
    mesh = problem_or_mesh if isinstance(problem_or_mesh, fem.Mesh) else fem.Mesh(problem_or_mesh)
    u = np.zeros(mesh.n_dofs) if u0 is None else np.array(u0, dtype=np.float64).reshape(-1).copy()
    n_newton = 0
    n_inner = 0
    free = ~mesh.mask
    for s in range(1, n_load_steps + 1):
        scale = s / n_load_steps
        u = fem.lifted(mesh, u, scale)
        ref = newton_reference(mesh, scale)
        for _ in range(max_newton + 1):
            r = fem.residual(mesh, u, scale)
            rel = float(np.linalg.norm(r)) / ref
            if log is not None:
                log.append((s, n_newton, rel))
            if rel <= tol:
                break
            if n_newton >= max_newton * n_load_steps:
                raise RuntimeError("Newton did not converge")
            K = fem.stiffness(mesh, u)
            Kff = K[free][:, free].tocsr()
            rf = r[free]
            if direct:
                delta = spla.spsolve(Kff.tocsc(), -rf)
            else:
                nr = float(np.linalg.norm(rf))
                delta, it = pcg(Kff, -rf, np.zeros_like(rf), Kff.diagonal(), inner_tol, nr, inner_max)
                n_inner += it
            t = 1.0
            for _ in range(11):
                trial = u.copy()
                trial[free] += t * delta
                if fem.min_jacobian(mesh, trial) > 0.0:
                    break
                t *= 0.5
            else:
                raise FloatingPointError("inverted element in every trial step")
            u = trial
            n_newton += 1
        else:
            raise RuntimeError("Newton did not converge")
    return u, n_newton, n_inner
