"""GPU parity of the ragged-batch energy loss (energy, gradient, Hessian-vector product in
one launch) and of its autograd Functions, against the FP64 CPU oracle and finite
differences.

Bars: FP32 element arithmetic -> relative L2 <= 1e-5 for gradient and Hessian action,
relative error <= 1e-5 for energies; FP64 path -> torch.autograd.gradcheck/gradgradcheck and
a central finite difference (h = 1e-4 on the FP64 energy, relative error <= 1e-6).
"""

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from oracle import fem
from tests.gpu_util import dev, host, pfem, rel_l2

pytestmark = pytest.mark.gpu


def _oracle_terms(p, u, v):
    m = fem.Mesh(p)
    e = fem.total_energy(m, u)
    g = fem.residual(m, u)
    K = fem.stiffness(m, u)
    free = (~m.mask).astype(np.float64)
    hv = free * (K @ (free * v.reshape(-1)))
    return e, g, hv


@pytest.fixture(scope="module")
def small_batch():
    items = pi.cfg4_batch(n_meshes=6, seed=14, lo=800, hi=8000)
    P = pfem()
    meshes = [P.Mesh(p) for p, _ in items]
    batch = P.Batch(meshes)
    u = np.concatenate([uu.reshape(-1) for _, uu in items]).astype(np.float32)
    v = np.random.default_rng(3).standard_normal(u.size).astype(np.float32)
    return items, meshes, batch, u, v


def test_batch_energy_grad_hvp_match_oracle(small_batch):
    items, meshes, batch, u, v = small_batch
    e, g, h = batch.eval(dev(u, torch.float32), dev(v, torch.float32), energy=True, grad=True, hvp=True)
    e, g, h = host(e), host(g), host(h)
    off = batch.offsets
    for k, (p, _) in enumerate(items):
        sl = slice(off[k], off[k + 1])
        eo, go, ho = _oracle_terms(p, u[sl].astype(np.float64), v[sl].astype(np.float64))
        assert abs(e[k] - eo) <= 1e-5 * (abs(eo) + abs(fem.strain_energy(fem.Mesh(p), u[sl].astype(np.float64))))
        assert rel_l2(g[sl], go) <= 1e-5
        assert rel_l2(h[sl], ho) <= 1e-5


def test_batch_matches_single_mesh_calls(small_batch):
    items, meshes, batch, u, v = small_batch
    P = pfem()
    _, g, _ = batch.eval(dev(u, torch.float32), energy=False, grad=True)
    g = host(g)
    off = batch.offsets
    for k, mesh in enumerate(meshes):
        r = host(P.pfem_residual(mesh, dev(u[off[k]:off[k + 1]], torch.float32)))
        assert rel_l2(g[off[k]:off[k + 1]], r) <= 1e-6


def test_batch_mesh_scale_and_autograd(small_batch):
    items, meshes, batch, u, v = small_batch
    P = pfem()
    ut = dev(u, torch.float32).requires_grad_(True)
    w = torch.linspace(0.5, 2.0, batch.n_meshes, dtype=torch.float64, device="cuda")
    loss = (P.batch_energy(ut, batch) * w).sum()
    (g,) = torch.autograd.grad(loss, ut, create_graph=True)
    _, g_ref, _ = batch.eval(ut.detach(), energy=False, grad=True)
    off = batch.offsets
    gh, gr = host(g), host(g_ref)
    wh = host(w)
    for k in range(batch.n_meshes):
        sl = slice(off[k], off[k + 1])
        assert rel_l2(gh[sl], wh[k] * gr[sl]) <= 1e-6
    vt = dev(v, torch.float32)
    (hv,) = torch.autograd.grad((g * vt).sum(), ut)
    _, _, h_ref = batch.eval(ut.detach(), vt, energy=False, hvp=True)
    hh, hr = host(hv), host(h_ref)
    for k in range(batch.n_meshes):
        sl = slice(off[k], off[k + 1])
        assert rel_l2(hh[sl], wh[k] * hr[sl]) <= 1e-6


def test_batch_deterministic(small_batch):
    items, meshes, batch, u, v = small_batch
    uu, vv = dev(u, torch.float32), dev(v, torch.float32)
    a = [t.clone() for t in batch.eval(uu, vv, grad=True, hvp=True)]
    b = [t.clone() for t in batch.eval(uu, vv, grad=True, hvp=True)]
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def _free_param(p):
    """u(w) = prescribed values + free DOFs w (gradcheck over the free DOFs only)."""
    mask = p["dirichlet_mask"].reshape(-1).astype(bool)
    idx = torch.as_tensor(np.flatnonzero(~mask), device="cuda")
    base = torch.as_tensor(np.where(mask, p["dirichlet_values"].reshape(-1), 0.0), device="cuda")

    def u_of(wf):
        return base.index_put((idx,), wf)

    return u_of, int((~mask).sum())


@pytest.mark.parametrize("kind", ["linear", "neohookean"])
def test_mesh_energy_gradcheck_fp64(kind):
    P = pfem()
    p = pi.small_problem(3, kind, n=2, seed=5)
    mesh = P.Mesh(p)
    u_of, nf = _free_param(p)
    rng = np.random.default_rng(2)
    w0 = torch.tensor(rng.normal(0, 0.02, nf), dtype=torch.float64, device="cuda", requires_grad=True)

    def f(wf):
        return P.mesh_energy(u_of(wf), mesh)

    assert torch.autograd.gradcheck(f, (w0,), eps=1e-6, atol=1e-8, rtol=1e-6)
    assert torch.autograd.gradgradcheck(f, (w0,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_energy_gradient_central_fd_and_oracle():
    """Directional central FD (h = 1e-4) of the FP64 energy matches the residual kernel, and
    the FP32 gradient matches the FP64 oracle gradient."""
    P = pfem()
    p, u = pi.cfg4_batch(n_meshes=1, seed=21, lo=4000, hi=6000)[0]
    mesh = P.Mesh(p)
    ud = u.astype(np.float64)
    # a direction of the field's own size, so h = 1e-4 is a relative step of 1e-4
    d = 0.01 * np.random.default_rng(9).standard_normal(ud.shape)
    d[p["dirichlet_mask"].astype(bool)] = 0.0
    h = 1e-4
    ep, _ = P.pfem_energy(mesh, dev(ud + h * d))
    em, _ = P.pfem_energy(mesh, dev(ud - h * d))
    fd = (ep - em) / (2 * h)
    r = host(P.pfem_residual(mesh, dev(ud)))
    an = float(r.reshape(-1) @ d.reshape(-1))
    assert abs(fd - an) <= 1e-6 * abs(an)
    m = fem.Mesh(p)
    g32 = host(P.pfem_residual(mesh, dev(ud, torch.float32)))
    assert rel_l2(g32, fem.residual(m, ud)) <= 1e-5


def test_full_cfg4_batch_sampled_meshes():
    """The 64-mesh batch (about 3 M tets) in one launch; 6 of its meshes checked in full
    against the oracle."""
    P = pfem()
    items = pi.cfg4_batch()
    meshes = [P.Mesh(p) for p, _ in items]
    batch = P.Batch(meshes)
    u = np.concatenate([uu.reshape(-1) for _, uu in items]).astype(np.float32)
    v = np.random.default_rng(4).standard_normal(u.size).astype(np.float32)
    e, g, h = batch.eval(dev(u, torch.float32), dev(v, torch.float32), energy=True, grad=True, hvp=True)
    e, g, h = host(e), host(g), host(h)
    off = batch.offsets
    sizes = [p["conn"].shape[0] for p, _ in items]
    pick = sorted(set([int(np.argmin(sizes)), int(np.argmax(sizes))] + list(range(0, 64, 16))))
    for k in pick:
        p = items[k][0]
        sl = slice(off[k], off[k + 1])
        eo, go, ho = _oracle_terms(p, u[sl].astype(np.float64), v[sl].astype(np.float64))
        assert abs(e[k] - eo) <= 1e-5 * (abs(eo) + abs(fem.strain_energy(fem.Mesh(p), u[sl].astype(np.float64))))
        assert rel_l2(g[sl], go) <= 1e-5
        assert rel_l2(h[sl], ho) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("kind", ["linear", "neohookean"])
def test_single_mesh_scaled_gradient_hvp_and_dot_match_oracle(kind, dtype):
    """The single-mesh autograd path's kernels: g = s P (f_int - f_ext), y = s P K P v (zero on
    prescribed DOFs), a . b, each against the oracle with the upstream factor s applied in the
    kernel (FP32 rel L2 <= 1e-5, FP64 <= 1e-12)."""
    P = pfem()
    tol = 1e-5 if dtype == torch.float32 else 1e-12
    p = pi.small_problem(3, kind, n=5, seed=17)
    mesh = P.Mesh(p)
    rng = np.random.default_rng(6)
    u = 0.01 * rng.standard_normal(p["coords"].size)
    v = rng.standard_normal(p["coords"].size)
    s = torch.tensor(-2.5, dtype=dtype, device="cuda")
    _, go, ho = _oracle_terms(p, u, v)
    g = host(P.pfem_energy_gradient(mesh, dev(u, dtype), scale=s))
    h = host(P.pfem_energy_hvp(mesh, dev(u, dtype), dev(v, dtype), scale=s))
    assert rel_l2(g, -2.5 * go) <= tol
    assert rel_l2(h, -2.5 * ho) <= tol
    assert np.all(h[p["dirichlet_mask"].reshape(-1).astype(bool)] == 0.0)
    g1 = host(P.pfem_energy_gradient(mesh, dev(u, dtype)))
    assert np.array_equal(g1, host(P.pfem_residual(mesh, dev(u, dtype))))
    d = float(host(P.pfem_dot(mesh, dev(g1, dtype), dev(v, dtype))))
    assert abs(d - float(go @ v)) <= tol * float(np.abs(go) @ np.abs(v))
    mesh.close()
