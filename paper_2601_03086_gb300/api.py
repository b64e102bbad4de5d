"""Python binding of the C ABI (same names as include/pfem.h).

Argument marshalling only: device vectors are torch CUDA tensors (float32 -> PFEM_F32,
float64 -> PFEM_F64, DOF-interleaved, contiguous) and every computation runs in libpfem's
CUDA kernels. A mesh is bound to the torch CUDA stream current at creation; its calls are
ordered on that stream.
"""

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import PFEM_F32, PFEM_F64, PFEM_LINEAR, PFEM_NEOHOOKEAN, check, lib

_KIND = {"linear": PFEM_LINEAR, "neohookean": PFEM_NEOHOOKEAN}


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _dtype_of(t, arith=None):
    """float32 -> PFEM_F32; float64 -> PFEM_F64, or PFEM_F64_F32 when arith == "f32"."""
    if t.dtype == torch.float32:
        return PFEM_F32
    if t.dtype == torch.float64:
        return _lib.PFEM_F64_F32 if arith == "f32" else PFEM_F64
    raise TypeError("vectors must be float32 or float64 CUDA tensors (got %s)" % t.dtype)


def _dev(t, n, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be contiguous with %d entries (got %d)" % (name, n, t.numel()))
    return C.c_void_p(t.data_ptr())


def _desc(problem):
    """MeshDesc plus the numpy arrays it points into (keep both alive during the call)."""
    dim = int(problem["dim"])
    fn = 3 if int(problem.get("npe", 0)) == 8 else dim  # ids per traction facet
    arrays = dict(
        coords=np.ascontiguousarray(problem["coords"], dtype=np.float64),
        conn=np.ascontiguousarray(problem["conn"], dtype=np.int32),
        mat_a=np.ascontiguousarray(problem["mat_a"], dtype=np.float64),
        mat_b=np.ascontiguousarray(problem["mat_b"], dtype=np.float64),
        mask=np.ascontiguousarray(problem["dirichlet_mask"], dtype=np.uint8),
        values=np.ascontiguousarray(problem["dirichlet_values"], dtype=np.float64),
        facets=np.ascontiguousarray(problem["facets"], dtype=np.int32).reshape(-1, fn),
        traction=np.ascontiguousarray(problem["traction"], dtype=np.float64).reshape(-1, dim),
        extra=None if problem.get("f_ext_extra") is None else np.ascontiguousarray(problem["f_ext_extra"],
                                                                                   dtype=np.float64),
    )
    a = arrays
    desc = _lib.MeshDesc()
    desc.dim = dim
    desc.n_nodes = a["coords"].shape[0]
    desc.coords = _ptr(a["coords"])
    desc.n_elems = a["conn"].shape[0]
    desc.conn = _ptr(a["conn"])
    desc.kind = _KIND[problem["kind"]]
    desc.mat_a = _ptr(a["mat_a"])
    desc.mat_b = _ptr(a["mat_b"])
    desc.dirichlet_mask = _ptr(a["mask"])
    desc.dirichlet_values = _ptr(a["values"])
    desc.n_facets = a["facets"].shape[0]
    desc.facets = _ptr(a["facets"])
    desc.traction = _ptr(a["traction"])
    desc.f_ext_extra = _ptr(a["extra"])
    return desc, arrays


def pfem_plan_check(problem):
    """Host-only validation + plan self-check; returns the plan statistics dict."""
    desc, arrays = _desc(problem)
    s = _lib.MeshStats()
    check(lib().pfem_plan_check(C.byref(desc), C.byref(s)))
    del arrays
    return {k: getattr(s, k) for k, _ in _lib.MeshStats._fields_}


class Mesh:
    """Owns a pfem_mesh_t (device plan) built from a problem dictionary (see pfem_inputs)."""

    def __init__(self, problem, stream=None):
        dim = int(problem["dim"])
        desc, self._arrays = _desc(problem)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        npe = int(problem.get("npe", 0))
        if npe:  # quadrilaterals
            check(lib().pfem_mesh_create_quad(C.byref(desc), npe, C.c_void_p(stream.cuda_stream), C.byref(h)))
        else:
            check(lib().pfem_mesh_create(C.byref(desc), C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.handle = h
        self.dim = dim
        self.kind = problem["kind"]
        self.n_nodes = int(desc.n_nodes)
        self.n_elems = int(desc.n_elems)
        self.n_dofs = self.n_nodes * dim
        self._arrays = None

    def stats(self):
        s = _lib.MeshStats()
        check(lib().pfem_mesh_stats_get(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.MeshStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().pfem_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pfem_mesh_create(problem, stream=None):
    return Mesh(problem, stream)


def pfem_mesh_destroy(mesh):
    mesh.close()


def pfem_mesh_set_load_scale(mesh, s):
    check(lib().pfem_mesh_set_load_scale(mesh.handle, float(s)))


def pfem_energy(mesh, u, arith=None):
    """(Pi(u), strain energy) as Python floats (synchronises the mesh stream)."""
    e = C.c_double()
    es = C.c_double()
    check(lib().pfem_energy(mesh.handle, _dtype_of(u, arith), _dev(u, mesh.n_dofs, "u"), C.byref(e), C.byref(es)))
    return e.value, es.value


def pfem_residual(mesh, u, r=None, arith=None):
    r = torch.empty_like(u) if r is None else r
    check(lib().pfem_residual(mesh.handle, _dtype_of(u, arith), _dev(u, mesh.n_dofs, "u"), _dev(r, mesh.n_dofs, "r")))
    return r


def pfem_tangent_apply(mesh, u, v, y=None, arith=None):
    y = torch.empty_like(v) if y is None else y
    up = _dev(u, mesh.n_dofs, "u") if u is not None else None
    check(lib().pfem_tangent_apply(mesh.handle, _dtype_of(v, arith), up, _dev(v, mesh.n_dofs, "v"), _dev(y, mesh.n_dofs, "y")))
    return y


def pfem_tangent_apply_multi(mesh, v, y=None, arith=None):
    """y[j] = A v[j] for the rows of v ((k, n_dofs) float32, or float64 with FP32 arithmetic)."""
    if v.dim() != 2 or v.shape[1] != mesh.n_dofs or not v.is_contiguous() or not v.is_cuda:
        raise ValueError("v must be a contiguous CUDA tensor of shape (k, %d)" % mesh.n_dofs)
    y = torch.empty_like(v) if y is None else y
    if y.shape != v.shape or not y.is_contiguous() or y.dtype != v.dtype:
        raise ValueError("y must match v")
    dt = PFEM_F32 if v.dtype == torch.float32 else _lib.PFEM_F64_F32
    check(lib().pfem_tangent_apply_multi(mesh.handle, dt, None, int(v.shape[0]), C.c_void_p(v.data_ptr()),
                                         C.c_void_p(y.data_ptr())))
    return y


def _scalar(s, like, name):
    """Device pointer of a one-entry tensor of the vector type (None = 1)."""
    if s is None:
        return None
    if not isinstance(s, torch.Tensor) or not s.is_cuda or s.numel() != 1 or s.dtype != like.dtype:
        raise TypeError("%s must be a one-entry CUDA tensor of dtype %s" % (name, like.dtype))
    return C.c_void_p(s.contiguous().data_ptr())


def pfem_energy_gradient(mesh, u, scale=None, g=None, arith=None):
    """g = scale * P (f_int(u) - f_ext), the upstream factor applied in the kernel."""
    g = torch.empty_like(u) if g is None else g
    check(lib().pfem_energy_gradient(mesh.handle, _dtype_of(u, arith), _dev(u, mesh.n_dofs, "u"),
                                     _scalar(scale, u, "scale"), _dev(g, mesh.n_dofs, "g")))
    return g


def pfem_energy_hvp(mesh, u, v, scale=None, y=None, arith=None):
    """y = scale * P K(u) P v (zero rows and columns on prescribed DOFs)."""
    y = torch.empty_like(v) if y is None else y
    up = _dev(u, mesh.n_dofs, "u") if u is not None else None
    check(lib().pfem_energy_hvp(mesh.handle, _dtype_of(v, arith), up, _dev(v, mesh.n_dofs, "v"),
                                _scalar(scale, v, "scale"), _dev(y, mesh.n_dofs, "y")))
    return y


def pfem_dot(mesh, a, b, out=None):
    """a . b as a 0-dim device tensor of the vectors' dtype (FP64 sums, fixed order)."""
    out = torch.empty((), dtype=a.dtype, device=a.device) if out is None else out
    check(lib().pfem_dot(mesh.handle, _dtype_of(a), _dev(a, mesh.n_dofs, "a"), _dev(b, mesh.n_dofs, "b"),
                         C.c_void_p(out.data_ptr())))
    return out


def pfem_jacobi_diag(mesh, u=None, d=None, dtype=torch.float32, arith=None):
    if d is None:
        d = torch.empty(mesh.n_dofs, dtype=u.dtype if u is not None else dtype, device="cuda")
    up = _dev(u, mesh.n_dofs, "u") if u is not None else None
    check(lib().pfem_jacobi_diag(mesh.handle, _dtype_of(d, arith), up, _dev(d, mesh.n_dofs, "d")))
    return d


def _info_dict(info):
    return {k: getattr(info, k) for k, _ in _lib.SolveInfo._fields_}


def pfem_solve_linear(mesh, u0=None, tol=1e-8, max_iter=100000, precision="f32", u_out=None, raise_on_error=True):
    """Warm-started Jacobi-PCG; returns (u float64 tensor, info dict)."""
    dt = PFEM_F32 if precision == "f32" else PFEM_F64
    u_out = torch.empty(mesh.n_dofs, dtype=torch.float64, device="cuda") if u_out is None else u_out
    u0p = _dev(u0, mesh.n_dofs, "u0") if u0 is not None else None
    info = _lib.SolveInfo()
    st = lib().pfem_solve_linear(mesh.handle, dt, u0p, float(tol), int(max_iter), _dev(u_out, mesh.n_dofs, "u_out"),
                                 C.byref(info))
    if raise_on_error:
        check(st)
    return u_out, _info_dict(info)


def pfem_solve_newton(mesh, u0=None, tol=1e-8, n_load_steps=1, max_newton=50, inner_tol=1e-8, precision="f32",
                      u_out=None, raise_on_error=True):
    """Newton-Raphson with load steps; returns (u float64 tensor, info dict)."""
    dt = PFEM_F32 if precision == "f32" else PFEM_F64
    u_out = torch.empty(mesh.n_dofs, dtype=torch.float64, device="cuda") if u_out is None else u_out
    u0p = _dev(u0, mesh.n_dofs, "u0") if u0 is not None else None
    info = _lib.SolveInfo()
    st = lib().pfem_solve_newton(mesh.handle, dt, u0p, float(tol), int(n_load_steps), int(max_newton),
                                 float(inner_tol), _dev(u_out, mesh.n_dofs, "u_out"), C.byref(info))
    if raise_on_error:
        check(st)
    return u_out, _info_dict(info)


def pfem_solve_linear_multi(mesh, b, u0=None, tol=1e-8, max_iter=100000, precision="f32", u_out=None,
                            raise_on_error=True):
    """k independent Jacobi-PCG solves sharing each operator application; b: (k, n_dofs)
    float64 CUDA tensor. Returns (u (k, n_dofs) float64, list of k info dicts)."""
    if b.dim() != 2 or b.shape[1] != mesh.n_dofs or b.dtype != torch.float64 or not b.is_contiguous():
        raise ValueError("b must be a contiguous float64 CUDA tensor of shape (k, %d)" % mesh.n_dofs)
    k = int(b.shape[0])
    u_out = torch.empty_like(b) if u_out is None else u_out
    u0p = None
    if u0 is not None:
        if u0.shape != b.shape or u0.dtype != torch.float64 or not u0.is_contiguous():
            raise ValueError("u0 must match b")
        u0p = C.c_void_p(u0.data_ptr())
    infos = (_lib.SolveInfo * k)()
    st = lib().pfem_solve_linear_multi(mesh.handle, PFEM_F32 if precision == "f32" else PFEM_F64, k,
                                       C.c_void_p(b.data_ptr()), u0p, float(tol), int(max_iter),
                                       C.c_void_p(u_out.data_ptr()), infos)
    if raise_on_error:
        check(st)
    return u_out, [_info_dict(i) for i in infos]


def pfem_mesh_set_springs(mesh, pairs, stiffness):
    """Penalty springs between node pairs ((n, 2) int array; empty removes them)."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    check(lib().pfem_mesh_set_springs(mesh.handle, int(pairs.shape[0]), _ptr(pairs) if pairs.size else None,
                                      float(stiffness)))


def pfem_homogenize(mesh, coords, xv0=None, tol=1e-8, max_iter=100000, precision="f32", raise_on_error=True):
    """Effective tensor of a periodic cell (springs set on the mesh). Returns (E^H 6x6 numpy,
    fluctuations (6, n_dofs) float64 CUDA tensor, list of 6 info dicts)."""
    xyz = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1)
    eh = np.zeros(36)
    xv = torch.empty((6, mesh.n_dofs), dtype=torch.float64, device="cuda")
    xv0p = None
    if xv0 is not None:
        if xv0.shape != xv.shape or xv0.dtype != torch.float64 or not xv0.is_contiguous():
            raise ValueError("xv0 must be a contiguous float64 CUDA tensor of shape (6, %d)" % mesh.n_dofs)
        xv0p = C.c_void_p(xv0.data_ptr())
    infos = (_lib.SolveInfo * 6)()
    st = lib().pfem_homogenize(mesh.handle, PFEM_F32 if precision == "f32" else PFEM_F64, _ptr(xyz), xv0p,
                               float(tol), int(max_iter), _ptr(eh), C.c_void_p(xv.data_ptr()), infos)
    if raise_on_error:
        check(st)
    return eh.reshape(6, 6), xv, [_info_dict(i) for i in infos]


def pfem_set_solver_mode(mode):
    check(lib().pfem_set_solver_mode(int(mode)))


def pfem_set_barrier_test(spin_limit=0, absent_cta=-1):
    check(lib().pfem_set_barrier_test(int(spin_limit), int(absent_cta)))


def pfem_set_kernel_timing(on):
    check(lib().pfem_set_kernel_timing(int(on)))


def pfem_version():
    return lib().pfem_version().decode()


# ---------------------------------------------------------------------------------------
# Ragged batches (one element launch for many meshes) and autograd Functions
# ---------------------------------------------------------------------------------------


class Batch:
    """Owns a pfem_batch_t over 3-D meshes (kept alive by this object)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (C.c_void_p * len(self.meshes))(*[m.handle.value for m in self.meshes])
        h = C.c_void_p()
        check(lib().pfem_batch_create(arr, len(self.meshes), C.byref(h)))
        self.handle = h
        off = (C.c_int64 * (len(self.meshes) + 1))()
        check(lib().pfem_batch_offsets(self.handle, off))
        self.offsets = [int(x) for x in off]
        self.n_meshes = len(self.meshes)
        self.n_dofs = self.offsets[-1]

    def eval(self, u, v=None, mesh_scale=None, energy=True, grad=False, hvp=False):
        """Returns (energy float64 (n_meshes,) or None, grad or None, hvp or None)."""
        n = self.n_dofs
        up = _dev(u, n, "u")
        if u.dtype != torch.float32:
            raise TypeError("batch vectors are float32")
        e = torch.empty(self.n_meshes, dtype=torch.float64, device=u.device) if energy else None
        g = torch.empty_like(u) if grad else None
        h = torch.empty_like(u) if hvp else None
        vp = _dev(v, n, "v") if v is not None else None
        sp = _dev(mesh_scale, self.n_meshes, "mesh_scale") if mesh_scale is not None else None
        check(lib().pfem_batch_eval(self.handle, up, vp, sp, C.c_void_p(e.data_ptr()) if e is not None else None,
                                    C.c_void_p(g.data_ptr()) if g is not None else None,
                                    C.c_void_p(h.data_ptr()) if h is not None else None, None))
        return e, g, h

    def close(self):
        if getattr(self, "handle", None):
            lib().pfem_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pfem_batch_create(meshes):
    return Batch(meshes)


def pfem_batch_destroy(batch):
    batch.close()


def pfem_batch_offsets(batch):
    return list(batch.offsets)


def pfem_batch_eval(batch, u, v=None, mesh_scale=None, energy=True, grad=False, hvp=False):
    return batch.eval(u, v, mesh_scale, energy, grad, hvp)


class _BatchGrad(torch.autograd.Function):
    """g = sum_m s_m dPi_m/du (residual kernel); its backward is the Hessian action."""

    @staticmethod
    def forward(ctx, u, s, batch):
        ctx.save_for_backward(u, s)
        ctx.batch = batch
        return batch.eval(u, mesh_scale=s, energy=False, grad=True)[1]

    @staticmethod
    def backward(ctx, w):
        u, s = ctx.saved_tensors
        hv = ctx.batch.eval(u, v=w.contiguous(), mesh_scale=s, energy=False, hvp=True)[2]
        return hv, None, None


class _BatchEnergy(torch.autograd.Function):
    """Per-mesh energies Pi_m(u) (FP64 sums of FP32 element terms)."""

    @staticmethod
    def forward(ctx, u, batch):
        ctx.save_for_backward(u)
        ctx.batch = batch
        return batch.eval(u, energy=True)[0]

    @staticmethod
    def backward(ctx, ge):
        (u,) = ctx.saved_tensors
        s = ge.detach().to(torch.float32).contiguous()
        return _BatchGrad.apply(u, s, ctx.batch), None


def batch_energy(u, batch):
    """Differentiable per-mesh FE energy loss of a ragged batch (float32 u, float64 output).

    backward = residual kernel (scaled per mesh by the upstream gradient inside the kernel),
    double backward = tangent kernel (Hessian-vector product); element quantities are
    recomputed in every pass, never stored.
    """
    return _BatchEnergy.apply(u, batch)


class _MeshGrad(torch.autograd.Function):
    """g = s dPi/du (gradient kernel, s applied in the kernel); its backward is the Hessian
    action (scaled in the kernel) and, for s, the unscaled gradient dotted with the upstream
    vector (dot kernel)."""

    @staticmethod
    def forward(ctx, u, s, mesh):
        ctx.save_for_backward(u, s)
        ctx.mesh = mesh
        return pfem_energy_gradient(mesh, u, scale=s)

    @staticmethod
    def backward(ctx, w):
        u, s = ctx.saved_tensors
        w = w.contiguous()
        hv = pfem_energy_hvp(ctx.mesh, u, w, scale=s)
        ds = None
        if ctx.needs_input_grad[1]:
            ds = pfem_dot(ctx.mesh, pfem_energy_gradient(ctx.mesh, u), w)
        return hv, ds, None


class _MeshEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, mesh):
        ctx.save_for_backward(u)
        ctx.mesh = mesh
        e, _ = pfem_energy(mesh, u)
        return torch.tensor(e, dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, ge):
        (u,) = ctx.saved_tensors
        return _MeshGrad.apply(u, ge.contiguous(), ctx.mesh), None


def mesh_energy(u, mesh):
    """Differentiable FE energy of one mesh (float32 or float64 u): backward = residual,
    double backward = tangent action, prescribed DOFs held fixed (zero gradient)."""
    return _MeshEnergy.apply(u, mesh)


# ---------------------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------------------

PFEM_SOLVE_LINEAR, PFEM_SOLVE_NEWTON = 0, 1
PFEM_PENDING = 8


class Server:
    """pfem_serve_*: continuous batching of warm-started solves on the current device."""

    def __init__(self, hbm_budget_bytes, max_slots=64):
        h = C.c_void_p()
        check(lib().pfem_serve_create(C.c_size_t(int(hbm_budget_bytes)), int(max_slots), C.byref(h)))
        self.handle = h
        self._dofs = {}

    def submit(self, problem, u0=None, tol=1e-8, solve="linear", n_load_steps=1):
        """Queue a solve (host arrays); returns its ticket."""
        desc, arrays = _desc(problem)
        u0a = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        t = C.c_uint64()
        kind = PFEM_SOLVE_LINEAR if solve == "linear" else PFEM_SOLVE_NEWTON
        check(lib().pfem_serve_submit(self.handle, C.byref(desc), kind, _ptr(u0a), float(tol), int(n_load_steps),
                                      C.byref(t)))
        del arrays
        self._dofs[t.value] = int(desc.n_nodes) * int(desc.dim)
        return t.value

    def poll(self, ticket):
        """None while pending, else (status, u float64 numpy, info dict)."""
        n = self._dofs[ticket]
        out = np.empty(n, dtype=np.float64)
        info = _lib.SolveInfo()
        st = lib().pfem_serve_poll(self.handle, C.c_uint64(ticket), out.ctypes.data_as(C.c_void_p), C.byref(info))
        if st == PFEM_PENDING:
            return None
        del self._dofs[ticket]
        return st, out, _info_dict(info)

    def drain(self, timeout_s=600.0):
        check(lib().pfem_serve_drain(self.handle, float(timeout_s)))

    def stats(self):
        """Worker-thread accounting (pfem_serve_stats): seconds waiting for the device after
        chunks, admitting, rebuilding tables, running the state machine; counts."""
        out = (C.c_double * 8)()
        check(lib().pfem_serve_stats(self.handle, out))
        keys = ("wait_s", "admit_s", "tables_s", "advance_s", "chunks", "rebuilds", "admitted")
        return {k: (int(out[i]) if i >= 4 else out[i]) for i, k in enumerate(keys)}

    def close(self):
        if getattr(self, "handle", None):
            lib().pfem_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pfem_serve_create(hbm_budget_bytes, max_slots=64):
    return Server(hbm_budget_bytes, max_slots)


def pfem_serve_submit(server, problem, u0=None, tol=1e-8, solve="linear", n_load_steps=1):
    return server.submit(problem, u0, tol, solve, n_load_steps)


def pfem_serve_poll(server, ticket):
    return server.poll(ticket)


def pfem_serve_stats(server):
    return server.stats()


def pfem_serve_drain(server, timeout_s=600.0):
    server.drain(timeout_s)


def pfem_serve_destroy(server):
    server.close()


# ---- physics attention ----------------------------------------------------------------

_ATTN_KEYS = ("wu", "bu", "wm", "bm", "wq", "bq", "wk", "bk", "wv", "bv")


class Attention:
    """Owns a pfem_attn_t: the physics-attention module with resident weights.  `params`
    maps wu, bu, wm, bm, wq, bq, wk, bk, wv, bv to arrays ((in, out) weights); they are
    copied (as float32) at creation.  Bound to the torch CUDA stream current at creation."""

    def __init__(self, params, n_heads, scale=1.0, stream=None):
        arrs = {k: np.ascontiguousarray(np.asarray(params[k], dtype=np.float32)) for k in _ATTN_KEYS}
        self.n_channels = int(arrs["wu"].shape[0])
        self.n_tokens = int(arrs["wm"].shape[1])
        self.s_pad = 64 if self.n_tokens <= 64 else 128
        w = _lib.AttnWeights(**{k: arrs[k].ctypes.data_as(C.c_void_p) for k in _ATTN_KEYS})
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        check(lib().pfem_attn_create(self.n_channels, self.n_tokens, int(n_heads), float(scale), C.byref(w),
                                     C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.handle = h

    def forward(self, x, xt=None, m=None, tokens=False):
        """x: bf16 CUDA tensor [N][C].  Returns xt (bf16 [N][C]); with tokens=True also the
        slice weights m (bf16 [N][S_pad]) and the tokens Z, Z^t (float32 [S][C])."""
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.bfloat16 and x.is_contiguous()
                and x.dim() == 2 and x.shape[1] == self.n_channels):
            raise TypeError("x must be a contiguous bf16 CUDA tensor of shape [N, %d]" % self.n_channels)
        n = int(x.shape[0])
        if xt is None:
            xt = torch.empty_like(x)
        if m is None and tokens:
            m = torch.empty((n, self.s_pad), dtype=torch.bfloat16, device=x.device)
        z = zt = None
        if tokens:
            z = torch.zeros((self.n_tokens, self.n_channels), dtype=torch.float32, device=x.device)
            zt = torch.zeros_like(z)
        check(lib().pfem_attn_forward(self.handle, n, C.c_void_p(x.data_ptr()), _dev(xt, x.numel(), "xt"),
                                      None if m is None else _dev(m, n * self.s_pad, "m"),
                                      None if z is None else C.c_void_p(z.data_ptr()),
                                      None if zt is None else C.c_void_p(zt.data_ptr())))
        return (xt, m, z, zt) if tokens else xt

    def sync(self):
        check(lib().pfem_attn_sync(self.handle))

    def set_timing(self, on):
        check(lib().pfem_attn_set_timing(self.handle, int(bool(on))))

    def kernel_ms(self):
        """Durations (ms) of the slice, token-sum, token-attention and deslice kernels of the
        last timed forward."""
        ms = (C.c_double * 4)()
        check(lib().pfem_attn_kernel_ms(self.handle, ms))
        return dict(zip(("slice", "reduce", "tokens", "deslice"), list(ms)))

    def close(self):
        if getattr(self, "handle", None):
            lib().pfem_attn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pfem_attn_create(params, n_heads, scale=1.0, stream=None):
    return Attention(params, n_heads, scale, stream)


def pfem_attn_forward(attn, x, xt=None, m=None, tokens=False):
    return attn.forward(x, xt, m, tokens)


def pfem_attn_sync(attn):
    attn.sync()


def pfem_attn_destroy(attn):
    attn.close()
