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
    arrays = dict(
        coords=np.ascontiguousarray(problem["coords"], dtype=np.float64),
        conn=np.ascontiguousarray(problem["conn"], dtype=np.int32),
        mat_a=np.ascontiguousarray(problem["mat_a"], dtype=np.float64),
        mat_b=np.ascontiguousarray(problem["mat_b"], dtype=np.float64),
        mask=np.ascontiguousarray(problem["dirichlet_mask"], dtype=np.uint8),
        values=np.ascontiguousarray(problem["dirichlet_values"], dtype=np.float64),
        facets=np.ascontiguousarray(problem["facets"], dtype=np.int32).reshape(-1, dim),
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


def pfem_set_solver_mode(mode):
    check(lib().pfem_set_solver_mode(int(mode)))


def pfem_version():
    return lib().pfem_version().decode()
