"""The bounds-checked build (libpfem_checked.so, compiled with PFEM_CHECKED) on the GPU: on a
valid mesh it raises no flag and gives the regular build's results bit for bit (in-kernel and
deferred halo completion); a node id corrupted on the device on purpose is caught: the flag
is raised and the kernel reads and writes node 0 instead, so nothing faults. The regular
build refuses the corruption hook."""

import ctypes as C

import pytest
import torch

import pfem_inputs as pi
from paper_2601_03086_gb300 import _lib, api, build
from tests.gpu_util import pfem

pytestmark = pytest.mark.gpu

_CHECKED = []


def _checked():
    if not _CHECKED:
        _CHECKED.append(_lib.load(build.build(checked=True)))
    return _CHECKED[0]


def _mesh(L, p):
    desc, arrays = api._desc(p)
    h = C.c_void_p()
    st = L.pfem_mesh_create(C.byref(desc), None, C.byref(h))
    assert st == 0, L.pfem_last_error()
    del arrays
    return h


def _apply(L, h, v):
    y = torch.empty_like(v)
    st = L.pfem_tangent_apply(h, _lib.PFEM_F32, None, C.c_void_p(v.data_ptr()), C.c_void_p(y.data_ptr()))
    assert st == 0, L.pfem_last_error()
    return y


def _word(L):
    w = C.c_uint32()
    assert L.pfem_check_status(C.byref(w)) == 0, L.pfem_last_error()
    return w.value


@pytest.mark.parametrize("n", [10, 56])  # 56: 1.1 M partials, halo nodes by the deferred pass
def test_checked_build_clean_and_bitwise_equal(n):
    P = pfem()
    L = _checked()
    p = pi.cube_problem(n, seed=3)
    mesh = P.Mesh(p)
    torch.manual_seed(n)
    v = torch.randn(mesh.n_dofs, dtype=torch.float32, device="cuda")
    y_ref = P.pfem_tangent_apply(mesh, None, v).clone()
    torch.cuda.synchronize()
    assert _word(L) == 0
    h = _mesh(L, p)
    y = _apply(L, h, v)
    assert _word(L) == 0
    assert torch.equal(y, y_ref)
    L.pfem_mesh_destroy(h)
    mesh.close()


def test_checked_build_flags_corrupted_node_id():
    P = pfem()
    L = _checked()
    p = pi.cube_problem(6, seed=1)
    h = _mesh(L, p)
    stats = _lib.MeshStats()
    assert L.pfem_mesh_stats_get(h, C.byref(stats)) == 0
    n_nodes = p["coords"].shape[0]
    v = torch.randn(n_nodes * 3, dtype=torch.float32, device="cuda")
    _apply(L, h, v)
    assert _word(L) == 0
    # one tile-node record pointed past the last node: caught, node 0 used instead
    assert L.pfem_debug_set_node_id(h, 5, n_nodes + 1000) == 0
    _apply(L, h, v)
    assert _word(L) & 1
    assert _word(L) == 0  # cleared by the read
    L.pfem_mesh_destroy(h)
    # the context is intact: a fresh mesh applies cleanly
    h2 = _mesh(L, p)
    _apply(L, h2, v)
    assert _word(L) == 0
    L.pfem_mesh_destroy(h2)
    # the regular build has neither the checks nor the hook
    mesh = P.Mesh(p)
    assert _lib.STATUS[_lib.lib().pfem_debug_set_node_id(mesh.handle, 5, n_nodes + 1000)] == "PFEM_ERR_UNSUPPORTED"
    w = C.c_uint32()
    assert _lib.STATUS[_lib.lib().pfem_check_status(C.byref(w))] == "PFEM_ERR_UNSUPPORTED"
    mesh.close()
