"""pfem_tangent_apply_noalloc: the tangent action for callers that cannot allocate.

Callers running with a frozen or exhausted device memory pool, inside allocator callbacks,
or in runtimes that only own memory handed to them up front cannot let a call allocate. The
no-alloc entry point keeps its per-call scratch in a fixed device array instead. These tests
call it through the C ABI (ctypes) and check it against pfem_tangent_apply, within the
operator tolerances of the other GPU tests, on two calls in a row with different inputs (so
stale contents of the shared array would show), and check that oversized meshes are refused.
This file is collected last on purpose.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from tests.gpu_util import dev, host, pfem, rel_l2

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-5, torch.float64: 1e-12}


def _noalloc(mesh, dtype_code, u, v, y):
    from paper_2601_03086_gb300._lib import lib

    up = C.c_void_p(u.data_ptr()) if u is not None else None
    return lib().pfem_tangent_apply_noalloc(mesh.handle, dtype_code, up, C.c_void_p(v.data_ptr()),
                                            C.c_void_p(y.data_ptr()))


@pytest.mark.parametrize("kind", ["linear", "neohookean"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_noalloc_matches_tangent_apply_twice(kind, dtype):
    P = pfem()
    from paper_2601_03086_gb300._lib import PFEM_F32, PFEM_F64

    p = pi.small_problem(3, kind, shape=(16, 8, 8), seed=41)  # several tiles, halo partials
    mesh = P.Mesh(p)
    assert mesh.stats()["n_partials"] > 0
    x = p["coords"][p["conn"]]
    h = float(np.mean(np.linalg.norm(x[:, 1] - x[:, 0], axis=1)))
    u = dev(np.random.default_rng(1).normal(0.0, 0.03 * h, p["coords"].shape), dtype)
    code = PFEM_F32 if dtype == torch.float32 else PFEM_F64
    for call in range(2):
        v = dev(np.random.default_rng(10 + call).standard_normal(p["coords"].shape), dtype)
        y_ref = P.pfem_tangent_apply(mesh, u, v)
        y = torch.full_like(v, float("nan"))
        assert _noalloc(mesh, code, u, v, y) == 0
        assert rel_l2(host(y), host(y_ref)) <= TOL[dtype]
    mesh.close()


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    P = pfem()
    from paper_2601_03086_gb300._lib import PFEM_F64

    p = pi.cube_problem(100, seed=2)  # 6 M tets: more halo partials than 16 MiB of FP64
    mesh = P.Mesh(p)
    need = mesh.stats()["n_partials"] * 3 * 8
    assert need > 16 << 20
    v = torch.zeros(mesh.n_dofs, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(v)
    assert _noalloc(mesh, PFEM_F64, None, v, y) == 1  # PFEM_ERR_INVALID_ARG
    mesh.close()
