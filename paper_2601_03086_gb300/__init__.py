"""GB300 (sm_103a) matrix-free P1 finite-element operator and warm-started solvers (PFEM).

The compute path is libpfem.so (hand-written CUDA, built in-tree by build.py); this package
is the Python binding of its C ABI. Importing it does not load the library; the first call
does, and raises if the library has not been built.
"""

from .api import (  # noqa: F401
    Attention,
    pfem_attn_create,
    pfem_attn_destroy,
    pfem_attn_forward,
    pfem_attn_sync,
    Batch,
    Mesh,
    Server,
    pfem_serve_create,
    pfem_serve_destroy,
    pfem_serve_drain,
    pfem_serve_poll,
    pfem_serve_submit,
    batch_energy,
    mesh_energy,
    pfem_batch_create,
    pfem_batch_destroy,
    pfem_batch_eval,
    pfem_batch_offsets,
    pfem_dot,
    pfem_energy,
    pfem_energy_gradient,
    pfem_energy_hvp,
    pfem_homogenize,
    pfem_jacobi_diag,
    pfem_mesh_create,
    pfem_mesh_destroy,
    pfem_mesh_set_load_scale,
    pfem_mesh_set_springs,
    pfem_plan_check,
    pfem_residual,
    pfem_set_barrier_test,
    pfem_set_kernel_timing,
    pfem_set_solver_mode,
    pfem_solve_linear,
    pfem_solve_linear_multi,
    pfem_solve_newton,
    pfem_tangent_apply,
    pfem_tangent_apply_multi,
    pfem_version,
)
