"""Seeded synthetic inputs for the PFEM element operator and its solves.

This package holds only input generation: structured and masked voxel meshes split into
P1 simplices, boundary facet extraction, per-element material sampling, Dirichlet sets,
the smooth warm-start perturbation shape and the workload descriptions of the five
benchmark problems. It contains none of the finite-element arithmetic (no shape
functions, stresses, forces or solvers); both the CPU oracle and the CUDA path consume
the same problem dictionaries produced here.

A *problem* is a plain dict:

    dim               2 (P1 triangles, plane strain) or 3 (P1 tetrahedra)
    coords            (n_nodes, dim) float64, reference coordinates X
    conn              (n_elems, dim+1) int32 node ids
    kind              "linear" (mat_a=E, mat_b=nu) or "neohookean" (mat_a=mu, mat_b=lambda)
    mat_a, mat_b      (n_elems,) float64 per-element material parameters
    dirichlet_mask    (n_nodes, dim) uint8, 1 = prescribed DOF
    dirichlet_values  (n_nodes, dim) float64, prescribed value at full load
    facets            (n_facets, dim) int32 boundary facets carrying a traction
    traction          (n_facets, dim) float64 traction vector per facet (reference config)
    f_ext_extra       None or (n_nodes, dim) float64 extra nodal force
    name, seed        bookkeeping
"""

from .meshes import (  # noqa: F401
    grid_tri,
    grid_tet,
    boundary_facets,
    jitter_nodes,
    permute_mesh,
    bbox,
)
from .problems import (  # noqa: F401
    cfg1_plate,
    cfg2_cube,
    cfg3_bar,
    cfg4_batch,
    cfg5_requests,
    cube_problem,
    bar_problem,
    request_problem,
    roofline_cube,
    small_problem,
    smooth_shape,
    make_warm_start,
    random_field,
    periodic_pairs,
    tpms_cell,
    laminate_cell,
)
from .quads import cook_membrane, nh_beam, quad_grid, quad_problem  # noqa: F401
