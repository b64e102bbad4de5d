"""ctypes declarations of the C ABI in include/pfem.h (argument marshalling only)."""

import ctypes as C
import os

_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_DIR, "libpfem.so")

PFEM_OK = 0
STATUS = {
    0: "PFEM_OK",
    1: "PFEM_ERR_INVALID_ARG",
    2: "PFEM_ERR_DEGENERATE_ELEMENT",
    3: "PFEM_ERR_INVERTED",
    4: "PFEM_ERR_NONFINITE",
    5: "PFEM_ERR_NOT_CONVERGED",
    6: "PFEM_ERR_OUT_OF_MEMORY",
    7: "PFEM_ERR_OVER_BUDGET",
    8: "PFEM_PENDING",
    9: "PFEM_ERR_TIMEOUT",
    10: "PFEM_ERR_CUDA",
    11: "PFEM_ERR_UNSUPPORTED",
}
PFEM_LINEAR, PFEM_NEOHOOKEAN = 0, 1
PFEM_F32, PFEM_F64, PFEM_F64_F32 = 0, 1, 2


class MeshDesc(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("n_nodes", C.c_int64),
        ("coords", C.c_void_p),
        ("n_elems", C.c_int64),
        ("conn", C.c_void_p),
        ("kind", C.c_int32),
        ("mat_a", C.c_void_p),
        ("mat_b", C.c_void_p),
        ("dirichlet_mask", C.c_void_p),
        ("dirichlet_values", C.c_void_p),
        ("n_facets", C.c_int64),
        ("facets", C.c_void_p),
        ("traction", C.c_void_p),
        ("f_ext_extra", C.c_void_p),
    ]


class MeshStats(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64),
        ("n_elems", C.c_int64),
        ("n_dofs", C.c_int64),
        ("n_free_dofs", C.c_int64),
        ("n_tiles", C.c_int64),
        ("n_local_nodes", C.c_int64),
        ("n_halo_nodes", C.c_int64),
        ("n_partials", C.c_int64),
        ("device_bytes", C.c_int64),
        ("max_tile_elems", C.c_int32),
        ("max_tile_nodes", C.c_int32),
        ("n_fans", C.c_int64),
        ("max_tile_slots", C.c_int32),
        ("reserved", C.c_int32),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32),
        ("newton_iterations", C.c_int32),
        ("replacements", C.c_int32),
        ("inverted_backtracks", C.c_int32),
        ("rel_residual_recursive", C.c_double),
        ("rel_residual_true_f64", C.c_double),
        ("initial_rel_residual", C.c_double),
        ("reference_norm", C.c_double),
        ("status", C.c_int32),
        ("kernel_launches", C.c_int64),
        ("queue_s", C.c_double),
        ("total_s", C.c_double),
        ("apply_ms", C.c_double),
        ("update_ms", C.c_double),
        ("timed_iterations", C.c_int32),
        ("load_step_cuts", C.c_int32),
    ]


class AttnWeights(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("wu", "bu", "wm", "bm", "wq", "bq", "wk", "bk", "wv", "bv")]


# name -> (restype, argtypes); every entry must be exported by libpfem.so
SIGNATURES = {
    "pfem_mesh_create": (C.c_int32, [C.POINTER(MeshDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "pfem_mesh_destroy": (None, [C.c_void_p]),
    "pfem_mesh_create_quad": (C.c_int32, [C.POINTER(MeshDesc), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pfem_plan_check": (C.c_int32, [C.POINTER(MeshDesc), C.POINTER(MeshStats)]),
    "pfem_mesh_stats_get": (C.c_int32, [C.c_void_p, C.POINTER(MeshStats)]),
    "pfem_mesh_set_load_scale": (C.c_int32, [C.c_void_p, C.c_double]),
    "pfem_energy": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pfem_residual": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "pfem_tangent_apply": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfem_tangent_apply_multi": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "pfem_tangent_apply_noalloc": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfem_jacobi_diag": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "pfem_energy_gradient": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfem_energy_hvp": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfem_dot": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfem_solve_linear": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                      C.POINTER(SolveInfo)]),
    "pfem_solve_newton": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_int32,
                                      C.c_double, C.c_void_p, C.POINTER(SolveInfo)]),
    "pfem_set_solver_mode": (C.c_int32, [C.c_int32]),
    "pfem_solve_linear_multi": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_double,
                                            C.c_int32, C.c_void_p, C.c_void_p]),
    "pfem_mesh_set_springs": (C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_double]),
    "pfem_homogenize": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "pfem_set_kernel_timing": (C.c_int32, [C.c_int32]),
    "pfem_set_barrier_test": (C.c_int32, [C.c_int64, C.c_int32]),
    "pfem_batch_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "pfem_batch_destroy": (None, [C.c_void_p]),
    "pfem_batch_offsets": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64)]),
    "pfem_batch_eval": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "pfem_serve_create": (C.c_int32, [C.c_size_t, C.c_int32, C.POINTER(C.c_void_p)]),
    "pfem_serve_submit": (C.c_int32, [C.c_void_p, C.POINTER(MeshDesc), C.c_int32, C.c_void_p, C.c_double, C.c_int32,
                                      C.POINTER(C.c_uint64)]),
    "pfem_serve_poll": (C.c_int32, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(SolveInfo)]),
    "pfem_serve_drain": (C.c_int32, [C.c_void_p, C.c_double]),
    "pfem_serve_stats": (C.c_int32, [C.c_void_p, C.POINTER(C.c_double)]),
    "pfem_serve_destroy": (None, [C.c_void_p]),
    "pfem_attn_create": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.POINTER(AttnWeights), C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "pfem_attn_forward": (C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "pfem_attn_sync": (C.c_int32, [C.c_void_p]),
    "pfem_attn_destroy": (None, [C.c_void_p]),
    "pfem_attn_set_timing": (C.c_int32, [C.c_void_p, C.c_int32]),
    "pfem_attn_kernel_ms": (C.c_int32, [C.c_void_p, C.POINTER(C.c_double)]),
    "pfem_check_status": (C.c_int32, [C.POINTER(C.c_uint32)]),
    "pfem_debug_set_node_id": (C.c_int32, [C.c_void_p, C.c_int64, C.c_int64]),
    "pfem_last_error": (C.c_char_p, []),
    "pfem_version": (C.c_char_p, []),
}

_LIB = None


class PfemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def load(path):
    """Open a build of the library at `path` (libpfem.so or the bounds-checked
    libpfem_checked.so) with every signature declared."""
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run paper_2601_03086_gb300.build.build() first" % os.path.basename(path))
    h = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(h, name)
        fn.restype = res
        fn.argtypes = args
    return h


def lib():
    """Load libpfem.so (raises if it has not been built: there is no fallback path)."""
    global _LIB
    if _LIB is None:
        _LIB = load(LIB_PATH)
    return _LIB


def check(status):
    if status != PFEM_OK:
        msg = lib().pfem_last_error()
        raise PfemError(status, msg.decode() if msg else "")
    return status
