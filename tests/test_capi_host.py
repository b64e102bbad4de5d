"""CPU tests of the C ABI: the library builds and loads, exports every symbol declared in
include/pfem.h, and the host-side validation and tile planner behave (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

import pfem_inputs as pi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpfem():
    from paper_2601_03086_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "pfem.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(pfem_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_symbols_exported(libpfem):
    names = _declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(libpfem, n), n


def test_checked_build_exports_header_and_reports_itself():
    """The bounds-checked twin exports the same C ABI; its version string says what it is,
    and the regular build answers pfem_check_status with UNSUPPORTED (no GPU call needed)."""
    from paper_2601_03086_gb300 import _lib, build

    checked = _lib.load(build.build(checked=True))
    for n in _declared_symbols():
        assert hasattr(checked, n), n
    assert b"bounds-checked" in checked.pfem_version()
    assert b"bounds-checked" not in _lib.lib().pfem_version()
    w = ctypes.c_uint32(7)
    assert _lib.STATUS[_lib.lib().pfem_check_status(ctypes.byref(w))] == "PFEM_ERR_UNSUPPORTED"
    assert w.value == 0


def test_python_binding_covers_header():
    from paper_2601_03086_gb300 import _lib

    for n in _declared_symbols():
        assert n in _lib.SIGNATURES, n


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["linear", "neohookean"])
@pytest.mark.parametrize("n", [1, 3, 9])
def test_plan_invariants_small(libpfem, dim, kind, n):
    from paper_2601_03086_gb300 import pfem_plan_check

    p = pi.small_problem(dim, kind, n=n, seed=n + dim)
    s = pfem_plan_check(p)
    assert s["n_elems"] == p["conn"].shape[0]
    assert s["max_tile_elems"] <= 1024 and s["max_tile_nodes"] <= 1024


def test_plan_invariants_cube_and_masked_domains(libpfem):
    from paper_2601_03086_gb300 import pfem_plan_check

    s = pfem_plan_check(pi.cube_problem(24, seed=2))
    assert s["n_tiles"] > 1 and s["n_halo_nodes"] > 0 and s["n_partials"] > 0
    for prob, _u in pi.cfg4_batch(n_meshes=3, seed=11, lo=2000, hi=20000):
        pfem_plan_check(prob)


def test_plan_orphan_nodes_and_empty_mesh(libpfem):
    from paper_2601_03086_gb300 import pfem_plan_check

    p = pi.small_problem(3, "linear", n=2, seed=1, permute=False)
    # add two nodes used by no element
    p["coords"] = np.vstack([p["coords"], [[5.0, 5.0, 5.0], [6.0, 5.0, 5.0]]])
    p["dirichlet_mask"] = np.vstack([p["dirichlet_mask"], np.zeros((2, 3), np.uint8)])
    p["dirichlet_values"] = np.vstack([p["dirichlet_values"], np.zeros((2, 3))])
    s0 = pfem_plan_check(pi.small_problem(3, "linear", n=2, seed=1, permute=False))
    s = pfem_plan_check(p)
    # orphans live in an element-free tile as complete nodes (the self-check covers them)
    assert s["n_tiles"] == s0["n_tiles"] + 1 and s["n_halo_nodes"] == s0["n_halo_nodes"]
    q = dict(p)
    q["conn"] = np.zeros((0, 4), np.int32)
    q["mat_a"] = np.zeros(0)
    q["mat_b"] = np.zeros(0)
    q["facets"] = np.zeros((0, 3), np.int32)
    q["traction"] = np.zeros((0, 3))
    s = pfem_plan_check(q)
    assert s["n_tiles"] == 1 and s["n_halo_nodes"] == 0 and s["max_tile_nodes"] == q["coords"].shape[0]


def _status(fn, p):
    from paper_2601_03086_gb300._lib import PfemError

    try:
        fn(p)
    except PfemError as e:
        return e.status
    return 0


def test_validation_errors(libpfem):
    from paper_2601_03086_gb300 import pfem_plan_check

    base = pi.small_problem(3, "linear", n=2, seed=3)
    p = dict(base)
    p["conn"] = base["conn"].copy()
    p["conn"][0, 1] = p["conn"][0, 0]  # repeated node -> zero volume
    assert _status(pfem_plan_check, p) == 2  # PFEM_ERR_DEGENERATE_ELEMENT
    p = dict(base)
    p["conn"] = base["conn"].copy()
    p["conn"][1, 2] = base["coords"].shape[0]  # out of range
    assert _status(pfem_plan_check, p) == 1
    p = dict(base)
    p["mat_b"] = base["mat_b"].copy()
    p["mat_b"][0] = 0.5  # incompressible linear material is rejected
    assert _status(pfem_plan_check, p) == 1
    p = dict(base)
    p["coords"] = base["coords"].copy()
    p["coords"][0, 0] = np.nan
    assert _status(pfem_plan_check, p) == 1
    p = dict(base)
    p["dim"] = 4
    p["coords"] = np.zeros((base["coords"].shape[0], 4))
    p["dirichlet_mask"] = np.zeros((base["coords"].shape[0], 4), np.uint8)
    p["dirichlet_values"] = np.zeros((base["coords"].shape[0], 4))
    p["facets"] = np.zeros((0, 4), np.int32)
    p["traction"] = np.zeros((0, 4))
    assert _status(pfem_plan_check, p) == 1
