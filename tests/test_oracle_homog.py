"""Pins of the homogenisation oracle (oracle/homog.py) against closed forms and invariants.

Periodicity is a penalty (springs of stiffness kappa between opposite-face nodes), so the
computed tensor carries an error of order 1/kappa: the opposite faces of even a homogeneous
cell carry equal and opposite loads that the springs only balance by stretching. As kappa
grows: a homogeneous cell converges to the material's own tensor, a periodic two-phase
laminate to the exact layered-medium tensor (its fluctuation is piecewise linear, so P1
elements on a mesh that follows the layers represent it exactly), with errors shrinking like
1/kappa. TPMS cells give symmetric, positive definite tensors below the Voigt bound with the
symmetries of their level sets."""

import numpy as np
import pytest

import pfem_inputs as pi
from oracle import fem, homog

KAPPA = 100.0  # penalty stiffness x E_solid x h of the tests' cells


def _eh(p, n):
    return homog.homogenized_tensor(p, KAPPA / n)


def test_homogeneous_cell_gives_material_tensor():
    n = 6
    p = pi.tpms_cell(n, "gyroid", void_ratio=1.0, E_solid=2.0, nu=0.3)
    C = homog.isotropic_tensor(2.0, 0.3)
    errs = []
    for kappa in (1e2, 1e3, 1e8):
        EH, X, F = homog.homogenized_tensor(p, kappa * 2.0 / n)
        errs.append(np.abs(EH - C).max() / np.abs(C).max())
    assert 7.0 < errs[0] / errs[1] < 13.0, errs  # penalty error ~ 1/kappa
    assert errs[2] < 1e-6, errs


@pytest.mark.parametrize("axis", [0, 2])
def test_laminate_matches_layered_closed_form(axis):
    n = 8
    p = pi.laminate_cell(n, layers=(1.0, 5.0), nus=(0.3, 0.2), axis=axis)
    C = homog.laminate_tensor((1.0, 5.0), (0.3, 0.2), p["phase_fraction"], axis=axis)
    errs = []
    for kappa in (1e2, 1e3, 1e8):
        EH, _, _ = homog.homogenized_tensor(p, kappa * 5.0 / n)
        errs.append(np.abs(EH - C).max() / np.abs(C).max())
    assert 7.0 < errs[0] / errs[1] < 13.0, errs
    assert errs[2] < 1e-6, errs


@pytest.mark.parametrize("family", ["primitive", "gyroid"])
def test_tpms_tensor_invariants(family):
    n = 8
    p = pi.tpms_cell(n, family)
    EH, _, _ = _eh(p, n)
    scale = np.abs(EH).max()
    assert np.allclose(EH, EH.T, atol=1e-10 * scale)
    assert np.linalg.eigvalsh(0.5 * (EH + EH.T)).min() > 0
    # the level set is invariant under a cyclic permutation of the axes, and so are the voxel
    # grid and the Kuhn split (diagonal (0,0,0)-(1,1,1)): cubic-type equalities
    d = np.diag(EH)
    assert np.allclose(d[:3], d[0], rtol=1e-9) and np.allclose(d[3:], d[3], rtol=1e-9)
    assert np.allclose([EH[0, 1], EH[1, 2], EH[0, 2]], EH[0, 1], rtol=1e-9)
    # Voigt bound: the cell is never stiffer than the volume average of its phases
    m = fem.Mesh(p)
    vol = m.vol.sum()
    avg = np.zeros((6, 6))
    for E in np.unique(p["mat_a"]):
        w = m.vol[p["mat_a"] == E].sum() / vol
        avg += w * homog.isotropic_tensor(float(E), 0.3)
    assert np.all(np.diag(EH) <= np.diag(avg) * (1 + 1e-12))
    assert 0.0 < p["volume_fraction"] < 1.0
