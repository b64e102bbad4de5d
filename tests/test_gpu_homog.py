"""GPU homogenisation (pfem_homogenize) against the FP64 oracle (oracle/homog.py) at the same
penalty stiffness: the six fluctuation fields within 1e-6 (rel L2) and E^H within 1e-6 of the
oracle's element-integral formula; a warm start near the solution needs fewer iterations for
the same tensor."""

import numpy as np
import pytest
import torch

import pfem_inputs as pi
from oracle import homog
from tests.gpu_util import host, pfem, rel_l2

pytestmark = pytest.mark.gpu


def _cell(kind, n):
    if kind == "laminate":
        return pi.laminate_cell(n, layers=(1.0, 5.0), nus=(0.3, 0.2), axis=1), 5.0
    return pi.tpms_cell(n, kind), 1.0


@pytest.mark.parametrize("kind", ["gyroid", "diamond", "laminate"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_homogenize_matches_oracle(kind, precision):
    P = pfem()
    n = 8
    p, e_max = _cell(kind, n)
    kappa = 100.0 * e_max / n
    EH_ref, X_ref, _ = homog.homogenized_tensor(p, kappa)
    mesh = P.Mesh(p)
    P.pfem_mesh_set_springs(mesh, p["pairs"], kappa)
    EH, xv, infos = P.pfem_homogenize(mesh, p["coords"], tol=1e-9, precision=precision)
    assert all(i["status"] == 0 for i in infos), infos
    X = host(xv).reshape(6, -1)
    for c in range(6):
        assert rel_l2(X[c], X_ref[c]) <= 1e-6, c
    assert np.abs(EH - EH_ref).max() <= 1e-6 * np.abs(EH_ref).max()
    mesh.close()


def test_homogenize_warm_start_saves_iterations():
    """PFEM warm start of the six fluctuations: the oracle's fields plus a smooth 1% error
    (the prediction of a pretrained operator) converge in fewer iterations to the same E^H."""
    P = pfem()
    n = 10
    p, _ = _cell("gyroid", n)
    kappa = 100.0 / n
    EH_ref, X_ref, _ = homog.homogenized_tensor(p, kappa)
    mesh = P.Mesh(p)
    P.pfem_mesh_set_springs(mesh, p["pairs"], kappa)
    _, _, cold = P.pfem_homogenize(mesh, p["coords"], tol=1e-8)
    warm = np.stack([pi.make_warm_start(p, X_ref[c], seed=40 + c) for c in range(6)])
    EH, _, hot = P.pfem_homogenize(mesh, p["coords"], xv0=torch.tensor(warm, device="cuda"), tol=1e-8)
    assert sum(i["iterations"] for i in hot) < sum(i["iterations"] for i in cold)
    assert np.abs(EH - EH_ref).max() <= 1e-6 * np.abs(EH_ref).max()
    mesh.close()
