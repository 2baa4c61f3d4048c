"""GPU parity of the smoother with even-odd preconditioned MR domain solves
(DD-alphaAMG's block solver) against the FP64 oracle, and the two-level solve
with it as the smoother."""
import numpy as np
import pytest

from helpers import TOL, fields, rel
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_cl = {}


def _clover(name):
    if name not in _cl:
        dims, block, eps, kappa, csw, U, psi = fields(name)
        Cl = O.clover(dims, kappa, csw, U)
        _cl[name] = (Cl, O.clover_inverse(dims, Cl))
    return _cl[name]


def _op(name, prec, compress=18):
    from paper_2112_00501_gb300 import api

    dims, block, eps, kappa, csw, U, psi = fields(name)
    lat = api.Lattice(dims, block, -1)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=prec, compress=compress)
    return api.CloverOperator(g, kappa, csw)


@pytest.mark.parametrize("prec,compress", [(64, 18), (32, 18), (32, 12), (16, 18), (16, 12)])
@pytest.mark.parametrize("name", ["c0_4^4", "mid_8^4", "ragged_8x4x12x8"])
def test_sap_eo_matches_oracle(name, prec, compress):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op = _op(name, prec if prec != 64 else 32, compress)
    got = op.sap_eo(torch.from_numpy(psi).cuda(), prec=prec, n_cy=4, n_mr=4).cpu().numpy()
    ref = O.sap_eo(dims, block, -1, kappa, U, Cl, Ci, psi, ncy=4, nmr=4)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_sap_eo_nonzero_guess_and_zero_steps(prec):
    from paper_2112_00501_gb300 import synth

    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op = _op(name, 32)
    x0 = synth.gaussian_spinor(dims, 111)
    for nmr in (0, 3):
        got = op.sap_eo(torch.from_numpy(psi).cuda(), prec=prec, n_cy=2, n_mr=nmr,
                        x0=torch.from_numpy(x0).cuda()).cpu().numpy()
        ref = O.sap_eo(dims, block, -1, kappa, U, Cl, Ci, psi, x0=x0, ncy=2, nmr=nmr)
        assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("smoother,compress", [(32, 18), (16, 12)])
def test_two_level_solve_with_eo_smoother(smoother, compress):
    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, _ = _clover(name)
    op = _op(name, smoother, compress)
    x, info = op.solve(torch.from_numpy(psi).cuda(), method=2, smoother_prec=smoother, sap_solver=2, tol=1e-10)
    assert info.status == 0 and info.true_res <= 1e-10
    r = psi - O.dirac(dims, -1, kappa, U, Cl, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(psi)


def test_bad_sap_solver_rejected():
    from paper_2112_00501_gb300._lib import MgcError

    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op = _op(name, 32)
    with pytest.raises(MgcError):
        op.solve(torch.from_numpy(psi).cuda(), sap_solver=1)
