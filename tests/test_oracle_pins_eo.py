"""Pins of the oracle's even-odd preconditioned block MR (DD-alphaAMG's SAP
domain solver, the f1 variant): the Schur complement MR steps in closed form
from the dense domain operator, convergence to the dense domain solve, and
the SAP sweep with converged domain solves."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_00501_gb300 import synth

from test_oracle_pins import dense

DIMS, BD = (4, 4, 4, 4), (2, 2, 2, 2)
KAPPA = 0.125


@pytest.fixture(scope="module")
def fields():
    U = synth.gauge_field(DIMS, 0.4, synth.gauge_seed(0))
    Cl = O.clover(DIMS, KAPPA, 1.0, U)
    Ci = O.clover_inverse(DIMS, Cl)
    return U, Cl, Ci


def _parity(bd):
    VB = int(np.prod(bd))
    par = []
    for l in range(VB):
        t, s = l, 0
        for b in bd:
            s += t % b
            t //= b
        par.append(s & 1)
    return np.repeat(np.array(par), 12)


@pytest.mark.parametrize("nmr", [1, 2, 3])
def test_eo_mr_closed_form(fields, nmr):
    """e_e = MR_k on Dh = D_ee - D_eo D_oo^-1 D_oe with rh = r_e - D_eo D_oo^-1 r_o,
    e_o = D_oo^-1 (r_o - D_oe e_e), with the blocks of the dense D_B."""
    U, Cl, Ci = fields
    bc = (1, 0, 0, 1)
    VB = int(np.prod(BD))
    D = dense(lambda v: O.dirac_block(DIMS, BD, bc, KAPPA, U, Cl, v.reshape(VB, 4, 3)), 12 * VB)
    par = _parity(BD)
    E, Od = np.where(par == 0)[0], np.where(par == 1)[0]
    Dee, Deo, Doe, Doo = D[np.ix_(E, E)], D[np.ix_(E, Od)], D[np.ix_(Od, E)], D[np.ix_(Od, Od)]
    Dooi = np.linalg.inv(Doo)
    Dh = Dee - Deo @ Dooi @ Doe
    r = synth.gaussian_spinor(BD, 101).reshape(-1)
    rho = r[E] - Deo @ Dooi @ r[Od]
    ee = np.zeros_like(rho)
    for _ in range(nmr):
        p = Dh @ rho
        alpha = np.vdot(p, rho) / np.vdot(p, p)
        ee = ee + alpha * rho
        rho = rho - alpha * p
    want = np.zeros_like(r)
    want[E] = ee
    want[Od] = Dooi @ (r[Od] - Doe @ ee)
    got = O.mr_eo_block(DIMS, BD, bc, KAPPA, U, Cl, Ci, r.reshape(VB, 4, 3), nmr).reshape(-1)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_eo_mr_converges_to_dense_solve(fields):
    U, Cl, Ci = fields
    bc = (0, 1, 1, 0)
    VB = int(np.prod(BD))
    D = dense(lambda v: O.dirac_block(DIMS, BD, bc, KAPPA, U, Cl, v.reshape(VB, 4, 3)), 12 * VB)
    r = synth.gaussian_spinor(BD, 102).reshape(-1)
    got = O.mr_eo_block(DIMS, BD, bc, KAPPA, U, Cl, Ci, r.reshape(VB, 4, 3), 200).reshape(-1)
    exact = np.linalg.solve(D, r)
    assert np.linalg.norm(got - exact) <= 1e-11 * np.linalg.norm(exact)


def test_sap_eo_with_converged_blocks_matches_exact_formula(fields):
    U, Cl, Ci = fields
    V = synth.volume(DIMS)
    D = dense(lambda v: O.dirac(DIMS, -1, KAPPA, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    K = [np.zeros((12 * V, 12 * V), np.complex128) for _ in range(2)]
    for bt in range(2):
        for bz in range(2):
            for by in range(2):
                for bx in range(2):
                    sites = O.block_sites(DIMS, BD, (bx, by, bz, bt))
                    idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
                    K[(bx + by + bz + bt) % 2][np.ix_(idx, idx)] = np.linalg.inv(D[np.ix_(idx, idx)])
    b = synth.gaussian_spinor(DIMS, 103).reshape(-1)
    x = np.zeros_like(b)
    x = x + K[0] @ (b - D @ x)
    x = x + K[1] @ (b - D @ x)
    got = O.sap_eo(DIMS, BD, -1, KAPPA, U, Cl, Ci, b.reshape(V, 4, 3), ncy=1, nmr=120)
    assert np.linalg.norm(got.reshape(-1) - x) <= 1e-11 * np.linalg.norm(x)
    # a few steps: the even-odd solver reduces the domain residual more than plain MR
    VB = int(np.prod(BD))
    bc = (1, 1, 0, 0)
    Db = dense(lambda v: O.dirac_block(DIMS, BD, bc, KAPPA, U, Cl, v.reshape(VB, 4, 3)), 12 * VB)
    r = synth.gaussian_spinor(BD, 104).reshape(-1)
    e_eo = O.mr_eo_block(DIMS, BD, bc, KAPPA, U, Cl, Ci, r.reshape(VB, 4, 3), 4).reshape(-1)
    e_mr = O.mr_block(DIMS, BD, bc, KAPPA, U, Cl, r.reshape(VB, 4, 3), 4).reshape(-1)
    assert np.linalg.norm(r - Db @ e_eo) < np.linalg.norm(r - Db @ e_mr)
