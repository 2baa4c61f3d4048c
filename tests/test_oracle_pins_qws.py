"""Pins of the oracle's QWS pieces (Sec. 2): the clover-preconditioned
operator A = C^-1 D, the fixed-count Jacobi domain solve on A_B, the SAP
sweep on A, and the QWS solver (Richardson around BiCGStab on A M_SAP)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_00501_gb300 import synth

from test_oracle_pins import dense

DIMS, BD = (4, 4, 4, 4), (2, 2, 2, 2)
KAPPA = 0.125


@pytest.fixture(scope="module")
def fields():
    V = synth.volume(DIMS)
    U = synth.gauge_field(DIMS, 0.4, synth.gauge_seed(0))
    Cl = O.clover(DIMS, KAPPA, 1.0, U)
    Ci = O.clover_inverse(DIMS, Cl)
    return V, U, Cl, Ci


def test_apply_A_is_one_minus_kappa_Cinv_H(fields):
    """A psi = psi - kappa C^-1 H psi, with kappa H psi taken from the c_SW = 0
    operator (C = 1: D0 = 1 - kappa H) and C^-1 by numpy."""
    V, U, Cl, Ci = fields
    psi = synth.gaussian_spinor(DIMS, 71)
    one = np.broadcast_to(np.eye(12, dtype=np.complex128), (V, 12, 12)).copy()
    kH = psi - O.dirac(DIMS, -1, KAPPA, U, one, psi)
    Cinv = np.linalg.inv(Cl)
    want = psi - np.einsum("xij,xj->xi", Cinv, kH.reshape(V, 12)).reshape(V, 4, 3)
    got = O.apply_A(DIMS, -1, KAPPA, U, Cl, Ci, psi)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
    # c_SW = 0: C = 1 and A = D
    C0 = O.clover(DIMS, KAPPA, 0.0, U)
    assert np.allclose(C0, one, atol=0)
    assert np.array_equal(O.apply_A(DIMS, -1, KAPPA, U, C0, C0, psi), O.dirac(DIMS, -1, KAPPA, U, C0, psi))


def _dense_AB(fields, bc):
    """Dense A_B = C_B^-1 D_B of one domain (local lexicographic order)."""
    V, U, Cl, Ci = fields
    VB = int(np.prod(BD))
    DB = dense(lambda v: O.dirac_block(DIMS, BD, bc, KAPPA, U, Cl, v.reshape(VB, 4, 3)), 12 * VB)
    sites = O.block_sites(DIMS, BD, bc)
    CB = np.zeros((12 * VB, 12 * VB), np.complex128)
    for l, s in enumerate(sites):
        CB[12 * l:12 * l + 12, 12 * l:12 * l + 12] = Cl[s]
    return np.linalg.inv(CB) @ DB


@pytest.mark.parametrize("nj", [1, 2, 5])
def test_jacobi_block_is_neumann_polynomial(fields, nj):
    """nj iterations from e = 0 give e = sum_{i<nj} (1 - A_B)^i r."""
    V, U, Cl, Ci = fields
    bc = (1, 0, 1, 0)
    A = _dense_AB(fields, bc)
    VB = int(np.prod(BD))
    r = synth.gaussian_spinor(BD, 72).reshape(-1)
    K = np.eye(12 * VB) - A
    want = np.zeros_like(r)
    term = r.copy()
    for _ in range(nj):
        want += term
        term = K @ term
    got = O.jacobi_block(DIMS, BD, bc, KAPPA, U, Cl, Ci, r.reshape(VB, 4, 3), nj).reshape(-1)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


def test_jacobi_block_converges_to_dense_solve(fields):
    V, U, Cl, Ci = fields
    bc = (0, 1, 1, 1)
    A = _dense_AB(fields, bc)
    VB = int(np.prod(BD))
    K = np.eye(12 * VB) - A
    rho = max(abs(np.linalg.eigvals(K)))
    assert rho < 0.9, rho  # the iteration converges on these fields
    r = synth.gaussian_spinor(BD, 73).reshape(-1)
    got = O.jacobi_block(DIMS, BD, bc, KAPPA, U, Cl, Ci, r.reshape(VB, 4, 3), 400).reshape(-1)
    exact = np.linalg.solve(A, r)
    assert np.linalg.norm(got - exact) <= 1e-11 * np.linalg.norm(exact)


def test_sap_A_matches_dense_polynomial_formula(fields):
    """Two sweeps with nj = 3: x <- x + J_c (b - A x), c = red then black,
    J_c = sum_{B of colour c} P_B [sum_{i<3} (1 - A_B)^i] P_B^T, built densely;
    the colour order is observable."""
    V, U, Cl, Ci = fields
    n = 12 * V
    A = dense(lambda v: O.apply_A(DIMS, -1, KAPPA, U, Cl, Ci, v.reshape(V, 4, 3)), n)
    J = [np.zeros((n, n), np.complex128) for _ in range(2)]
    for bt in range(2):
        for bz in range(2):
            for by in range(2):
                for bx in range(2):
                    bc = (bx, by, bz, bt)
                    sites = O.block_sites(DIMS, BD, bc)
                    idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
                    AB = A[np.ix_(idx, idx)]
                    KB = np.eye(len(idx)) - AB
                    P = np.eye(len(idx)) + KB + KB @ KB
                    J[(bx + by + bz + bt) % 2][np.ix_(idx, idx)] = P
    b = synth.gaussian_spinor(DIMS, 74).reshape(-1)
    x0 = synth.gaussian_spinor(DIMS, 75).reshape(-1)
    x = x0.copy()
    for _ in range(2):
        x = x + J[0] @ (b - A @ x)
        x = x + J[1] @ (b - A @ x)
    got = O.sap_A(DIMS, BD, -1, KAPPA, U, Cl, Ci, b.reshape(V, 4, 3), x0.reshape(V, 4, 3), ncy=2, nj=3)
    assert np.linalg.norm(got.reshape(-1) - x) <= 1e-12 * np.linalg.norm(x)
    xr = x0 + J[1] @ (b - A @ x0)
    xr = xr + J[0] @ (b - A @ xr)
    one = O.sap_A(DIMS, BD, -1, KAPPA, U, Cl, Ci, b.reshape(V, 4, 3), x0.reshape(V, 4, 3), ncy=1, nj=3)
    assert np.linalg.norm(one.reshape(-1) - xr) > 1e-3 * np.linalg.norm(xr)


def test_qws_solver_matches_dense_lu(fields):
    V, U, Cl, Ci = fields
    b = synth.gaussian_spinor(DIMS, synth.source_seed(0))
    x, st, it, res = O.solve_qws(DIMS, BD, -1, KAPPA, U, Cl, Ci, b, ncy=4, nj=4, tol=1e-10, inner_tol=1e-6)
    assert st == 0 and res <= 1e-10
    D = dense(lambda v: O.dirac(DIMS, -1, KAPPA, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    r = b.reshape(-1) - D @ x.reshape(-1)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    exact = np.linalg.solve(D, b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - exact) <= 2e-10 * np.linalg.cond(D) * np.linalg.norm(exact)


def test_jacobi_block_at_equals_jacobi_block(fields):
    V, U, Cl, Ci = fields
    bc = (1, 1, 0, 1)
    VB = int(np.prod(BD))
    r = synth.gaussian_spinor(BD, 76)
    a = O.jacobi_block(DIMS, BD, bc, KAPPA, U, Cl, Ci, r, 4)
    b = O.jacobi_block_at(DIMS, BD, bc, KAPPA, 1.0, U, r, 4)
    assert np.array_equal(a, b)
    assert a.shape == (VB, 4, 3)
