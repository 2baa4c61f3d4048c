"""Pins of the oracle's two-level multigrid (Sec. 3): block-orthonormal
null-vector basis, restriction R = P^dagger and prolongation P, the coarse
operator D_c = R D P as a 9-point stencil (including coarse extents 1 and 2),
its gamma5-hermiticity, the coarse BiCGStab, the two-level preconditioner,
the setup and the multigrid solve."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_00501_gb300 import synth

from test_oracle_pins import dense

DIMS, BD = (4, 4, 4, 4), (2, 2, 2, 2)
KAPPA = 0.125
NVEC = 3
# (2,2,2,2): coarse 2^4; (4,2,2,4): coarse extents 1,2,2,1 (self-neighbours)
AGGS = [(2, 2, 2, 2), (4, 2, 2, 4)]


@pytest.fixture(scope="module")
def fields():
    V = synth.volume(DIMS)
    U = synth.gauge_field(DIMS, 0.4, synth.gauge_seed(0))
    Cl = O.clover(DIMS, KAPPA, 1.0, U)
    Ci = O.clover_inverse(DIMS, Cl)
    Vin = synth.gaussian_spinor(DIMS, 90, nrhs=NVEC)
    return V, U, Cl, Ci, Vin


def _agg_masks(agg):
    """List of (site index array) per aggregate, coarse lexicographic order."""
    Lc = [d // a for d, a in zip(DIMS, agg)]
    out = []
    for at in range(Lc[3]):
        for az in range(Lc[2]):
            for ay in range(Lc[1]):
                for ax in range(Lc[0]):
                    out.append(O.block_sites(DIMS, agg, (ax, ay, az, at)))
    return out


@pytest.mark.parametrize("agg", AGGS)
def test_basis_orthonormal_and_same_span(fields, agg):
    V, U, Cl, Ci, Vin = fields
    W, bad = O.mg_basis(DIMS, agg, Vin)
    assert bad == 0
    for sites in _agg_masks(agg):
        for chi in range(2):
            sl = slice(2 * chi, 2 * chi + 2)
            Wb = W[:, sites, sl, :].reshape(NVEC, -1)
            Vb = Vin[:, sites, sl, :].reshape(NVEC, -1)
            assert np.allclose(Wb.conj() @ Wb.T, np.eye(NVEC), atol=1e-13)
            # V restricted lies in the span of W restricted
            proj = (Vb @ Wb.conj().T) @ Wb
            assert np.linalg.norm(proj - Vb) <= 1e-12 * np.linalg.norm(Vb)
            # Gram-Schmidt order: W_0 is V_0 normalised
            assert np.allclose(Wb[0], Vb[0] / np.linalg.norm(Vb[0]), atol=1e-13)


@pytest.mark.parametrize("agg", AGGS)
def test_restrict_is_adjoint_of_prolong(fields, agg):
    V, U, Cl, Ci, Vin = fields
    W, _ = O.mg_basis(DIMS, agg, Vin)
    Vc = O.coarse_volume(DIMS, agg)
    g = synth.rng(91)
    u = g.normal(size=(Vc, 2, NVEC)) + 1j * g.normal(size=(Vc, 2, NVEC))
    v = synth.gaussian_spinor(DIMS, 92)
    lhs = np.vdot(u, O.mg_restrict(DIMS, agg, W, v))
    rhs = np.vdot(O.mg_prolong(DIMS, agg, W, u), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert np.allclose(O.mg_restrict(DIMS, agg, W, O.mg_prolong(DIMS, agg, W, u)), u, atol=1e-13)


@pytest.mark.parametrize("agg", AGGS)
def test_coarse_operator_is_galerkin(fields, agg):
    """D_c u = R D P u for random u: the stencil assembled per hop direction
    reproduces the Galerkin operator, also when a coarse extent is 1 or 2."""
    V, U, Cl, Ci, Vin = fields
    W, _ = O.mg_basis(DIMS, agg, Vin)
    Dc = O.mg_coarse_op(DIMS, agg, -1, KAPPA, U, Cl, W)
    Vc = O.coarse_volume(DIMS, agg)
    g = synth.rng(93)
    for _ in range(2):
        u = g.normal(size=(Vc, 2, NVEC)) + 1j * g.normal(size=(Vc, 2, NVEC))
        want = O.mg_restrict(DIMS, agg, W, O.dirac(DIMS, -1, KAPPA, U, Cl, O.mg_prolong(DIMS, agg, W, u)))
        got = O.mg_coarse_apply(DIMS, agg, Dc, u)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_coarse_operator_gamma5_hermitian(fields):
    """With chirality-split aggregates gamma5 P = P Gamma5_c, so
    Gamma5_c D_c Gamma5_c = D_c^dagger."""
    V, U, Cl, Ci, Vin = fields
    agg = AGGS[0]
    W, _ = O.mg_basis(DIMS, agg, Vin)
    Dc = O.mg_coarse_op(DIMS, agg, -1, KAPPA, U, Cl, W)
    Vc = O.coarse_volume(DIMS, agg)
    n = Vc * 2 * NVEC
    M = dense(lambda u: O.mg_coarse_apply(DIMS, agg, Dc, u.reshape(Vc, 2, NVEC)), n)
    g5 = np.tile(np.repeat([1.0, -1.0], NVEC), Vc)
    assert np.linalg.norm(g5[:, None] * M * g5[None, :] - M.conj().T) <= 1e-12 * np.linalg.norm(M)


def test_coarse_bicgstab_matches_dense_solve(fields):
    V, U, Cl, Ci, Vin = fields
    agg = AGGS[0]
    W, _ = O.mg_basis(DIMS, agg, Vin)
    Dc = O.mg_coarse_op(DIMS, agg, -1, KAPPA, U, Cl, W)
    Vc = O.coarse_volume(DIMS, agg)
    n = Vc * 2 * NVEC
    M = dense(lambda u: O.mg_coarse_apply(DIMS, agg, Dc, u.reshape(Vc, 2, NVEC)), n)
    g = synth.rng(94)
    b = g.normal(size=n) + 1j * g.normal(size=n)
    x, st, it = O.mg_coarse_solve(DIMS, agg, Dc, b.reshape(Vc, 2, NVEC), tol=1e-12, maxit=2000)
    assert st == 0
    exact = np.linalg.solve(M, b)
    assert np.linalg.norm(x.reshape(-1) - exact) <= 1e-10 * np.linalg.cond(M) * np.linalg.norm(exact)


def test_two_level_preconditioner_composition(fields):
    """With an exact coarse solve, B v = x0 + M_A(C^-1 (v - D x0)), x0 = P D_c^-1 R v,
    M_A = n_cy sweeps of the SAP for A from zero (each piece pinned on its own)."""
    V, U, Cl, Ci, Vin = fields
    agg = AGGS[0]
    W, _ = O.mg_basis(DIMS, agg, Vin)
    Dc = O.mg_coarse_op(DIMS, agg, -1, KAPPA, U, Cl, W)
    Vc = O.coarse_volume(DIMS, agg)
    n = Vc * 2 * NVEC
    M = dense(lambda u: O.mg_coarse_apply(DIMS, agg, Dc, u.reshape(Vc, 2, NVEC)), n)
    v = synth.gaussian_spinor(DIMS, 95)
    uc = np.linalg.solve(M, O.mg_restrict(DIMS, agg, W, v).reshape(-1))
    x0 = O.mg_prolong(DIMS, agg, W, uc.reshape(Vc, 2, NVEC))
    r = v - O.dirac(DIMS, -1, KAPPA, U, Cl, x0)
    ra = np.einsum("xij,xj->xi", np.linalg.inv(Cl), r.reshape(V, 12)).reshape(V, 4, 3)
    want = x0 + O.sap_A(DIMS, BD, -1, KAPPA, U, Cl, Ci, ra, ncy=2, nj=3)
    got = O.mg_precond(DIMS, BD, agg, -1, KAPPA, U, Cl, Ci, W, Dc, v, ncy=2, nj=3, ctol=1e-14, cmaxit=5000)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_setup_is_sap_then_adaptive_passes(fields):
    V, U, Cl, Ci, Vin = fields
    agg = AGGS[0]
    eta = synth.gaussian_spinor(DIMS, 96, nrhs=NVEC)
    # no adaptive pass: W from V_i = M_SAP(C^-1 eta_i)
    W0, Dc0, bad = O.mg_setup(DIMS, BD, agg, -1, KAPPA, U, Cl, Ci, eta, ncy=2, nj=3, n_adapt=0)
    assert bad == 0
    Cinv = np.linalg.inv(Cl)
    V0 = np.stack([O.sap_A(DIMS, BD, -1, KAPPA, U, Cl, Ci,
                           np.einsum("xij,xj->xi", Cinv, e.reshape(V, 12)).reshape(V, 4, 3), ncy=2, nj=3)
                   for e in eta])
    Wr, _ = O.mg_basis(DIMS, agg, V0)
    assert np.linalg.norm(W0 - Wr) <= 1e-12 * np.linalg.norm(Wr)
    assert np.linalg.norm(Dc0 - O.mg_coarse_op(DIMS, agg, -1, KAPPA, U, Cl, Wr)) <= 1e-12 * np.linalg.norm(Dc0)
    # one adaptive pass: V_i <- B V_i with the first basis, then rebuild
    W1, Dc1, _ = O.mg_setup(DIMS, BD, agg, -1, KAPPA, U, Cl, Ci, eta, ncy=2, nj=3, n_adapt=1, ctol=1e-3)
    V1 = np.stack([O.mg_precond(DIMS, BD, agg, -1, KAPPA, U, Cl, Ci, W0, Dc0, v, ncy=2, nj=3, ctol=1e-3)
                   for v in V0])
    W1r, _ = O.mg_basis(DIMS, agg, V1)
    assert np.linalg.norm(W1 - W1r) <= 1e-12 * np.linalg.norm(W1r)


def test_multigrid_solve_matches_dense_lu(fields):
    V, U, Cl, Ci, Vin = fields
    agg = AGGS[0]
    eta = synth.gaussian_spinor(DIMS, 97, nrhs=NVEC)
    W, Dc, _ = O.mg_setup(DIMS, BD, agg, -1, KAPPA, U, Cl, Ci, eta, ncy=2, nj=3, n_adapt=2)
    b = synth.gaussian_spinor(DIMS, synth.source_seed(0))
    x, st, it, res = O.solve_mg(DIMS, BD, agg, -1, KAPPA, U, Cl, Ci, W, Dc, b, ncy=2, nj=3, tol=1e-10)
    assert st == 0 and res <= 1e-10
    D = dense(lambda v: O.dirac(DIMS, -1, KAPPA, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    r = b.reshape(-1) - D @ x.reshape(-1)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    exact = np.linalg.solve(D, b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - exact) <= 2e-10 * np.linalg.cond(D) * np.linalg.norm(exact)


def test_coarse_operator_is_galerkin_extent_4():
    """A coarse extent of 4 (t) separates the +mu and -mu neighbours and puts
    the antiperiodic boundary between distinct aggregates."""
    dims, agg = (4, 4, 4, 8), (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(7))
    Cl = O.clover(dims, KAPPA, 1.0, U)
    W, bad = O.mg_basis(dims, agg, synth.gaussian_spinor(dims, 98, nrhs=NVEC))
    assert bad == 0
    Dc = O.mg_coarse_op(dims, agg, -1, KAPPA, U, Cl, W)
    Vc = O.coarse_volume(dims, agg)
    g = synth.rng(99)
    u = g.normal(size=(Vc, 2, NVEC)) + 1j * g.normal(size=(Vc, 2, NVEC))
    want = O.mg_restrict(dims, agg, W, O.dirac(dims, -1, KAPPA, U, Cl, O.mg_prolong(dims, agg, W, u)))
    got = O.mg_coarse_apply(dims, agg, Dc, u)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
