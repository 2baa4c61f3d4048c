"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

The paper prints no worked example, so each part of the oracle is pinned by a
closed form, an identity of the mathematics, brute-force dense linear algebra
or finite differences:
  - gamma algebra (Clifford relations) and the chiral-basis structure;
  - the free-field (unit link) spectrum in momentum space, which fixes the
    hopping sign, projectors, kappa normalisation and the antiperiodic t
    boundary;
  - D^dagger as the conjugate transpose, and gamma5-hermiticity, which fix the
    placement of U versus U^dagger in the two hops;
  - covariance under a random SU(3) gauge transformation (hopping and clover);
  - the constant abelian field, which fixes the clover normalisation of
    Eq. (1) (sigma, F, the 1/8 and the factor i kappa c_SW);
  - dense block matrices and dense LU solves for the Dirichlet block operator,
    the minimal-residual block solve, the multiplicative SAP sweep and the
    outer solvers;
  - central finite differences of S for the force;
  - the degenerate parameters (kappa = 0: D = 1; c_SW = 0: C = 1; a zero
    field), where the operator, the smoother and the solve reduce to the
    identity.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_00501_gb300 import synth


def dense(apply, n):
    """Dense matrix of a linear map on C^n, column by column."""
    M = np.zeros((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = apply(e).reshape(n)
    return M


def coords(dims):
    V = synth.volume(dims)
    s = np.arange(V)
    c = np.zeros((V, 4), int)
    for mu in range(4):
        c[:, mu] = s % dims[mu]
        s = s // dims[mu]
    return c


# ---------------------------------------------------------------- gamma basis

def test_gamma_clifford_and_chiral_basis():
    g = O.gamma()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]), atol=1e-15)
    sig = O.sigma()
    for mu in range(4):
        for nu in range(4):
            s = sig[mu, nu]
            assert np.allclose(s, s.conj().T)
            # chiral basis: every sigma_{mu nu} commutes with gamma5 (block diagonal)
            assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)
            assert np.allclose(s, -sig[nu, mu])


# ---------------------------------------------------------------- free field

@pytest.mark.parametrize("tbc", [-1, 1])
def test_free_field_spectrum(tbc):
    """U = 1 (so F = 0, C = 1): the eigenvalues of D are
    1 - 2 kappa sum cos p_mu +- 2 i kappa sqrt(sum sin^2 p_mu), six-fold each,
    with p_k = 2 pi n / L_k and p_t = (2n + 1) pi / L_t when antiperiodic."""
    dims = (3, 4, 2, 4)
    kappa = 0.11
    V = synth.volume(dims)
    U = synth.unit_gauge(dims)
    Cl = O.clover(dims, kappa, 1.0, U)
    assert np.allclose(Cl, np.eye(12)[None], atol=1e-15)
    D = dense(lambda v: O.dirac(dims, tbc, kappa, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    ev = np.linalg.eigvals(D)
    pred = []
    shift = 0.5 if tbc == -1 else 0.0
    for nx in range(dims[0]):
        for ny in range(dims[1]):
            for nz in range(dims[2]):
                for nt in range(dims[3]):
                    p = 2 * np.pi * np.array([nx / dims[0], ny / dims[1], nz / dims[2],
                                              (nt + shift) / dims[3]])
                    a = 1 - 2 * kappa * np.cos(p).sum()
                    b = 2 * kappa * np.sqrt((np.sin(p) ** 2).sum())
                    pred += [a + 1j * b] * 6 + [a - 1j * b] * 6
    pred = np.array(pred)
    key = lambda z: np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))
    assert np.allclose(ev[key(ev)], pred[key(pred)], atol=1e-10)


def test_free_field_plane_wave():
    """D (u e^{ipx}) = (1 - 2 kappa sum cos p + 2 i kappa sum gamma_mu sin p_mu) u e^{ipx}."""
    dims = (4, 6, 4, 8)
    kappa = 0.13
    V = synth.volume(dims)
    U = synth.unit_gauge(dims)
    Cl = O.clover(dims, kappa, 1.0, U)
    g = O.gamma()
    c = coords(dims)
    rng = synth.rng(5)
    for n in [(1, 2, 3, 0), (0, 1, 1, 3), (3, 5, 2, 7)]:
        p = 2 * np.pi * np.array([n[0] / 4, n[1] / 6, n[2] / 4, (n[3] + 0.5) / 8])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * c @ p)
        psi = phase[:, None, None] * u[None]
        Dp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
            g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (Dp @ u)[None]
        got = O.dirac(dims, -1, kappa, U, Cl, psi)
        assert np.allclose(got, expect, atol=1e-12)


# ---------------------------------------------------------------- adjoint / gamma5

def test_dagger_is_adjoint_and_gamma5_hermiticity():
    dims = (2, 2, 2, 2)
    V = synth.volume(dims)
    kappa, csw = 0.13, 1.3
    U = synth.gauge_field(dims, 0.6, 11)
    Cl = O.clover(dims, kappa, csw, U)
    D = dense(lambda v: O.dirac(dims, -1, kappa, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    Dd = dense(lambda v: O.dirac(dims, -1, kappa, U, Cl, v.reshape(V, 4, 3), dagger=True), 12 * V)
    assert np.allclose(Dd, D.conj().T, atol=1e-14)
    g5 = np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.allclose(g5 @ D @ g5, D.conj().T, atol=1e-14)
    # and on a larger lattice through inner products
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.4, 12)
    Cl = O.clover(dims, kappa, csw, U)
    phi = synth.gaussian_spinor(dims, 13)
    psi = synth.gaussian_spinor(dims, 14)
    lhs = np.vdot(phi, O.dirac(dims, -1, kappa, U, Cl, psi))
    rhs = np.vdot(O.gamma5(O.dirac(dims, -1, kappa, U, Cl, O.gamma5(phi))), psi)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- gauge covariance

def test_gauge_covariance():
    """U'_mu(x) = W(x) U_mu(x) W(x+mu)^dagger implies D[U'] (W psi) = W D[U] psi,
    clover term included (the leaves are closed loops at x)."""
    dims = (4, 4, 4, 4)
    V = synth.volume(dims)
    kappa, csw = 0.125, 1.0
    U = synth.gauge_field(dims, 0.4, 21)
    W = synth.random_su3(V, synth.rng(22))
    c = coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        cp = c.copy()
        cp[:, mu] = (cp[:, mu] + 1) % dims[mu]
        fwd = cp[:, 0] + dims[0] * (cp[:, 1] + dims[1] * (cp[:, 2] + dims[2] * cp[:, 3]))
        Up[:, mu] = W @ U[:, mu] @ np.conj(np.swapaxes(W[fwd], 1, 2))
    psi = synth.gaussian_spinor(dims, 23)
    Cl = O.clover(dims, kappa, csw, U)
    Clp = O.clover(dims, kappa, csw, Up)
    lhs = O.dirac(dims, -1, kappa, Up, Clp, np.einsum("sab,sib->sia", W, psi))
    rhs = np.einsum("sab,sib->sia", W, O.dirac(dims, -1, kappa, U, Cl, psi))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)
    # the clover alone transforms as W C W^dagger
    W12 = np.einsum("ij,sab->siajb", np.eye(4), W).reshape(V, 12, 12)
    assert np.allclose(Clp, W12 @ Cl @ np.conj(np.swapaxes(W12, 1, 2)), atol=1e-13)


# ---------------------------------------------------------------- clover

@pytest.mark.parametrize("n", [1, 2])
def test_clover_constant_abelian_field(n):
    """U_x(x) = diag(e^{i phi y}, e^{-i phi y}, 1), phi = 2 pi n / L_y, all other
    links 1.  Every x-y plaquette is diag(e^{-i phi}, e^{i phi}, 1), so
    Q_xy = 4 diag(e^{-i phi}, e^{i phi}, 1), F_xy = -i sin(phi) diag(1, -1, 0)
    and every other plane has F = 0.  Then C - 1 = kappa c_SW sin(phi)
    sigma_xy (x) diag(1, -1, 0), whose eigenvalues are +-kappa c_SW sin(phi)
    (four each) and 0 (four)."""
    dims = (4, 6, 4, 4)
    Ly = dims[1]
    phi = 2 * np.pi * n / Ly
    kappa, csw = 0.13, 1.7
    U = synth.unit_gauge(dims)
    c = coords(dims)
    U[:, 0, 0, 0] = np.exp(1j * phi * c[:, 1])
    U[:, 0, 1, 1] = np.exp(-1j * phi * c[:, 1])
    for site in [0, 17, 55, 300]:
        F = O.field_strength_site(dims, U, site)
        expect = np.zeros((6, 3, 3), np.complex128)
        expect[0] = -1j * np.sin(phi) * np.diag([1, -1, 0])
        assert np.allclose(F, expect, atol=1e-14)
    Cl = O.clover(dims, kappa, csw, U)
    sig = O.sigma()
    expectC = np.eye(12) + kappa * csw * np.sin(phi) * np.kron(sig[0, 1], np.diag([1, -1, 0]))
    assert np.allclose(Cl, expectC[None], atol=1e-14)
    ev = np.sort(np.linalg.eigvalsh(Cl[0] - np.eye(12)))
    a = kappa * csw * np.sin(phi)
    assert np.allclose(ev, np.sort([-a] * 4 + [0] * 4 + [a] * 4), atol=1e-14)


def test_clover_structure_and_inverse():
    dims = (4, 4, 4, 4)
    kappa = 0.125
    U = synth.gauge_field(dims, 0.4, 31)
    C1 = O.clover(dims, kappa, 1.0, U)
    C2 = O.clover(dims, kappa, 2.5, U)
    # Hermitian, chirally block diagonal, linear in c_SW
    assert np.allclose(C1, np.conj(np.swapaxes(C1, 1, 2)), atol=1e-15)
    assert np.allclose(C1[:, :6, 6:], 0, atol=0) and np.allclose(C1[:, 6:, :6], 0, atol=0)
    assert np.allclose(C2 - np.eye(12), 2.5 * (C1 - np.eye(12)), atol=1e-14)
    Ci = O.clover_inverse(dims, C1)
    assert np.allclose(C1 @ Ci, np.eye(12)[None], atol=1e-14)
    ref = np.linalg.inv(C1[:8])
    assert np.allclose(Ci[:8], ref, atol=1e-13)


# ---------------------------------------------------------------- block operator

def test_dirichlet_block_operator_2x4_blocks():
    """With 2^4 blocks on a 4^4 lattice no hop inside a block wraps, so D_B is
    exactly the block-site submatrix of the dense D."""
    dims, bd = (4, 4, 4, 4), (2, 2, 2, 2)
    V = synth.volume(dims)
    kappa = 0.125
    U = synth.gauge_field(dims, 0.4, 41)
    Cl = O.clover(dims, kappa, 1.0, U)
    D = dense(lambda v: O.dirac(dims, -1, kappa, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    for bc in [(0, 0, 0, 0), (1, 0, 1, 1), (1, 1, 1, 1)]:
        sites = O.block_sites(dims, bd, bc)
        idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
        DB = dense(lambda v: O.dirac_block(dims, bd, bc, kappa, U, Cl, v.reshape(16, 4, 3)), 192)
        assert np.allclose(DB, D[np.ix_(idx, idx)], atol=1e-15)
        DBd = dense(lambda v: O.dirac_block(dims, bd, bc, kappa, U, Cl, v.reshape(16, 4, 3),
                                            dagger=True), 192)
        assert np.allclose(DBd, DB.conj().T, atol=1e-15)


@pytest.fixture(scope="module")
def single_block_4x4():
    """One 4^4 block covering a 4^4 lattice (every wrap-around hop cut)."""
    dims = (4, 4, 4, 4)
    V = synth.volume(dims)
    kappa = 0.125
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(0))
    Cl = O.clover(dims, kappa, 1.0, U)
    DB = dense(lambda v: O.dirac_block(dims, dims, (0, 0, 0, 0), kappa, U, Cl,
                                       v.reshape(V, 4, 3)), 12 * V)
    return dims, V, kappa, U, Cl, DB


def test_dirichlet_block_operator_single_block(single_block_4x4):
    """D_B equals the dense D with exactly the wrap-around hop entries removed."""
    dims, V, kappa, U, Cl, DB = single_block_4x4
    D = dense(lambda v: O.dirac(dims, -1, kappa, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    c = coords(dims)
    diff = np.abs(c[:, None, :] - c[None, :, :])
    wrap = np.any(diff == 3, axis=2)              # neighbours only across the boundary
    mask = np.kron(wrap, np.ones((12, 12), bool))
    assert np.count_nonzero(D[mask]) > 0
    assert np.allclose(DB[~mask], D[~mask], atol=1e-15)
    assert np.all(DB[mask] == 0)


def test_mr_converges_to_dense_lu(single_block_4x4):
    """Many MR steps on the 4^4 block reach the dense LU solution of D_B e = r,
    and the MR residual norm never increases."""
    dims, V, kappa, U, Cl, DB = single_block_4x4
    r = synth.gaussian_spinor(dims, 51)
    exact = np.linalg.solve(DB, r.reshape(-1))
    e = O.mr_block(dims, dims, (0, 0, 0, 0), kappa, U, Cl, r, 300)
    assert np.linalg.norm(e.reshape(-1) - exact) <= 1e-11 * np.linalg.norm(exact)
    norms = []
    for k in range(0, 8):
        _, rk = O.mr_block(dims, dims, (0, 0, 0, 0), kappa, U, Cl, r, k, return_residual=True)
        norms.append(np.linalg.norm(rk))
        # the residual the iteration carries is the true block residual
        ek = O.mr_block(dims, dims, (0, 0, 0, 0), kappa, U, Cl, r, k)
        assert np.allclose(rk.reshape(-1), r.reshape(-1) - DB @ ek.reshape(-1), atol=1e-12)
    assert all(b <= a * (1 + 1e-14) for a, b in zip(norms, norms[1:]))
    assert norms[-1] < 0.5 * norms[0]


def test_mr_one_step_minimises_along_r(single_block_4x4):
    """After one step, r1 = r - alpha D_B r is orthogonal to D_B r (the defining
    property of the minimal-residual step length)."""
    dims, V, kappa, U, Cl, DB = single_block_4x4
    r = synth.gaussian_spinor(dims, 52).reshape(-1)
    _, r1 = O.mr_block(dims, dims, (0, 0, 0, 0), kappa, U, Cl, r.reshape(V, 4, 3), 1,
                       return_residual=True)
    p = DB @ r
    assert abs(np.vdot(p, r1.reshape(-1))) <= 1e-12 * np.linalg.norm(p) * np.linalg.norm(r)


# ---------------------------------------------------------------- SAP

def test_sap_sweep_matches_exact_block_formula():
    """With converged block solves, one multiplicative sweep is
    x1 = x0 + K_red (b - D x0), x2 = x1 + K_black (b - D x1) with
    K_c = sum_{B of colour c} P_B D_B^-1 P_B^T, built densely."""
    dims, bd = (4, 4, 4, 4), (2, 2, 2, 2)
    V = synth.volume(dims)
    kappa = 0.125
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(0))
    Cl = O.clover(dims, kappa, 1.0, U)
    D = dense(lambda v: O.dirac(dims, -1, kappa, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    K = [np.zeros((12 * V, 12 * V), np.complex128) for _ in range(2)]
    for bt in range(2):
        for bz in range(2):
            for by in range(2):
                for bx in range(2):
                    sites = O.block_sites(dims, bd, (bx, by, bz, bt))
                    idx = (sites[:, None] * 12 + np.arange(12)[None]).reshape(-1)
                    col = (bx + by + bz + bt) % 2
                    K[col][np.ix_(idx, idx)] = np.linalg.inv(D[np.ix_(idx, idx)])
    b = synth.gaussian_spinor(dims, synth.source_seed(0)).reshape(-1)
    x0 = synth.gaussian_spinor(dims, 61).reshape(-1)
    x = x0.copy()
    for _ in range(2):
        x = x + K[0] @ (b - D @ x)
        x = x + K[1] @ (b - D @ x)
    got = O.sap(dims, bd, -1, kappa, U, Cl, b.reshape(V, 4, 3), x0.reshape(V, 4, 3), ncy=2,
                nmr=120)
    assert np.linalg.norm(got.reshape(-1) - x) <= 1e-11 * np.linalg.norm(x)
    # black-then-red is a different operator: the colour order is observable
    xr = x0.copy()
    xr = xr + K[1] @ (b - D @ xr)
    xr = xr + K[0] @ (b - D @ xr)
    one = O.sap(dims, bd, -1, kappa, U, Cl, b.reshape(V, 4, 3), x0.reshape(V, 4, 3), ncy=1,
                nmr=120)
    assert np.linalg.norm(one.reshape(-1) - xr) > 1e-3 * np.linalg.norm(xr)


# ---------------------------------------------------------------- solvers

@pytest.mark.parametrize("method", ["fgcr", "fbicgstab"])
@pytest.mark.parametrize("precond", ["sap", "none"])
def test_solver_matches_dense_lu(method, precond):
    dims, bd = (4, 4, 4, 4), (2, 2, 2, 2)
    V = synth.volume(dims)
    kappa = 0.125
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(0))
    Cl = O.clover(dims, kappa, 1.0, U)
    b = synth.gaussian_spinor(dims, synth.source_seed(0))
    x, st, it, res = O.solve(dims, bd, -1, kappa, U, Cl, b, method=method, precond=precond,
                             tol=1e-10, max_iter=2000)
    assert st == 0 and res <= 1e-10
    r = b - O.dirac(dims, -1, kappa, U, Cl, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    D = dense(lambda v: O.dirac(dims, -1, kappa, U, Cl, v.reshape(V, 4, 3)), 12 * V)
    exact = np.linalg.solve(D, b.reshape(-1))
    cond = np.linalg.cond(D)
    assert np.linalg.norm(x.reshape(-1) - exact) <= 2e-10 * cond * np.linalg.norm(exact)


# ---------------------------------------------------------------- force

def _su3_direction(rng):
    h = synth.random_traceless_hermitian(1, rng)[0]
    return h / np.linalg.norm(h)


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_force_matches_central_differences(csw):
    """dS/dh at h = 0 for U_mu(x) -> exp(i h T) U_mu(x) (T traceless Hermitian)
    and for single real / imaginary entries, by central differences with
    h = 1e-5, against Re sum conj(g) dU/dh from the analytic force."""
    dims, bd = (4, 4, 4, 4), (2, 2, 2, 2)
    kappa, tbc = 0.125, -1
    U = synth.gauge_field(dims, 0.4, 71)
    phi = synth.gaussian_spinor(dims, 72)
    Cl = O.clover(dims, kappa, csw, U)
    X, Y = O.force_solves(dims, bd, tbc, kappa, U, Cl, phi)
    g = O.force(dims, tbc, kappa, csw, U, X, Y)
    rng = synth.rng(73)
    V = synth.volume(dims)
    h = 1e-5
    cases = []
    # links on the antiperiodic t boundary and in the bulk
    for _ in range(4):
        cases.append((int(rng.integers(V)), int(rng.integers(4)), "su3"))
    cases.append((V - 1, 3, "su3"))
    cases.append((int(rng.integers(V)), int(rng.integers(4)), "re"))
    cases.append((int(rng.integers(V)), int(rng.integers(4)), "im"))
    for site, mu, kind in cases:
        if kind == "su3":
            T = _su3_direction(rng)
            dU = 1j * T @ U[site, mu]

            def pert(hh):
                w, v = np.linalg.eigh(T)
                E = (v * np.exp(1j * hh * w)) @ v.conj().T
                Up = U.copy()
                Up[site, mu] = E @ U[site, mu]
                return Up
        else:
            a, b = rng.integers(3), rng.integers(3)
            dU = np.zeros((3, 3), np.complex128)
            dU[a, b] = 1.0 if kind == "re" else 1j

            def pert(hh, dU=dU):
                Up = U.copy()
                Up[site, mu] = U[site, mu] + hh * dU
                return Up
        fd = (O.action(dims, bd, tbc, kappa, csw, pert(h), phi)
              - O.action(dims, bd, tbc, kappa, csw, pert(-h), phi)) / (2 * h)
        an = np.real(np.sum(np.conj(g[site, mu]) * dU))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(g).max()), (site, mu, kind, fd, an)


def test_mr_block_at_equals_mr_block():
    """The on-the-fly-clover MR used for sampled large-lattice checks is the same
    computation as MR with the stored clover field."""
    dims, bd = (8, 8, 4, 8), (4, 4, 2, 4)
    kappa, csw = 0.1355, 1.0
    U = synth.gauge_field(dims, 0.4, 81)
    Cl = O.clover(dims, kappa, csw, U)
    r = synth.gaussian_spinor(bd, 82)
    for bc in [(0, 1, 1, 0), (1, 1, 0, 1)]:
        a = O.mr_block(dims, bd, bc, kappa, U, Cl, r, 4)
        b = O.mr_block_at(dims, bd, bc, kappa, csw, U, r, 4)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tbc", [-1, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_at_equals_dirac(tbc, dagger):
    """The sampled operator that checks the full-size Dslash and solves (its
    clover term built on the fly at each listed site) is the same computation as
    the pinned whole-lattice D, bit for bit: on every site of a non-cubic
    lattice, and on a list with repeats, both t boundaries and the x wrap."""
    dims = (4, 6, 4, 8)
    kappa, csw = 0.1355, 1.0
    U = synth.gauge_field(dims, 0.4, 91)
    Cl = O.clover(dims, kappa, csw, U)
    psi = synth.gaussian_spinor(dims, 92)
    V = synth.volume(dims)
    full = O.dirac(dims, tbc, kappa, U, Cl, psi, dagger=dagger)
    assert np.array_equal(O.dirac_at(dims, tbc, kappa, csw, U, psi, np.arange(V), dagger=dagger), full)
    Lx, Ly, Lz, Lt = dims
    idx = lambda x, y, z, t: x + Lx * (y + Ly * (z + Lz * t))  # noqa: E731
    sites = [idx(0, 0, 0, 0), idx(Lx - 1, 2, 1, Lt - 1), idx(3, Ly - 1, Lz - 1, 0), idx(1, 1, 1, 3), 7, 7]
    assert np.array_equal(O.dirac_at(dims, tbc, kappa, csw, U, psi, sites, dagger=dagger), full[sites])


# ---------------------------------------------------------------- degenerate parameters

def test_degenerate_parameters():
    """kappa = 0 makes C = 1 and D = 1 exactly, so one MR step solves every
    domain (p = r, alpha = 1) and one SAP sweep returns x = b, and the solve
    returns b; c_SW = 0 makes C = 1 exactly (D = 1 - kappa H, whose hopping
    part is pinned by the free-field and gauge-covariance tests); a zero field
    stays zero."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    V = synth.volume(dims)
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(0))
    psi = synth.gaussian_spinor(dims, synth.source_seed(0))
    eye = np.broadcast_to(np.eye(12, dtype=np.complex128), (V, 12, 12))
    C0 = O.clover(dims, 0.0, 1.3, U)
    assert np.array_equal(C0, eye)
    assert np.array_equal(O.clover(dims, 0.13, 0.0, U), eye)
    assert np.array_equal(O.dirac(dims, -1, 0.0, U, C0, psi), psi)
    x = O.sap(dims, block, -1, 0.0, U, C0, psi, ncy=1, nmr=1)
    assert np.abs(x - psi).max() <= 1e-14 * np.abs(psi).max()
    xs, st, it, res = O.solve(dims, block, -1, 0.0, U, C0, psi, tol=1e-12)
    assert st == 0 and np.abs(xs - psi).max() <= 1e-12 * np.abs(psi).max()
    Cl = O.clover(dims, 0.13, 1.0, U)
    z = np.zeros_like(psi)
    assert np.array_equal(O.dirac(dims, -1, 0.13, U, Cl, z), z)
    assert np.array_equal(O.sap(dims, block, -1, 0.13, U, Cl, z, ncy=2, nmr=3), z)


def test_sap_same_colour_block_order_invariance():
    """Blocks of one colour share no hop, so a sweep does not depend on the
    order it visits them in: a sweep composed from the pinned block MR over
    each colour's blocks in a shuffled order (each block's residual from the
    current x) equals the oracle's sweep, with a finite MR step count."""
    dims, bd = (4, 4, 8, 4), (2, 2, 2, 2)
    V = synth.volume(dims)
    kappa = 0.13
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(2))
    Cl = O.clover(dims, kappa, 1.0, U)
    b = synth.gaussian_spinor(dims, synth.source_seed(2))
    x0 = synth.gaussian_spinor(dims, 62)
    nb = [d // k for d, k in zip(dims, bd)]
    blocks = [[], []]
    for bt in range(nb[3]):
        for bz in range(nb[2]):
            for by in range(nb[1]):
                for bx in range(nb[0]):
                    blocks[(bx + by + bz + bt) % 2].append((bx, by, bz, bt))
    rng = synth.rng(63)
    for trial in range(2):
        x = x0.copy()
        for col in (0, 1):
            order = list(blocks[col])
            rng.shuffle(order)
            for bc in order:
                sites = O.block_sites(dims, bd, bc)
                r = (b - O.dirac(dims, -1, kappa, U, Cl, x))[sites]
                x[sites] += O.mr_block(dims, bd, bc, kappa, U, Cl, r, 3).reshape(len(sites), 4, 3)
        want = O.sap(dims, bd, -1, kappa, U, Cl, b, x0, ncy=1, nmr=3)
        assert np.linalg.norm(x - want) <= 1e-13 * np.linalg.norm(want), trial


def test_force_richardson_cross_check():
    """The force against differences at larger steps, where rounding in S is
    negligible: central differences at h = 1e-3 and 1e-4 combined by
    Richardson extrapolation (error O(h^4)) along random su(3) directions,
    with the clover term on, agree with the analytic force to 1e-7."""
    dims, bd = (4, 4, 4, 4), (2, 2, 2, 2)
    kappa, csw, tbc = 0.125, 1.0, -1
    U = synth.gauge_field(dims, 0.4, 81)
    phi = synth.gaussian_spinor(dims, 82)
    Cl = O.clover(dims, kappa, csw, U)
    X, Y = O.force_solves(dims, bd, tbc, kappa, U, Cl, phi)
    g = O.force(dims, tbc, kappa, csw, U, X, Y)
    rng = synth.rng(83)
    V = synth.volume(dims)
    for _ in range(3):
        site, mu = int(rng.integers(V)), int(rng.integers(4))
        T = _su3_direction(rng)
        w, v = np.linalg.eigh(T)

        def S(hh):
            Up = U.copy()
            Up[site, mu] = ((v * np.exp(1j * hh * w)) @ v.conj().T) @ U[site, mu]
            return O.action(dims, bd, tbc, kappa, csw, Up, phi)

        d = {h: (S(h) - S(-h)) / (2 * h) for h in (1e-3, 1e-4)}
        fd = (100.0 * d[1e-4] - d[1e-3]) / 99.0
        an = np.real(np.sum(np.conj(g[site, mu]) * (1j * T @ U[site, mu])))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * np.abs(g).max()), (site, mu, fd, an)
