"""The link force dS/dU of S = phi^+ (D^+ D)^-1 phi: against the oracle's
analytic force, against central finite differences of S (step 1e-5, 64 random
links of an 8^4 lattice plus four along directions only the clover-leaf term
feels, each derivative within 1e-6 relative; S taken beyond double precision so
that the differences keep their digits), and through torch.autograd."""
import numpy as np
import pytest

from helpers import fields, rel
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _op(dims, block, U, kappa, csw):
    from paper_2112_00501_gb300 import api

    lat = api.Lattice(dims, block, -1)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=64)
    return api.CloverOperator(g, kappa, csw), lat


PARAMS = dict(method=0, smoother_prec=64, tol=1e-13, max_iter=2000)


@pytest.mark.parametrize("name", ["c0_4^4", "c4_8^4"])
def test_force_matches_oracle(name):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(dims, block, U, kappa, csw)
    g, S, info = op.force(torch.from_numpy(psi).cuda(), **PARAMS)
    Cl = O.clover(dims, kappa, csw, U)
    X, Y = O.force_solves(dims, block, -1, kappa, U, Cl, psi, tol=1e-13)
    go = O.force(dims, -1, kappa, csw, U, X, Y)
    assert rel(g.cpu().numpy(), go) < 1e-9
    So = 2 * np.real(np.vdot(psi, X)) - np.linalg.norm(O.dirac(dims, -1, kappa, U, Cl, X)) ** 2
    assert abs(S - So) <= 1e-11 * abs(So)


def _gell_mann():
    """The eight Gell-Mann matrices: a basis of the traceless Hermitian 3x3 matrices."""
    L = np.zeros((8, 3, 3), np.complex128)
    L[0][0, 1] = L[0][1, 0] = 1
    L[1][0, 1], L[1][1, 0] = -1j, 1j
    L[2][0, 0], L[2][1, 1] = 1, -1
    L[3][0, 2] = L[3][2, 0] = 1
    L[4][0, 2], L[4][2, 0] = -1j, 1j
    L[5][1, 2] = L[5][2, 1] = 1
    L[6][1, 2], L[6][2, 1] = -1j, 1j
    L[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return L


def test_force_central_differences_8x4():
    """Each directional derivative on its own: |fd - an| <= 1e-6 max(|an|, 1e-3 max|g|)
    (the oracle pin's criterion), on 64 random links along random su(3)
    directions, plus four links along directions orthogonal to the hopping
    term's gradient there, so that their derivative comes from the clover-leaf
    term alone."""
    from paper_2112_00501_gb300 import api, synth

    name = "c4_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(dims, block, U, kappa, csw)
    phi = torch.from_numpy(psi).cuda()
    g, S0, _ = op.force(phi, **PARAMS)
    g = g.cpu().numpy()
    V = synth.volume(dims)
    rng = synth.rng(4444)
    h = 1e-5
    floor = 1e-3 * np.abs(g).max()

    def action(Uh):
        """S as (S rounded to double, remainder): S ~ 5e4 here, whose ulp
        (7e-12) divided by 2h would be 2e-6 of a derivative of 0.2"""
        o, _ = _op(dims, block, Uh, kappa, csw)
        _, S, info = o.force(phi, action_parts=True, **PARAMS)
        assert info.status == 0
        return S

    def check(site, mu, T, what):
        w, v = np.linalg.eigh(T)
        plus, minus = U.copy(), U.copy()
        plus[site, mu] = (v * np.exp(1j * h * w)) @ v.conj().T @ U[site, mu]
        minus[site, mu] = (v * np.exp(-1j * h * w)) @ v.conj().T @ U[site, mu]
        (p0, p1), (m0, m1) = action(plus), action(minus)
        fd = ((p0 - m0) + (p1 - m1)) / (2 * h)  # p0 - m0 is exact (Sterbenz)
        an = np.real(np.sum(np.conj(g[site, mu]) * (1j * T @ U[site, mu])))
        assert abs(fd - an) <= 1e-6 * max(abs(an), floor), (what, site, mu, fd, an)
        return an

    for k in range(64):
        site, mu = int(rng.integers(V)), int(rng.integers(4))
        T = synth.random_traceless_hermitian(1, rng)[0]
        check(site, mu, T / np.linalg.norm(T), "random")

    # the hopping part of the gradient: the oracle's force with the same X, Y
    # and c_SW = 0 (its clover-leaf term vanishes, the hopping term does not
    # depend on c_SW)
    Cl = O.clover(dims, kappa, csw, U)
    X, Y = O.force_solves(dims, block, -1, kappa, U, Cl, psi, tol=1e-13)
    g_hop = O.force(dims, -1, kappa, 0.0, U, X, Y)
    g_all = O.force(dims, -1, kappa, csw, U, X, Y)
    lam = _gell_mann()
    for k in range(4):
        site, mu = int(rng.integers(V)), int(rng.integers(4))
        f = np.array([np.real(np.sum(np.conj(g_hop[site, mu]) * (1j * la @ U[site, mu]))) for la in lam])
        t = rng.normal(size=8)
        t -= (t @ f) / (f @ f) * f  # no hopping contribution along T
        T = np.einsum("a,aij->ij", t, lam)
        T /= np.linalg.norm(T)
        dU = 1j * T @ U[site, mu]
        assert abs(np.real(np.sum(np.conj(g_hop[site, mu]) * dU))) <= 1e-12 * np.abs(g_hop).max()
        clover_part = np.real(np.sum(np.conj(g_all[site, mu]) * dU))
        assert abs(clover_part) > 1e-2 * floor  # the clover-leaf term carries a derivative here
        an = check(site, mu, T, "clover-leaf only")
        assert abs(an - clover_part) <= 1e-9 * np.abs(g).max()


def test_autograd_function():
    from paper_2112_00501_gb300 import api
    from paper_2112_00501_gb300.autograd import fermion_action

    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    lat = api.Lattice(dims, block, -1)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    phi = torch.from_numpy(psi).cuda()
    S = fermion_action(Ut, phi, lat, kappa, csw, **PARAMS)
    (grad,) = torch.autograd.grad(S, Ut)
    op, _ = _op(dims, block, U, kappa, csw)
    g, S2, _ = op.force(phi, **PARAMS)
    assert abs(float(S.detach()) - S2) <= 1e-12 * abs(S2)
    assert rel(grad.cpu().numpy(), g.cpu().numpy()) < 1e-12
