"""The link force dS/dU of S = phi^+ (D^+ D)^-1 phi: against the oracle's
analytic force, against central finite differences of S (step 1e-5, 64 random
links of an 8^4 lattice, relative agreement 1e-6), and through torch.autograd."""
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


def test_force_central_differences_8x4():
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

    def action(Uh):
        o, _ = _op(dims, block, Uh, kappa, csw)
        _, S, info = o.force(phi, **PARAMS)
        assert info.status == 0
        return S

    fds, ans = [], []
    for k in range(64):
        site, mu = int(rng.integers(V)), int(rng.integers(4))
        T = synth.random_traceless_hermitian(1, rng)[0]
        T /= np.linalg.norm(T)
        w, v = np.linalg.eigh(T)
        plus, minus = U.copy(), U.copy()
        plus[site, mu] = (v * np.exp(1j * h * w)) @ v.conj().T @ U[site, mu]
        minus[site, mu] = (v * np.exp(-1j * h * w)) @ v.conj().T @ U[site, mu]
        fds.append((action(plus) - action(minus)) / (2 * h))
        ans.append(np.real(np.sum(np.conj(g[site, mu]) * (1j * T @ U[site, mu]))))
    # relative L2 agreement over the 64 directional derivatives
    assert rel(np.array(fds), np.array(ans)) < 1e-6


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
