"""The operator, the smoother and the solve at the method's degenerate
parameters, on the GPU against results that Eq. (1) and the minimal-residual
step of Sec. 2 fix in closed form (not only against the oracle):

- kappa = 0: C = 1 and D = 1, so D psi = psi, and one MR step solves every
  Dirichlet domain exactly (p = r, alpha = 1): one sweep gives x = b;
- c_SW = 0: C = 1 exactly and D = 1 - kappa H;
- the free field (every link the identity): every plaquette is 1, so F = 0
  and C = 1 exactly, and a plane wave u e^{ipx} (t momentum shifted by half a
  unit for the antiperiodic t boundary) is an eigenvector of D whose 4x4
  symbol 1 - 2 kappa sum_mu cos p_mu + 2 i kappa sum_mu gamma_mu sin p_mu
  acts on u;
- a zero field: D 0 = 0 and the smoother leaves x = 0, at every storage.
"""
import numpy as np
import pytest

from helpers import TOL, fields, rel
from oracle import oracle as O
from paper_2112_00501_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STORAGES = [(64, 18), (32, 18), (32, 12), (16, 18), (16, 12)]


def _op(dims, block, U, kappa, csw, prec, compress, tbc=-1):
    from paper_2112_00501_gb300 import api

    lat = api.Lattice(dims, block, tbc)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=prec, compress=compress)
    return api.CloverOperator(g, kappa, csw)


def _identity_clover(V):
    return np.broadcast_to(np.eye(12, dtype=np.complex128), (V, 12, 12))


@pytest.mark.parametrize("prec,compress", STORAGES)
def test_kappa_zero_is_the_identity(prec, compress):
    """kappa = 0: C = 1 bit for bit, D psi = psi (exactly at FP64, to the
    storage's rounding otherwise), and one sweep of one MR step gives x = b."""
    dims, block, eps, kappa, csw, U, psi = fields("ragged_8x4x12x8")
    op = _op(dims, block, U, 0.0, csw, prec, compress)
    V = synth.volume(dims)
    assert np.array_equal(op.export_clover().cpu().numpy(), _identity_clover(V))
    assert np.array_equal(op.export_clover(inverse=True).cpu().numpy(), _identity_clover(V))
    for dagger in (False, True):
        got = op.D(torch.from_numpy(psi).cuda(), prec=prec, dagger=dagger).cpu().numpy()
        if prec == 64:
            assert np.array_equal(got, psi)
        else:
            assert rel(got, psi) < TOL[prec]
    x = op.sap(torch.from_numpy(psi).cuda(), prec=prec, n_cy=1, n_mr=1).cpu().numpy()
    assert rel(x, psi) < (1e-14 if prec == 64 else TOL[prec])


@pytest.mark.parametrize("prec,compress", STORAGES)
def test_csw_zero_is_plain_wilson(prec, compress):
    """c_SW = 0: C = 1 bit for bit and D = 1 - kappa H, against the oracle's
    operator with the unit clover term; the smoother likewise."""
    dims, block, eps, kappa, csw, U, psi = fields("mid_8^4")
    op = _op(dims, block, U, kappa, 0.0, prec, compress)
    V = synth.volume(dims)
    assert np.array_equal(op.export_clover().cpu().numpy(), _identity_clover(V))
    Cl = O.clover(dims, kappa, 0.0, U)
    assert np.array_equal(Cl.reshape(V, 12, 12), _identity_clover(V))
    got = op.D(torch.from_numpy(psi).cuda(), prec=prec).cpu().numpy()
    assert rel(got, O.dirac(dims, -1, kappa, U, Cl, psi)) < TOL[prec]
    x = op.sap(torch.from_numpy(psi).cuda(), prec=prec, n_cy=2, n_mr=4).cpu().numpy()
    assert rel(x, O.sap(dims, block, -1, kappa, U, Cl, psi, ncy=2, nmr=4)) < TOL[prec]


@pytest.mark.parametrize("prec,compress", STORAGES)
def test_free_field_plane_waves(prec, compress):
    """Unit links: C = 1 for any c_SW, and D maps u e^{ipx} to (D(p) u) e^{ipx}
    with the closed-form symbol above, D^dagger to (D(p)^dagger u) e^{ipx}."""
    dims, block = (8, 4, 12, 8), (2, 2, 2, 2)
    kappa, csw = 0.13, 1.7
    V = synth.volume(dims)
    U = synth.unit_gauge(dims)
    op = _op(dims, block, U, kappa, csw, prec, compress)
    assert np.array_equal(op.export_clover().cpu().numpy(), _identity_clover(V))
    s = np.arange(V)
    c = np.zeros((V, 4), int)
    for mu in range(4):
        c[:, mu] = s % dims[mu]
        s = s // dims[mu]
    g = O.gamma()
    rng = synth.rng(77)
    for n in [(1, 2, 3, 0), (0, 1, 5, 3), (7, 3, 2, 7), (0, 0, 0, 0)]:
        p = 2 * np.pi * np.array([n[0] / dims[0], n[1] / dims[1], n[2] / dims[2], (n[3] + 0.5) / dims[3]])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (c @ p))
        psi = phase[:, None, None] * u[None]
        Dp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
            g[mu] * np.sin(p[mu]) for mu in range(4))
        for dagger, M in ((False, Dp), (True, Dp.conj().T)):
            got = op.D(torch.from_numpy(psi).cuda(), prec=prec, dagger=dagger).cpu().numpy()
            expect = phase[:, None, None] * (M @ u)[None]
            assert rel(got, expect) < TOL[prec], (n, dagger)


@pytest.mark.parametrize("prec,compress", STORAGES)
def test_zero_field_stays_zero(prec, compress):
    """D 0 = 0 and the smoother on b = 0 gives x = 0 exactly (the FP16 storage's
    per-site scale is 0 there, never a division by it)."""
    dims, block, eps, kappa, csw, U, psi = fields("c0_4^4")
    op = _op(dims, block, U, kappa, csw, prec, compress)
    z = torch.zeros((synth.volume(dims), 4, 3), dtype=torch.complex128, device="cuda")
    for dagger in (False, True):
        assert float(op.D(z, prec=prec, dagger=dagger).abs().max()) == 0.0
    assert float(op.sap(z, prec=prec, n_cy=2, n_mr=3).abs().max()) == 0.0


@pytest.mark.parametrize("method,prec,compress", [(0, 16, 12), (1, 32, 18), (2, 16, 12), (2, 32, 18), (3, 16, 12)])
def test_kappa_zero_solve_returns_the_source(method, prec, compress):
    """kappa = 0 (D = 1, A = C^-1 D = 1): every solver converges, and its x is
    b to 1e-10 (a smoother that solves every domain to its storage's precision
    must not break the Krylov recurrences)."""
    dims, block, eps, kappa, csw, U, psi = fields("mid_8^4")
    op = _op(dims, block, U, 0.0, csw, prec, compress)
    x, info = op.solve(torch.from_numpy(psi).cuda(), method=method, smoother_prec=prec, tol=1e-10)
    assert info.status == 0
    assert rel(x.cpu().numpy(), psi) <= 1e-10
