"""GPU parity of QWS's pieces (Sec. 2) against the FP64 oracle, through the
C ABI: the clover-preconditioned operator A = C^-1 D, the clover inverse at
every precision, the SAP smoother for A with a fixed number of Jacobi
iterations per domain, and the QWS solve (FP64 Richardson around an FP32
BiCGStab on A M_SAP) to a true residual of 1e-10."""
import numpy as np
import pytest

from helpers import TOL, block_coords_of_colour, fields, rel
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
    return api.CloverOperator(g, kappa, csw), lat


CASES = [(64, 18), (32, 18), (32, 12), (16, 18), (16, 12)]
NAMES = ["c0_4^4", "mid_8^4", "ragged_8x4x12x8"]


@pytest.mark.parametrize("prec,compress", CASES)
@pytest.mark.parametrize("name", NAMES)
def test_apply_A_matches_oracle(name, prec, compress):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, prec if prec != 64 else 32, compress)
    got = op.A(torch.from_numpy(psi).cuda(), prec=prec).cpu().numpy()
    ref = O.apply_A(dims, -1, kappa, U, Cl, Ci, psi)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [64, 32, 16])
def test_clover_inverse_every_precision(prec):
    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, prec if prec != 64 else 32)
    x = lat.pack(torch.from_numpy(psi).cuda(), prec)
    got = lat.unpack(op.apply_clover(x, prec, inverse=True), prec).cpu().numpy()
    ref = np.einsum("xij,xj->xi", Ci, psi.reshape(-1, 12)).reshape(psi.shape)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec,compress", CASES)
@pytest.mark.parametrize("name", NAMES)
def test_sap_A_matches_oracle(name, prec, compress):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, prec if prec != 64 else 32, compress)
    got = op.sap_A(torch.from_numpy(psi).cuda(), prec=prec, n_cy=4, n_jacobi=4).cpu().numpy()
    ref = O.sap_A(dims, block, -1, kappa, U, Cl, Ci, psi, ncy=4, nj=4)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_sap_A_nonzero_guess_and_degenerate_counts(prec):
    from paper_2112_00501_gb300 import synth

    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, 32)
    x0 = synth.gaussian_spinor(dims, 81)
    got = op.sap_A(torch.from_numpy(psi).cuda(), prec=prec, n_cy=2, n_jacobi=3,
                   x0=torch.from_numpy(x0).cuda()).cpu().numpy()
    ref = O.sap_A(dims, block, -1, kappa, U, Cl, Ci, psi, x0=x0, ncy=2, nj=3)
    assert rel(got, ref) < TOL[prec]
    # one Jacobi iteration is e = r_B; zero iterations leave x unchanged
    for nj in (0, 1):
        got = op.sap_A(torch.from_numpy(psi).cuda(), prec=prec, n_cy=1, n_jacobi=nj,
                       x0=torch.from_numpy(x0).cuda()).cpu().numpy()
        ref = O.sap_A(dims, block, -1, kappa, U, Cl, Ci, psi, x0=x0, ncy=1, nj=nj)
        assert rel(got, ref) < TOL[prec]
    assert np.array_equal(O.sap_A(dims, block, -1, kappa, U, Cl, Ci, psi, x0=x0, ncy=1, nj=0), x0)


def test_sap_A_many_jacobi_steps_reach_block_solves():
    """With many iterations the Jacobi domain solve converges, so one colour
    launch from x = 0 leaves x_B = A_B^-1 b_B on every red domain."""
    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, 32)
    got = op.sap_A(torch.from_numpy(psi).cuda(), prec=64, n_cy=1, n_jacobi=200).cpu().numpy()
    ref = O.sap_A(dims, block, -1, kappa, U, Cl, Ci, psi, ncy=1, nj=200)
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("prec,compress", [(16, 12), (32, 18)])
def test_full_size_32c64_sap_A_sampled_domains(prec, compress):
    """One sweep from x = 0 on 32^3 x 64 in the benchmark's storage format: a
    red domain's result is Jacobi(A_B, b_B); a black domain's needs its eight
    red neighbours first.  Sampled domains are recomputed by the oracle."""
    from paper_2112_00501_gb300 import synth

    name = "c2_32^3x64"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, prec, compress)
    nj = 4
    got = op.sap_A(torch.from_numpy(psi).cuda(), prec=prec, n_cy=1, n_jacobi=nj).cpu().numpy()
    g = synth.rng(98)
    red = block_coords_of_colour(dims, block, 0)
    black = block_coords_of_colour(dims, block, 1)
    pairs = []
    for k in g.choice(len(red), 3, replace=False):
        bc = red[k]
        sites = O.block_sites(dims, block, bc)
        pairs.append((got[sites], O.jacobi_block_at(dims, block, bc, kappa, csw, U, psi[sites], nj)))
    nb = [d // b for d, b in zip(dims, block)]
    for k in g.choice(len(black), 2, replace=False):
        bc = black[k]
        x = np.zeros_like(psi)
        for mu in range(4):
            for d in (-1, 1):
                nbc = list(bc)
                nbc[mu] = (nbc[mu] + d) % nb[mu]
                s = O.block_sites(dims, block, nbc)
                x[s] = O.jacobi_block_at(dims, block, nbc, kappa, csw, U, psi[s], nj)
        sites = O.block_sites(dims, block, bc)
        Dx = O.dirac_at(dims, -1, kappa, csw, U, x, sites)
        Ax = np.stack([O.invert(O.clover_site(dims, kappa, csw, U, s)) @ Dx[q].reshape(12)
                       for q, s in enumerate(sites)]).reshape(Dx.shape)
        pairs.append((got[sites], O.jacobi_block_at(dims, block, bc, kappa, csw, U, psi[sites] - Ax, nj)))
    a = np.concatenate([p for p, _ in pairs])
    b = np.concatenate([q for _, q in pairs])
    assert rel(a, b) < TOL[prec]


@pytest.mark.parametrize("smoother,compress", [(32, 18), (16, 12)])
@pytest.mark.parametrize("name", ["c0_4^4", "mid_8^4"])
def test_qws_solve_reaches_1e10(name, smoother, compress):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, smoother, compress)
    x, info = op.solve(torch.from_numpy(psi).cuda(), method=3, smoother_prec=smoother, n_mr=4, tol=1e-10)
    assert info.status == 0 and info.true_res <= 1e-10
    xr = x.cpu().numpy()
    r = psi - O.dirac(dims, -1, kappa, U, Cl, xr)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(psi)
    xo, st, it, res = O.solve_qws(dims, block, -1, kappa, U, Cl, Ci, psi, ncy=4, nj=4, tol=1e-12)
    assert st == 0
    assert rel(xr, xo) < 1e-8


def test_qws_solve_host_pointers_guess_and_bad_params():
    from paper_2112_00501_gb300._lib import MgcError

    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    Cl, Ci = _clover(name)
    op, lat = _op(name, 32)
    x, info = op.solve(psi, method=3, smoother_prec=32)
    assert not x.is_cuda and info.status == 0
    x2, info2 = op.solve(psi, method=3, smoother_prec=32, x0=x)
    assert info2.status == 0 and info2.iters == 0
    with pytest.raises(MgcError):
        op.solve(torch.from_numpy(psi).cuda(), method=3, precond=0)
    with pytest.raises(MgcError):
        op.solve(torch.from_numpy(psi).cuda(), method=3, smoother_prec=64)
