"""GPU parity of the multiplicative SAP smoother (Sec. 2, M_SAP) against the
FP64 oracle: n_cy red/black sweeps, n_mr minimal-residual steps per domain on
the Dirichlet domain operator."""
import numpy as np
import pytest

from helpers import TOL, block_coords_of_colour, fields, rel
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _op(name, prec, compress):
    from paper_2112_00501_gb300 import api

    dims, block, eps, kappa, csw, U, psi = fields(name)
    lat = api.Lattice(dims, block, -1)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=prec, compress=compress)
    return api.CloverOperator(g, kappa, csw), lat


@pytest.mark.parametrize("prec,compress", [(64, 18), (32, 18), (32, 12), (16, 18), (16, 12)])
@pytest.mark.parametrize("name", ["c0_4^4", "mid_8^4", "ragged_8x4x12x8"])
def test_sap_matches_oracle(name, prec, compress):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, prec, compress)
    got = op.sap(torch.from_numpy(psi).cuda(), prec=prec, n_cy=4, n_mr=4).cpu().numpy()
    ref = O.sap(dims, block, -1, kappa, U, O.clover(dims, kappa, csw, U), psi, ncy=4, nmr=4)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec,compress", [(64, 18), (32, 18), (16, 12)])
def test_sap_from_nonzero_guess(prec, compress):
    from paper_2112_00501_gb300 import synth

    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, prec, compress)
    x0 = synth.gaussian_spinor(dims, 321)
    got = op.sap(torch.from_numpy(psi).cuda(), prec=prec, n_cy=2, n_mr=3,
                 x0=torch.from_numpy(x0).cuda()).cpu().numpy()
    ref = O.sap(dims, block, -1, kappa, U, O.clover(dims, kappa, csw, U), psi, x0=x0, ncy=2, nmr=3)
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec,compress", [(32, 18), (16, 12), (16, 18)])
def test_sap_several_rhs_in_one_call(prec, compress):
    """Three right-hand sides in one call (one thread block per domain and
    right-hand side, the FP16 scales of each field after all their planes):
    each against the oracle's smoother on its own source."""
    from paper_2112_00501_gb300 import synth

    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, prec, compress)
    bs = synth.gaussian_spinor(dims, 4321, nrhs=3)
    bs[1] *= 1e-3  # a right-hand side of another magnitude
    got = op.sap(torch.from_numpy(bs).cuda(), prec=prec, n_cy=2, n_mr=4).cpu().numpy()
    Cl = O.clover(dims, kappa, csw, U)
    for q in range(3):
        ref = O.sap(dims, block, -1, kappa, U, Cl, bs[q], ncy=2, nmr=4)
        assert rel(got[q], ref) < TOL[prec], q


def test_sap_degenerate_counts():
    """n_cy = 0 leaves x alone; n_mr = 0 adds nothing."""
    from paper_2112_00501_gb300 import synth

    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, 64, 18)
    x0 = synth.gaussian_spinor(dims, 5)
    for n_cy, n_mr in [(0, 4), (3, 0)]:
        got = op.sap(torch.from_numpy(psi).cuda(), prec=64, n_cy=n_cy, n_mr=n_mr,
                     x0=torch.from_numpy(x0).cuda()).cpu().numpy()
        assert np.array_equal(got, x0)


def test_sap_many_mr_steps_reach_block_solves():
    """With many MR steps each domain solve converges: one sweep from 0 then
    satisfies the SAP error-propagation identity checked by the oracle pins,
    so GPU and oracle agree after 40 MR steps too."""
    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, 64, 18)
    got = op.sap(torch.from_numpy(psi).cuda(), prec=64, n_cy=1, n_mr=40).cpu().numpy()
    ref = O.sap(dims, block, -1, kappa, U, O.clover(dims, kappa, csw, U), psi, ncy=1, nmr=40)
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("prec,compress", [(16, 12), (32, 18)])
def test_full_size_32c64_one_sweep_sampled_domains(prec, compress):
    """One sweep from x = 0 on 32^3 x 64 (8192 domains) in the benchmark's
    storage format.  A red domain's result is MR_k(D_B, b_B); a black domain's
    needs its eight red neighbours first.  The oracle recomputes sampled domains
    of both colours one by one."""
    from paper_2112_00501_gb300 import synth

    name = "c2_32^3x64"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, prec, compress)
    got = op.sap(torch.from_numpy(psi).cuda(), prec=prec, n_cy=1, n_mr=4).cpu().numpy()
    g = synth.rng(99)
    red = block_coords_of_colour(dims, block, 0)
    black = block_coords_of_colour(dims, block, 1)
    nmr = 4
    errs = []
    for k in g.choice(len(red), 3, replace=False):
        bc = red[k]
        sites = O.block_sites(dims, block, bc)
        e = O.mr_block_at(dims, block, bc, kappa, csw, U, psi[sites], nmr)
        errs.append((got[sites], e))
    nb = [d // b for d, b in zip(dims, block)]
    for k in g.choice(len(black), 2, replace=False):
        bc = black[k]
        x = np.zeros_like(psi)
        for mu in range(4):
            for d in (-1, 1):
                nbc = list(bc)
                nbc[mu] = (nbc[mu] + d) % nb[mu]
                s = O.block_sites(dims, block, nbc)
                x[s] = O.mr_block_at(dims, block, nbc, kappa, csw, U, psi[s], nmr)
        sites = O.block_sites(dims, block, bc)
        r = psi[sites] - O.dirac_at(dims, -1, kappa, csw, U, x, sites)
        e = O.mr_block_at(dims, block, bc, kappa, csw, U, r, nmr)
        errs.append((got[sites], e))
    a = np.concatenate([x for x, _ in errs])
    b = np.concatenate([y for _, y in errs])
    assert rel(a, b) < TOL[prec]
