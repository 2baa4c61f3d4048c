"""GPU parity of the clover term, D and D^dagger against the FP64 oracle (Eq. (1)).

Relative L2 tolerances: 1e-12 (FP64), 1e-5 (FP32 storage), 2e-3 (FP16
storage with per-site scale), each against the FP64 oracle on the original
fields.
"""
import numpy as np
import pytest

from helpers import TOL, fields, rel
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _op(name, prec, compress, tbc=-1):
    from paper_2112_00501_gb300 import api

    dims, block, eps, kappa, csw, U, psi = fields(name)
    lat = api.Lattice(dims, block, tbc)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=prec, compress=compress)
    return api.CloverOperator(g, kappa, csw), lat


@pytest.mark.parametrize("name", ["c0_4^4", "ragged_8x4x12x8", "mid_8^4"])
def test_clover_and_inverse_match_oracle(name):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, _ = _op(name, 64, 18)
    Cg = op.export_clover().cpu().numpy()
    Co = O.clover(dims, kappa, csw, U)
    assert rel(Cg, Co) < 1e-14
    Cig = op.export_clover(inverse=True).cpu().numpy()
    assert rel(Cig, O.clover_inverse(dims, Co)) < 1e-13


@pytest.mark.parametrize("name", ["c0_4^4", "ragged_8x4x12x8", "mid_8^4"])
@pytest.mark.parametrize("tbc", [-1, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_fp64(name, tbc, dagger):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, _ = _op(name, 64, 18, tbc)
    got = op.D(torch.from_numpy(psi).cuda(), prec=64, dagger=dagger).cpu().numpy()
    ref = O.dirac(dims, tbc, kappa, U, O.clover(dims, kappa, csw, U), psi, dagger=dagger)
    assert rel(got, ref) < TOL[64]


@pytest.mark.parametrize("prec,compress", [(32, 18), (32, 12), (16, 18), (16, 12)])
@pytest.mark.parametrize("name", ["c0_4^4", "mid_8^4"])
@pytest.mark.parametrize("dagger", [False, True])
def test_dirac_low_precision(name, prec, compress, dagger):
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, _ = _op(name, prec, compress)
    got = op.D(torch.from_numpy(psi).cuda(), prec=prec, dagger=dagger).cpu().numpy()
    ref = O.dirac(dims, -1, kappa, U, O.clover(dims, kappa, csw, U), psi, dagger=dagger)
    assert rel(got, ref) < TOL[prec]


def test_multi_rhs_batch_equals_single():
    from paper_2112_00501_gb300 import synth

    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, 32, 12)
    psis = synth.gaussian_spinor(dims, 900, nrhs=3)
    batch = op.D(torch.from_numpy(psis).cuda(), prec=32).cpu().numpy()
    Cl = O.clover(dims, kappa, csw, U)
    for k in range(3):
        single = op.D(torch.from_numpy(psis[k]).cuda(), prec=32).cpu().numpy()
        assert np.array_equal(batch[k], single)
        assert rel(batch[k], O.dirac(dims, -1, kappa, U, Cl, psis[k])) < TOL[32]


def test_pack_roundtrip_and_clover_inverse_apply():
    name = "mid_8^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, 16, 12)
    x = torch.from_numpy(psi).cuda()
    assert torch.equal(lat.unpack(lat.pack(x, 64), 64), x)
    assert rel(lat.unpack(lat.pack(x, 32), 32).cpu().numpy(), psi) < 1e-7
    assert rel(lat.unpack(lat.pack(x, 16), 16).cpu().numpy(), psi) < 1e-3
    p = lat.pack(x, 64)
    back = lat.unpack(op.apply_clover(op.apply_clover(p, 64), 64, inverse=True), 64)
    assert rel(back.cpu().numpy(), psi) < 1e-14
    Cl = O.clover(dims, kappa, csw, U)
    c16 = lat.unpack(op.apply_clover(lat.pack(x, 16), 16), 16).cpu().numpy()
    assert rel(c16, np.einsum("sij,sj->si", Cl, psi.reshape(-1, 12)).reshape(psi.shape)) < TOL[16]


def test_gauge_create_rejects_non_su3_for_12_real():
    from paper_2112_00501_gb300 import _lib, api

    dims, block, eps, kappa, csw, U, psi = fields("c0_4^4")
    lat = api.Lattice(dims, block, -1)
    bad = U.copy()
    bad[5, 2] *= 1.01
    with pytest.raises(_lib.MgcError) as e:
        api.Gauge(lat, torch.from_numpy(bad).cuda(), storage_prec=16, compress=12)
    assert e.value.status == _lib.MGC_ERR_NOT_UNITARY
    api.Gauge(lat, torch.from_numpy(bad).cuda(), storage_prec=16, compress=18)


@pytest.mark.parametrize("prec,compress", [(64, 18), (32, 12), (16, 12), (16, 18)])
def test_full_size_32c64_sampled_sites(prec, compress):
    """32^3 x 64 in each storage format the benchmark times, on 2048 sampled
    sites the oracle computes one by one (its clover built on the fly)."""
    from paper_2112_00501_gb300 import synth

    name = "c2_32^3x64"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    op, lat = _op(name, prec, compress)
    got = op.D(torch.from_numpy(psi).cuda(), prec=prec).cpu().numpy()
    sites = synth.rng(77).choice(synth.volume(dims), 2048, replace=False)
    sites = np.concatenate([sites, [0, synth.volume(dims) - 1]])
    ref = O.dirac_at(dims, -1, kappa, csw, U, psi, sites)
    assert rel(got[sites], ref) < TOL[prec]
