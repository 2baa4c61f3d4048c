"""Batches of lattices through the C ABI: one launch covering every
right-hand side of every lattice.

- batched D (every launch shape the autotuner chooses among) equals the
  single-lattice D bit for bit and the FP64 oracle within each precision's
  tolerance;
- the batched smoother (captured into a CUDA graph, then replayed) equals the
  single-lattice smoother bit for bit;
- the lock-step batched two-level solve reaches ||b - D x|| / ||b|| <= 1e-10 on
  every system, measured by the oracle.
"""
import numpy as np
import pytest

from helpers import TOL, rel
from oracle import oracle as O
from paper_2112_00501_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (dims, nrhs, gauge seed index) -- same domain shape 4^4, eps 0.4, kappa 0.1355, c_sw 1
BATCH = [((8, 8, 8, 8), 3, 30), ((8, 8, 16, 8), 2, 31), ((16, 8, 8, 8), 1, 32)]
BLOCK = (4, 4, 4, 4)
EPS, KAPPA, CSW = 0.4, 0.1355, 1.0

_cache = {}


def _fields():
    if "f" not in _cache:
        out = []
        for dims, nr, ci in BATCH:
            U = synth.gauge_field(dims, EPS, synth.gauge_seed(ci))
            psi = synth.gaussian_spinor(dims, synth.source_seed(ci), nrhs=nr)
            out.append((dims, nr, U, psi))
        _cache["f"] = out
    return _cache["f"]


def _ops(prec, compress=18):
    from paper_2112_00501_gb300 import api

    ops = []
    for dims, nr, U, psi in _fields():
        lat = api.Lattice(dims, BLOCK, -1)
        g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=prec, compress=compress)
        ops.append(api.CloverOperator(g, KAPPA, CSW))
    return ops


def _oracle_D(dims, U, psi, dagger=False):
    C = O.clover(dims, KAPPA, CSW, U)
    return np.stack([O.dirac(dims, -1, KAPPA, U, C, p, dagger=dagger) for p in psi])


SHAPES = [(rb, th, rf) for rb in (1, 2, 4) for th in (128, 256) for rf in (0, 1)]


@pytest.mark.parametrize("prec,compress", [(64, 18), (32, 18), (32, 12), (16, 18), (16, 12)])
def test_batched_D_every_shape(prec, compress):
    from paper_2112_00501_gb300 import api

    ops = _ops(prec if prec != 64 else 32, compress)
    fl = _fields()
    nrhs = [nr for _, nr, _, _ in fl]
    B = api.Batch(ops, nrhs)
    assert B.systems == sum(nrhs)
    xs = [op.lattice.pack(torch.from_numpy(psi).cuda(), prec) for op, (_, _, _, psi) in zip(ops, fl)]
    for dagger in (False, True):
        ref = [(op.apply_Ddag if dagger else op.apply_D)(x, prec, nr) for op, x, nr in zip(ops, xs, nrhs)]
        want = [_oracle_D(dims, U, psi, dagger) for dims, _, U, psi in fl]
        for rb, th, rf in SHAPES:
            B.set_shape(prec, rb, th, rf, 1)
            out = B.apply_D(xs, prec, dagger=dagger)
            torch.cuda.synchronize()
            for k, (op, nr) in enumerate(zip(ops, nrhs)):
                assert torch.equal(out[k], ref[k]), (k, rb, th, rf, dagger)
                got = op.lattice.unpack(out[k], prec, nr).cpu().numpy().reshape(want[k].shape)
                assert rel(got, want[k]) < TOL[prec], (k, rb, th, rf, dagger)


def test_batched_D_autotuned():
    from paper_2112_00501_gb300 import api

    ops = _ops(16, 12)
    fl = _fields()
    nrhs = [nr for _, nr, _, _ in fl]
    B = api.Batch(ops, nrhs)
    shape = B.tune(16)
    assert shape["rhs_per_thread"] in (1, 2, 4) and shape["threads"] in (128, 256)
    assert B.tune(16) == shape  # cached
    xs = [op.lattice.pack(torch.from_numpy(psi).cuda(), 16) for op, (_, _, _, psi) in zip(ops, fl)]
    out = B.apply_D(xs, 16)
    for k, (op, nr) in enumerate(zip(ops, nrhs)):
        assert torch.equal(out[k], op.apply_D(xs[k], 16, nr))


@pytest.mark.parametrize("prec,compress", [(32, 18), (32, 12), (16, 12), (16, 18)])
def test_batched_sap_graph_equals_single(prec, compress):
    from paper_2112_00501_gb300 import api

    ops = _ops(prec, compress)
    fl = _fields()
    nrhs = [nr for _, nr, _, _ in fl]
    B = api.Batch(ops, nrhs)
    bs = [op.lattice.pack(torch.from_numpy(psi).cuda(), prec) for op, (_, _, _, psi) in zip(ops, fl)]
    for rf in (0, 1):
        B.set_shape(prec, 1, 256, 1, rf)
        xs = B.zeros_packed(prec)
        xr = [op.lattice.zeros_packed(prec, nr) for op, nr in zip(ops, nrhs)]
        # first call captures the graph, the second replays it on the updated x
        for rep in range(2):
            B.sap_smooth(bs, xs, prec, n_cy=2, n_mr=4, x_is_zero=(rep == 0))
            for op, b, x, nr in zip(ops, bs, xr, nrhs):
                op.sap_smooth(b, x, prec, nr, n_cy=2, n_mr=4, x_is_zero=(rep == 0))
            torch.cuda.synchronize()
            for k in range(len(ops)):
                assert torch.equal(xs[k], xr[k]), (k, rf, rep)
    # the smoother reduces the residual of every system
    for op, (dims, nr, U, psi), x in zip(ops, fl, xs):
        got = op.lattice.unpack(x, prec, nr).cpu().numpy().reshape(nr, -1, 4, 3)
        r = psi - _oracle_D(dims, U, got)
        for q in range(nr):
            assert np.linalg.norm(r[q]) < 0.5 * np.linalg.norm(psi[q])


def _true_res(dims, U, psi, x):
    Dx = _oracle_D(dims, U, x)
    return [float(np.linalg.norm(psi[q] - Dx[q]) / np.linalg.norm(psi[q])) for q in range(len(psi))]


@pytest.mark.parametrize("smoother,compress", [(32, 18), (16, 12)])
def test_batched_solve_reaches_1e10(smoother, compress):
    from paper_2112_00501_gb300 import api

    ops = _ops(smoother, compress)
    fl = _fields()
    nrhs = [nr for _, nr, _, _ in fl]
    B = api.Batch(ops, nrhs)
    bs = [torch.from_numpy(psi).cuda() for _, _, _, psi in fl]
    xs, infos = B.solve(bs, method=2, smoother_prec=smoother, tol=1e-10)
    assert len(infos) == sum(nrhs)
    i = 0
    for (dims, nr, U, psi), x in zip(fl, xs):
        res = _true_res(dims, U, psi, x.cpu().numpy().reshape(psi.shape))
        for q in range(nr):
            assert infos[i].status == 0 and infos[i].true_res <= 1e-10, (i, infos[i].true_res)
            assert res[q] <= 1e-10, (i, res[q])
            i += 1


def test_batched_solve_sources_far_from_unit_scale():
    """Systems whose sources are scaled by 2^-400 and 2^+400 in one batch (each
    system's inner solve works on its residual normalised to unit norm): every
    system still reaches 1e-10, and x scales with its source."""
    from paper_2112_00501_gb300 import api

    ops = _ops(16, 12)
    fl = _fields()
    nrhs = [nr for _, nr, _, _ in fl]
    B = api.Batch(ops, nrhs)
    fac = [2.0 ** -400, 2.0 ** 400, 1.0]
    bs = [torch.from_numpy(psi * f).cuda() for (_, _, _, psi), f in zip(fl, fac)]
    xs, infos = B.solve(bs, method=2, smoother_prec=16, tol=1e-10)
    assert all(i.status == 0 and i.true_res <= 1e-10 for i in infos)
    for (dims, nr, U, psi), x, f in zip(fl, xs, fac):
        res = _true_res(dims, U, psi, x.cpu().numpy().reshape(psi.shape) / f)
        assert max(res) <= 1e-10, res


def test_batched_solve_guess_zero_rhs_and_host_pointers():
    from paper_2112_00501_gb300 import api

    ops = _ops(32)
    fl = _fields()
    nrhs = [nr for _, nr, _, _ in fl]
    B = api.Batch(ops, nrhs)
    bs = [psi.copy() for _, _, _, psi in fl]
    bs[0][1] = 0.0  # one system with b = 0: its solution is 0
    xs, infos = B.solve([torch.from_numpy(b) for b in bs], method=2, smoother_prec=32, tol=1e-10)
    assert not xs[0].is_cuda
    assert infos[1].status == 0 and infos[1].iters == 0
    assert np.all(xs[0][1].numpy() == 0)
    i = 0
    for (dims, nr, U, _), b, x in zip(fl, bs, xs):
        for q in range(nr):
            if i != 1:
                xq = x.numpy()[q:q + 1]
                assert _true_res(dims, U, b[q:q + 1], xq)[0] <= 1e-10
            i += 1
    # restart from the solution: nothing left to do
    xg, ig = B.solve([torch.from_numpy(b) for b in bs], x0=xs, method=2, smoother_prec=32, tol=1e-10)
    assert all(inf.status == 0 and inf.iters == 0 for inf in ig)
    for a, b in zip(xg, xs):
        assert torch.equal(a, b)


def test_batch_rejects_mixed_formats_and_methods():
    from paper_2112_00501_gb300 import api
    from paper_2112_00501_gb300._lib import MgcError

    fl = _fields()
    a = _ops(32)
    b = _ops(16)
    with pytest.raises(MgcError):
        api.Batch([a[0], b[1]], [1, 1])  # storage precisions differ
    dims, nr, U, psi = fl[0]
    lat2 = api.Lattice(dims, (2, 2, 2, 2), -1)
    op2 = api.CloverOperator(api.Gauge(lat2, torch.from_numpy(U).cuda(), storage_prec=32), KAPPA, CSW)
    with pytest.raises(MgcError) as e:
        api.Batch([a[0], op2], [1, 1])  # SAP domain shapes differ
    assert e.value.status == 2
    B = api.Batch(a[:1], [nr])
    with pytest.raises(MgcError):
        B.solve([torch.from_numpy(psi).cuda()], method=1)
    with pytest.raises(MgcError):
        B.apply_D([a[0].lattice.zeros_packed(16, nr)], 16)  # no FP16 copy


# the benchmark's batch: 12 RHS on 24^3 x 48, 8 on 16^4, 8 on 8^4 (FP32 storage,
# 18-real links, 4^4 domains), in the launch shape bench.py times
C3 = [((24, 24, 24, 48), 12), ((16, 16, 16, 16), 8), ((8, 8, 8, 8), 8)]


def test_full_size_batched_D_sampled_sites():
    """The full-size batch in one launch (two RHS per thread, 128-thread
    blocks, the RHS groups of a site block adjacent): bit for bit the
    per-lattice operator, and on sampled sites of every RHS the oracle's D
    computed site by site."""
    from paper_2112_00501_gb300 import api

    ops, xs, fields = [], [], []
    for k, (dims, nr) in enumerate(C3):
        U = synth.gauge_field(dims, EPS, synth.gauge_seed(40 + k))
        psi = synth.gaussian_spinor(dims, synth.source_seed(40 + k), nrhs=nr)
        lat = api.Lattice(dims, BLOCK, -1)
        g = api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=32, compress=18)
        ops.append(api.CloverOperator(g, KAPPA, CSW))
        xs.append(lat.pack(torch.from_numpy(psi).cuda(), 32))
        fields.append((dims, nr, U, psi))
    B = api.Batch(ops, [nr for _, nr in C3])
    B.set_shape(32, 2, 128, 1, 1)
    out = B.apply_D(xs, 32)
    torch.cuda.synchronize()
    for k, (op, (dims, nr, U, psi)) in enumerate(zip(ops, fields)):
        assert torch.equal(out[k], op.apply_D(xs[k], 32, nr)), k
        V = synth.volume(dims)
        sites = synth.rng(90 + k).choice(V, 96, replace=False)
        sites = np.concatenate([sites, [0, V - 1]])
        got = op.lattice.unpack(out[k], 32, nr).reshape(nr, V, 4, 3)[:, torch.from_numpy(sites).cuda()]
        got = got.cpu().numpy()
        for q in range(nr):
            ref = O.dirac_at(dims, -1, KAPPA, CSW, U, psi[q], sites)
            assert rel(got[q], ref) < TOL[32], (k, q)
        del psi
