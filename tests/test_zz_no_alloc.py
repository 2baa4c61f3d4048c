"""mgc_solve_noalloc, the allocation-free variant of mgc_solve, for callers that
cannot call cudaMalloc at solve time (their device memory is all held by
another allocator, or a cudaMalloc/cudaFree pair would synchronise the device
inside a loop that must not stall).

Called through the C ABI twice in a row on a freshly created operator (the
second call finds the previous call's contents in the shared scratch array),
with the device's free memory unchanged by each call; each solution is checked
against the oracle (its true residual recomputed with the oracle's D) and
against mgc_solve's solution of the same system with the same method, which is
called only afterwards so that none of its lazily created workspace exists
while the allocation-free calls run.  Its size limit and method restriction are
checked too.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from helpers import TOL, fields, rel
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _operator(dims, block, U, kappa, csw):
    from paper_2112_00501_gb300 import api

    lat = api.Lattice(dims, block, -1)
    gauge = api.Gauge(lat, torch.as_tensor(U).cuda(), storage_prec=16, compress=12)
    return api.CloverOperator(gauge, kappa, csw), gauge, lat


def _noalloc(lib, op, b, x, stream, **kw):
    from paper_2112_00501_gb300 import _lib, api

    p = api.solve_params(method=1, smoother_prec=16, tol=1e-10, on_device=1, **kw)
    info = _lib.SolveInfo()
    st = lib.mgc_solve_noalloc(op.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(p),
                               C.byref(info), stream)
    return st, info


def test_noalloc_solve_matches_oracle_and_mgc_solve_on_two_calls():
    from paper_2112_00501_gb300 import _lib, api

    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    dims, block, eps, kappa, csw, U, psi = fields("mid_8^4")  # 4096 sites: the stated maximum

    # a first call on another operator of the same shape, so that loading the
    # kernels it launches and looking up the scratch array's address happen
    # before the measured calls
    op0, g0, l0 = _operator(dims, block, U, kappa, csw)
    b0 = torch.from_numpy(psi).cuda()
    x0 = torch.zeros_like(b0)
    st, info = _noalloc(lib, op0, b0, x0, stream)
    assert st == _lib.MGC_OK, lib.mgc_last_error()
    del op0, g0, l0

    op, gauge, lat = _operator(dims, block, U, kappa, csw)  # fresh: no solver workspace yet
    b = torch.from_numpy(psi).cuda()
    xs = [torch.full_like(b, float("nan")) for _ in range(2)]  # x is ignored without a guess
    Cl = O.clover(dims, kappa, csw, U)
    torch.cuda.synchronize()
    for call, x in enumerate(xs):
        free_before, _ = torch.cuda.mem_get_info()
        st, info = _noalloc(lib, op, b, x, stream)
        torch.cuda.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        assert st == _lib.MGC_OK, (call, lib.mgc_last_error())
        assert free_after == free_before, (call, free_before - free_after)
        assert info.status == _lib.MGC_OK and info.true_res <= 1e-10
        xh = x.cpu().numpy()
        r = psi - O.dirac(dims, -1, kappa, U, Cl, xh)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(psi), call

    # the existing entry point, same method and parameters, called last
    ref, ref_info = op.solve(b, api.solve_params(method=1, smoother_prec=16, tol=1e-10))
    assert ref_info.status == _lib.MGC_OK and ref_info.true_res <= 1e-10
    ref = ref.cpu().numpy()
    for call, x in enumerate(xs):
        assert rel(x.cpu().numpy(), ref) < TOL[64], call


def test_noalloc_solve_rejects_what_it_cannot_do():
    from paper_2112_00501_gb300 import _lib, synth

    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # more sites than MGC_NOALLOC_MAX_SITES
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    op, gauge, lat = _operator(dims, block, synth.unit_gauge(dims), 0.12, 1.0)
    b = torch.from_numpy(synth.gaussian_spinor(dims, 3)).cuda()
    x = torch.zeros_like(b)
    st, info = _noalloc(lib, op, b, x, stream)
    assert st == _lib.MGC_ERR_UNSUPPORTED_SHAPE and b"MGC_NOALLOC_MAX_SITES" in lib.mgc_last_error()
    # only flexible BiCGStab
    dims, block, eps, kappa, csw, U, psi = fields("c0_4^4")
    op, gauge, lat = _operator(dims, block, U, kappa, csw)
    b = torch.from_numpy(psi).cuda()
    x = torch.zeros_like(b)
    from paper_2112_00501_gb300 import api

    p = api.solve_params(method=2, smoother_prec=16, on_device=1)
    info = _lib.SolveInfo()
    st = lib.mgc_solve_noalloc(op.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(p),
                               C.byref(info), stream)
    assert st == _lib.MGC_ERR_INVALID_ARG
