"""mgc_solve_noalloc, the allocation-free variant of mgc_solve for callers that
cannot call cudaMalloc at solve time: called through the C ABI twice in a row
(the second call finds the previous call's contents in the shared scratch
array), each time checked against mgc_solve's solution of the same system with
the same method, and its size limit and method restriction checked.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import pytest

from helpers import TOL, fields, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _operator(dims, block, U, kappa, csw):
    from paper_2112_00501_gb300 import api

    lat = api.Lattice(dims, block, -1)
    gauge = api.Gauge(lat, torch.as_tensor(U).cuda(), storage_prec=16, compress=12)
    return api.CloverOperator(gauge, kappa, csw), gauge, lat


def test_noalloc_solve_matches_mgc_solve_on_two_calls():
    from paper_2112_00501_gb300 import _lib, api

    lib = _lib.load()
    dims, block, eps, kappa, csw, U, psi = fields("mid_8^4")  # 4096 sites: the stated maximum
    op, gauge, lat = _operator(dims, block, U, kappa, csw)
    b = torch.from_numpy(psi).cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    # the existing entry point, same method and parameters
    ref, ref_info = op.solve(b, api.solve_params(method=1, smoother_prec=16, tol=1e-10))
    assert ref_info.status == _lib.MGC_OK and ref_info.true_res <= 1e-10
    ref = ref.cpu().numpy()

    for call in range(2):
        p = api.solve_params(method=1, smoother_prec=16, tol=1e-10, on_device=1)
        x = torch.full_like(b, float("nan"))  # whatever x holds is ignored without a guess
        info = _lib.SolveInfo()
        st = lib.mgc_solve_noalloc(op.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(p),
                                   C.byref(info), stream)
        assert st == _lib.MGC_OK, (call, lib.mgc_last_error())
        assert info.status == _lib.MGC_OK and info.true_res <= 1e-10
        assert rel(x.cpu().numpy(), ref) < TOL[64], call


def test_noalloc_solve_rejects_what_it_cannot_do():
    from paper_2112_00501_gb300 import _lib, api, synth

    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # more sites than MGC_NOALLOC_MAX_SITES
    dims, block = (8, 8, 8, 16), (4, 4, 4, 4)
    op, gauge, lat = _operator(dims, block, synth.unit_gauge(dims), 0.12, 1.0)
    b = torch.from_numpy(synth.gaussian_spinor(dims, 3)).cuda()
    x = torch.zeros_like(b)
    info = _lib.SolveInfo()
    p = api.solve_params(method=1, smoother_prec=16, on_device=1)
    st = lib.mgc_solve_noalloc(op.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(p),
                               C.byref(info), stream)
    assert st == _lib.MGC_ERR_UNSUPPORTED_SHAPE and b"MGC_NOALLOC_MAX_SITES" in lib.mgc_last_error()
    # only flexible BiCGStab
    dims, block, eps, kappa, csw, U, psi = fields("c0_4^4")
    op, gauge, lat = _operator(dims, block, U, kappa, csw)
    b = torch.from_numpy(psi).cuda()
    x = torch.zeros_like(b)
    p = api.solve_params(method=2, smoother_prec=16, on_device=1)
    st = lib.mgc_solve_noalloc(op.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(p),
                               C.byref(info), stream)
    assert st == _lib.MGC_ERR_INVALID_ARG
