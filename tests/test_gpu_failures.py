"""Failure detection without a GPU fault: the bounded wait of the staged SAP
kernel gives up, reports MGC_ERR_TIMEOUT through a status word the host reads,
and leaves the context usable."""
import ctypes as C

import pytest

from helpers import TOL, fields, rel
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_runs_out_and_context_survives():
    from paper_2112_00501_gb300 import _lib, api

    lib = _lib.load()
    flag = C.c_int(0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a barrier that completes
    assert lib.mgc_selftest_bounded_wait(20_000_000, 1, C.byref(flag), stream) == _lib.MGC_OK
    assert flag.value == 0
    # a barrier nothing arrives at: the 20 ms limit runs out
    assert lib.mgc_selftest_bounded_wait(20_000_000, 0, C.byref(flag), stream) == _lib.MGC_ERR_TIMEOUT
    assert flag.value != 0
    assert b"ran out" in lib.mgc_last_error()
    # the context is still usable: a smoother run afterwards matches the oracle
    name = "c0_4^4"
    dims, block, eps, kappa, csw, U, psi = fields(name)
    lat = api.Lattice(dims, block, -1)
    op = api.CloverOperator(api.Gauge(lat, torch.from_numpy(U).cuda(), storage_prec=16, compress=12), kappa, csw)
    got = op.sap(torch.from_numpy(psi).cuda(), prec=16, n_cy=2, n_mr=3).cpu().numpy()
    ref = O.sap(dims, block, -1, kappa, U, O.clover(dims, kappa, csw, U), psi, ncy=2, nmr=3)
    assert rel(got, ref) < TOL[16]
    flags = C.c_int(-1)
    assert lib.mgc_device_status(op.handle, C.byref(flags), 1, stream) == _lib.MGC_OK
    assert flags.value == 0
