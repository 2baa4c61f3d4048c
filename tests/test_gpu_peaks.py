"""The measured FMA rates (mgc_fma_peak) that the roofline of the
arithmetic-bound kernels divides by."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_fma_peak_probe():
    """FP32 and FP64 rates finite and positive, FP32 far above FP64 on this
    part; a precision other than 32 or 64 is refused."""
    from paper_2112_00501_gb300 import _lib

    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    f32, f64 = C.c_double(0), C.c_double(0)
    assert lib.mgc_fma_peak(32, C.byref(f32), stream) == _lib.MGC_OK
    assert lib.mgc_fma_peak(64, C.byref(f64), stream) == _lib.MGC_OK
    assert 1e12 < f32.value < 1e15 and 1e10 < f64.value < f32.value
    assert lib.mgc_fma_peak(16, C.byref(f32), stream) == _lib.MGC_ERR_INVALID_ARG
