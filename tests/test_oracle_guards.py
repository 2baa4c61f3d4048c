"""The oracle's front end refuses arrays of the wrong size instead of letting
its C routines index past them, and its results do not depend on how many
threads it runs on."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_00501_gb300 import synth


def test_wrong_sizes_raise():
    dims = (4, 4, 4, 4)
    V = 256
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[:, :, [0, 1, 2], [0, 1, 2]] = 1.0
    Cl = O.clover(dims, 0.1, 1.0, U)
    psi = np.ones((V, 4, 3), np.complex128)
    O.dirac(dims, -1, 0.1, U, Cl, psi)
    with pytest.raises(ValueError):
        O.dirac(dims, -1, 0.1, U, Cl, psi[:1])
    with pytest.raises(ValueError):
        O.dirac(dims, -1, 0.1, U[:-1], Cl, psi)
    with pytest.raises(ValueError):
        O.clover(dims, 0.1, 1.0, U[:7])
    with pytest.raises(ValueError):
        O.dirac_at(dims, -1, 0.1, 1.0, U, psi, [V])
    with pytest.raises(ValueError):
        O.sap(dims, (2, 2, 2, 2), -1, 0.1, U, Cl, psi[:3])
    with pytest.raises(ValueError):
        O.mr_block(dims, (2, 2, 2, 2), (0, 0, 0, 0), 0.1, U, Cl, psi, 2)


def test_results_do_not_depend_on_the_thread_count():
    """The CPU baseline times the oracle on one thread and on all cores; its
    parallel loops are per site or per domain, so both give the same bits."""
    dims, bd = (4, 4, 4, 8), (2, 2, 2, 2)
    kappa, csw = 0.1355, 1.0
    U = synth.gauge_field(dims, 0.4, 61)
    b = synth.gaussian_spinor(dims, 62)
    n0 = O.threads()
    out = []
    try:
        for n in (1, max(2, n0)):
            O.set_threads(n)
            Cl = O.clover(dims, kappa, csw, U)
            d = O.dirac(dims, -1, kappa, U, Cl, b)
            s = O.sap(dims, bd, -1, kappa, U, Cl, b, ncy=2, nmr=3)
            out.append((Cl, d, s))
    finally:
        O.set_threads(n0)
    for a, c in zip(out[0], out[1]):
        assert np.array_equal(a, c)
