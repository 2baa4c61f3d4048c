"""The oracle's front end refuses arrays of the wrong size instead of letting
its C routines index past them."""
import numpy as np
import pytest

from oracle import oracle as O


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
