"""The seeded input generators: the properties the input recipe states for the
stand-in gauge fields and sources (disordered SU(3) links exp(i eps H) with H
traceless Hermitian, complex Gaussian sources), and that every input is
reproducible from its seed alone."""
import numpy as np

from paper_2112_00501_gb300 import synth


def test_traceless_hermitian_generator():
    g = synth.rng(11)
    h = synth.random_traceless_hermitian(20000, g)
    assert np.abs(h - np.conj(np.swapaxes(h, 1, 2))).max() == 0.0
    assert np.abs(np.trace(h, axis1=1, axis2=2)).max() < 1e-14
    # off-diagonal real and imaginary parts N(0, 1/2); diagonal N(0, 1) before
    # the trace subtraction, which leaves variance 1 - 1/3 on each diagonal entry
    off = h[:, 0, 1]
    assert abs(np.var(off.real) - 0.5) < 0.02 and abs(np.var(off.imag) - 0.5) < 0.02
    assert abs(np.var(h[:, 0, 0].real) - 2.0 / 3.0) < 0.03


def test_gauge_field_is_su3_and_reproducible():
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, 0.4, synth.gauge_seed(0))
    assert U.shape == (synth.volume(dims), 4, 3, 3)
    u = U.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(u @ np.conj(np.swapaxes(u, 1, 2)) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-14
    # eps sets the disorder: the links stay within eps * |H| of the identity
    assert np.abs(u - eye).max() < 0.4 * 4
    assert np.array_equal(U, synth.gauge_field(dims, 0.4, synth.gauge_seed(0)))
    assert not np.array_equal(U, synth.gauge_field(dims, 0.4, synth.gauge_seed(1)))


def test_small_eps_approaches_the_free_field():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 1e-6, 5)
    assert np.abs(U - synth.unit_gauge(dims)).max() < 1e-5


def test_reunitarise_projects_onto_su3():
    g = synth.rng(3)
    a = g.standard_normal((500, 3, 3)) + 1j * g.standard_normal((500, 3, 3))
    u = synth.reunitarise(a)
    assert np.abs(u @ np.conj(np.swapaxes(u, 1, 2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-14
    # an SU(3) matrix is left as it is
    v = synth.random_su3(500, g)
    assert np.abs(synth.reunitarise(v) - v).max() < 1e-14


def test_gaussian_spinor_statistics_and_batches():
    dims = (8, 8, 8, 8)
    psi = synth.gaussian_spinor(dims, synth.source_seed(2))
    assert psi.shape == (synth.volume(dims), 4, 3) and psi.dtype == np.complex128
    assert abs(psi.real.mean()) < 0.01 and abs(psi.imag.mean()) < 0.01
    assert abs(psi.real.var() - 0.5) < 0.01 and abs(psi.imag.var() - 0.5) < 0.01
    b = synth.gaussian_spinor(dims, 70, nrhs=3)
    assert b.shape == (3,) + psi.shape
    for k in range(3):
        assert np.array_equal(b[k], synth.gaussian_spinor(dims, 70 + k))


def test_seeds_of_the_workloads():
    assert synth.gauge_seed(2) == 1002
    assert synth.source_seed(2) == 2002 and synth.source_seed(2, 3) == 2005
