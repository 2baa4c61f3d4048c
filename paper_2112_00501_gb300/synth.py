"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws random numbers and shapes them into lattice fields; it holds
none of the Dirac-operator, smoother or solver arithmetic.  It imports numpy
only, so both the oracle-side tests and the CUDA-side code can use it without
importing each other.

The paper measures on Japan Lattice Data Grid configurations (Sec. 4, sets A, B
and C) that are not available here.  The stand-ins are disordered SU(3) fields
U = exp(i*eps*H) with H a random traceless Hermitian 3x3 matrix per link.

Canonical layouts (all complex128, C order):
  site index   s = x + Lx*(y + Ly*(z + Lz*t))
  gauge field  U[s, mu, a, b]   mu = 0..3 for x, y, z, t; U_mu(s) links s to s+mu
  spinor       psi[s, spin, colour]  (4 spins x 3 colours); a batch adds a
               leading right-hand-side axis.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "rng",
    "random_traceless_hermitian",
    "reunitarise",
    "random_su3",
    "gauge_field",
    "gaussian_spinor",
    "unit_gauge",
    "gauge_seed",
    "source_seed",
]


def volume(dims) -> int:
    """Number of sites of a lattice with extents dims = (Lx, Ly, Lz, Lt)."""
    v = 1
    for d in dims:
        v *= int(d)
    return v


def rng(seed: int) -> np.random.Generator:
    """The one generator every input uses: numpy PCG64 seeded with `seed`."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def gauge_seed(config_index: int) -> int:
    """Seed of the gauge field of workload `config_index`."""
    return 1000 + int(config_index)


def source_seed(config_index: int, rhs: int = 0) -> int:
    """Seed of right-hand side `rhs` of workload `config_index`."""
    return 2000 + int(config_index) + int(rhs)


def random_traceless_hermitian(n: int, g: np.random.Generator) -> np.ndarray:
    """n random traceless Hermitian 3x3 matrices.

    Diagonal entries are N(0, 1); above the diagonal the real and imaginary
    parts are independent N(0, 1/2), mirrored below by conjugation; the trace
    divided by 3 is then subtracted from the diagonal.
    """
    h = np.zeros((n, 3, 3), dtype=np.complex128)
    d = g.standard_normal((n, 3))
    h[:, [0, 1, 2], [0, 1, 2]] = d
    o = g.standard_normal((n, 3, 2)) * np.sqrt(0.5)
    iu = ([0, 0, 1], [1, 2, 2])
    h[:, iu[0], iu[1]] = o[..., 0] + 1j * o[..., 1]
    h[:, iu[1], iu[0]] = o[..., 0] - 1j * o[..., 1]
    tr = (d.sum(axis=1) / 3.0)[:, None]
    h[:, [0, 1, 2], [0, 1, 2]] -= tr
    return h


def reunitarise(u: np.ndarray) -> np.ndarray:
    """Project 3x3 matrices back onto SU(3) by row Gram-Schmidt.

    Row 0 is normalised, row 1 is orthogonalised against row 0 and
    normalised, and row 2 is the complex conjugate of row0 x row1, which
    makes the determinant exactly one up to rounding.
    """
    u = np.array(u, dtype=np.complex128, copy=True)
    r0 = u[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=1)[:, None]
    r1 = u[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=1)[:, None] * r0
    r1 = r1 / np.linalg.norm(r1, axis=1)[:, None]
    r2 = np.conj(np.cross(r0, r1))
    u[:, 0, :] = r0
    u[:, 1, :] = r1
    u[:, 2, :] = r2
    return u


def _expi(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*h) for Hermitian h, through its eigen-decomposition."""
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(v, 1, 2))


def random_su3(n: int, g: np.random.Generator, eps: float = 1.0) -> np.ndarray:
    """n SU(3) matrices exp(i*eps*H), H from random_traceless_hermitian."""
    return reunitarise(_expi(random_traceless_hermitian(n, g), eps))


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """Disordered SU(3) gauge field U[s, mu] = exp(i*eps*H), reunitarised.

    Links are drawn in canonical order (site-major, then mu) in chunks of
    `chunk` links; each chunk draws its diagonal normals, then its
    off-diagonal normals.  The chunk size is therefore part of the field's
    definition: keep the default to reproduce a field.
    """
    v = volume(dims)
    n = 4 * v
    g = rng(seed)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        out[lo:hi] = random_su3(hi - lo, g, eps)
    return out.reshape(v, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    """The free field: every link the 3x3 identity."""
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, [0, 1, 2], [0, 1, 2]] = 1.0
    return u


def gaussian_spinor(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian spinor field(s), real and imaginary parts N(0, 1/2).

    Returns shape (V, 4, 3), or (nrhs, V, 4, 3) when nrhs is given; with nrhs
    given, right-hand side k is drawn from its own generator seeded seed + k.
    """
    v = volume(dims)
    if nrhs is None:
        g = rng(seed)
        z = g.standard_normal((v, 4, 3, 2)) * np.sqrt(0.5)
        return z[..., 0] + 1j * z[..., 1]
    return np.stack([gaussian_spinor(dims, seed + k) for k in range(nrhs)])
