"""Shared workload definitions and helpers for the GPU parity tests.

The synthetic workloads stand in for the paper's lattices (Sec. 4): disordered
SU(3) fields U = exp(i eps H) with Gaussian sources, on the lattice shapes and
parameters below.
"""
import numpy as np

from paper_2112_00501_gb300 import synth

# name: (dims, SAP block, eps, kappa, c_sw, config index for the seeds)
WORKLOADS = {
    "c0_4^4": ((4, 4, 4, 4), (2, 2, 2, 2), 0.4, 0.125, 1.0, 0),
    "c1_16^3x32": ((16, 16, 16, 32), (4, 4, 4, 4), 0.4, 0.1355, 1.0, 1),
    "c2_32^3x64": ((32, 32, 32, 64), (4, 4, 4, 4), 0.5, 0.1370, 1.0, 2),
    "c3_24^3x48": ((24, 24, 24, 48), (4, 4, 4, 4), 0.4, 0.1355, 1.0, 3),
    "c3_16^4": ((16, 16, 16, 16), (4, 4, 4, 4), 0.4, 0.1355, 1.0, 3),
    "c3_8^4": ((8, 8, 8, 8), (4, 4, 4, 4), 0.4, 0.1355, 1.0, 3),
    "c4_8^4": ((8, 8, 8, 8), (4, 4, 4, 4), 0.4, 0.1355, 1.0, 4),
    "mid_8^4": ((8, 8, 8, 8), (4, 4, 4, 4), 0.4, 0.1355, 1.0, 5),
    "ragged_8x4x12x8": ((8, 4, 12, 8), (2, 2, 2, 2), 0.4, 0.13, 1.0, 6),
}

TOL = {64: 1e-12, 32: 1e-5, 16: 2e-3}

_cache = {}


def fields(name):
    """(dims, block, eps, kappa, csw, U, psi) of a workload, cached."""
    if name not in _cache:
        dims, block, eps, kappa, csw, ci = WORKLOADS[name]
        U = synth.gauge_field(dims, eps, synth.gauge_seed(ci))
        psi = synth.gaussian_spinor(dims, synth.source_seed(ci))
        _cache[name] = (dims, block, eps, kappa, csw, U, psi)
    return _cache[name]


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def block_coords_of_colour(dims, block, colour):
    nb = [d // b for d, b in zip(dims, block)]
    out = []
    for bt in range(nb[3]):
        for bz in range(nb[2]):
            for by in range(nb[1]):
                for bx in range(nb[0]):
                    if (bx + by + bz + bt) % 2 == colour:
                        out.append((bx, by, bz, bt))
    return out
