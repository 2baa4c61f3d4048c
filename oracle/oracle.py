"""numpy front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg call this module; the CUDA library never does.  It imports
nothing from the CUDA package.

All fields are complex128 in the canonical layouts:
  spinor psi[V, 4, 3]; gauge U[V, 4, 3, 3]; clover C[V, 12, 12] with index
  spin*3 + colour; force g[V, 4, 3, 3].
Site s = x + Lx*(y + Ly*(z + Lz*t)).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

_i4 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i8 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_c16 = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_gamma.argtypes = [_c16]
        L.or_sigma.argtypes = [_c16]
        L.or_threads.restype = C.c_int
        L.or_set_threads.restype = None
        L.or_set_threads.argtypes = [C.c_int]
        L.or_field_strength_site.argtypes = [_i4, _c16, C.c_long, _c16]
        L.or_clover_site.argtypes = [_i4, C.c_double, C.c_double, _c16, C.c_long, _c16]
        L.or_clover_build.argtypes = [_i4, C.c_double, C.c_double, _c16, _c16]
        L.or_invert.argtypes = [C.c_int, _c16, _c16]
        L.or_invert.restype = C.c_int
        L.or_clover_invert.argtypes = [_i4, _c16, _c16]
        L.or_clover_invert.restype = C.c_int
        L.or_dirac.argtypes = [_i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, C.c_int]
        L.or_dirac_at.argtypes = [_i4, C.c_int, C.c_double, C.c_double, _c16, _c16, C.c_long,
                                  _i8, _c16, C.c_int]
        L.or_dirac_block.argtypes = [_i4, _i4, _i4, C.c_double, _c16, _c16, _c16, _c16, C.c_int]
        L.or_mr_block.argtypes = [_i4, _i4, _i4, C.c_double, _c16, _c16, _c16, _c16, C.c_void_p,
                                  C.c_int]
        L.or_mr_block_at.argtypes = [_i4, _i4, _i4, C.c_double, C.c_double, _c16, _c16, _c16,
                                     C.c_int]
        L.or_sap.argtypes = [_i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, C.c_int, C.c_int]
        L.or_solve.argtypes = [_i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, C.c_int,
                               C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                               C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.or_solve.restype = C.c_int
        L.or_force.argtypes = [_i4, C.c_int, C.c_double, C.c_double, _c16, _c16, _c16, _c16]
        L.or_mr_eo_block.argtypes = [_i4, _i4, _i4, C.c_double, _c16, _c16, _c16, _c16, _c16, C.c_int]
        L.or_sap_eo.argtypes = [_i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, _c16, C.c_int, C.c_int]
        L.or_apply_A.argtypes = [_i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, _c16]
        L.or_jacobi_block.argtypes = [_i4, _i4, _i4, C.c_double, _c16, _c16, _c16, _c16, _c16, C.c_int]
        L.or_jacobi_block_at.argtypes = [_i4, _i4, _i4, C.c_double, C.c_double, _c16, _c16, _c16, C.c_int]
        L.or_sap_A.argtypes = [_i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, _c16, C.c_int, C.c_int]
        L.or_solve_qws.argtypes = [_i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, _c16, _c16, C.c_int,
                                   C.c_int, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]
        L.or_solve_qws.restype = C.c_int
        L.or_mg_basis.argtypes = [_i4, _i4, C.c_int, _c16, _c16]
        L.or_mg_basis.restype = C.c_int
        L.or_mg_restrict.argtypes = [_i4, _i4, C.c_int, _c16, _c16, _c16]
        L.or_mg_prolong.argtypes = [_i4, _i4, C.c_int, _c16, _c16, _c16]
        L.or_mg_coarse_op.argtypes = [_i4, _i4, C.c_int, C.c_double, _c16, _c16, C.c_int, _c16, _c16]
        L.or_mg_coarse_apply.argtypes = [_i4, _i4, C.c_int, _c16, _c16, _c16]
        L.or_mg_coarse_solve.argtypes = [_i4, _i4, C.c_int, _c16, _c16, _c16, C.c_double, C.c_int,
                                         C.POINTER(C.c_int)]
        L.or_mg_coarse_solve.restype = C.c_int
        L.or_mg_precond.argtypes = [_i4, _i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, C.c_int, _c16, _c16,
                                    C.c_int, C.c_int, C.c_double, C.c_int, _c16, _c16]
        L.or_mg_setup.argtypes = [_i4, _i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, C.c_int, _c16, C.c_int,
                                  C.c_int, C.c_int, C.c_double, C.c_int, _c16, _c16]
        L.or_mg_setup.restype = C.c_int
        L.or_solve_mg.argtypes = [_i4, _i4, _i4, C.c_int, C.c_double, _c16, _c16, _c16, C.c_int, _c16, _c16,
                                  C.c_int, C.c_int, C.c_double, C.c_int, _c16, _c16, C.c_double, C.c_int,
                                  C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.or_solve_mg.restype = C.c_int
        _lib = L
    return _lib


def _dims(d):
    return np.ascontiguousarray(np.asarray(d, dtype=np.int32).reshape(4))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _sized(a, n, what):
    """a as contiguous complex128, refusing any size but n entries: the C
    routines index whole-lattice arrays without knowing their length."""
    a = _c(a)
    if a.size != n:
        raise ValueError(f"{what}: expected {n} complex entries, got {a.size} (shape {a.shape})")
    return a


def _vol(dims):
    return int(np.prod([int(d) for d in dims]))


def _vb(bdims):
    return int(np.prod([int(b) for b in bdims]))


def threads() -> int:
    """Number of OpenMP threads the oracle uses (1 without OpenMP)."""
    return int(lib().or_threads())


def set_threads(n: int) -> None:
    """Run the oracle's parallel loops on n threads from here on."""
    lib().or_set_threads(int(n))


def gamma():
    """(gamma_x, gamma_y, gamma_z, gamma_t, gamma_5) as a (5, 4, 4) array."""
    out = np.zeros((5, 4, 4), np.complex128)
    lib().or_gamma(out)
    return out


def sigma():
    """sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] as a (4, 4, 4, 4) array."""
    out = np.zeros((4, 4, 4, 4), np.complex128)
    lib().or_sigma(out)
    return out


def field_strength_site(dims, U, site):
    """F_{mu nu}(x) for the planes (01, 02, 03, 12, 13, 23), shape (6, 3, 3)."""
    out = np.zeros((6, 3, 3), np.complex128)
    if not 0 <= int(site) < _vol(dims):
        raise ValueError("site out of range")
    lib().or_field_strength_site(_dims(dims), _sized(U, _vol(dims) * 36, "U"), int(site), out)
    return out


def clover_site(dims, kappa, csw, U, site):
    out = np.zeros((12, 12), np.complex128)
    if not 0 <= int(site) < _vol(dims):
        raise ValueError("site out of range")
    lib().or_clover_site(_dims(dims), float(kappa), float(csw), _sized(U, _vol(dims) * 36, "U"), int(site), out)
    return out


def clover(dims, kappa, csw, U):
    """C(x) = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x), (V, 12, 12)."""
    V = int(np.prod(dims))
    out = np.zeros((V, 12, 12), np.complex128)
    lib().or_clover_build(_dims(dims), float(kappa), float(csw), _sized(U, V * 36, "U"), out)
    return out


def invert(A):
    A = _c(A)
    n = A.shape[0]
    out = np.zeros_like(A)
    if lib().or_invert(n, A, out) != 0:
        raise ZeroDivisionError("singular matrix")
    return out


def clover_inverse(dims, Cl):
    Cl = _sized(Cl, _vol(dims) * 144, "Cl")
    out = np.zeros_like(Cl)
    if lib().or_clover_invert(_dims(dims), Cl, out) != 0:
        raise ZeroDivisionError("singular clover block")
    return out


def dirac(dims, tbc, kappa, U, Cl, psi, dagger=False):
    """D psi (or D^dagger psi) on the whole lattice; psi (V, 4, 3)."""
    V = _vol(dims)
    psi = _sized(psi, V * 12, "psi")
    out = np.zeros_like(psi)
    lib().or_dirac(_dims(dims), int(tbc), float(kappa), _sized(U, V * 36, "U"), _sized(Cl, V * 144, "Cl"), psi,
                   out, int(bool(dagger)))
    return out


def dirac_at(dims, tbc, kappa, csw, U, psi, sites, dagger=False):
    """D psi at the listed sites only (clover built on the fly); (n, 4, 3)."""
    V = _vol(dims)
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int64).reshape(-1))
    if sites.size and (sites.min() < 0 or sites.max() >= V):
        raise ValueError("site out of range")
    out = np.zeros((len(sites), 4, 3), np.complex128)
    lib().or_dirac_at(_dims(dims), int(tbc), float(kappa), float(csw), _sized(U, V * 36, "U"),
                      _sized(psi, V * 12, "psi"),
                      len(sites), sites, out, int(bool(dagger)))
    return out


def block_sites(dims, bdims, bc):
    """Global sites of block bc in local lexicographic order."""
    bdims = [int(b) for b in bdims]
    out = []
    for lt in range(bdims[3]):
        for lz in range(bdims[2]):
            for ly in range(bdims[1]):
                for lx in range(bdims[0]):
                    c = [bc[0] * bdims[0] + lx, bc[1] * bdims[1] + ly,
                         bc[2] * bdims[2] + lz, bc[3] * bdims[3] + lt]
                    out.append(c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3])))
    return np.array(out, dtype=np.int64)


def dirac_block(dims, bdims, bc, kappa, U, Cl, v, dagger=False):
    """Dirichlet block operator D_B on a block vector v (V_B, 4, 3)."""
    V = _vol(dims)
    v = _sized(v, _vb(bdims) * 12, "v")
    out = np.zeros_like(v)
    lib().or_dirac_block(_dims(dims), _dims(bdims), _dims(bc), float(kappa), _sized(U, V * 36, "U"),
                         _sized(Cl, V * 144, "Cl"), v,
                         out, int(bool(dagger)))
    return out


def mr_block(dims, bdims, bc, kappa, U, Cl, r, nmr, return_residual=False):
    """k = nmr minimal-residual steps on D_B e = r from e = 0."""
    V = _vol(dims)
    r = _sized(r, _vb(bdims) * 12, "r")
    e = np.zeros_like(r)
    rout = np.zeros_like(r) if return_residual else None
    lib().or_mr_block(_dims(dims), _dims(bdims), _dims(bc), float(kappa), _sized(U, V * 36, "U"),
                      _sized(Cl, V * 144, "Cl"), r, e,
                      None if rout is None else rout.ctypes.data, int(nmr))
    return (e, rout) if return_residual else e


def mr_block_at(dims, bdims, bc, kappa, csw, U, r, nmr):
    """MR on one block with its clover built on the fly (no full clover field)."""
    r = _sized(r, _vb(bdims) * 12, "r")
    e = np.zeros_like(r)
    lib().or_mr_block_at(_dims(dims), _dims(bdims), _dims(bc), float(kappa), float(csw),
                         _sized(U, _vol(dims) * 36, "U"), r, e,
                         int(nmr))
    return e


def sap(dims, bdims, tbc, kappa, U, Cl, b, x0=None, ncy=4, nmr=4):
    """n_cy multiplicative SAP sweeps on D x = b; returns the updated x."""
    V = _vol(dims)
    b = _sized(b, V * 12, "b")
    x = np.zeros_like(b) if x0 is None else _sized(np.array(x0, dtype=np.complex128, copy=True), V * 12, "x0")
    lib().or_sap(_dims(dims), _dims(bdims), int(tbc), float(kappa), _sized(U, V * 36, "U"), _sized(Cl, V * 144, "Cl"),
                 b, x,
                 int(ncy), int(nmr))
    return x


def mr_eo_block(dims, bdims, bc, kappa, U, Cl, Ci, r, nmr):
    """Even-odd preconditioned MR on one domain (Schur complement on even sites)."""
    V = _vol(dims)
    r = _sized(r, _vb(bdims) * 12, "r")
    e = np.zeros_like(r)
    lib().or_mr_eo_block(_dims(dims), _dims(bdims), _dims(bc), float(kappa), _sized(U, V * 36, "U"),
                         _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), r, e, int(nmr))
    return e


def sap_eo(dims, bdims, tbc, kappa, U, Cl, Ci, b, x0=None, ncy=4, nmr=4):
    """n_cy SAP sweeps on D x = b with even-odd preconditioned MR domain solves."""
    V = _vol(dims)
    b = _sized(b, V * 12, "b")
    x = np.zeros_like(b) if x0 is None else _sized(np.array(x0, dtype=np.complex128, copy=True), V * 12, "x0")
    lib().or_sap_eo(_dims(dims), _dims(bdims), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                    _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), b, x, int(ncy), int(nmr))
    return x


def solve(dims, bdims, tbc, kappa, U, Cl, b, method="fgcr", precond="sap", ncy=4, nmr=4,
          m=16, tol=1e-10, max_iter=1000, x0=None):
    """Solve D x = b.  Returns (x, status, iterations, true relative residual)."""
    V = _vol(dims)
    b = _sized(b, V * 12, "b")
    x = np.zeros_like(b) if x0 is None else _sized(np.array(x0, dtype=np.complex128, copy=True), V * 12, "x0")
    it = C.c_int(0)
    res = C.c_double(0)
    st = lib().or_solve(_dims(dims), _dims(bdims), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                        _sized(Cl, V * 144, "Cl"), b, x,
                        {"fgcr": 0, "fbicgstab": 1}[method], {"none": 0, "sap": 1}[precond],
                        int(ncy), int(nmr), int(m), float(tol), int(max_iter), C.byref(it),
                        C.byref(res))
    return x, int(st), int(it.value), float(res.value)


def apply_A(dims, tbc, kappa, U, Cl, Ci, psi):
    """A psi with A = C^-1 D (the clover-preconditioned operator of Sec. 2)."""
    V = _vol(dims)
    psi = _sized(psi, V * 12, "psi")
    out = np.zeros_like(psi)
    lib().or_apply_A(_dims(dims), int(tbc), float(kappa), _sized(U, V * 36, "U"), _sized(Cl, V * 144, "Cl"),
                     _sized(Ci, V * 144, "Ci"), psi, out)
    return out


def jacobi_block(dims, bdims, bc, kappa, U, Cl, Ci, r, nj):
    """nj Jacobi iterations e <- e + (r - A_B e) from e = 0 on one domain."""
    V = _vol(dims)
    r = _sized(r, _vb(bdims) * 12, "r")
    e = np.zeros_like(r)
    lib().or_jacobi_block(_dims(dims), _dims(bdims), _dims(bc), float(kappa), _sized(U, V * 36, "U"),
                          _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), r, e, int(nj))
    return e


def jacobi_block_at(dims, bdims, bc, kappa, csw, U, r, nj):
    """Jacobi on one domain with its C and C^-1 built on the fly (no full clover field)."""
    r = _sized(r, _vb(bdims) * 12, "r")
    e = np.zeros_like(r)
    lib().or_jacobi_block_at(_dims(dims), _dims(bdims), _dims(bc), float(kappa), float(csw),
                             _sized(U, _vol(dims) * 36, "U"), r, e, int(nj))
    return e


def sap_A(dims, bdims, tbc, kappa, U, Cl, Ci, b, x0=None, ncy=4, nj=4):
    """n_cy multiplicative SAP sweeps on A x = b with nj Jacobi iterations per domain."""
    V = _vol(dims)
    b = _sized(b, V * 12, "b")
    x = np.zeros_like(b) if x0 is None else _sized(np.array(x0, dtype=np.complex128, copy=True), V * 12, "x0")
    lib().or_sap_A(_dims(dims), _dims(bdims), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                   _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), b, x, int(ncy), int(nj))
    return x


def solve_qws(dims, bdims, tbc, kappa, U, Cl, Ci, b, ncy=4, nj=4, tol=1e-10, inner_tol=1e-6, max_iter=1000):
    """The QWS solver of Sec. 2 for D x = b.  Returns (x, status, BiCGStab iterations, true residual)."""
    V = _vol(dims)
    b = _sized(b, V * 12, "b")
    x = np.zeros_like(b)
    it = C.c_int(0)
    res = C.c_double(0)
    st = lib().or_solve_qws(_dims(dims), _dims(bdims), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                            _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), b, x, int(ncy), int(nj),
                            float(tol), float(inner_tol), int(max_iter), C.byref(it), C.byref(res))
    return x, int(st), int(it.value), float(res.value)


# ---------------------------------------------------------------- multigrid (Sec. 3)
# W: (nvec, V, 4, 3) block-orthonormal null vectors; coarse vectors u: (Vc, 2, nvec);
# coarse operator Dc: (Vc, 9, 2 nvec, 2 nvec), stencil order self, +x, -x, +y, -y, +z, -z, +t, -t.

def coarse_volume(dims, agg):
    return int(np.prod([int(d) // int(a) for d, a in zip(dims, agg)]))


def mg_basis(dims, agg, Vin):
    """Block modified Gram-Schmidt per (aggregate, chirality).  Returns (W, n_dependent)."""
    Vin = _c(Vin)
    nvec = Vin.shape[0]
    _sized(Vin, nvec * _vol(dims) * 12, "V")
    W = np.zeros_like(Vin)
    bad = lib().or_mg_basis(_dims(dims), _dims(agg), nvec, Vin, W)
    return W, int(bad)


def mg_restrict(dims, agg, W, v):
    W = _c(W)
    nvec = W.shape[0]
    u = np.zeros((coarse_volume(dims, agg), 2, nvec), np.complex128)
    lib().or_mg_restrict(_dims(dims), _dims(agg), nvec, _sized(W, nvec * _vol(dims) * 12, "W"),
                         _sized(v, _vol(dims) * 12, "v"), u)
    return u


def mg_prolong(dims, agg, W, u):
    W = _c(W)
    nvec = W.shape[0]
    v = np.zeros((_vol(dims), 4, 3), np.complex128)
    lib().or_mg_prolong(_dims(dims), _dims(agg), nvec, _sized(W, nvec * _vol(dims) * 12, "W"),
                        _sized(u, coarse_volume(dims, agg) * 2 * nvec, "u"), v)
    return v


def mg_coarse_op(dims, agg, tbc, kappa, U, Cl, W):
    W = _c(W)
    nvec = W.shape[0]
    V = _vol(dims)
    Dc = np.zeros((coarse_volume(dims, agg), 9, 2 * nvec, 2 * nvec), np.complex128)
    lib().or_mg_coarse_op(_dims(dims), _dims(agg), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                          _sized(Cl, V * 144, "Cl"), nvec, _sized(W, nvec * V * 12, "W"), Dc)
    return Dc


def mg_coarse_apply(dims, agg, Dc, u):
    Dc = _c(Dc)
    nvec = Dc.shape[-1] // 2
    Vc = coarse_volume(dims, agg)
    out = np.zeros((Vc, 2, nvec), np.complex128)
    lib().or_mg_coarse_apply(_dims(dims), _dims(agg), nvec, _sized(Dc, Vc * 9 * 4 * nvec * nvec, "Dc"),
                             _sized(u, Vc * 2 * nvec, "u"), out)
    return out


def mg_coarse_solve(dims, agg, Dc, b, tol=1e-10, maxit=1000):
    Dc = _c(Dc)
    nvec = Dc.shape[-1] // 2
    Vc = coarse_volume(dims, agg)
    x = np.zeros((Vc, 2, nvec), np.complex128)
    it = C.c_int(0)
    st = lib().or_mg_coarse_solve(_dims(dims), _dims(agg), nvec, _sized(Dc, Vc * 9 * 4 * nvec * nvec, "Dc"),
                                  _sized(b, Vc * 2 * nvec, "b"), x, float(tol), int(maxit), C.byref(it))
    return x, int(st), int(it.value)


def mg_precond(dims, bdims, agg, tbc, kappa, U, Cl, Ci, W, Dc, v, ncy=2, nj=4, ctol=1e-2, cmaxit=100):
    """The two-level preconditioner applied to v: coarse correction, then SAP post-smoothing."""
    W = _c(W)
    nvec = W.shape[0]
    V = _vol(dims)
    x = np.zeros((V, 4, 3), np.complex128)
    lib().or_mg_precond(_dims(dims), _dims(bdims), _dims(agg), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                        _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), nvec, _sized(W, nvec * V * 12, "W"),
                        _sized(Dc, coarse_volume(dims, agg) * 36 * nvec * nvec, "Dc"), int(ncy), int(nj),
                        float(ctol), int(cmaxit), _sized(v, V * 12, "v"), x)
    return x


def mg_setup(dims, bdims, agg, tbc, kappa, U, Cl, Ci, eta, ncy=2, nj=4, n_adapt=4, ctol=1e-2, cmaxit=100):
    """Null vectors from M_SAP on the random vectors eta, then n_adapt adaptive passes.
    Returns (W, Dc, n_dependent)."""
    eta = _c(eta)
    nvec = eta.shape[0]
    V = _vol(dims)
    W = np.zeros((nvec, V, 4, 3), np.complex128)
    Dc = np.zeros((coarse_volume(dims, agg), 9, 2 * nvec, 2 * nvec), np.complex128)
    bad = lib().or_mg_setup(_dims(dims), _dims(bdims), _dims(agg), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                            _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), nvec,
                            _sized(eta, nvec * V * 12, "eta"), int(ncy), int(nj), int(n_adapt), float(ctol),
                            int(cmaxit), W, Dc)
    return W, Dc, int(bad)


def solve_mg(dims, bdims, agg, tbc, kappa, U, Cl, Ci, W, Dc, b, ncy=2, nj=4, ctol=1e-2, cmaxit=100, tol=1e-10,
             max_iter=500):
    """Flexible BiCGStab with the two-level preconditioner.  Returns (x, status, iterations, true residual)."""
    W = _c(W)
    nvec = W.shape[0]
    V = _vol(dims)
    x = np.zeros((V, 4, 3), np.complex128)
    it = C.c_int(0)
    res = C.c_double(0)
    st = lib().or_solve_mg(_dims(dims), _dims(bdims), _dims(agg), int(tbc), float(kappa), _sized(U, V * 36, "U"),
                           _sized(Cl, V * 144, "Cl"), _sized(Ci, V * 144, "Ci"), nvec, _sized(W, nvec * V * 12, "W"),
                           _sized(Dc, coarse_volume(dims, agg) * 36 * nvec * nvec, "Dc"), int(ncy), int(nj),
                           float(ctol), int(cmaxit), _sized(b, V * 12, "b"), x, float(tol), int(max_iter),
                           C.byref(it), C.byref(res))
    return x, int(st), int(it.value), float(res.value)


def gamma5(psi):
    """gamma_5 = diag(1, 1, -1, -1) on the spin index."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    out[..., 2:, :] *= -1
    return out


def force(dims, tbc, kappa, csw, U, X, Y):
    """dS/dRe U + i dS/dIm U for S = ||Y||^2, Y = D^-dagger phi, X = D^-1 Y."""
    V = int(np.prod(dims))
    g = np.zeros((V, 4, 3, 3), np.complex128)
    lib().or_force(_dims(dims), int(tbc), float(kappa), float(csw), _sized(U, V * 36, "U"), _sized(X, V * 12, "X"),
                   _sized(Y, V * 12, "Y"), g)
    return g


def force_solves(dims, bdims, tbc, kappa, U, Cl, phi, tol=1e-13, **kw):
    """Y = D^-dagger phi (as gamma5 D^-1 gamma5 phi) and X = D^-1 Y."""
    y5, st1, _, _ = solve(dims, bdims, tbc, kappa, U, Cl, gamma5(phi), tol=tol, **kw)
    Y = gamma5(y5)
    X, st2, _, _ = solve(dims, bdims, tbc, kappa, U, Cl, Y, tol=tol, **kw)
    if st1 or st2:
        raise RuntimeError("oracle solve did not converge")
    return X, Y


def action(dims, bdims, tbc, kappa, csw, U, phi, tol=1e-13, **kw):
    """S = phi^dagger (D^dagger D)^-1 phi, evaluated as 2 Re(phi^dagger X) - ||D X||^2,
    whose error is second order in the solver error of X."""
    Cl = clover(dims, kappa, csw, U)
    X, Y = force_solves(dims, bdims, tbc, kappa, U, Cl, phi, tol=tol, **kw)
    DX = dirac(dims, tbc, kappa, U, Cl, X)
    return 2.0 * np.real(np.vdot(phi, X)) - np.real(np.vdot(DX, DX))
