"""Python binding of the C ABI with torch tensors for device memory and streams.

Names follow include/mgc.h.  Tensors are passed as raw pointers; the library
does all the work.  Canonical fields are complex128 tensors:
  spinor (V, 4, 3) or (nrhs, V, 4, 3); gauge (V, 4, 3, 3); clover (V, 12, 12).
Packed fields are uint8 tensors of Lattice.spinor_bytes(prec, nrhs) bytes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import MgParams, SolveInfo, SolveParams, check


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _canon(t, device) -> torch.Tensor:
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(t, dtype=np.complex128))
    t = t.to(device=device, dtype=torch.complex128)
    return t.contiguous()


class Lattice:
    """Lattice extents, SAP domain extents and the t boundary condition."""

    def __init__(self, dims, block, t_bc: int = -1):
        self.lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in block)
        self.t_bc = int(t_bc)
        h = C.c_void_p()
        d = (C.c_int * 4)(*self.dims)
        b = (C.c_int * 4)(*self.block)
        check(self.lib.mgc_lattice_create(d, b, self.t_bc, C.byref(h)), "mgc_lattice_create")
        self.handle = h
        self.volume = int(self.lib.mgc_lattice_volume(h))

    def spinor_bytes(self, prec: int, nrhs: int = 1) -> int:
        return int(self.lib.mgc_spinor_bytes(self.handle, prec, nrhs))

    def empty_packed(self, prec: int, nrhs: int = 1, device="cuda") -> torch.Tensor:
        return torch.empty(self.spinor_bytes(prec, nrhs), dtype=torch.uint8, device=device)

    def zeros_packed(self, prec: int, nrhs: int = 1, device="cuda") -> torch.Tensor:
        return torch.zeros(self.spinor_bytes(prec, nrhs), dtype=torch.uint8, device=device)

    def pack(self, psi, prec: int, out=None, stream=None) -> torch.Tensor:
        """canonical complex128 (device) -> packed at prec"""
        psi = _canon(psi, "cuda")
        nrhs = 1 if psi.dim() == 3 else psi.shape[0]
        if out is None:
            out = self.empty_packed(prec, nrhs)
        check(self.lib.mgc_spinor_pack(self.handle, prec, nrhs, _ptr(psi), _ptr(out), _stream(stream)),
              "mgc_spinor_pack")
        return out

    def unpack(self, packed: torch.Tensor, prec: int, nrhs: int = 1, out=None, stream=None) -> torch.Tensor:
        if out is None:
            shape = (self.volume, 4, 3) if nrhs == 1 else (nrhs, self.volume, 4, 3)
            out = torch.empty(shape, dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_spinor_unpack(self.handle, prec, nrhs, _ptr(packed), _ptr(out), _stream(stream)),
              "mgc_spinor_unpack")
        return out

    def convert(self, packed: torch.Tensor, prec_in: int, prec_out: int, nrhs: int = 1, out=None, stream=None):
        if out is None:
            out = self.empty_packed(prec_out, nrhs)
        check(self.lib.mgc_spinor_convert(self.handle, nrhs, prec_in, _ptr(packed), prec_out, _ptr(out),
                                          _stream(stream)), "mgc_spinor_convert")
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.mgc_lattice_destroy(h)
            self.handle = None


class Gauge:
    """Packed copies of a gauge field: FP64 plus one at storage_prec (18 or 12 reals)."""

    def __init__(self, lattice: Lattice, U, storage_prec: int = 32, compress: int = 18, stream=None):
        self.lib = lattice.lib
        self.lattice = lattice
        self.prec = int(storage_prec)
        self.compress = int(compress)
        on_device = isinstance(U, torch.Tensor) and U.is_cuda
        if on_device:
            Ut = U.to(torch.complex128).contiguous()
        else:
            Ut = torch.from_numpy(np.ascontiguousarray(np.asarray(U), dtype=np.complex128))
        h = C.c_void_p()
        check(self.lib.mgc_gauge_create(lattice.handle, _ptr(Ut), int(on_device), self.prec, self.compress,
                                        _stream(stream), C.byref(h)), "mgc_gauge_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.mgc_gauge_destroy(h)
            self.handle = None


def solve_params(**kw) -> SolveParams:
    p = SolveParams()
    _lib.load().mgc_solve_params_default(C.byref(p))
    names = {f[0] for f in SolveParams._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown solver parameter {k}")
        setattr(p, k, v)
    return p


class CloverOperator:
    """D = C - kappa H with the clover term of the gauge field (the ABI's mgc_clover_t)."""

    def __init__(self, gauge: Gauge, kappa: float, csw: float, stream=None):
        self.lib = gauge.lib
        self.gauge = gauge
        self.lattice = gauge.lattice
        self.kappa = float(kappa)
        self.csw = float(csw)
        h = C.c_void_p()
        check(self.lib.mgc_clover_create(gauge.handle, self.kappa, self.csw, _stream(stream), C.byref(h)),
              "mgc_clover_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.mgc_clover_destroy(h)
            self.handle = None

    # -- operator applications on packed fields --------------------------------
    def apply_D(self, x: torch.Tensor, prec: int, nrhs: int = 1, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = self.lattice.empty_packed(prec, nrhs)
        check(self.lib.mgc_apply_D(self.handle, _ptr(x), _ptr(out), nrhs, prec, _stream(stream)), "mgc_apply_D")
        return out

    def apply_Ddag(self, x: torch.Tensor, prec: int, nrhs: int = 1, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = self.lattice.empty_packed(prec, nrhs)
        check(self.lib.mgc_apply_Ddag(self.handle, _ptr(x), _ptr(out), nrhs, prec, _stream(stream)),
              "mgc_apply_Ddag")
        return out

    def apply_clover(self, x: torch.Tensor, prec: int, nrhs: int = 1, inverse=False, out=None, stream=None):
        if out is None:
            out = self.lattice.empty_packed(prec, nrhs)
        check(self.lib.mgc_apply_clover(self.handle, _ptr(x), _ptr(out), nrhs, prec, int(bool(inverse)),
                                        _stream(stream)), "mgc_apply_clover")
        return out

    def sap_smooth(self, b: torch.Tensor, x: torch.Tensor, prec: int, nrhs: int = 1, n_cy: int = 4,
                   n_mr: int = 4, x_is_zero: bool = False, stream=None) -> torch.Tensor:
        check(self.lib.mgc_sap_smooth(self.handle, _ptr(b), _ptr(x), nrhs, n_cy, n_mr, prec, int(bool(x_is_zero)),
                                      _stream(stream)), "mgc_sap_smooth")
        return x

    def sap_smooth_eo(self, b: torch.Tensor, x: torch.Tensor, prec: int, nrhs: int = 1, n_cy: int = 4,
                      n_mr: int = 4, x_is_zero: bool = False, stream=None) -> torch.Tensor:
        """SAP sweeps with even-odd preconditioned MR domain solves, packed fields."""
        check(self.lib.mgc_sap_smooth_eo(self.handle, _ptr(b), _ptr(x), nrhs, n_cy, n_mr, prec,
                                         int(bool(x_is_zero)), _stream(stream)), "mgc_sap_smooth_eo")
        return x

    def sap_eo(self, b, prec: int = 64, n_cy: int = 4, n_mr: int = 4, x0=None) -> torch.Tensor:
        """n_cy SAP sweeps with even-odd MR domain solves on D x = b, canonical in and out."""
        b = _canon(b, "cuda")
        nrhs = 1 if b.dim() == 3 else b.shape[0]
        bp = self.lattice.pack(b, prec)
        xp = self.lattice.zeros_packed(prec, nrhs) if x0 is None else self.lattice.pack(_canon(x0, "cuda"), prec)
        self.sap_smooth_eo(bp, xp, prec, nrhs, n_cy, n_mr, x_is_zero=x0 is None)
        return self.lattice.unpack(xp, prec, nrhs)

    def apply_A(self, x: torch.Tensor, prec: int, nrhs: int = 1, out=None, stream=None) -> torch.Tensor:
        """A x with A = C^-1 D (QWS's operator), packed fields."""
        if out is None:
            out = self.lattice.empty_packed(prec, nrhs)
        check(self.lib.mgc_apply_A(self.handle, _ptr(x), _ptr(out), nrhs, prec, _stream(stream)), "mgc_apply_A")
        return out

    def sap_smooth_A(self, b: torch.Tensor, x: torch.Tensor, prec: int, nrhs: int = 1, n_cy: int = 4,
                     n_jacobi: int = 4, x_is_zero: bool = False, stream=None) -> torch.Tensor:
        """QWS's M_SAP for A: n_cy sweeps with n_jacobi Jacobi iterations per domain, packed fields."""
        check(self.lib.mgc_sap_smooth_A(self.handle, _ptr(b), _ptr(x), nrhs, n_cy, n_jacobi, prec,
                                        int(bool(x_is_zero)), _stream(stream)), "mgc_sap_smooth_A")
        return x

    def A(self, psi, prec: int = 64) -> torch.Tensor:
        """A psi for canonical complex128 field(s), computed at prec."""
        psi = _canon(psi, "cuda")
        nrhs = 1 if psi.dim() == 3 else psi.shape[0]
        x = self.lattice.pack(psi, prec)
        return self.lattice.unpack(self.apply_A(x, prec, nrhs), prec, nrhs)

    def sap_A(self, b, prec: int = 64, n_cy: int = 4, n_jacobi: int = 4, x0=None) -> torch.Tensor:
        """n_cy SAP sweeps on A x = b from x0 (default 0), canonical in and out."""
        b = _canon(b, "cuda")
        nrhs = 1 if b.dim() == 3 else b.shape[0]
        bp = self.lattice.pack(b, prec)
        xp = self.lattice.zeros_packed(prec, nrhs) if x0 is None else self.lattice.pack(_canon(x0, "cuda"), prec)
        self.sap_smooth_A(bp, xp, prec, nrhs, n_cy, n_jacobi, x_is_zero=x0 is None)
        return self.lattice.unpack(xp, prec, nrhs)

    def export_clover(self, inverse=False, stream=None) -> torch.Tensor:
        out = torch.empty((self.lattice.volume, 12, 12), dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_clover_export(self.handle, int(bool(inverse)), _ptr(out), _stream(stream)),
              "mgc_clover_export")
        return out

    # -- canonical-field conveniences --------------------------------------------
    def D(self, psi, prec: int = 64, dagger=False) -> torch.Tensor:
        """D psi (or D^dagger psi) for canonical complex128 field(s), computed at prec."""
        psi = _canon(psi, "cuda")
        nrhs = 1 if psi.dim() == 3 else psi.shape[0]
        x = self.lattice.pack(psi, prec)
        y = (self.apply_Ddag if dagger else self.apply_D)(x, prec, nrhs)
        return self.lattice.unpack(y, prec, nrhs)

    def sap(self, b, prec: int = 64, n_cy: int = 4, n_mr: int = 4, x0=None) -> torch.Tensor:
        """n_cy SAP sweeps on D x = b from x0 (default 0), canonical in and out."""
        b = _canon(b, "cuda")
        nrhs = 1 if b.dim() == 3 else b.shape[0]
        bp = self.lattice.pack(b, prec)
        if x0 is None:
            xp = self.lattice.zeros_packed(prec, nrhs)
        else:
            xp = self.lattice.pack(_canon(x0, "cuda"), prec)
        self.sap_smooth(bp, xp, prec, nrhs, n_cy, n_mr, x_is_zero=x0 is None)
        return self.lattice.unpack(xp, prec, nrhs)

    def solve(self, b, params: SolveParams | None = None, x0=None, stream=None, out=None, **kw):
        """Solve D x = b.  b: canonical complex128 on the GPU (on_device = 1) or a
        host tensor / array (on_device = 0).  `out` (optional) receives x and
        must live where b lives (pinned for host b).  Returns (x, info)."""
        p = params if params is not None else solve_params(**kw)
        host = not (isinstance(b, torch.Tensor) and b.is_cuda)
        if host:
            bt = _canon(b, "cpu")
            if not bt.is_pinned():
                bt = bt.pin_memory()
        else:
            bt = _canon(b, "cuda")
        p.on_device = 0 if host else 1
        nrhs = 1 if bt.dim() == 3 else bt.shape[0]
        if x0 is not None:
            x = _canon(x0, bt.device).clone()
            p.x_is_guess = 1
        elif out is not None:
            if out.shape != bt.shape or out.dtype != torch.complex128 or out.device != bt.device:
                raise ValueError("out must match b in shape, dtype and device")
            x = out
            p.x_is_guess = 0
        else:
            x = torch.zeros_like(bt)
            if host:
                x = x.pin_memory()
            p.x_is_guess = 0
        info = SolveInfo()
        st = self.lib.mgc_solve(self.handle, _ptr(bt), _ptr(x), nrhs, C.byref(p), C.byref(info), _stream(stream))
        if st not in (_lib.MGC_OK, _lib.MGC_NOT_CONVERGED):
            check(st, "mgc_solve")
        return x, info

    def force(self, phi, params: SolveParams | None = None, stream=None, action_parts=False, **kw):
        """dS/dU for S = phi^+ (D^+ D)^-1 phi; returns (g (V, 4, 3, 3) complex128, S, info).
        With action_parts, S is the pair (S rounded to double, remainder)."""
        p = params if params is not None else solve_params(**kw)
        on_device = isinstance(phi, torch.Tensor) and phi.is_cuda
        ph = _canon(phi, "cuda" if on_device else "cpu")
        p.on_device = int(on_device)
        g = torch.empty((self.lattice.volume, 4, 3, 3), dtype=torch.complex128, device=ph.device)
        info = SolveInfo()
        S = (C.c_double * 2)(0.0, 0.0)
        check(self.lib.mgc_force(self.handle, _ptr(ph), _ptr(g), C.byref(p), C.byref(info), S,
                                 _stream(stream)), "mgc_force")
        if action_parts:
            return g, (float(S[0]), float(S[1])), info
        return g, float(S[0]), info


def _ptr_array(ts):
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


class Batch:
    """Several operators (same storage format and SAP domain shape) with nrhs[k]
    right-hand sides each, driven by one launch per step (the ABI's mgc_batch_t).
    Field arguments are lists with one tensor per operator."""

    def __init__(self, ops, nrhs):
        if len(ops) != len(nrhs) or not 1 <= len(ops) <= _lib.MGC_BATCH_MAX:
            raise ValueError(f"need 1..{_lib.MGC_BATCH_MAX} operators, one nrhs each")
        self.lib = ops[0].lib
        self.ops = list(ops)
        self.nrhs = [int(n) for n in nrhs]
        h = C.c_void_p()
        hs = (C.c_void_p * len(ops))(*[op.handle.value for op in ops])
        nr = (C.c_int * len(ops))(*self.nrhs)
        check(self.lib.mgc_batch_create(hs, nr, len(ops), C.byref(h)), "mgc_batch_create")
        self.handle = h
        self.systems = int(self.lib.mgc_batch_systems(h))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.mgc_batch_destroy(h)
            self.handle = None

    def empty_packed(self, prec: int):
        return [op.lattice.empty_packed(prec, n) for op, n in zip(self.ops, self.nrhs)]

    def zeros_packed(self, prec: int):
        return [op.lattice.zeros_packed(prec, n) for op, n in zip(self.ops, self.nrhs)]

    def apply_D(self, xs, prec: int, dagger=False, out=None, stream=None):
        out = self.empty_packed(prec) if out is None else out
        check(self.lib.mgc_batch_apply_D(self.handle, _ptr_array(xs), _ptr_array(out), prec, int(bool(dagger)),
                                         _stream(stream)), "mgc_batch_apply_D")
        return out

    def sap_smooth(self, bs, xs, prec: int, n_cy: int = 4, n_mr: int = 4, x_is_zero=False, stream=None):
        check(self.lib.mgc_batch_sap_smooth(self.handle, _ptr_array(bs), _ptr_array(xs), n_cy, n_mr, prec,
                                            int(bool(x_is_zero)), _stream(stream)), "mgc_batch_sap_smooth")
        return xs

    def tune(self, prec: int, force=False, stream=None) -> dict:
        v = [C.c_int(0) for _ in range(4)]
        check(self.lib.mgc_batch_tune(self.handle, prec, int(bool(force)), *[C.byref(x) for x in v],
                                      _stream(stream)), "mgc_batch_tune")
        return {"rhs_per_thread": v[0].value, "threads": v[1].value, "rhs_fast_d": v[2].value,
                "rhs_fast_sap": v[3].value}

    def set_shape(self, prec: int, rhs_per_thread: int, threads: int, rhs_fast_d: int, rhs_fast_sap: int):
        check(self.lib.mgc_batch_set_shape(self.handle, prec, rhs_per_thread, threads, rhs_fast_d, rhs_fast_sap),
              "mgc_batch_set_shape")

    def solve(self, bs, params: SolveParams | None = None, x0=None, out=None, stream=None, **kw):
        """Solve every system; bs[k]: canonical (nrhs[k], V, 4, 3) complex128, all on
        the GPU or all on the host (pinned).  Returns (xs, infos) with one info per
        system, operator-major."""
        p = params if params is not None else solve_params(**kw)
        host = not (isinstance(bs[0], torch.Tensor) and bs[0].is_cuda)
        dev = "cpu" if host else "cuda"
        bt = []
        for b, op, n in zip(bs, self.ops, self.nrhs):
            t = _canon(b, dev).reshape(n, op.lattice.volume, 4, 3)
            if host and not t.is_pinned():
                t = t.pin_memory()
            bt.append(t)
        p.on_device = 0 if host else 1
        if x0 is not None:
            xs = [_canon(x, dev).reshape(t.shape).clone() for x, t in zip(x0, bt)]
            if host:
                xs = [x.pin_memory() for x in xs]
            p.x_is_guess = 1
        elif out is not None:
            xs = list(out)
            p.x_is_guess = 0
        else:
            xs = [torch.zeros_like(t) for t in bt]
            if host:
                xs = [x.pin_memory() for x in xs]
            p.x_is_guess = 0
        infos = (SolveInfo * self.systems)()
        st = self.lib.mgc_batch_solve(self.handle, _ptr_array(bt), _ptr_array(xs), C.byref(p), infos,
                                      _stream(stream))
        if st not in (_lib.MGC_OK, _lib.MGC_NOT_CONVERGED):
            check(st, "mgc_batch_solve")
        return xs, list(infos)


def mg_params(**kw) -> MgParams:
    p = MgParams()
    _lib.load().mgc_mg_params_default(C.byref(p))
    names = {f[0] for f in MgParams._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown multigrid parameter {k}")
        setattr(p, k, v)
    return p


class Multigrid:
    """Two-level multigrid on one operator (the ABI's mgc_mg_t): aggregates of
    agg sites split by chirality, nvec null vectors.  Canonical fields are
    complex128 torch tensors on the GPU: fine (V, 4, 3), coarse (Vc, 2, nvec)."""

    def __init__(self, op: CloverOperator, agg, nvec: int):
        self.lib = op.lib
        self.op = op
        self.agg = tuple(int(a) for a in agg)
        self.nvec = int(nvec)
        h = C.c_void_p()
        check(self.lib.mgc_mg_create(op.handle, (C.c_int * 4)(*self.agg), self.nvec, C.byref(h)), "mgc_mg_create")
        self.handle = h
        self.coarse_volume = int(self.lib.mgc_mg_coarse_volume(h))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.mgc_mg_destroy(h)
            self.handle = None

    def _fine(self, v):
        return _canon(v, "cuda").reshape(self.op.lattice.volume, 4, 3)

    def _coarse(self, u):
        return _canon(u, "cuda").reshape(self.coarse_volume, 2, self.nvec)

    def setup(self, eta, params: MgParams | None = None, stream=None, **kw):
        p = params if params is not None else mg_params(**kw)
        e = _canon(eta, "cuda").reshape(self.nvec, self.op.lattice.volume, 4, 3)
        check(self.lib.mgc_mg_setup(self.handle, _ptr(e), C.byref(p), _stream(stream)), "mgc_mg_setup")

    def set_vectors(self, V, stream=None):
        v = _canon(V, "cuda").reshape(self.nvec, self.op.lattice.volume, 4, 3)
        check(self.lib.mgc_mg_set_vectors(self.handle, _ptr(v), _stream(stream)), "mgc_mg_set_vectors")

    def export(self, stream=None):
        W = torch.empty((self.nvec, self.op.lattice.volume, 4, 3), dtype=torch.complex128, device="cuda")
        n2 = 2 * self.nvec
        Dc = torch.empty((self.coarse_volume, 9, n2, n2), dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_mg_export(self.handle, _ptr(W), _ptr(Dc), _stream(stream)), "mgc_mg_export")
        return W, Dc

    def restrict(self, v, stream=None):
        u = torch.empty((self.coarse_volume, 2, self.nvec), dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_mg_restrict(self.handle, _ptr(self._fine(v)), _ptr(u), _stream(stream)), "mgc_mg_restrict")
        return u

    def prolong(self, u, stream=None):
        v = torch.empty((self.op.lattice.volume, 4, 3), dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_mg_prolong(self.handle, _ptr(self._coarse(u)), _ptr(v), _stream(stream)), "mgc_mg_prolong")
        return v

    def coarse_apply(self, u, stream=None):
        out = torch.empty((self.coarse_volume, 2, self.nvec), dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_mg_coarse_apply(self.handle, _ptr(self._coarse(u)), _ptr(out), _stream(stream)),
              "mgc_mg_coarse_apply")
        return out

    def coarse_solve(self, b, tol=1e-6, maxit=1000, stream=None):
        x = torch.empty((self.coarse_volume, 2, self.nvec), dtype=torch.complex128, device="cuda")
        it = C.c_int(0)
        check(self.lib.mgc_mg_coarse_solve(self.handle, _ptr(self._coarse(b)), _ptr(x), float(tol), int(maxit),
                                           C.byref(it), _stream(stream)), "mgc_mg_coarse_solve")
        return x, int(it.value)

    def precond(self, v, params: MgParams | None = None, stream=None, **kw):
        p = params if params is not None else mg_params(**kw)
        x = torch.empty((self.op.lattice.volume, 4, 3), dtype=torch.complex128, device="cuda")
        check(self.lib.mgc_mg_precond(self.handle, _ptr(self._fine(v)), _ptr(x), C.byref(p), _stream(stream)),
              "mgc_mg_precond")
        return x

    def solve(self, b, params: SolveParams | None = None, mg: MgParams | None = None, out=None, stream=None,
              **kw):
        """Flexible BiCGStab preconditioned by the two-level preconditioner.  Returns (x, info)."""
        p = params if params is not None else solve_params(**kw)
        m = mg if mg is not None else mg_params()
        host = not (isinstance(b, torch.Tensor) and b.is_cuda)
        bt = _canon(b, "cpu" if host else "cuda")
        if host and not bt.is_pinned():
            bt = bt.pin_memory()
        p.on_device = 0 if host else 1
        p.x_is_guess = 0
        x = out if out is not None else torch.zeros_like(bt)
        if host and out is None:
            x = x.pin_memory()
        info = SolveInfo()
        st = self.lib.mgc_mg_solve(self.handle, _ptr(bt), _ptr(x), C.byref(p), C.byref(m), C.byref(info),
                                   _stream(stream))
        if st not in (_lib.MGC_OK, _lib.MGC_NOT_CONVERGED):
            check(st, "mgc_mg_solve")
        return x, info
