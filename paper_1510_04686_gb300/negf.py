"""ctypes binding of the C ABI in include/negf.h.

Argument marshalling only: tensors must already live on the GPU with the documented dtype and
layout; every computation happens in libnegf.so.  A missing library raises, there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_size_t, c_void_p

import torch

from . import _build

PREC_FP64 = 0
PREC_MIXED = 1       # tensor cores, 48-bit operand values
PREC_MIXED_40 = 2    # tensor cores, 40-bit operand values
PREC_MIXED_56 = 3    # tensor cores, 56-bit operand values
PREC_AUTO = -1       # lead_precision: FP64 for the FP64 form, else 56-bit (48 beyond b = 7008)
SIGMA_ORBITAL_DIAG = 0  # scattering self-energies: one value per orbital
SIGMA_ATOM_BLOCK = 1    # scattering self-energies: one atom_orbitals^2 block per atom
WS_LEAD, WS_RGF, WS_ADJOINT, WS_ADJOINT_CKPT = 0, 1, 2, 3

_STATUS = {
    0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "workspace too small",
    4: "lead decimation did not converge", 5: "zero pivot", 6: "non-finite output",
    7: "timeout", 8: "unsupported option or size",
}


class NegfError(RuntimeError):
    def __init__(self, code, where, detail=""):
        msg = f"{where}: negf status {code} ({_STATUS.get(code, 'unknown')})"
        super().__init__(msg + (f": {detail}" if detail else ""))
        self.code = code


class _Dev(ctypes.Structure):
    _fields_ = [("n_sys", c_int32), ("n_slabs", c_int32), ("block", c_int32),
                ("iface_rows", c_int32), ("H_diag", c_void_p), ("H_up", c_void_p),
                ("iface_cols", c_int32), ("reserved", c_int32)]


class _Opt(ctypes.Structure):
    _fields_ = [("eta_lead", c_double), ("eta_device", c_double), ("mu_L", c_double),
                ("mu_R", c_double), ("kT", c_double), ("sr_tol", c_double),
                ("sr_max_iter", c_int32), ("precision", c_int32), ("refine_steps", c_int32),
                ("chunk", c_int32), ("sr_host_check", c_int32), ("adjoint_segment", c_int32),
                ("lead_precision", c_int32), ("refine_max", c_int32),
                ("sigma_structure", c_int32), ("atom_orbitals", c_int32)]


def sigma_width(opt) -> int:
    """Entries per orbital of a scattering self-energy / diag-G row: 1, or the atom block
    width under SIGMA_ATOM_BLOCK (rows hold N b A entries)."""
    return int(opt.atom_orbitals) if opt.sigma_structure == SIGMA_ATOM_BLOCK else 1


_LIB = None
EXPORTS = ("negf_default_options", "negf_abi_version", "negf_status_string",
           "negf_workspace_size", "negf_lead_selfenergy", "negf_rgf_solve", "negf_scba_step",
           "negf_rgf_adjoint", "negf_integrate", "negf_zgemm_workspace_size",
           "negf_zgemm_batched", "negf_zinv_workspace_size", "negf_zinv_batched",
           "negf_profile_enable", "negf_profile_reset", "negf_profile_read", "negf_profile_flops",
           "negf_launch_count", "negf_zinv_batched_noalloc", "negf_tc_config_count",
           "negf_tc_config_set", "negf_tc_config_get", "negf_last_cuda_error",
           "negf_fp64_fallback_count", "negf_debug_fail_waits", "negf_poisson_apply",
           "negf_orbitals_to_atoms", "negf_atoms_to_orbitals", "negf_scba_step_mesh",
           "negf_checkpoint_bytes")


def library():
    """Load libnegf.so (built in-tree by __graft_entry__.build / _build.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libnegf.so not found at {path}; build it with "
                           "paper_1510_04686_gb300._build.build()")
    lib = ctypes.CDLL(path)
    P = c_void_p
    lib.negf_default_options.argtypes = [POINTER(_Opt)]
    lib.negf_default_options.restype = None
    lib.negf_abi_version.restype = c_int32
    lib.negf_status_string.argtypes = [c_int32]
    lib.negf_status_string.restype = ctypes.c_char_p
    lib.negf_workspace_size.argtypes = [POINTER(_Dev), c_int32, POINTER(_Opt), c_int32]
    lib.negf_workspace_size.restype = c_size_t
    lib.negf_lead_selfenergy.argtypes = [POINTER(_Dev), c_int32, P, P, POINTER(_Opt), P, P, P, P,
                                         P, c_size_t, P]
    lib.negf_lead_selfenergy.restype = c_int32
    lib.negf_rgf_solve.argtypes = [POINTER(_Dev), c_int32, P, P, P, P, P, P, P, P, c_int32,
                                   POINTER(_Opt), P, P, P, P, P, P, P, P, c_size_t, P]
    lib.negf_rgf_solve.restype = c_int32
    lib.negf_scba_step.argtypes = [c_int32, c_int32, c_int32, P, c_double, c_double, c_int32,
                                   c_double, c_double, P, P, P, P, P, P]
    lib.negf_scba_step.restype = c_int32
    lib.negf_rgf_adjoint.argtypes = [POINTER(_Dev), c_int32, P, P, P, P, P, P, P, P, c_int32,
                                     POINTER(_Opt), P, P, P, P, P, P, c_size_t, P]
    lib.negf_checkpoint_bytes.argtypes = [POINTER(_Dev), c_int32]
    lib.negf_checkpoint_bytes.restype = c_size_t
    lib.negf_rgf_adjoint.restype = c_int32
    lib.negf_integrate.argtypes = [c_int32, c_int32, c_int32, P, P, P, P, P]
    lib.negf_integrate.restype = c_int32
    lib.negf_zgemm_workspace_size.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32]
    lib.negf_zgemm_workspace_size.restype = c_size_t
    i64 = ctypes.c_int64
    lib.negf_zgemm_batched.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, c_double,
                                       c_double, P, i64, c_int32, c_int32, P, i64, c_int32,
                                       c_int32, c_double, c_double, P, i64, c_int32, P, c_size_t,
                                       P]
    lib.negf_zgemm_batched.restype = c_int32
    lib.negf_zinv_workspace_size.argtypes = [c_int32, c_int32, c_int32]
    lib.negf_zinv_workspace_size.restype = c_size_t
    lib.negf_zinv_batched.argtypes = [c_int32, c_int32, c_int32, P, P, c_int32, P, P, c_size_t,
                                      P]
    lib.negf_zinv_batched.restype = c_int32
    lib.negf_profile_enable.argtypes = [c_int32]
    lib.negf_profile_enable.restype = None
    lib.negf_profile_reset.argtypes = []
    lib.negf_profile_reset.restype = None
    lib.negf_profile_read.argtypes = [c_int32, POINTER(ctypes.c_longlong), POINTER(c_double)]
    lib.negf_profile_read.restype = c_int32
    lib.negf_profile_flops.argtypes = [c_int32, POINTER(c_double), POINTER(c_double)]
    lib.negf_profile_flops.restype = c_int32
    lib.negf_launch_count.argtypes = []
    lib.negf_launch_count.restype = ctypes.c_longlong
    lib.negf_zinv_batched_noalloc.argtypes = [c_int32, c_int32, P, P, P, P]
    lib.negf_zinv_batched_noalloc.restype = c_int32
    lib.negf_tc_config_count.argtypes = []
    lib.negf_tc_config_count.restype = c_int32
    lib.negf_tc_config_set.argtypes = [c_int32]
    lib.negf_tc_config_set.restype = c_int32
    lib.negf_tc_config_get.argtypes = []
    lib.negf_tc_config_get.restype = c_int32
    lib.negf_last_cuda_error.argtypes = []
    lib.negf_last_cuda_error.restype = ctypes.c_char_p
    lib.negf_scba_step_mesh.argtypes = [c_int32, c_int32, c_int32, P, P, c_double, c_double,
                                        c_double, c_double, c_double, P, P, P, P, P, P]
    lib.negf_scba_step_mesh.restype = c_int32
    lib.negf_poisson_apply.argtypes = [c_int32, c_int32, c_double, c_double, c_double, c_double,
                                       c_double, P, P, P, P, P]
    lib.negf_poisson_apply.restype = c_int32
    lib.negf_orbitals_to_atoms.argtypes = [c_int32, c_int32, c_int32, c_int32, P, P, P]
    lib.negf_orbitals_to_atoms.restype = c_int32
    lib.negf_atoms_to_orbitals.argtypes = [c_int32, c_int32, c_int32, P, P, P]
    lib.negf_atoms_to_orbitals.restype = c_int32
    lib.negf_debug_fail_waits.argtypes = [c_int32]
    lib.negf_debug_fail_waits.restype = None
    lib.negf_fp64_fallback_count.argtypes = []
    lib.negf_fp64_fallback_count.restype = ctypes.c_longlong
    _LIB = lib
    return lib


def options(**kw) -> _Opt:
    """negf_options with the library defaults, overridden by keyword."""
    o = _Opt()
    library().negf_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _need(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _rows(scat):
    return 0 if scat is None else int(scat.shape[0])


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


class Device:
    """Block-tridiagonal Hamiltonians H_diag [n_sys,N,b,b], H_up [n_sys,N-1,b,b] (complex128).

    iface=(r, c): every H_{i,i+1} is nonzero only in its last r rows and first c columns (the
    facing atoms of neighbouring slabs); the sweeps then contract over r or c instead of b."""

    def __init__(self, H_diag: torch.Tensor, H_up: torch.Tensor | None, iface=None):
        _need(H_diag, torch.complex128, "H_diag")
        if H_diag.dim() != 4 or H_diag.shape[2] != H_diag.shape[3]:
            raise ValueError("H_diag must be [n_sys, N, b, b]")
        n_sys, N, b, _ = H_diag.shape
        if N > 1:
            _need(H_up, torch.complex128, "H_up", (n_sys, N - 1, b, b))
        self.H_diag, self.H_up = H_diag, H_up
        self.n_sys, self.N, self.b = int(n_sys), int(N), int(b)
        r, c = (0, 0) if iface is None else (int(iface[0]), int(iface[1]))
        self.iface = iface
        self.c = _Dev(self.n_sys, self.N, self.b, r, H_diag.data_ptr(),
                      H_up.data_ptr() if (H_up is not None and N > 1) else None, c, 0)


_WS = {}


def _workspace(nbytes, device):
    # one buffer per (device, stream): calls on different streams may run concurrently
    key = (str(device), torch.cuda.current_stream(device).cuda_stream)
    buf = _WS.get(key)
    if buf is None or buf.numel() < nbytes:
        _WS.pop(key, None)
        buf = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
        _WS[key] = buf
    return buf


def workspace_size(dev: Device, n_pts: int, opt: _Opt, which: int) -> int:
    return int(library().negf_workspace_size(ctypes.byref(dev.c), n_pts, ctypes.byref(opt), which))


def _check(code, where):
    if code != 0:
        detail = ""
        if code == 2:  # NEGF_ERR_CUDA: name the CUDA runtime error behind it
            detail = library().negf_last_cuda_error().decode()
        raise NegfError(code, where, detail)


def lead_selfenergy(dev: Device, E: torch.Tensor, sys_idx: torch.Tensor, opt: _Opt):
    """Sancho-Rubio lead self-energies: returns dict(sigma_R, sigma_L [n,2,b,b], iters, status)."""
    _need(E, torch.float64, "E")
    n = E.numel()
    _need(sys_idx, torch.int32, "sys_idx", (n,))
    b = dev.b
    dv = E.device
    sR = torch.empty((n, 2, b, b), dtype=torch.complex128, device=dv)
    sL = torch.empty_like(sR)
    it = torch.empty((n, 2), dtype=torch.int32, device=dv)
    st = torch.empty((n,), dtype=torch.int32, device=dv)
    nb = workspace_size(dev, max(n, 1), opt, WS_LEAD)
    ws = _workspace(nb, dv)
    _check(library().negf_lead_selfenergy(ctypes.byref(dev.c), n, _ptr(E), _ptr(sys_idx),
                                          ctypes.byref(opt), _ptr(sR), _ptr(sL), _ptr(it),
                                          _ptr(st), _ptr(ws), nb, _stream()),
           "negf_lead_selfenergy")
    return dict(sigma_R=sR, sigma_L=sL, iters=it, status=st)


def checkpoint_buffer(dev: Device, n_pts: int, device=None):
    """A buffer for the sweep checkpoints negf_rgf_solve hands to negf_rgf_adjoint:
    complex128 [5, N, n_pts, b, b] (5 N b^2 complex numbers per point)."""
    nb = int(library().negf_checkpoint_bytes(ctypes.byref(dev.c), int(n_pts)))
    if nb == 0:
        raise ValueError("no checkpoints for this device / point count")
    return torch.empty((5, dev.N, n_pts, dev.b, dev.b), dtype=torch.complex128,
                       device=device if device is not None else dev.H_diag.device)


def rgf_solve(dev: Device, E, sys_idx, sigma_R, sigma_L, opt, V=None, scat_R=None, scat_L=None,
              e_idx=None, outputs=("density", "current", "transmission"), diag=False,
              checkpoints=None):
    """Forward/backward RGF sweeps and observables for every point (negf_rgf_solve).

    checkpoints: an optional buffer from checkpoint_buffer(dev, n) that receives the sweep blocks
    for a later rgf_adjoint of the same points."""
    _need(E, torch.float64, "E")
    n = E.numel()
    N, b = dev.N, dev.b
    _need(sys_idx, torch.int32, "sys_idx", (n,))
    _need(sigma_R, torch.complex128, "sigma_R", (n, 2, b, b))
    _need(sigma_L, torch.complex128, "sigma_L", (n, 2, b, b))
    if V is not None:
        _need(V, torch.float64, "V", (N, b))
    A = sigma_width(opt)
    if scat_R is not None:
        _need(scat_R, torch.complex128, "scat_R")
        _need(scat_L, torch.complex128, "scat_L", tuple(scat_R.shape))
        if scat_R.shape[-1] != N * b * A:
            raise ValueError(f"scat_R rows must hold N*b*{A} entries")
    if e_idx is not None:
        _need(e_idx, torch.int32, "e_idx", (n,))
    if checkpoints is not None:
        _need(checkpoints, torch.complex128, "checkpoints", (5, N, n, b, b))
    dv = E.device
    out = {}
    dens = torch.empty((n, N * b), dtype=torch.float64, device=dv) if "density" in outputs else None
    cur = (torch.empty((n, max(N - 1, 0)), dtype=torch.float64, device=dv)
           if "current" in outputs else None)
    tr = torch.empty((n,), dtype=torch.float64, device=dv) if "transmission" in outputs else None
    dGR = torch.empty((n, N * b * A), dtype=torch.complex128, device=dv) if diag else None
    dGL = torch.empty((n, N * b * A), dtype=torch.complex128, device=dv) if diag else None
    st = torch.empty((n,), dtype=torch.int32, device=dv)
    nb = workspace_size(dev, max(n, 1), opt, WS_RGF)
    ws = _workspace(nb, dv)
    _check(library().negf_rgf_solve(ctypes.byref(dev.c), n, _ptr(E), _ptr(sys_idx), _ptr(V),
                                    _ptr(sigma_R), _ptr(sigma_L), _ptr(scat_R), _ptr(scat_L),
                                    _ptr(e_idx), _rows(scat_R), ctypes.byref(opt), _ptr(dens),
                                    _ptr(cur),
                                    _ptr(tr), _ptr(dGR), _ptr(dGL), _ptr(checkpoints), _ptr(st),
                                    _ptr(ws), nb, _stream()), "negf_rgf_solve")
    out.update(density=dens, current=cur, transmission=tr, diagGR=dGR, diagGL=dGL, status=st)
    return out


def scba_step(diagGR, diagGL, w_k, sigma_R, sigma_L, D_ac, D_op, shift, n0, mix=1.0):
    """One Born update (negf_scba_step); sigma_R/L [n_E, n_orb] are updated in place.

    diagGR/diagGL are [n_k, n_E, n_orb] complex128; returns the device scalar max|dSigma|."""
    _need(diagGR, torch.complex128, "diagGR")
    n_k, n_E, n_orb = diagGR.shape
    _need(diagGL, torch.complex128, "diagGL", (n_k, n_E, n_orb))
    _need(w_k, torch.float64, "w_k", (n_k,))
    _need(sigma_R, torch.complex128, "sigma_R", (n_E, n_orb))
    _need(sigma_L, torch.complex128, "sigma_L", (n_E, n_orb))
    delta = torch.empty((1,), dtype=torch.float64, device=diagGR.device)
    _check(library().negf_scba_step(n_k, n_E, n_orb, _ptr(w_k), float(D_ac), float(D_op),
                                    int(shift), float(n0), float(mix), _ptr(diagGR),
                                    _ptr(diagGL), _ptr(sigma_R), _ptr(sigma_L), _ptr(delta),
                                    _stream()), "negf_scba_step")
    return delta


def scba_step_mesh(diagGR, diagGL, w_k, E, sigma_R, sigma_L, D_ac, D_op, hw, n0, mix=1.0):
    """Born update on a non-uniform energy mesh E [n_E] (negf_scba_step_mesh): optical terms at
    E +- hw by linear interpolation; sigma_R/L [n_E, n_orb] are updated in place.  Returns the
    device scalar max|dSigma|."""
    _need(diagGR, torch.complex128, "diagGR")
    n_k, n_E, n_orb = diagGR.shape
    _need(diagGL, torch.complex128, "diagGL", (n_k, n_E, n_orb))
    _need(w_k, torch.float64, "w_k", (n_k,))
    _need(E, torch.float64, "E", (n_E,))
    _need(sigma_R, torch.complex128, "sigma_R", (n_E, n_orb))
    _need(sigma_L, torch.complex128, "sigma_L", (n_E, n_orb))
    delta = torch.empty((1,), dtype=torch.float64, device=diagGR.device)
    _check(library().negf_scba_step_mesh(n_k, n_E, n_orb, _ptr(E), _ptr(w_k), float(D_ac),
                                         float(D_op), float(hw), float(n0), float(mix),
                                         _ptr(diagGR), _ptr(diagGL), _ptr(sigma_R),
                                         _ptr(sigma_L), _ptr(delta), _stream()),
           "negf_scba_step_mesh")
    return delta


def rgf_adjoint(dev: Device, E, sys_idx, sigma_R, sigma_L, opt, density_bar=None,
                current_bar=None, V=None, scat_R=None, scat_L=None, e_idx=None,
                checkpoints=None):
    """dL/dV for cotangents of density [n, N*b] and current [n, N-1] (negf_rgf_adjoint).

    checkpoints: the buffer an rgf_solve of the same points, V and options filled; the sweeps
    are then not recomputed."""
    _need(E, torch.float64, "E")
    n = E.numel()
    N, b = dev.N, dev.b
    if density_bar is not None:
        _need(density_bar, torch.float64, "density_bar", (n, N * b))
    if current_bar is not None:
        _need(current_bar, torch.float64, "current_bar", (n, N - 1))
    if V is not None:
        _need(V, torch.float64, "V", (N, b))
    if scat_R is not None and scat_R.shape[-1] != N * b * sigma_width(opt):
        raise ValueError(f"scat_R rows must hold N*b*{sigma_width(opt)} entries")
    if checkpoints is not None:
        _need(checkpoints, torch.complex128, "checkpoints", (5, N, n, b, b))
    dv = E.device
    Vbar = torch.empty((N, b), dtype=torch.float64, device=dv)
    st = torch.empty((n,), dtype=torch.int32, device=dv)
    nb = workspace_size(dev, max(n, 1), opt, WS_ADJOINT if checkpoints is None else WS_ADJOINT_CKPT)
    ws = _workspace(nb, dv)
    _check(library().negf_rgf_adjoint(ctypes.byref(dev.c), n, _ptr(E), _ptr(sys_idx), _ptr(V),
                                      _ptr(sigma_R), _ptr(sigma_L), _ptr(scat_R), _ptr(scat_L),
                                      _ptr(e_idx), _rows(scat_R), ctypes.byref(opt),
                                      _ptr(checkpoints), _ptr(density_bar),
                                      _ptr(current_bar), _ptr(Vbar), _ptr(st), _ptr(ws), nb,
                                      _stream()), "negf_rgf_adjoint")
    return Vbar, st


def integrate(values, w, group=None, n_groups=1):
    """out[g] = sum_{p in g} w[p] values[p] in FP64, fixed order (negf_integrate)."""
    _need(values, torch.float64, "values")
    n = values.shape[0]
    ln = values[0].numel() if n else 0
    _need(w, torch.float64, "w", (n,))
    out = torch.empty((n_groups,) + tuple(values.shape[1:]), dtype=torch.float64,
                      device=values.device)
    _check(library().negf_integrate(n, ln, n_groups, _ptr(w), _ptr(group), _ptr(values),
                                    _ptr(out), _stream()), "negf_integrate")
    return out


_OPS = {"N": 0, "T": 1, "C": 2}


def zgemm(A, B, C=None, alpha=1.0, beta=0.0, opA="N", opB="N", precision=PREC_FP64):
    """Batched C = alpha op(A) op(B) + beta C on [n, rows, cols] complex128 CUDA tensors.

    A or B may be 2-D (shared by every batch item)."""
    def bview(X, name):
        _need(X, torch.complex128, name)
        if X.dim() == 2:
            return X, 0
        return X, X.shape[1] * X.shape[2]
    A, sA = bview(A, "A")
    B, sB = bview(B, "B")
    nb = max(A.shape[0] if A.dim() == 3 else 1, B.shape[0] if B.dim() == 3 else 1)
    ra, ca = A.shape[-2], A.shape[-1]
    rb, cb = B.shape[-2], B.shape[-1]
    M, K = (ra, ca) if opA == "N" else (ca, ra)
    K2, N = (rb, cb) if opB == "N" else (cb, rb)
    if K != K2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((nb, M, N), dtype=torch.complex128, device=A.device)
    _need(C, torch.complex128, "C", (nb, M, N))
    ws_n = int(library().negf_zgemm_workspace_size(precision, nb, M, N, K))
    ws = _workspace(ws_n, A.device)
    a = complex(alpha)
    b = complex(beta)
    _check(library().negf_zgemm_batched(precision, nb, M, N, K, a.real, a.imag, _ptr(A), sA,
                                        A.shape[-1], _OPS[opA], _ptr(B), sB, B.shape[-1],
                                        _OPS[opB], b.real, b.imag, _ptr(C), M * N, N, _ptr(ws),
                                        ws_n, _stream()), "negf_zgemm_batched")
    return C


def zinv(M, precision=PREC_FP64, refine_steps=2):
    """Batched inverse of [n, b, b] complex128; returns (X, status).  M is consumed in FP64."""
    _need(M, torch.complex128, "M")
    nb, n, _ = M.shape
    X = torch.empty_like(M)
    st = torch.empty((nb,), dtype=torch.int32, device=M.device)
    ws_n = int(library().negf_zinv_workspace_size(precision, nb, n))
    ws = _workspace(ws_n, M.device)
    _check(library().negf_zinv_batched(precision, nb, n, _ptr(M), _ptr(X), refine_steps,
                                       _ptr(st), _ptr(ws), ws_n, _stream()),
           "negf_zinv_batched")
    return X, st


PROF_TC_GEMM, PROF_SLICE, PROF_INV, PROF_GJ_PANEL = 0, 1, 2, 3


def profile(enable: bool):
    library().negf_profile_enable(1 if enable else 0)


def profile_reset():
    library().negf_profile_reset()


def profile_read(kind=PROF_TC_GEMM):
    """(launches, total_ms, algorithmic_flops, issued_bf16_flops) of a kernel kind."""
    n = ctypes.c_longlong(0)
    ms = c_double(0.0)
    _check(library().negf_profile_read(kind, ctypes.byref(n), ctypes.byref(ms)), "profile_read")
    a = c_double(0.0)
    h = c_double(0.0)
    _check(library().negf_profile_flops(kind, ctypes.byref(a), ctypes.byref(h)), "profile_flops")
    return int(n.value), float(ms.value), float(a.value), float(h.value)


def launch_count() -> int:
    return int(library().negf_launch_count())


def fp64_fallback_count() -> int:
    """Mixed-form block inverses recomputed in FP64 since load (synchronises the device)."""
    return int(library().negf_fp64_fallback_count())


class RGFFunction(torch.autograd.Function):
    """(density [n, N*b], current [n, N-1]) = RGF(V [N, b]) with a hand-written adjoint.

    Forward runs negf_rgf_solve; backward runs negf_rgf_adjoint with the incoming cotangents, so
    autograd returns dL/dV for any scalar L built from the density and current (the gradient a
    Newton-Poisson loop needs).  Lead and scattering self-energies are held fixed.  With
    keep_sweeps the forward pass keeps the sweep checkpoints (5 N b^2 complex per point) and the
    backward pass recomputes no sweep."""

    @staticmethod
    def forward(ctx, V, dev, E, sys_idx, sigma_R, sigma_L, opt, scat_R=None, scat_L=None,
                e_idx=None, keep_sweeps=False):
        ck = checkpoint_buffer(dev, E.numel(), E.device) if keep_sweeps else None
        out = rgf_solve(dev, E, sys_idx, sigma_R, sigma_L, opt, V=V.detach().contiguous(),
                        scat_R=scat_R, scat_L=scat_L, e_idx=e_idx,
                        outputs=("density", "current"), checkpoints=ck)
        ctx.args = (dev, E, sys_idx, sigma_R, sigma_L, opt, scat_R, scat_L, e_idx, ck)
        ctx.save_for_backward(V.detach())
        return out["density"], out["current"]

    @staticmethod
    def backward(ctx, g_density, g_current):
        (V,) = ctx.saved_tensors
        dev, E, sys_idx, sigma_R, sigma_L, opt, scat_R, scat_L, e_idx, ck = ctx.args
        gd = None if g_density is None else g_density.contiguous()
        gc = None if g_current is None else g_current.contiguous()
        Vbar, _ = rgf_adjoint(dev, E, sys_idx, sigma_R, sigma_L, opt, density_bar=gd,
                              current_bar=gc, V=V, scat_R=scat_R, scat_L=scat_L, e_idx=e_idx,
                              checkpoints=ck)
        return (Vbar,) + (None,) * 10


def rgf(V, dev, E, sys_idx, sigma_R, sigma_L, opt, scat_R=None, scat_L=None, e_idx=None,
        keep_sweeps=False):
    """Differentiable (density, current) of the points with respect to V; keep_sweeps hands the
    solve's sweep blocks to the adjoint instead of recomputing them."""
    return RGFFunction.apply(V, dev, E, sys_idx, sigma_R, sigma_L, opt, scat_R, scat_L, e_idx,
                             keep_sweeps)


def tc_config(idx=None):
    """Get (and with idx, set) the tensor-core GEMM kernel configuration."""
    lib = library()
    if idx is not None:
        _check(lib.negf_tc_config_set(int(idx)), "negf_tc_config_set")
    return int(lib.negf_tc_config_get())


def tc_config_count():
    return int(library().negf_tc_config_count())


class GraphSolve:
    """A lead + RGF solve of fixed points captured once in a CUDA graph and replayed.

    The decimation runs a fixed sr_max_iter steps with converged points masked on the device
    (sr_host_check = 0), so the captured sequence has no host synchronisation.  Inputs are the
    tensors given here; change their contents in place and call replay() to solve again (for
    example once per Born iteration with updated scattering self-energies).
    """

    def __init__(self, dev: Device, E, sys_idx, opt: _Opt, sr_steps: int = 40, V=None,
                 scat_R=None, scat_L=None, e_idx=None, diag=False):
        o = _Opt()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opt), ctypes.sizeof(_Opt))
        o.sr_host_check = 0
        o.sr_max_iter = sr_steps
        self.opt = o
        args = (dev, E, sys_idx)
        kw = dict(V=V, scat_R=scat_R, scat_L=scat_L, e_idx=e_idx, diag=diag)
        # warm-up outside capture: workspace allocation, kernel attributes, tensor-map encoder
        lead = lead_selfenergy(*args, o)
        rgf_solve(*args, lead["sigma_R"], lead["sigma_L"], o, **kw)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(self.graph, stream=s):
                self.lead = lead_selfenergy(*args, o)
                self.out = rgf_solve(*args, self.lead["sigma_R"], self.lead["sigma_L"], o, **kw)
        torch.cuda.current_stream().wait_stream(s)

    def replay(self):
        self.graph.replay()
        return self.out


_RAGGED_STREAMS = {}


def solve_ragged(systems, opt: _Opt, outputs=("density", "current", "transmission"),
                 concurrent=True):
    """Solve many systems of different block sizes: ``systems`` is a list of
    (H_diag [N,b,b], H_up [N-1,b,b], E [n]) complex128 / float64 CUDA tensors.

    Systems with the same (N, b) are stacked into one device (one batched lead + sweep chain per
    group, points of every system of the group in one call); groups run on separate CUDA streams
    so that small and large block sizes overlap.  Returns one result dict per system."""
    groups = {}
    for i, (Hd, Hu, E) in enumerate(systems):
        groups.setdefault((int(Hd.shape[0]), int(Hd.shape[1])), []).append(i)
    results = [None] * len(systems)
    cur = torch.cuda.current_stream()
    # the side streams are kept across calls: each owns a cached workspace
    pool = _RAGGED_STREAMS.setdefault(str(cur.device), [])
    streams = []
    for g, ((N, b), idx) in enumerate(sorted(groups.items(), key=lambda kv: -kv[0][1])):
        if concurrent:
            while len(pool) <= g:
                pool.append(torch.cuda.Stream(device=cur.device))
            st = pool[g]
        else:
            st = cur
        st.wait_stream(cur)
        streams.append(st)
        with torch.cuda.stream(st):
            Hd = torch.stack([systems[i][0] for i in idx])
            Hu = torch.stack([systems[i][1] for i in idx]) if N > 1 else None
            dev = Device(Hd, Hu)
            E = torch.cat([systems[i][2] for i in idx])
            sys_idx = torch.cat([torch.full((systems[i][2].numel(),), j, dtype=torch.int32,
                                            device=E.device) for j, i in enumerate(idx)])
            lead = lead_selfenergy(dev, E, sys_idx, opt)
            out = rgf_solve(dev, E, sys_idx, lead["sigma_R"], lead["sigma_L"], opt,
                            outputs=outputs)
            off = 0
            for i in idx:
                n = systems[i][2].numel()
                results[i] = {k: (v[off:off + n] if isinstance(v, torch.Tensor) else v)
                              for k, v in out.items()}
                off += n
    for st in streams:
        cur.wait_stream(st)
    return results


class RaggedGraph:
    """A batch of systems with different block sizes solved by one CUDA graph.

    ``systems`` is a list of (H_diag [N,b,b], H_up [N-1,b,b], E [n]) complex128 / float64 CUDA
    tensors (for example alloy samples of different cross-sections, each with its energy list).
    Systems of equal (N, b) are stacked into one device; each such group's lead decimation and
    RGF sweeps are one batched launch chain on a stream of its own, and the chains of all groups
    are captured together in one CUDA graph (fork from and join to the capturing stream), so a
    replay launches the whole ragged batch at once and the groups overlap on the GPU.  The
    decimation runs a fixed ``sr_steps`` steps with converged points masked on the device, so
    the capture has no host synchronisation.  The Hamiltonians are stacked (copied) once, here;
    the energy tensors given here are read again by every replay(), so changing them in place
    and calling replay() solves the new energies.  replay() returns one result dict per system
    (views into the group outputs).  Results equal those of solve_ragged with the same fixed
    decimation steps.
    """

    def __init__(self, systems, opt: _Opt, sr_steps: int = 40,
                 outputs=("density", "current", "transmission")):
        o = _Opt()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opt), ctypes.sizeof(_Opt))
        o.sr_host_check = 0
        o.sr_max_iter = sr_steps
        self.opt = o
        groups = {}
        for i, (Hd, Hu, E) in enumerate(systems):
            groups.setdefault((int(Hd.shape[0]), int(Hd.shape[1])), []).append(i)
        cur = torch.cuda.current_stream()
        self.groups = []
        for (N, b), idx in sorted(groups.items(), key=lambda kv: -kv[0][1]):
            Hd = torch.stack([systems[i][0] for i in idx])
            Hu = torch.stack([systems[i][1] for i in idx]) if N > 1 else None
            E = torch.cat([systems[i][2] for i in idx])
            sys_idx = torch.cat([torch.full((systems[i][2].numel(),), j, dtype=torch.int32,
                                            device=E.device) for j, i in enumerate(idx)])
            self.groups.append(dict(dev=Device(Hd, Hu), E=E, sys=sys_idx, idx=idx,
                                    stream=torch.cuda.Stream(device=E.device)))
        self.n_systems = len(systems)
        self.energies = [systems[i][2] for i in range(len(systems))]
        self.sizes = [E.numel() for E in self.energies]

        def run():
            for gr in self.groups:
                gr["stream"].wait_stream(torch.cuda.current_stream())
            for gr in self.groups:
                with torch.cuda.stream(gr["stream"]):
                    lead = lead_selfenergy(gr["dev"], gr["E"], gr["sys"], o)
                    gr["out"] = rgf_solve(gr["dev"], gr["E"], gr["sys"], lead["sigma_R"],
                                          lead["sigma_L"], o, outputs=outputs)
                    gr["lead_status"] = lead["status"]
            for gr in self.groups:
                torch.cuda.current_stream().wait_stream(gr["stream"])

        # warm-up outside the capture: workspaces (one per stream), kernel attributes, tensor
        # maps' encoder
        run()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=cur.device)
        cap.wait_stream(cur)
        with torch.cuda.stream(cap):
            with torch.cuda.graph(self.graph, stream=cap):
                run()
        cur.wait_stream(cap)

    def replay(self):
        for gr in self.groups:  # the callers' current energies into the captured buffers
            gr["E"].copy_(torch.cat([self.energies[i] for i in gr["idx"]]))
        self.graph.replay()
        results = [None] * self.n_systems
        for gr in self.groups:
            off = 0
            for i in gr["idx"]:
                n = self.sizes[i]
                r = {k: (v[off:off + n] if isinstance(v, torch.Tensor) else v)
                     for k, v in gr["out"].items()}
                r["lead_status"] = gr["lead_status"][off:off + n]
                results[i] = r
                off += n
        return results


ORBITALS_PER_ATOM = 10


def poisson_apply(U, c_x, c_y, U_L=0.0, U_R=0.0, kappa=0.0, n=None, n_D=None):
    """Residual of Eq. 9 on the atom grid, F = K U - boundary terms - kappa (n - n_D)
    (negf_poisson_apply); U, n, n_D are [N, A] float64 CUDA tensors (n, n_D nullable)."""
    _need(U, torch.float64, "U")
    N, A = U.shape
    for t, name in ((n, "n"), (n_D, "n_D")):
        if t is not None:
            _need(t, torch.float64, name, (N, A))
    out = torch.empty_like(U)
    _check(library().negf_poisson_apply(N, A, float(c_x), float(c_y), float(U_L), float(U_R),
                                        float(kappa), _ptr(U), _ptr(n), _ptr(n_D), _ptr(out),
                                        _stream()), "negf_poisson_apply")
    return out


def orbitals_to_atoms(orb, N, b, per=ORBITALS_PER_ATOM):
    """[groups, N*b] (or [N*b]) per-orbital values -> [groups, N, A] per-atom sums."""
    _need(orb, torch.float64, "orb")
    groups = orb.numel() // (N * b)
    A = -(-b // per)
    out = torch.empty((groups, N, A), dtype=torch.float64, device=orb.device)
    _check(library().negf_orbitals_to_atoms(groups, N, b, per, _ptr(orb), _ptr(out), _stream()),
           "negf_orbitals_to_atoms")
    return out


def atoms_to_orbitals(U, b, per=ORBITALS_PER_ATOM):
    """[N, A] per-atom values -> [N, b] per-orbital values."""
    _need(U, torch.float64, "U")
    N = U.shape[0]
    out = torch.empty((N, b), dtype=torch.float64, device=U.device)
    _check(library().negf_atoms_to_orbitals(N, b, per, _ptr(U), _ptr(out), _stream()),
           "negf_atoms_to_orbitals")
    return out


def poisson_newton(dev: Device, E, w, sys_idx, opt: _Opt, n_D, kappa, c_x, c_y, U_L=0.0,
                   U_R=0.0, U0=None, tol=1e-9, max_iter=30, per=ORBITALS_PER_ATOM,
                   keep_sweeps=True):
    """Self-consistent NEGF-Poisson solution (Eqs. 1, 7 and 9): Newton's method on
    F(U) = K U - boundary terms - kappa (n(U) - n_D) = 0 for the potential energy U [N, A] per
    atom, the electrons per atom n(U) = sum_p w[p] n(E_p, U) summed over each atom's orbitals.

    Every step runs in the library: the RGF densities with U in Eq. 1 (negf_rgf_solve, V = U on
    each atom's orbitals), the FP64 quadrature, the Poisson residual, and the Jacobian
    J = K - kappa dn/dU, whose row for atom a is one adjoint sweep (negf_rgf_adjoint, the
    backward of RGFFunction) with the cotangent w[p] on atom a's orbitals; the Newton step is
    J^-1 (-F) by the FP64 block inverse and GEMM.  Lead self-energies do not depend on U and
    are computed once.  With keep_sweeps (5 N b^2 complex per point) the step's solve hands its
    sweep blocks to every adjoint sweep of the step, which then run only their reverse passes.
    Returns (U, list of max |F| per iteration)."""
    N, b = dev.N, dev.b
    A = -(-b // per)
    n_pts = E.numel()
    dv = E.device
    _need(w, torch.float64, "w", (n_pts,))
    _need(n_D, torch.float64, "n_D", (N, A))
    lead = lead_selfenergy(dev, E, sys_idx, opt)
    U = torch.zeros((N, A), dtype=torch.float64, device=dv) if U0 is None else U0.clone()
    # K: the linear part of the residual, column by column (grounded contacts, no charge)
    NA = N * A
    K = torch.empty((NA, NA), dtype=torch.float64, device=dv)
    unit = torch.zeros((N, A), dtype=torch.float64, device=dv)
    for j in range(NA):
        unit.view(-1)[j] = 1.0
        K[:, j] = poisson_apply(unit, c_x, c_y).view(-1)
        unit.view(-1)[j] = 0.0
    hist = []
    cot = torch.zeros((n_pts, N * b), dtype=torch.float64, device=dv)
    # the sweep blocks of each Newton step's solve serve all of its adjoint sweeps
    ck = checkpoint_buffer(dev, n_pts, dv) if keep_sweeps else None
    for _ in range(max_iter):
        V = atoms_to_orbitals(U, b, per)
        out = rgf_solve(dev, E, sys_idx, lead["sigma_R"], lead["sigma_L"], opt, V=V,
                        outputs=("density",), checkpoints=ck)
        n = orbitals_to_atoms(integrate(out["density"], w), N, b, per)[0]
        F = poisson_apply(U, c_x, c_y, U_L, U_R, kappa, n, n_D)
        hist.append(float(F.abs().max().item()))
        if hist[-1] < tol:
            break
        chi = torch.empty((NA, NA), dtype=torch.float64, device=dv)
        for i in range(N):
            for a in range(A):
                lo, hi = i * b + per * a, i * b + min(per * a + per, b)
                cot[:, lo:hi] = w[:, None]
                Vbar, _ = rgf_adjoint(dev, E, sys_idx, lead["sigma_R"], lead["sigma_L"], opt,
                                      density_bar=cot, V=V, checkpoints=ck)
                cot[:, lo:hi] = 0.0
                chi[i * A + a] = orbitals_to_atoms(Vbar, N, b, per).view(-1)
        # J = K - kappa chi  (as complex128 for the block kernels); delta = -J^-1 F
        J = K.to(torch.complex128)[None].contiguous()
        zgemm(chi.to(torch.complex128)[None].contiguous(),
              torch.eye(NA, dtype=torch.complex128, device=dv), J, alpha=-float(kappa), beta=1.0)
        Jinv, st = zinv(J, precision=PREC_FP64)
        if int(st.abs().sum().item()) != 0:
            raise NegfError(5, "poisson_newton", "singular Jacobian")
        d = zgemm(Jinv, F.reshape(1, NA, 1).to(torch.complex128).contiguous(), alpha=-1.0)
        U = U + d.real.reshape(N, A)
    return U, hist
