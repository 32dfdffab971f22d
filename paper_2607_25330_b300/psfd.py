"""Thin ctypes binding of libpsfd (the C ABI in include/psfd.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  torch provides device memory and the stream.  The binding
fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpsfd.so")

PSFD_OK, PSFD_ERR_ARG, PSFD_ERR_CUDA, PSFD_NOT_CONVERGED, PSFD_ERR_BREAKDOWN, PSFD_ERR_TIMEOUT, PSFD_ERR_STATE = range(7)
PSFD_TE, PSFD_TM = 0, 1
PSFD_PRECOND, PSFD_HYBRID, PSFD_ADJOINT, PSFD_LAYERED = 1, 2, 4, 8
LAY_C64, LAY_HALF = 0, 1
LAY_FORM_AUTO, LAY_FORM_SCHUR = 0, 1
# use_precond values of the solves: identity, spectral damping M, layered-background P
PC_NONE, PC_DAMPING, PC_LAYERED = 0, 1, 2
PSFD_BICGSTAB, PSFD_GMRES = 0, 1


class PsfdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"psfd error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("nrhs", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("lam", C.c_double),
                ("theta_deg", C.c_double), ("phi_deg", C.c_double),
                ("pml_planes", C.c_int), ("pml_R0", C.c_double), ("pml_backing", C.c_double), ("z_ml", C.c_int),
                ("eps_abs_re", C.c_double), ("eps_abs_im", C.c_double),
                ("m_min", C.c_double), ("k_ref", C.c_double), ("gamma", C.c_double), ("damp_eps_rel", C.c_double),
                ("sigma_px", C.c_double), ("stream", C.c_void_p)]


class Stack(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("n_re", C.POINTER(C.c_double)), ("n_im", C.POINTER(C.c_double)),
                ("d", C.POINTER(C.c_double)), ("sub_re", C.c_double), ("sub_im", C.c_double)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("r_rel", C.c_double),
                ("r_rel_recursive", C.c_double), ("r_rel_initial", C.c_double),
                ("outer", C.c_int), ("r_rel_output", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("method", C.c_int), ("restart", C.c_int),
                ("use_precond", C.c_int), ("refine", C.c_int), ("inner_tol", C.c_double), ("max_outer", C.c_int),
                ("out_c128", C.c_int)]


class FnoWeights(C.Structure):
    _fields_ = [("dv", C.c_int), ("dh", C.c_int), ("layers", C.c_int), ("mx", C.c_int), ("my", C.c_int),
                ("mz", C.c_int), ("dq", C.c_int)] + \
               [(n, C.c_void_p) for n in ("lift_w", "lift_b", "kxy", "kz", "w1", "b1", "w2", "b2",
                                          "q1", "qb1", "q2", "qb2")]


class FnoGrads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("lift_w", "lift_b", "kxy", "kz", "w1", "b1", "w2", "b2",
                                          "q1", "qb1", "q2", "qb2")]


FNO_PARAM_NAMES = ("lift_w", "lift_b", "kxy", "kz", "w1", "b1", "w2", "b2", "q1", "qb1", "q2", "qb2")

_lib = None


def lib() -> C.CDLL:
    """Load libpsfd.so (built by paper_2607_25330_b300.build); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpsfd.so not built ({LIB_PATH}); run paper_2607_25330_b300/build.py")
    L = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "psfd_plan_create": (i, [C.POINTER(vp), C.POINTER(Params)]),
        "psfd_plan_destroy": (i, [vp]),
        "psfd_supported": (i, [i, i, i]),
        "psfd_mask_fill": (i, [vp, vp, C.POINTER(C.c_float), vp]),
        "psfd_background": (i, [vp, C.POINTER(Stack), vp, C.POINTER(C.c_int), vp]),
        "psfd_reflection_tables": (i, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "psfd_apply": (i, [vp, vp, vp, i]),
        "psfd_precond": (i, [vp, vp, vp, i]),
        "psfd_apply64": (i, [vp, vp, vp, i]),
        "psfd_physics_loss_workspace_size": (sz, [vp]),
        "psfd_physics_loss": (i, [vp, vp, vp, d, d, d, C.POINTER(C.c_double), vp, vp, sz]),
        "psfd_solve": (i, [vp, vp, vp, vp, d, i, i, i, i, C.POINTER(Info), vp, sz]),
        "psfd_solve_workspace_size": (sz, [vp, i, i]),
        "psfd_set_history": (i, [vp, C.POINTER(C.c_double), i]),
        "psfd_solve_ex": (i, [vp, vp, vp, vp, C.POINTER(SolveOpts), C.POINTER(Info), vp, sz]),
        "psfd_solve_ex_workspace_size": (sz, [vp, C.POINTER(SolveOpts)]),
        "psfd_autotune": (i, [vp, C.POINTER(C.c_int)]),
        "psfd_layered_build": (i, [vp]),
        "psfd_layered_storage": (i, [vp, i]),
        "psfd_layered_form": (i, [vp, i]),
        "psfd_width_metric": (i, [vp, vp, vp, i, i, i, C.c_float, i, d, C.POINTER(C.c_double)]),
        "psfd_set_plane_contrast": (i, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "psfd_set_layer_stack_contrast": (i, [vp, C.POINTER(Stack), d, C.POINTER(C.c_float)]),
        "psfd_layered_refresh": (i, [vp, d, C.POINTER(C.c_int)]),
        "psfd_layered_bytes": (sz, [vp]),
        "psfd_device_status": (i, [vp]),
        "psfd_solve_batched": (i, [C.POINTER(vp), i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(SolveOpts),
                                   C.POINTER(Info), i]),
        "fno_workspace_size": (sz, [C.POINTER(FnoWeights), i, i, i, i]),
        "fno_forward": (i, [C.POINTER(FnoWeights), vp, i, i, i, i, vp, vp, sz, vp]),
        "fno_train_workspace_size": (sz, [C.POINTER(FnoWeights), i, i, i, i, i]),
        "fno_forward_train": (i, [C.POINTER(FnoWeights), vp, i, i, i, i, vp, vp, sz, i, vp]),
        "fno_backward": (i, [C.POINTER(FnoWeights), C.POINTER(FnoGrads), vp, i, i, i, i, vp, vp, sz, i, vp]),
        "psfd_spectral_upsample": (i, [vp, i, i, i, i, vp, i, i, i, vp]),
        "psfd_spectral_upsample_static": (i, [vp, i, i, i, i, vp, i, i, i, vp]),
        "psfd_launch_count": (C.c_longlong, []),
        "psfd_timing_enable": (i, [i]),
        "psfd_timing_read": (i, [C.POINTER(C.c_double), C.POINTER(C.c_longlong), i]),
        "psfd_timing_read_bytes": (i, [C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double), i]),
        "psfd_last_error": (C.c_char_p, []),
        "psfd_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_symbols() -> List[str]:
    """Names of the functions the binding expects the library to export."""
    return ["psfd_plan_create", "psfd_plan_destroy", "psfd_supported", "psfd_mask_fill", "psfd_background",
            "psfd_reflection_tables", "psfd_apply", "psfd_apply64", "psfd_physics_loss_workspace_size",
            "psfd_physics_loss", "psfd_precond", "psfd_solve", "psfd_solve_workspace_size",
            "psfd_set_history", "psfd_solve_ex", "psfd_solve_ex_workspace_size", "psfd_autotune", "psfd_solve_batched",
            "psfd_layered_build", "psfd_layered_refresh", "psfd_layered_bytes", "psfd_width_metric",
            "psfd_layered_storage", "psfd_layered_form", "psfd_device_status",
            "psfd_set_plane_contrast", "psfd_set_layer_stack_contrast",
            "fno_workspace_size", "fno_forward", "fno_train_workspace_size", "fno_forward_train", "fno_backward",
            "psfd_spectral_upsample",
            "psfd_spectral_upsample_static", "psfd_launch_count", "psfd_timing_enable", "psfd_timing_read", "psfd_timing_read_bytes", "psfd_last_error", "psfd_version"]


def _pc(precond) -> int:
    """Solver preconditioner selector: False/0 none, True/1 spectral damping M, 2 layered P."""
    v = int(precond)
    if v not in (PC_NONE, PC_DAMPING, PC_LAYERED):
        raise ValueError(f"precond must be 0, 1 or 2, got {precond!r}")
    return v


def _check(code: int, what: str, allow=()):
    if code != PSFD_OK and code not in allow:
        raise PsfdError(code, f"{what}: {lib().psfd_last_error().decode()}")
    return code


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_stack(stack: Dict):
    n = [complex(v) for v in stack["n"]]
    nl = len(n)
    nre = (C.c_double * max(nl, 1))(*[v.real for v in n])
    nim = (C.c_double * max(nl, 1))(*[v.imag for v in n])
    d = (C.c_double * max(nl, 1))(*[float(v) for v in stack["d"]])
    sub = complex(stack["n_sub"])
    st = Stack(nl, C.cast(nre, C.POINTER(C.c_double)), C.cast(nim, C.POINTER(C.c_double)),
               C.cast(d, C.POINTER(C.c_double)), sub.real, sub.imag)
    st._keep = (nre, nim, d)
    return st


class Plan:
    """One PSFD operator (grid, angle, PML, damping) shared by nrhs right-hand sides."""

    def __init__(self, prob, nrhs: Optional[int] = None, stream: Optional[torch.cuda.Stream] = None):
        L = lib()
        self.prob = prob
        self.nrhs = nrhs if nrhs is not None else len(prob.pols)
        self.stream = stream
        eps = prob.eps_abs
        self.params = Params(prob.nx, prob.ny, prob.nz, self.nrhs, prob.dx, prob.dy, prob.dz, prob.lam,
                             prob.theta_deg, prob.phi_deg, prob.pml_planes, prob.pml_R0, prob.pml_backing, prob.z_ml,
                             eps.real, eps.imag, prob.m_min, prob.k_ref, prob.gamma, prob.damp_eps_rel,
                             prob.sigma_px, _stream_handle(stream))
        h = C.c_void_p()
        _check(L.psfd_plan_create(C.byref(h), C.byref(self.params)), "psfd_plan_create")
        self.h = h
        self.shape = (self.nrhs, 3, prob.nz, prob.ny, prob.nx)
        self.fill = None

    def close(self):
        if getattr(self, "h", None):
            lib().psfd_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self) -> torch.Tensor:
        return torch.empty(self.shape, dtype=torch.complex64, device="cuda")

    def mask_fill(self, a_bin: torch.Tensor, zprof: Sequence[float]) -> torch.Tensor:
        p = self.prob
        a = a_bin.to(device="cuda", dtype=torch.uint8).contiguous()
        zp = (C.c_float * p.nz)(*[float(v) for v in zprof])
        fill = torch.empty((p.nz, p.ny, p.nx), dtype=torch.float32, device="cuda")
        _check(lib().psfd_mask_fill(self.h, _ptr(a), zp, _ptr(fill)), "psfd_mask_fill")
        return fill

    def background(self, stack: Dict, fill: torch.Tensor, pols: Sequence[int]) -> torch.Tensor:
        st = make_stack(stack)
        pol = (C.c_int * self.nrhs)(*[int(v) for v in pols])
        b = self.empty()
        self.fill = fill
        _check(lib().psfd_background(self.h, C.byref(st), _ptr(fill), pol, _ptr(b)), "psfd_background")
        return b

    def reflection_tables(self):
        p = self.prob
        n = p.nx * p.ny
        bufs = [np.zeros(2 * n, dtype=np.float64) for _ in range(3)]
        ptrs = [b.ctypes.data_as(C.POINTER(C.c_double)) for b in bufs]
        _check(lib().psfd_reflection_tables(self.h, *ptrs), "psfd_reflection_tables")
        return [(b[0::2] + 1j * b[1::2]).reshape(p.ny, p.nx) for b in bufs]

    def apply(self, x: torch.Tensor, flags: int = 0, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        y = self.empty() if out is None else out
        _check(lib().psfd_apply(self.h, _ptr(x), _ptr(y), flags), "psfd_apply")
        return y

    def apply64(self, x: torch.Tensor, flags: int = 0, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """y = A x in FP64 (complex128 device tensors); flags 0 or PSFD_HYBRID."""
        if x.dtype != torch.complex128:
            raise ValueError("complex128 x expected")
        y = torch.empty(self.shape, dtype=torch.complex128, device="cuda") if out is None else out
        _check(lib().psfd_apply64(self.h, _ptr(x), _ptr(y), flags), "psfd_apply64")
        return y

    def physics_loss(self, E: torch.Tensor, b: torch.Tensor, lam_hf: float = 0.1, w0: float = 1.0,
                     eta_hf: float = 1.0, grad: bool = True):
        """Eq. loss per right-hand side (host float64 array [nrhs]) and, with grad, its gradient
        dJ/dRe E + i dJ/dIm E (device complex64, same shape as E); both from the library."""
        n = int(lib().psfd_physics_loss_workspace_size(self.h))
        if getattr(self, "_loss_ws", None) is None or self._loss_ws.numel() < n:
            self._loss_ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        J = np.zeros(self.nrhs, dtype=np.float64)
        g = torch.empty(self.shape, dtype=torch.complex64, device="cuda") if grad else None
        _check(lib().psfd_physics_loss(self.h, _ptr(E.contiguous()), _ptr(b.contiguous()), lam_hf, w0, eta_hf,
                                       J.ctypes.data_as(C.POINTER(C.c_double)), _ptr(g), _ptr(self._loss_ws),
                                       self._loss_ws.numel()), "psfd_physics_loss")
        return J, g

    def precond(self, x: torch.Tensor, flags: int = 0, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        y = self.empty() if out is None else out
        _check(lib().psfd_precond(self.h, _ptr(x), _ptr(y), flags), "psfd_precond")
        return y

    def solve_ex(self, b: torch.Tensor, x0: Optional[torch.Tensor] = None, tol: float = 1e-6, maxit: int = 20000,
                 method: int = PSFD_GMRES, restart: int = 30, precond: bool = True, refine: bool = True,
                 inner_tol: float = 1e-2, max_outer: int = 0, out: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None, out_c128: bool = False):
        """Mixed-precision solve (FP64 outer residual and field, complex64 inner Krylov).

        out_c128: return the FP64 field as complex128 instead of its complex64 rounding."""
        if out is None:
            E = torch.empty(self.shape, dtype=torch.complex128 if out_c128 else torch.complex64, device="cuda")
        else:
            E = out
            assert E.dtype == (torch.complex128 if out_c128 else torch.complex64)
        info = (Info * self.nrhs)()
        o = SolveOpts(tol, maxit, method, restart, _pc(precond), 1 if refine else 0, inner_tol, max_outer,
                      1 if out_c128 else 0)
        ws, wsb = None, 0
        if workspace is not None:
            ws, wsb = _ptr(workspace), workspace.numel() * workspace.element_size()
        code = lib().psfd_solve_ex(self.h, _ptr(b), _ptr(x0), _ptr(E), C.byref(o), info, ws, wsb)
        _check(code, "psfd_solve_ex", allow=(PSFD_NOT_CONVERGED, PSFD_ERR_BREAKDOWN))
        return {"E": E, "info": [info_dict(i) for i in info], "code": code}

    def layered_build(self) -> None:
        """Assemble and invert the per-column blocks of the layered-background preconditioner."""
        _check(lib().psfd_layered_build(self.h), "psfd_layered_build")

    def device_status(self) -> None:
        """Raise PsfdError (PSFD_ERR_TIMEOUT) if a bounded device-side wait gave up since the last check."""
        _check(lib().psfd_device_status(self.h), "psfd_device_status")

    def layered_refresh(self, max_shift: float) -> bool:
        """Rebuild the blocks only if a plane's mean fill moved by more than max_shift; True if rebuilt."""
        r = C.c_int(0)
        _check(lib().psfd_layered_refresh(self.h, max_shift, C.byref(r)), "psfd_layered_refresh")
        return bool(r.value)

    def width_metric(self, E: torch.Tensor, E_ref: torch.Tensor, z: int, rhs: int = 0, comp: int = 1,
                     I_th: float = 0.15, n_lines: int = 100, demag: float = 4.0) -> Dict:
        """Threshold-contour width deviation of E from E_ref on plane z (Sec. 4), wafer units (nm)."""
        out = (C.c_double * 6)()
        _check(lib().psfd_width_metric(self.h, _ptr(E.contiguous()), _ptr(E_ref.contiguous()), rhs, comp, z, I_th,
                                       n_lines, demag, out), "psfd_width_metric")
        return {"mean": out[0], "std": out[1], "max": out[2], "matched": int(out[3]), "unresolved": int(out[4]),
                "frac_above_1nm": out[5]}

    def set_plane_contrast(self, c: Optional[Sequence[complex]]) -> None:
        """deps = fill * c[z] per plane (None restores eps_abs - 1); call background() afterwards."""
        if c is None:
            _check(lib().psfd_set_plane_contrast(self.h, None, None), "psfd_set_plane_contrast")
            return
        c = np.asarray(c, dtype=np.complex128)
        assert c.shape == (self.prob.nz,)
        re = np.ascontiguousarray(c.real)
        im = np.ascontiguousarray(c.imag)
        _check(lib().psfd_set_plane_contrast(self.h, re.ctypes.data_as(C.POINTER(C.c_double)),
                                             im.ctypes.data_as(C.POINTER(C.c_double))), "psfd_set_plane_contrast")

    def set_layer_stack_contrast(self, stack: Dict, z_top: float) -> np.ndarray:
        """Mesh a layer stack (top face at z_top nm) into the per-plane contrast; returns the plane mask."""
        st = make_stack(stack)
        zm = np.zeros(self.prob.nz, dtype=np.float32)
        _check(lib().psfd_set_layer_stack_contrast(self.h, C.byref(st), z_top,
                                                   zm.ctypes.data_as(C.POINTER(C.c_float))),
               "psfd_set_layer_stack_contrast")
        return zm

    def layered_storage(self, half: bool) -> None:
        """Store the layered blocks in half precision (True) or complex64 (False) from the next build."""
        _check(lib().psfd_layered_storage(self.h, LAY_HALF if half else LAY_C64), "psfd_layered_storage")

    def layered_form(self, schur: bool) -> None:
        """Schur form of the blocks for nz a multiple of 32 (True), or the default rule (False), from the
        next build."""
        _check(lib().psfd_layered_form(self.h, LAY_FORM_SCHUR if schur else LAY_FORM_AUTO), "psfd_layered_form")

    def layered_bytes(self) -> int:
        return int(lib().psfd_layered_bytes(self.h))

    def autotune(self) -> int:
        T = C.c_int(0)
        _check(lib().psfd_autotune(self.h, C.byref(T)), "psfd_autotune")
        return T.value

    def workspace_size_ex(self, method: int = PSFD_GMRES, restart: int = 30, refine: bool = True) -> int:
        o = SolveOpts(1e-6, 1, method, restart, 1, 1 if refine else 0, 1e-2, 0, 0)
        return int(lib().psfd_solve_ex_workspace_size(self.h, C.byref(o)))

    def workspace_size(self, method: int = PSFD_BICGSTAB, restart: int = 30) -> int:
        return int(lib().psfd_solve_workspace_size(self.h, method, restart))

    def solve(self, b: torch.Tensor, x0: Optional[torch.Tensor] = None, tol: float = 1e-6, maxit: int = 1000,
              method: int = PSFD_BICGSTAB, restart: int = 30, precond: bool = True,
              out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
              history: int = 0):
        E = self.empty() if out is None else out
        info = (Info * self.nrhs)()
        hist = None
        if history > 0:
            hist = np.zeros(self.nrhs * history, dtype=np.float64)
            _check(lib().psfd_set_history(self.h, hist.ctypes.data_as(C.POINTER(C.c_double)), history),
                   "psfd_set_history")
        ws, wsb = None, 0
        if workspace is not None:
            ws, wsb = _ptr(workspace), workspace.numel() * workspace.element_size()
        code = lib().psfd_solve(self.h, _ptr(b), _ptr(x0), _ptr(E), tol, maxit, method, restart,
                                _pc(precond), info, ws, wsb)
        if history > 0:
            lib().psfd_set_history(self.h, None, 0)
        _check(code, "psfd_solve", allow=(PSFD_NOT_CONVERGED, PSFD_ERR_BREAKDOWN))
        res = [info_dict(i) for i in info]
        out_d = {"E": E, "info": res, "code": code}
        if hist is not None:
            out_d["history"] = hist.reshape(self.nrhs, history)
        return out_d


def info_dict(i: Info) -> Dict:
    return {"iters": i.iters, "status": i.status, "r_rel": i.r_rel, "r_rel_recursive": i.r_rel_recursive,
            "r_rel_initial": i.r_rel_initial, "outer": i.outer, "r_rel_output": i.r_rel_output}


def fno_struct(w: Dict[str, torch.Tensor], shape) -> FnoWeights:
    """Device weights (dict of CUDA tensors, complex kernels as complex64) -> fno_weights_t."""
    s = FnoWeights(shape.dv, shape.dh, shape.layers, shape.mx, shape.my, shape.mz, shape.dq,
                   *[_ptr(w[n]) for n in FNO_PARAM_NAMES])
    s._keep = w
    return s


def fno_forward(wt: FnoWeights, a: torch.Tensor, out: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    B, nz, ny, nx = a.shape
    E = torch.empty((B, 3, nz, ny, nx), dtype=torch.complex64, device="cuda") if out is None else out
    L = lib()
    n = int(L.fno_workspace_size(C.byref(wt), B, nx, ny, nz))
    ws = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    _check(L.fno_forward(C.byref(wt), _ptr(a.contiguous()), B, nx, ny, nz, _ptr(E), _ptr(ws), n,
                         _stream_handle(stream)), "fno_forward")
    return E


class FnoTrainer:
    """Owns the workspace of a training pass (fno_forward_train / fno_backward) for one (B, grid).

    checkpoint=True keeps only the layer inputs and recomputes the spectral branches in the backward.
    """

    def __init__(self, wt: FnoWeights, B: int, nz: int, ny: int, nx: int, checkpoint: bool = False):
        self.wt, self.B, self.shape, self.ckpt = wt, B, (nz, ny, nx), int(bool(checkpoint))
        self.n = int(lib().fno_train_workspace_size(C.byref(wt), B, nx, ny, nz, self.ckpt))
        self.ws = torch.empty(max(self.n, 1), dtype=torch.uint8, device="cuda")

    def forward(self, a: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        nz, ny, nx = self.shape
        assert a.shape == (self.B, nz, ny, nx) and a.dtype == torch.float32 and a.is_contiguous()
        E = torch.empty((self.B, 3, nz, ny, nx), dtype=torch.complex64, device="cuda")
        _check(lib().fno_forward_train(C.byref(self.wt), _ptr(a), self.B, nx, ny, nz, _ptr(E), _ptr(self.ws),
                                       self.n, self.ckpt, _stream_handle(stream)), "fno_forward_train")
        return E

    def backward(self, a: torch.Tensor, dE: torch.Tensor, grads: Dict[str, torch.Tensor],
                 stream: Optional[torch.cuda.Stream] = None) -> None:
        """Add the parameter gradients of the last forward, given dE = dJ/dRe E + i dJ/dIm E, into grads."""
        nz, ny, nx = self.shape
        dE = dE.contiguous()
        assert dE.dtype == torch.complex64 and dE.shape == (self.B, 3, nz, ny, nx)
        g = FnoGrads(*[_ptr(grads[n]) for n in FNO_PARAM_NAMES])
        _check(lib().fno_backward(C.byref(self.wt), C.byref(g), _ptr(a), self.B, nx, ny, nz, _ptr(dE),
                                  _ptr(self.ws), self.n, self.ckpt, _stream_handle(stream)), "fno_backward")


def spectral_upsample(src: torch.Tensor, nz: int, ny: int, nx: int,
                      stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    nb = int(np.prod(src.shape[:-3]))
    nz0, ny0, nx0 = src.shape[-3:]
    dst = torch.empty(src.shape[:-3] + (nz, ny, nx), dtype=torch.complex64, device="cuda")
    _check(lib().psfd_spectral_upsample(_ptr(src.contiguous()), nb, nx0, ny0, nz0, _ptr(dst), nx, ny, nz,
                                        _stream_handle(stream)), "psfd_spectral_upsample")
    return dst


def spectral_upsample_static(src: torch.Tensor, nz: int, ny: int, nx: int,
                             stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """Same result as spectral_upsample; the library call allocates no device memory (its scratch
    is a fixed 16 MiB array inside the library; overlapping calls race).  The output tensor is
    allocated here, by the caller, as for every other call."""
    nb = int(np.prod(src.shape[:-3]))
    nz0, ny0, nx0 = src.shape[-3:]
    dst = torch.empty(src.shape[:-3] + (nz, ny, nx), dtype=torch.complex64, device="cuda")
    _check(lib().psfd_spectral_upsample_static(_ptr(src.contiguous()), nb, nx0, ny0, nz0, _ptr(dst), nx, ny, nz,
                                               _stream_handle(stream)), "psfd_spectral_upsample_static")
    return dst


def solve_batched(plans: Sequence["Plan"], bs: Sequence[torch.Tensor], x0s=None, tol: float = 1e-6,
                  maxit: int = 20000, method: int = PSFD_GMRES, restart: int = 30, precond: bool = True,
                  refine: bool = False, inner_tol: float = 1e-2, nworkers: int = 8):
    """Solve independent problems concurrently (one stream per plan); returns (fields, infos)."""
    n = len(plans)
    Es = [p.empty() for p in plans]
    arr = lambda ts: (C.c_void_p * n)(*[t.data_ptr() if t is not None else None for t in ts])
    total = sum(p.nrhs for p in plans)
    info = (Info * total)()
    o = SolveOpts(tol, maxit, method, restart, _pc(precond), 1 if refine else 0, inner_tol, 0, 0)
    for t in list(bs) + ([t for t in x0s if t is not None] if x0s else []):
        _ptr(t)
    code = lib().psfd_solve_batched((C.c_void_p * n)(*[p.h for p in plans]), n, arr(bs),
                                    arr(x0s) if x0s is not None else None, arr(Es), C.byref(o), info, nworkers)
    _check(code, "psfd_solve_batched", allow=(PSFD_NOT_CONVERGED, PSFD_ERR_BREAKDOWN))
    infos, k = [], 0
    for p in plans:
        infos.append([info_dict(info[k + r]) for r in range(p.nrhs)])
        k += p.nrhs
    return Es, infos


STAGES = ("axial", "contrast", "krylov", "transform", "fno", "precond", "lay_build")


def launch_count() -> int:
    return int(lib().psfd_launch_count())


def timing_enable(on: bool = True):
    lib().psfd_timing_enable(1 if on else 0)


def timing_read() -> Dict[str, Dict[str, float]]:
    """Per stage: summed ms, number of timed launch groups, summed algorithmic bytes."""
    ms = (C.c_double * len(STAGES))()
    calls = (C.c_longlong * len(STAGES))()
    nbytes = (C.c_double * len(STAGES))()
    lib().psfd_timing_read_bytes(ms, calls, nbytes, len(STAGES))
    return {s: {"ms": ms[i], "calls": int(calls[i]), "bytes": nbytes[i]} for i, s in enumerate(STAGES)}
