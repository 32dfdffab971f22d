"""Oracle: Krylov solves of A E = b with right preconditioning and an affine warm start.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Eq. right_correction_solution / right_preconditioned_system: with a base field
  E_base, solve (A M) y = b - A E_base and return E = E_base + M y; with
  E_base = 0 this is Eq. right_preconditioned, A M x = b.
* Convergence is measured by Eq. relative_residual, ||b - A E|| / ||b|| with the
  original b, also when warm-started.  For right preconditioning the Krylov
  residual of the y-system equals b - A E, so the recursive residual is that
  quantity up to rounding; the true residual is recomputed at exit.
* BiCGSTAB (van der Vorst, the paper's solver) and restarted GMRES(m) with
  modified Gram-Schmidt and Givens rotations.
* ``dense_matrix`` assembles A column by column on tiny grids and
  ``dense_solve`` solves it by LU with partial pivoting (torch.linalg.solve);
  this is the pin for both Krylov solvers.
"""
from __future__ import annotations

from typing import Callable, Dict, Optional

import torch

C128 = torch.complex128


def _nrm(x):
    return float(torch.linalg.vector_norm(x))


def bicgstab(B: Callable, c: torch.Tensor, bnorm: float, tol: float, maxit: int,
             history: Optional[list] = None):
    """Unpreconditioned BiCGSTAB on B y = c (B already contains A M), y0 = 0.

    Stops when ||r|| / bnorm <= tol.  Returns (y, iterations, status) with
    status 0 converged, 1 not converged, 2 breakdown.
    """
    y = torch.zeros_like(c)
    r = c.clone()
    rhat = r.clone()
    if _nrm(r) / bnorm <= tol:
        return y, 0, 0
    rho_old = alpha = omega = 1.0 + 0j
    v = torch.zeros_like(c)
    p = torch.zeros_like(c)
    for it in range(1, maxit + 1):
        rho = complex(torch.vdot(rhat.flatten(), r.flatten()))
        if abs(rho) < 1e-300:
            return y, it, 2
        if it == 1:
            p = r.clone()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = B(p)
        den = complex(torch.vdot(rhat.flatten(), v.flatten()))
        if abs(den) < 1e-300:
            return y, it, 2
        alpha = rho / den
        s = r - alpha * v
        if _nrm(s) / bnorm <= tol:
            y = y + alpha * p
            if history is not None:
                history.append(_nrm(s) / bnorm)
            return y, it, 0
        t = B(s)
        tt = complex(torch.vdot(t.flatten(), t.flatten()))
        if abs(tt) < 1e-300:
            return y, it, 2
        omega = complex(torch.vdot(t.flatten(), s.flatten())) / tt
        y = y + alpha * p + omega * s
        r = s - omega * t
        rn = _nrm(r) / bnorm
        if history is not None:
            history.append(rn)
        if rn <= tol:
            return y, it, 0
        if abs(omega) < 1e-300:
            return y, it, 2
        rho_old = rho
    return y, maxit, 1


def gmres(B: Callable, c: torch.Tensor, bnorm: float, tol: float, maxit: int, restart: int = 30,
          history: Optional[list] = None):
    """Restarted GMRES(m) on B y = c, y0 = 0; maxit counts operator applications."""
    y = torch.zeros_like(c)
    it = 0
    r = c.clone()
    while True:
        beta = _nrm(r)
        if beta / bnorm <= tol:
            return y, it, 0
        if it >= maxit:
            return y, it, 1
        V = [r / beta]
        H = torch.zeros(restart + 1, restart, dtype=C128)
        cs = torch.zeros(restart, dtype=C128)
        sn = torch.zeros(restart, dtype=C128)
        g = torch.zeros(restart + 1, dtype=C128)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            w = B(V[j])
            it += 1
            for i in range(j + 1):                         # modified Gram-Schmidt
                H[i, j] = torch.vdot(V[i].flatten(), w.flatten())
                w = w - H[i, j] * V[i]
            H[j + 1, j] = _nrm(w)
            V.append(w / H[j + 1, j] if abs(H[j + 1, j]) > 0 else w)
            for i in range(j):                             # apply earlier rotations
                a, b_ = H[i, j].clone(), H[i + 1, j].clone()
                H[i, j] = cs[i].conj() * a + sn[i].conj() * b_
                H[i + 1, j] = -sn[i] * a + cs[i] * b_
            a, b_ = H[j, j].clone(), H[j + 1, j].clone()
            den = torch.sqrt(abs(a) ** 2 + abs(b_) ** 2)
            cs[j] = a / den if abs(den) > 0 else 1.0
            sn[j] = b_ / den if abs(den) > 0 else 0.0
            H[j, j] = cs[j].conj() * a + sn[j].conj() * b_
            H[j + 1, j] = 0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j].conj() * g[j]
            j_done = j + 1
            res = float(abs(g[j + 1])) / bnorm
            if history is not None:
                history.append(res)
            if res <= tol or it >= maxit:
                break
        z = torch.linalg.solve_triangular(H[:j_done, :j_done], g[:j_done, None], upper=True)[:, 0]
        for i in range(j_done):
            y = y + z[i] * V[i]
        r = c - B(y)


def solve(A: Callable, M: Optional[Callable], b: torch.Tensor, E_base: Optional[torch.Tensor] = None,
          tol: float = 1e-6, maxit: int = 1000, method: str = "bicgstab", restart: int = 30,
          history: Optional[list] = None) -> Dict:
    """E = E_base + M y with A M y = b - A E_base (M = identity when None)."""
    b = b.to(C128)
    bnorm = _nrm(b)
    Mop = (lambda x: x) if M is None else M
    if bnorm == 0.0:
        E = torch.zeros_like(b) if E_base is None else E_base.clone()
        return {"E": E, "iters": 0, "status": 0, "r_rel": 0.0}
    if E_base is None:
        c = b.clone()
    else:
        c = b - A(E_base.to(C128))
    Bop = lambda y: A(Mop(y))
    if method == "bicgstab":
        y, it, st = bicgstab(Bop, c, bnorm, tol, maxit, history)
    elif method == "gmres":
        y, it, st = gmres(Bop, c, bnorm, tol, maxit, restart, history)
    else:
        raise ValueError(method)
    E = Mop(y) if E_base is None else E_base.to(C128) + Mop(y)
    r_rel = _nrm(b - A(E)) / bnorm
    return {"E": E, "iters": it, "status": st, "r_rel": r_rel}


def dense_matrix(A: Callable, shape) -> torch.Tensor:
    """Assemble the matrix of a linear map by applying it to unit vectors (tiny grids only)."""
    n = 1
    for s in shape:
        n *= s
    cols = []
    for j in range(n):
        e = torch.zeros(n, dtype=C128)
        e[j] = 1.0
        cols.append(A(e.reshape(shape)).reshape(n))
    return torch.stack(cols, dim=1)


def dense_solve(Amat: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """LU with partial pivoting."""
    return torch.linalg.solve(Amat, b.reshape(-1).to(C128)).reshape(b.shape)
