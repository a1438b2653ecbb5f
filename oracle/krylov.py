"""Restarted (flexible) GMRES (oracle; test infrastructure).

Paper Sec. 2: the outer solver is flexible GMRES preconditioned by the
multigrid operator M, and the coarse-grid solver is (even-odd preconditioned)
GMRES stopped at a relative residual of 5e-2.  The paper gives no restart
length or orthogonalisation; the reading here is the textbook method:
Arnoldi with modified Gram-Schmidt, complex Givens rotations on the
Hessenberg matrix, stop when the recurrence residual ``|g_{k+1}|`` reaches
``tol * ||b||``, restart from the true residual ``b - A x``.  With a
preconditioner the basis ``Z`` of preconditioned vectors is kept (flexible
variant) and the update is ``x += Z y``.
"""
from __future__ import annotations

import math

import torch


def _givens(h1: complex, h2: complex):
    """Rotation with ``[c, s; -conj(s), c] [h1; h2] = [rho; 0]`` (c real)."""
    a1, a2 = abs(h1), abs(h2)
    if a2 == 0.0:
        return 1.0, 0.0j, h1
    if a1 == 0.0:
        return 0.0, h2.conjugate() / a2, complex(a2)
    rho = math.hypot(a1, a2)
    ph = h1 / a1
    return a1 / rho, ph * h2.conjugate() / rho, ph * rho


def gmres_steps(apply_A, b, tol, restart, maxiter, precond=None):
    """Generator form of :func:`gmres`: yields the running iteration count
    after every Arnoldi step and returns ``(x, iterations, converged)`` (as
    the value of ``StopIteration``).  The arithmetic is that of gmres."""
    x = torch.zeros_like(b)
    bnorm = torch.linalg.vector_norm(b).item()
    if bnorm == 0.0:
        return x, 0, True
    total = 0
    r = b.clone()
    while True:
        beta = torch.linalg.vector_norm(r).item()
        if beta <= tol * bnorm:
            return x, total, True
        if total >= maxiter:
            return x, total, False
        m = restart
        Vb = [r / beta]
        Zb = []
        H = [[0j] * m for _ in range(m + 1)]
        cs = [0.0] * m
        sn = [0j] * m
        g = [0j] * (m + 1)
        g[0] = complex(beta)
        k_done = 0
        for k in range(m):
            z = precond(Vb[k]) if precond is not None else Vb[k]
            Zb.append(z)
            w = apply_A(z)
            for j in range(k + 1):
                H[j][k] = torch.vdot(Vb[j].reshape(-1), w.reshape(-1)).item()
                w = w - H[j][k] * Vb[j]
            hn = torch.linalg.vector_norm(w).item()
            H[k + 1][k] = complex(hn)
            Vb.append(w / hn if hn > 0 else w)
            for j in range(k):
                t = cs[j] * H[j][k] + sn[j] * H[j + 1][k]
                H[j + 1][k] = -sn[j].conjugate() * H[j][k] + cs[j] * H[j + 1][k]
                H[j][k] = t
            cs[k], sn[k], H[k][k] = _givens(H[k][k], H[k + 1][k])
            H[k + 1][k] = 0j
            g[k + 1] = -sn[k].conjugate() * g[k]
            g[k] = cs[k] * g[k]
            total += 1
            k_done = k + 1
            yield total
            if abs(g[k + 1]) <= tol * bnorm or total >= maxiter or hn == 0:
                break
        y = [0j] * k_done
        for i in range(k_done - 1, -1, -1):
            acc = g[i]
            for j in range(i + 1, k_done):
                acc -= H[i][j] * y[j]
            y[i] = acc / H[i][i]
        for i in range(k_done):
            x = x + y[i] * Zb[i]
        r = b - apply_A(x)


def gmres(apply_A, b, tol, restart, maxiter, precond=None):
    """Solve ``A x = b`` from ``x = 0``.  Returns ``(x, iterations, converged)``.

    ``precond`` (optional) is applied on the right, each basis vector may be
    preconditioned differently (flexible GMRES).
    """
    it = gmres_steps(apply_A, b, tol, restart, maxiter, precond)
    while True:
        try:
            next(it)
        except StopIteration as done:
            return done.value
