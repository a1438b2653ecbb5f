"""Choosing a bare mass by the cost of the unpreconditioned solve.

A workload can be defined as "m0 such that conjugate gradients on the normal
equations D^H D x = D^H b need more than N iterations to reach a relative
residual ||b - D x|| / ||b|| <= tol" (a light quark, where the multigrid
preconditioner matters).  This module measures that count with the library's
own D (``DDAMG.apply_D``; D^H = g5 D g5 for the Wilson-clover operator) and
scans m0 downward until the count exceeds N (or, where no mass reaches N,
to the mass of the largest count).  The scan estimates the count
from a short run first: the CG coefficients of k iterations define the Lanczos
tridiagonal matrix of D^H D, whose extreme eigenvalues bound its condition
number kappa, and CG needs about sqrt(kappa)/2 * ln(2/tol) iterations.  The
chosen mass is then confirmed by a full count in FP64.

The CG vectors are device tensors updated by torch; every application of D
is the library's kernel.  This is a workload-definition tool, not part of the
solver.
"""
from __future__ import annotations

import math

import numpy as np

from ._ddamg import FP32, FP64


def _g5(v):
    """g5 = diag(1, 1, -1, -1) on the spin index of a [V][4][3] field."""
    w = v.clone()
    w[:, 2:] = -w[:, 2:]
    return w


def cg_normal_equations(h, b, tol=1e-10, max_iter=6000, precision=FP64):
    """CG on D^H D x = D^H b from x = 0 (CGNR); stops when the recurrence
    residual ||b - D x|| / ||b|| reaches tol or after max_iter iterations.

    Returns (iterations, reached residual, alphas, betas, x); the
    coefficients give the Lanczos matrix of D^H D (:func:`lanczos_extremes`)."""
    import torch
    bn = torch.linalg.vector_norm(b).item()
    res = b.clone()                                   # b - D x
    r = _g5(h.apply_D(_g5(res), precision))           # D^H (b - D x)
    p = r.clone()
    x = torch.zeros_like(b)
    rr = torch.vdot(r.flatten(), r.flatten()).real.item()
    alphas, betas = [], []
    k = 0
    resid = 1.0
    while k < max_iter:
        q = h.apply_D(p, precision)
        qq = torch.vdot(q.flatten(), q.flatten()).real.item()
        alpha = rr / qq
        x.add_(p, alpha=alpha)
        res.sub_(q, alpha=alpha)
        k += 1
        alphas.append(alpha)
        resid = torch.linalg.vector_norm(res).item() / bn
        if resid <= tol:
            break
        r = _g5(h.apply_D(_g5(res), precision))
        rr_new = torch.vdot(r.flatten(), r.flatten()).real.item()
        beta = rr_new / rr
        betas.append(beta)
        rr = rr_new
        p.mul_(beta).add_(r)
    return k, resid, alphas, betas, x


def lanczos_extremes(alphas, betas):
    """Smallest and largest eigenvalue of the Lanczos matrix that k CG steps
    build: diagonal 1/a_0, 1/a_j + b_{j-1}/a_{j-1}; off-diagonal
    sqrt(b_j)/a_j.  They lie inside the spectrum of D^H D, so the ratio is a
    lower bound on its condition number that tightens with k."""
    k = len(alphas)
    diag = np.empty(k)
    off = np.empty(max(k - 1, 0))
    for j in range(k):
        diag[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < k - 1:
            off[j] = math.sqrt(betas[j]) / alphas[j]
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def predicted_iterations(kappa, tol):
    """The CG iteration bound sqrt(kappa)/2 * ln(2/tol)."""
    return 0.5 * math.sqrt(kappa) * math.log(2.0 / tol)


def scan_mass(h, b, target=5000, m0_start=0.0, step=0.01, probe_iters=400, probe_tol=1e-6, tol=1e-10,
              m0_floor=-2.0, patience=5, confirm=True, confirm_cap=None):
    """Lower m0 from m0_start in steps of `step` until the predicted CG count
    of the normal equations exceeds `target`.

    Each probe runs at most `probe_iters` CG steps with the FP32 operator and
    stops at the relative residual `probe_tol` (beyond the FP32 rounding
    floor the coefficients carry no information).  Near-unit links and an
    antiperiodic time direction keep the smallest singular value of D away
    from zero, so the count has a maximum over m0 (the most critical mass)
    that may lie below the target: once `patience` probes in a row stay
    below the largest prediction, the scan has passed that maximum and
    returns the mass of the largest prediction, with target_reached False.
    If `confirm`, the count at the chosen mass is then taken in FP64 (at most
    `confirm_cap` iterations).  The handle's mass is changed
    (``update_mass``).  Returns a dict with the chosen m0, the scan's
    estimates and the confirmed count."""
    csw = h.p.csw
    scan = []
    m0 = m0_start
    best_m0, best = m0_start, -1.0
    behind = 0
    reached = False
    while m0 >= m0_floor - 1e-12:
        h.update_mass(m0, csw)
        _, _, a, bt, _ = cg_normal_equations(h, b, tol=probe_tol, max_iter=probe_iters, precision=FP32)
        lo, hi = lanczos_extremes(a, bt)
        pred = predicted_iterations(hi / lo, tol) if lo > 0 else float("inf")
        scan.append({"m0": round(m0, 6), "lambda_min": lo, "lambda_max": hi, "predicted": pred,
                     "probe_iters": len(a)})
        if pred > best:
            best_m0, best, behind = m0, pred, 0
        else:
            behind += 1
        if pred > target:
            reached = True
            break
        if behind >= patience:
            break
        m0 -= step
    chosen = m0 if reached else best_m0
    out = {"m0": round(chosen, 6), "target": target, "target_reached": reached, "scan": scan}
    if confirm:
        cap = confirm_cap or 3 * target
        h.update_mass(chosen, csw)
        its, resid, _, _, _ = cg_normal_equations(h, b, tol=tol, max_iter=cap, precision=FP64)
        out.update(cg_iterations=its, cg_residual=resid, capped=resid > tol)
    return out
