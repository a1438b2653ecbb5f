"""Two-level DD-alpha-AMG: preconditioner, outer solver, adaptive setup
(oracle; test infrastructure).

Paper Sec. 2:

* Eq. 5, post-smoothing only:
  ``M = P D_c^-1 R + S (1 - D P D_c^-1 R)``, S the SAP smoother;
  applied to r as ``x1 = P D_c^-1 R r``, ``x = x1 + SAP(r - D x1)``;
* the outer solver is flexible GMRES right-preconditioned by M;
* adaptive setup: the first test vectors come from an approximate solver
  applied to random vectors; then, a tunable number of times (4 in the
  paper), M is built from the current vectors and (part of) the multigrid
  solver is applied to every vector to enrich its low modes.

Readings: the initial approximate solver is the SAP smoother with the random
vector as right-hand side and a zero start; the update step is
``lambda_i <- M lambda_i`` (one preconditioner application) after the
vectors have been orthonormalised per (X, s) and D_c rebuilt; after the last
update the vectors are orthonormalised once more and D_c is rebuilt.  The
result of the setup is not unique (it depends on rounding) and is pinned
only through the invariants of what it builds ("parity unpinned" as a unique
result).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import torch

from .coarse import (Aggregation, CoarseOperator, coarse_operator,
                     orthonormalise, prolong, restrict)
from .dirac import WilsonClover
from .krylov import gmres, gmres_steps
from .sap import SchwarzSmoother


@dataclass
class Params:
    L: tuple
    sap_block: tuple
    agg_block: tuple
    n_v: int
    m0: float
    csw: float
    setup_iters: int = 4
    n_sap: int = 4
    mr_iters: int = 4
    coarse_tol: float = 5e-2
    coarse_restart: int = 30
    coarse_maxiter: int = 300
    outer_restart: int = 30
    outer_maxiter: int = 1000


class TwoLevelMG:
    def __init__(self, U, p: Params):
        self.p = p
        self.op = WilsonClover(U, p.L, p.m0, p.csw)
        self.sap = SchwarzSmoother(self.op, p.sap_block)
        self.agg = Aggregation(self.op.geom, p.agg_block)
        for mu in range(4):
            if self.agg.blk.grid[mu] % 2:
                raise ValueError("coarse lattice extents must be even")
        self.lam = None
        self.cop = None
        self.coarse_iters = []

    # -- pieces ---------------------------------------------------------------
    def set_test_vectors(self, lam, orthonormalised=False):
        self.lam = lam if orthonormalised else orthonormalise(lam, self.agg)
        self.cop = CoarseOperator(coarse_operator(self.op, self.lam, self.agg),
                                  self.agg.coarse)

    def smoother(self, r):
        """SAP on every field of ``r`` ``[..., V, 4, 3]`` (one field at a time)."""
        if r.dim() == 3:
            return self.sap.apply(r, self.p.n_sap, self.p.mr_iters)
        return torch.stack([self.smoother(v) for v in r])

    def coarse_correction(self, r):
        """P D_c^-1 R r with the approximate coarse solve (per right-hand side)."""
        bc = restrict(self.lam, self.agg, r)
        xc = torch.empty_like(bc)
        for idx in itertools.product(*(range(k) for k in bc.shape[:-2])):
            xc[idx], its = self.cop.solve(bc[idx], self.p.coarse_tol,
                                          self.p.coarse_restart, self.p.coarse_maxiter)
            self.coarse_iters.append(its)
        return prolong(self.lam, self.agg, xc)

    def apply_M(self, r):
        """Eq. 5 applied to r (post-smoothing only), one field at a time."""
        if r.dim() > 3:
            return torch.stack([self.apply_M(v) for v in r])
        x1 = self.coarse_correction(r)
        return x1 + self.smoother(r - self.op.apply(x1))

    # -- setup and solve ------------------------------------------------------
    def setup(self, lam0):
        """Adaptive setup from the random vectors ``lam0`` ``[n][V][4][3]``."""
        lam = self.smoother(torch.as_tensor(lam0).to(torch.complex128))
        for _ in range(self.p.setup_iters):
            self.set_test_vectors(lam)
            lam = self.apply_M(self.lam)
        self.set_test_vectors(lam)

    def solve(self, b, tol):
        """Outer FGMRES preconditioned by M; returns ``(x, iterations, converged)``."""
        return gmres(self.op.apply, b, tol, self.p.outer_restart,
                     self.p.outer_maxiter, precond=self.apply_M)

    def solve_steps(self, b, tol):
        """:meth:`solve` as a generator that yields after every outer
        iteration (for timing the solver one iteration at a time)."""
        return gmres_steps(self.op.apply, b, tol, self.p.outer_restart,
                           self.p.outer_maxiter, precond=self.apply_M)

    def true_residual(self, b, x):
        return (torch.linalg.vector_norm(b - self.op.apply(x))
                / torch.linalg.vector_norm(b)).item()
