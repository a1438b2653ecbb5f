"""Three-level DD-alpha-AMG (oracle; test infrastructure).

Sec. 1 of the paper counts among the merits of the multigrid method that its
coarse-grid solver can itself be given a coarse grid, recursively; Sec. 2
and Sec. 3 then restrict the algorithm and its tuning to two levels.  This
module states the third level in the terms the paper uses for the second
(smoother, test vectors, aggregation, Galerkin coarse operator, Eq. 1-5),
applied to the coarse operator D_c instead of D.

Readings (none of this is in the paper):

* level 2 is the coarse lattice of level 1 with D_c (Eq. 2) as its 9-point
  operator; a coarse site carries 2n components ``s*n + i`` and the coarse
  chirality is ``G5 = diag(1_n, -1_n)``;
* the level-2 smoother is the same multiplicative red/black Schwarz sweep
  over blocks of coarse sites; a block solve eliminates the odd coarse sites
  of the block (coarse parity) and runs MR on
  ``S = A_ee - D_eo A_oo^-1 D_oe`` with the self blocks as A, as the fine
  block solve does with the clover blocks;
* the level-2 test vectors (n2 of them, vectors on the coarse lattice) come
  from the same adaptive setup run on D_c: random vectors smoothed by the
  level-2 SAP, then ``setup_iters`` times {orthonormalise per (X', s),
  rebuild D_cc, lambda2 <- M2 lambda2}, then a last orthonormalisation and
  D_cc.  The setup runs level by level: the fine level's test vectors are
  those of the two-level setup; the level-2 setup follows on the D_c they
  give;
* aggregates of level 2 are blocks of coarse sites; the projection onto
  (X', s) keeps the components of coarse chirality s on the sites of X'
  (Eq. 1 with G5 in place of g5); ``D_cc = P2^H D_c P2`` is assembled term
  by term of the coarse stencil with forward and backward links kept as
  separate blocks, as on level 1;
* M2 is Eq. 5 on level 2 (post-smoothing only); the coarsest system is
  solved by the even-odd GMRES of the level-1 coarse solver, to its own
  relative tolerance;
* in the three-level M the level-1 coarse solve is flexible GMRES on D_c,
  right-preconditioned by M2, stopped at the same relative residual as the
  two-level coarse solve (5e-2).

The setup's result is not unique (it depends on rounding): "parity
unpinned" as a unique result, pinned through the invariants it builds
(orthonormality, D_cc = P2^H D_c P2, G5-hermiticity) and through the solve.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import torch

from .coarse import CoarseOperator, prolong, restrict
from .krylov import gmres
from .lattice import Blocking, Geometry
from .solver import Params, TwoLevelMG

C128 = torch.complex128


class CoarseSchwarz:
    """Multiplicative Schwarz smoother on a coarse level (blocks of coarse
    sites of extent ``block``), block solves by even-odd MR."""

    def __init__(self, cop: CoarseOperator, block):
        self.cop = cop
        self.blk = Blocking(cop.geom, block)
        for mu in range(4):
            if self.blk.b[mu] % 2:
                raise ValueError("coarse Schwarz block extents must be even")
            if self.blk.grid[mu] % 2:
                raise ValueError("the number of coarse blocks along each axis must be even")
        par = cop.geom.parity
        col = self.blk.colour_of_site
        self.mask = {}
        for c in (0, 1):
            for p in (0, 1):
                self.mask[c, p] = ((col == c) & (par == p)).to(C128)[:, None]
            self.mask[c, None] = (col == c).to(C128)[:, None]

    def _hop_block(self, v, c):
        """Off-diagonal part of D_c restricted to the blocks of colour c."""
        m = self.mask[c, None]
        return m * self.cop.hop(m * v)

    def _block_dot(self, u, v, c):
        d = (u.conj() * v).sum(dim=-1)                            # [..., NX]
        per_block = d[..., self.blk.sites].sum(dim=-1)
        return per_block[..., self.blk.block_of_site][..., None]

    def block_solve(self, r, c, mr_iters):
        """Approximate inverse of D_c on every block of colour c (zero elsewhere)."""
        me, mo = self.mask[c, 0], self.mask[c, 1]
        r_e, r_o = me * r, mo * r

        def D_eo(v):
            return me * self._hop_block(mo * v, c)

        def D_oe(v):
            return mo * self._hop_block(me * v, c)

        def Ainv_o(v):
            return mo * self.cop.self_term(v, inverse=True)

        def S(v):
            return me * self.cop.self_term(me * v) - D_eo(Ainv_o(D_oe(v)))

        rhs = r_e - D_eo(Ainv_o(r_o))
        x_e = torch.zeros_like(r)
        res = rhs
        for _ in range(mr_iters):
            p = S(res)
            pr = self._block_dot(p, res, c)
            pp = self._block_dot(p, p, c).real
            ok = pp > torch.finfo(torch.float64).tiny
            alpha = torch.where(ok, pr / torch.where(ok, pp, 1.0), 0.0)
            x_e = x_e + alpha * res
            res = res - alpha * p
        x_o = Ainv_o(r_o - D_oe(x_e))
        return x_e + x_o

    def apply(self, b, n_sap, mr_iters):
        """``n_sap`` cycles (colour 0, then 1) from a zero start."""
        x = torch.zeros_like(b)
        for _ in range(n_sap):
            for c in (0, 1):
                x = x + self.block_solve(b - self.cop.apply(x), c, mr_iters)
        return x


class CoarseAggregation:
    """Aggregates of coarse sites; ``n1`` components per chirality below."""

    def __init__(self, geom: Geometry, block, n1: int):
        self.blk = Blocking(geom, block)
        self.coarse = self.blk.coarse
        self.agg_of_site = self.blk.block_of_site
        self.sites = self.blk.sites
        self.NX = self.blk.n_blocks
        self.Va = self.blk.block_volume
        self.n1 = n1


def orthonormalise_c(lam: torch.Tensor, agg: CoarseAggregation) -> torch.Tensor:
    """Classical Gram-Schmidt, twice, of the n2 vectors ``[n2][NX][2 n1]``
    inside every (X', s), in the order i = 1..n2."""
    n2, n1 = lam.shape[0], agg.n1
    out = torch.empty_like(lam)
    for s in (0, 1):
        sub = lam[:, agg.sites, s * n1:(s + 1) * n1]             # [n2][NX'][Va'][n1]
        M = sub.reshape(n2, agg.NX, agg.Va * n1).transpose(0, 1).clone()
        for i in range(n2):
            v = M[:, i]
            for _ in range(2):
                if i:
                    c = torch.einsum("xjk,xk->xj", M[:, :i].conj(), v)
                    v = v - torch.einsum("xj,xjk->xk", c, M[:, :i])
            M[:, i] = v / torch.linalg.vector_norm(v, dim=1)[:, None]
        out[:, agg.sites, s * n1:(s + 1) * n1] = M.transpose(0, 1).reshape(n2, agg.NX, agg.Va, n1)
    return out


def restrict_c(lam: torch.Tensor, agg: CoarseAggregation, b: torch.Tensor) -> torch.Tensor:
    """Eq. 3 on level 2: ``[..., NX, 2 n1] -> [..., NX', 2 n2]``,
    component ``s*n2 + i`` = <lambda2_i(X', s) | b>."""
    n1 = agg.n1
    parts = []
    for s in (0, 1):
        ls = lam[:, :, s * n1:(s + 1) * n1].conj()
        prod = torch.einsum("ixc,...xc->...ix", ls, b[..., s * n1:(s + 1) * n1])
        parts.append(prod[..., agg.sites].sum(dim=-1))
    return torch.cat(parts, dim=-2).transpose(-1, -2).contiguous()


def prolong_c(lam: torch.Tensor, agg: CoarseAggregation, xc: torch.Tensor) -> torch.Tensor:
    """Eq. 4 on level 2: ``x = sum_{X', s, i} x_c[X', s*n2 + i] lambda2_i(X', s)``."""
    n2, n1 = lam.shape[0], agg.n1
    out = torch.zeros(xc.shape[:-2] + (lam.shape[1], 2 * n1), dtype=C128)
    for s in (0, 1):
        coeff = xc[..., agg.agg_of_site, s * n2:(s + 1) * n2]
        out[..., s * n1:(s + 1) * n1] = torch.einsum("...xi,ixc->...xc", coeff,
                                                      lam[:, :, s * n1:(s + 1) * n1])
    return out


def coarse_coarse_operator(cop: CoarseOperator, lam: torch.Tensor, agg: CoarseAggregation) -> torch.Tensor:
    """Eq. 2 on level 2, ``[NX'][9][2 n2][2 n2]``: every term ``d`` of the
    coarse stencil (self block, link to X +- mu) is applied to the
    chirality-t projection of lambda2_j and contracted at X with lambda2_i of
    chirality s; the self term and links that stay inside the aggregate of X
    go to the self block of X', a link that leaves it to the link block of
    the same direction."""
    n2, n1 = lam.shape[0], agg.n1
    NX = lam.shape[1]
    Dcc = torch.zeros((agg.NX, 9, 2 * n2, 2 * n2), dtype=C128)
    Xp = agg.agg_of_site
    proj = []
    for t in (0, 1):
        p = torch.zeros_like(lam)
        p[:, :, t * n1:(t + 1) * n1] = lam[:, :, t * n1:(t + 1) * n1]
        proj.append(p)
    lam_c = lam.conj()
    for d in range(9):
        y = cop.nbr[d]
        W = [torch.einsum("xab,jxb->jxa", cop.Dc[:, d], proj[t][:, y]) for t in (0, 1)]
        G = torch.zeros((NX, 2 * n2, 2 * n2), dtype=C128)
        for s in (0, 1):
            Ls = lam_c[:, :, s * n1:(s + 1) * n1].permute(1, 0, 2)           # [NX][n2][n1]
            for t in (0, 1):
                Wt = W[t][:, :, s * n1:(s + 1) * n1].permute(1, 2, 0)         # [NX][n1][n2]
                G[:, s * n2:(s + 1) * n2, t * n2:(t + 1) * n2] = Ls @ Wt
        target = torch.zeros(NX, dtype=torch.int64) if d == 0 else torch.where(Xp[y] == Xp, 0, d)
        Dcc.index_put_((Xp, target), G, accumulate=True)
    return Dcc


@dataclass
class Level2Params:
    sap_block: tuple = (2, 2, 2, 2)        # blocks of coarse sites
    agg_block: tuple = (2, 2, 2, 2)        # aggregates of coarse sites
    n_v: int = 8
    setup_iters: int = 2
    n_sap: int = 4
    mr_iters: int = 4
    coarsest_tol: float = 5e-2
    coarsest_restart: int = 30
    coarsest_maxiter: int = 300
    restart: int = 30                      # FGMRES of the level-1 coarse solve


class ThreeLevelMG:
    """The two-level method of :mod:`oracle.solver` with its coarse solve
    replaced by FGMRES on D_c preconditioned by the level-2 method."""

    def __init__(self, U, p: Params, p2: Level2Params, two: TwoLevelMG = None):
        self.two = TwoLevelMG(U, p) if two is None else two
        self.p, self.p2 = self.two.p, p2
        self.op = self.two.op
        self.lam2 = None
        self.cop2 = None
        self.sap2 = None
        self.agg2 = None
        self.level1_iters = []

    @classmethod
    def on(cls, two: TwoLevelMG, p2: Level2Params):
        """A three-level method over an existing two-level one (its fine
        test vectors and D_c), with the level-2 geometry laid out."""
        mg = cls(None, two.p, p2, two=two)
        mg._level2_geometry()
        return mg

    # -- level 2 --------------------------------------------------------------
    def _level2_geometry(self):
        cop = self.two.cop
        self.sap2 = CoarseSchwarz(cop, self.p2.sap_block)
        self.agg2 = CoarseAggregation(cop.geom, self.p2.agg_block, self.p.n_v)
        for mu in range(4):
            if self.agg2.blk.grid[mu] % 2:
                raise ValueError("coarsest lattice extents must be even")

    def set_level2_vectors(self, lam2, orthonormalised=False):
        self.lam2 = lam2 if orthonormalised else orthonormalise_c(lam2, self.agg2)
        self.cop2 = CoarseOperator(coarse_coarse_operator(self.two.cop, self.lam2, self.agg2),
                                   self.agg2.coarse)

    def smoother2(self, r):
        if r.dim() == 2:
            return self.sap2.apply(r, self.p2.n_sap, self.p2.mr_iters)
        return torch.stack([self.smoother2(v) for v in r])

    def apply_M2(self, r):
        """Eq. 5 on level 2, one coarse field ``[NX][2n]`` at a time."""
        if r.dim() > 2:
            return torch.stack([self.apply_M2(v) for v in r])
        bc = restrict_c(self.lam2, self.agg2, r)
        xc, _ = self.cop2.solve(bc, self.p2.coarsest_tol, self.p2.coarsest_restart,
                                self.p2.coarsest_maxiter)
        x1 = prolong_c(self.lam2, self.agg2, xc)
        return x1 + self.smoother2(r - self.two.cop.apply(x1))

    def setup_level2(self, lam2_0):
        """Adaptive setup on D_c from random coarse vectors ``[n2][NX][2n]``."""
        self._level2_geometry()
        lam2 = self.smoother2(torch.as_tensor(lam2_0).to(C128))
        for _ in range(self.p2.setup_iters):
            self.set_level2_vectors(lam2)
            lam2 = self.apply_M2(self.lam2)
        self.set_level2_vectors(lam2)

    def setup(self, lam0, lam2_0):
        """Level by level: the two-level setup of the fine test vectors,
        then the adaptive setup of level 2 on the D_c they give."""
        self.two.setup(lam0)
        self.setup_level2(lam2_0)

    # -- level 1 with the level-2 coarse solve --------------------------------
    def coarse_solve(self, bc, tol=None):
        """FGMRES on D_c preconditioned by M2, to ``tol`` (default: the
        two-level coarse tolerance); returns ``(x_c, iterations)``."""
        tol = self.p.coarse_tol if tol is None else tol
        x, its, _ = gmres(self.two.cop.apply, bc, tol, self.p2.restart, self.p.coarse_maxiter,
                          precond=self.apply_M2)
        return x, its

    def coarse_correction(self, r, tol=None):
        bc = restrict(self.two.lam, self.two.agg, r)
        xc = torch.empty_like(bc)
        for idx in itertools.product(*(range(k) for k in bc.shape[:-2])):
            xc[idx], its = self.coarse_solve(bc[idx], tol)
            self.level1_iters.append(its)
        return prolong(self.two.lam, self.two.agg, xc)

    def apply_M(self, r, tol=None):
        """Eq. 5 with the three-level coarse correction."""
        if r.dim() > 3:
            return torch.stack([self.apply_M(v, tol) for v in r])
        x1 = self.coarse_correction(r, tol)
        return x1 + self.two.smoother(r - self.op.apply(x1))

    def solve(self, b, tol):
        """Outer FGMRES preconditioned by the three-level M."""
        return gmres(self.op.apply, b, tol, self.p.outer_restart, self.p.outer_maxiter,
                     precond=self.apply_M)

    def true_residual(self, b, x):
        return self.two.true_residual(b, x)
