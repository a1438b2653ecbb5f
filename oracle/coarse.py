"""Coarse grid of the 2-level method (oracle; test infrastructure).

Paper Sec. 2 and Fig. 1:

* Eq. 1: the test vectors ``lambda_i`` (i = 1..n) are projected onto an
  aggregate ``X`` and a chirality ``s``: ``lambda_i(X, s) = (1 +- g5)/2
  lambda_i`` on the sites of ``X``, zero elsewhere;
* Eq. 2: ``D_c(X,s,i; Y,t,j) = <lambda_i(X,s)| D |lambda_j(Y,t)>``; every
  aggregate is one coarse site carrying ``2n`` components (chirality x i);
* Eq. 3: restriction ``b_c(X,s,i) = <lambda_i(X,s)|b>``;
* Eq. 4: prolongation ``x = sum_{X,s,i} x_c(X,s,i) |lambda_i(X,s)>``;
* the coarse solver is even-odd preconditioned GMRES to 5e-2.

Readings: the projected vectors are made orthonormal inside every (X, s)
by classical Gram-Schmidt applied twice, in the order i = 1..n, so that
``R = P^H`` and ``P^H P = 1``.  Coarse component index is ``s*n + i``.
The coarse operator is stored per coarse site as nine ``2n x 2n`` blocks:
``d = 0`` the self ("clover") block, ``d = 1 + 2 mu`` the link to ``X + mu``,
``d = 2 + 2 mu`` the link to ``X - mu``; forward and backward links stay
separate blocks even where a coarse extent is 2 and both reach the same
aggregate.  The coarse even-odd split uses the parity of the aggregate
coordinates; GMRES runs on the Schur complement
``S = A_ee - D_eo A_oo^-1 D_oe`` (A = self blocks) with right-hand side
``b_e - D_eo A_oo^-1 b_o`` and stops when its residual reaches
``tol * ||rhs||``; then ``x_o = A_oo^-1 (b_o - D_oe x_e)``.
"""
from __future__ import annotations

import torch

from .dirac import GAMMA, WilsonClover
from .krylov import gmres
from .lattice import Blocking, Geometry


class Aggregation:
    def __init__(self, geom: Geometry, agg_block):
        self.blk = Blocking(geom, agg_block)
        self.coarse = self.blk.coarse
        self.agg_of_site = self.blk.block_of_site
        self.sites = self.blk.sites                     # [NX][Va]
        self.NX = self.blk.n_blocks
        self.Va = self.blk.block_volume


def orthonormalise(lam: torch.Tensor, agg: Aggregation) -> torch.Tensor:
    """Gram-Schmidt (classical, twice) of the n vectors inside every (X, s)."""
    n = lam.shape[0]
    out = torch.empty_like(lam)
    for s in (0, 1):
        sub = lam[:, agg.sites, 2 * s:2 * s + 2, :]             # [n][NX][Va][2][3]
        M = sub.reshape(n, agg.NX, agg.Va * 6).transpose(0, 1).clone()
        for i in range(n):
            v = M[:, i]
            for _ in range(2):
                if i:
                    c = torch.einsum("xjk,xk->xj", M[:, :i].conj(), v)
                    v = v - torch.einsum("xj,xjk->xk", c, M[:, :i])
            v = v / torch.linalg.vector_norm(v, dim=1)[:, None]
            M[:, i] = v
        out[:, agg.sites, 2 * s:2 * s + 2, :] = (
            M.transpose(0, 1).reshape(n, agg.NX, agg.Va, 2, 3))
    return out


def restrict(lam: torch.Tensor, agg: Aggregation, b: torch.Tensor) -> torch.Tensor:
    """Eq. 3: ``b_c[..., X, s*n + i] = <lambda_i(X, s) | b>``."""
    n = lam.shape[0]
    parts = []
    for s in (0, 1):
        ls = lam[:, :, 2 * s:2 * s + 2, :].conj()
        prod = torch.einsum("ixsc,...xsc->...ix", ls, b[..., 2 * s:2 * s + 2, :])
        parts.append(prod[..., agg.sites].sum(dim=-1))          # [..., n, NX]
    out = torch.cat(parts, dim=-2)                              # [..., 2n, NX]
    return out.transpose(-1, -2).contiguous()


def prolong(lam: torch.Tensor, agg: Aggregation, xc: torch.Tensor) -> torch.Tensor:
    """Eq. 4: ``x = sum_{X, s, i} x_c[X, s*n + i] lambda_i(X, s)``."""
    n = lam.shape[0]
    V = lam.shape[1]
    out = torch.zeros(xc.shape[:-2] + (V, 4, 3), dtype=torch.complex128)
    for s in (0, 1):
        coeff = xc[..., agg.agg_of_site, s * n:(s + 1) * n]       # [..., V, n]
        out[..., 2 * s:2 * s + 2, :] = torch.einsum(
            "...xi,ixsc->...xsc", coeff, lam[:, :, 2 * s:2 * s + 2, :])
    return out


def coarse_operator(op: WilsonClover, lam: torch.Tensor, agg: Aggregation,
                    aggregates=None) -> torch.Tensor:
    """Eq. 2 evaluated term by term of D, ``[NX][9][2n][2n]``.

    D = A(x) + sum_mu (forward hop + backward hop).  For the chirality-t
    projection of lambda_j, every term is applied at the sites x of the
    requested aggregates and contracted at x with lambda_i(x) of chirality s;
    the site term and hops that stay inside the aggregate of x go to the self
    block, a forward (backward) hop that leaves it goes to the block of the
    link to X + mu (X - mu).  ``aggregates`` restricts the evaluation to a
    list of coarse sites (the other blocks stay zero).
    """
    g = op.geom
    n = lam.shape[0]
    NX = agg.NX
    if aggregates is None:
        xs = torch.arange(g.V)
    else:
        xs = torch.sort(agg.sites[torch.as_tensor(aggregates)].reshape(-1)).values
    X = agg.agg_of_site[xs]
    nx = len(xs)
    Dc = torch.zeros((NX, 9, 2 * n, 2 * n), dtype=torch.complex128)
    lam_c = lam[:, xs].conj()                                   # [n][xs][4][3]
    proj = []
    for t in (0, 1):
        p = torch.zeros_like(lam)
        p[:, :, 2 * t:2 * t + 2, :] = lam[:, :, 2 * t:2 * t + 2, :]
        proj.append(p)

    def contract(W_t, target):
        # W_t[t]: [n][xs][4][3] = term applied to P_t lambda_j, evaluated at xs
        G = torch.zeros((nx, 2 * n, 2 * n), dtype=torch.complex128)
        for s in (0, 1):
            Ls = lam_c[:, :, 2 * s:2 * s + 2, :].reshape(n, nx, 6).permute(1, 0, 2)
            for t in (0, 1):
                Wt = W_t[t][:, :, 2 * s:2 * s + 2, :].reshape(n, nx, 6).permute(1, 2, 0)
                G[:, s * n:(s + 1) * n, t * n:(t + 1) * n] = Ls @ Wt
        Dc.index_put_((X, target), G, accumulate=True)

    # site term A(x)
    W = [torch.einsum("xab,jxb->jxa", op.A[xs], proj[t][:, xs].reshape(n, nx, 12))
         .reshape(n, nx, 4, 3) for t in (0, 1)]
    contract(W, torch.zeros(nx, dtype=torch.int64))
    one = torch.eye(4, dtype=torch.complex128)
    for mu in range(4):
        # forward hop: -1/2 (1 - g_mu) U_mu(x) psi(x + mu)
        y = g.fwd[mu][xs]
        W = []
        for t in (0, 1):
            up = proj[t][:, y] @ op.U[xs, mu].transpose(-1, -2)
            up = up * op.fsign[mu][xs]
            W.append(-0.5 * ((one - GAMMA[mu]) @ up))
        same = agg.agg_of_site[y] == X
        contract(W, torch.where(same, 0, 1 + 2 * mu))
        # backward hop: -1/2 (1 + g_mu) U_mu(x - mu)^H psi(x - mu)
        y = g.bwd[mu][xs]
        Ud = op.U[y, mu].conj().transpose(-1, -2)
        W = []
        for t in (0, 1):
            dn = proj[t][:, y] @ Ud.transpose(-1, -2)
            dn = dn * op.bsign[mu][xs]
            W.append(-0.5 * ((one + GAMMA[mu]) @ dn))
        same = agg.agg_of_site[y] == X
        contract(W, torch.where(same, 0, 2 + 2 * mu))
    return Dc


class CoarseOperator:
    """The 9-point coarse stencil and its even-odd preconditioned GMRES."""

    def __init__(self, Dc: torch.Tensor, coarse: Geometry):
        self.Dc = Dc
        self.geom = coarse
        self.NX = coarse.V
        self.nbr = torch.empty((9, self.NX), dtype=torch.int64)
        self.nbr[0] = torch.arange(self.NX)
        for mu in range(4):
            self.nbr[1 + 2 * mu] = coarse.fwd[mu]
            self.nbr[2 + 2 * mu] = coarse.bwd[mu]
        self.even = (coarse.parity == 0).to(torch.complex128)[:, None]
        self.odd = (coarse.parity == 1).to(torch.complex128)[:, None]
        self.self_inv = torch.linalg.inv(Dc[:, 0])

    def hop(self, v):
        out = torch.zeros_like(v)
        for d in range(1, 9):
            out += (self.Dc[:, d] @ v[..., self.nbr[d], :, None])[..., 0]
        return out

    def self_term(self, v, inverse=False):
        M = self.self_inv if inverse else self.Dc[:, 0]
        return (M @ v[..., None])[..., 0]

    def apply(self, v):
        """y(X) = sum_d D_c[X, d] v(nbr_d(X))."""
        return self.self_term(v) + self.hop(v)

    def dense(self) -> torch.Tensor:
        """The stencil as a dense matrix: block (X, nbr_d(X)) collects
        D_c[X, d] for every d (blocks whose neighbours coincide add up)."""
        n2 = self.Dc.shape[-1]
        B = torch.zeros((self.NX, self.NX, n2, n2), dtype=torch.complex128)   # [X][Y][row][col]
        rows = torch.arange(self.NX)
        for d in range(9):
            B.index_put_((rows, self.nbr[d]), self.Dc[:, d], accumulate=True)
        return B.permute(0, 2, 1, 3).reshape(self.NX * n2, self.NX * n2)

    def solve(self, b, tol, restart, maxiter):
        """Even-odd preconditioned GMRES; returns ``(x, iterations)``."""
        me, mo = self.even, self.odd

        def D_oe(v):
            return mo * self.hop(me * v)

        def D_eo(v):
            return me * self.hop(mo * v)

        def Aoo_inv(v):
            return mo * self.self_term(v, inverse=True)

        def S(v):
            return me * self.self_term(me * v) - D_eo(Aoo_inv(D_oe(v)))

        rhs = me * b - D_eo(Aoo_inv(mo * b))
        x_e, its, _ = gmres(S, rhs, tol, restart, maxiter)
        x_o = Aoo_inv(mo * b - D_oe(x_e))
        return me * x_e + x_o, its
