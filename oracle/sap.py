"""Schwarz alternating procedure smoother (oracle; test infrastructure).

Paper Sec. 2: the smoother is a multiplicative SAP over domains; inside every
domain the block system is solved approximately by site even-odd
preconditioned minimal residual (MR) with a fixed number of iterations.
Sec. 4 uses 4^4 domains and N_SAP = 4 cycles; loops over domains are the
parallel dimension.

Readings (the paper does not spell these out):

* the block operator D_B is D with both rows and columns restricted to the
  block (hops that leave the block are cut);
* one SAP cycle sweeps the blocks of colour 0, then those of colour 1; for a
  colour c, ``x <- x + sum_{B of colour c} I_B K_B I_B^T (b - D x)`` with
  ``K_B`` the approximate block inverse below;
  the SAP solution starts from ``x = 0``;
* the block solve eliminates the odd sites: with ``D_B = [[A_ee, D_eo],
  [D_oe, A_oo]]`` it runs MR on ``S = A_ee - D_eo A_oo^-1 D_oe`` with
  right-hand side ``r_e - D_eo A_oo^-1 r_o``, starting from zero, then sets
  ``e_o = A_oo^-1 (r_o - D_oe e_e)``;
* MR step: ``p = S r; alpha = <p, r> / <p, p>; x += alpha r; r -= alpha p``
  with ``<u, v> = sum conj(u) v`` over the block.

Blocks of one colour never touch each other (every block-grid extent is
even), so all blocks of a colour are processed at once on masked
full-lattice fields: ``mask * hop(mask * v)`` is the block-diagonal hop.
"""
from __future__ import annotations

import torch

from .dirac import WilsonClover
from .lattice import Blocking


class SchwarzSmoother:
    def __init__(self, op: WilsonClover, sap_block):
        self.op = op
        self.blk = Blocking(op.geom, sap_block)
        for mu in range(4):
            if self.blk.b[mu] % 2:
                raise ValueError("Schwarz block extents must be even")
            if self.blk.grid[mu] % 2:
                raise ValueError("the number of blocks along each axis must be even")
        par = op.geom.parity
        col = self.blk.colour_of_site
        self.mask = {}
        for c in (0, 1):
            for p in (0, 1):
                self.mask[c, p] = ((col == c) & (par == p)).to(torch.complex128)[:, None, None]
            self.mask[c, None] = (col == c).to(torch.complex128)[:, None, None]

    # block-local pieces ------------------------------------------------------
    def _hop_block(self, v, c):
        """-1/2 hop restricted to the blocks of colour c (hops leaving a block cut)."""
        m = self.mask[c, None]
        return m * (-0.5 * self.op.hop(m * v))

    def _block_dot(self, u, v, c):
        """<u, v> per block of colour c, returned as a per-site broadcastable field."""
        d = (u.conj() * v).sum(dim=(-1, -2))                     # [..., V]
        per_block = d[..., self.blk.sites].sum(dim=-1)           # [..., n_blocks]
        return per_block[..., self.blk.block_of_site][..., None, None]

    def block_solve(self, r, c, mr_iters):
        """Approximate D_B^-1 r on every block of colour c (zero elsewhere)."""
        op = self.op
        me, mo = self.mask[c, 0], self.mask[c, 1]
        r_e, r_o = me * r, mo * r

        def D_eo(v_o):
            return me * self._hop_block(mo * v_o, c)

        def D_oe(v_e):
            return mo * self._hop_block(me * v_e, c)

        def Ainv_o(v):
            return mo * op.site(v, inverse=True)

        def S(v_e):
            return me * op.site(v_e) - D_eo(Ainv_o(D_oe(v_e)))

        rhs = r_e - D_eo(Ainv_o(r_o))
        x_e = torch.zeros_like(r)
        res = rhs
        for _ in range(mr_iters):
            p = S(res)
            pr = self._block_dot(p, res, c)
            pp = self._block_dot(p, p, c).real
            # a block whose residual has vanished (or underflowed) stays put
            ok = pp > torch.finfo(torch.float64).tiny
            alpha = torch.where(ok, pr / torch.where(ok, pp, 1.0), 0.0)
            x_e = x_e + alpha * res
            res = res - alpha * p
        x_o = Ainv_o(r_o - D_oe(x_e))
        return x_e + x_o

    def sweep(self, b, x, c, mr_iters):
        """One colour of one SAP cycle: x + blockdiag solve of (b - D x)."""
        r = b - self.op.apply(x)
        return x + self.block_solve(r, c, mr_iters)

    def apply(self, b, n_sap, mr_iters):
        """SAP from a zero initial guess: ``n_sap`` cycles of colour 0 then 1."""
        x = torch.zeros_like(b)
        for _ in range(n_sap):
            for c in (0, 1):
                x = self.sweep(b, x, c, mr_iters)
        return x
