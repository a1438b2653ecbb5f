"""Index maps of the fine and coarse lattices (oracle; test infrastructure).

Paper Sec. 2 and Fig. 1: the fine lattice is cut into domains (Schwarz
blocks for the SAP smoother, aggregates for the coarse grid); every aggregate
becomes one coarse site.  Sec. 4 uses 4^4 domains for both.

Conventions restated here (the paper fixes none of them):

* lexicographic site index ``x + Lx*(y + Ly*(z + Lz*t))``;
* site parity ``(x+y+z+t) mod 2`` (site even-odd preconditioning, Sec. 2);
* block index = lexicographic index of ``floor(coord / block)`` on the block
  grid, block colour = parity of the block coordinates (the red/black order
  of the multiplicative Schwarz sweep);
* aggregate index = the same map with the aggregate extents; the coarse site
  ``X`` of a fine site is its aggregate index, and the coarse parity is the
  parity of the aggregate coordinates.

Index arrays are int64 torch tensors (CPU).
"""
from __future__ import annotations

import torch


class Geometry:
    """A periodic 4-D lattice ``L = (Lx, Ly, Lz, Lt)`` with neighbour tables."""

    def __init__(self, L):
        self.L = tuple(int(v) for v in L)
        Lx, Ly, Lz, Lt = self.L
        self.V = Lx * Ly * Lz * Lt
        idx = torch.arange(self.V)
        x = idx % Lx
        y = (idx // Lx) % Ly
        z = (idx // (Lx * Ly)) % Lz
        t = idx // (Lx * Ly * Lz)
        self.coords = torch.stack([x, y, z, t], dim=1)
        self.parity = (x + y + z + t) % 2
        self.fwd = torch.empty((4, self.V), dtype=torch.int64)
        self.bwd = torch.empty((4, self.V), dtype=torch.int64)
        for mu in range(4):
            c = self.coords.clone()
            c[:, mu] = (c[:, mu] + 1) % self.L[mu]
            self.fwd[mu] = self.index(c)
            c = self.coords.clone()
            c[:, mu] = (c[:, mu] - 1) % self.L[mu]
            self.bwd[mu] = self.index(c)

    def index(self, c) -> torch.Tensor:
        Lx, Ly, Lz, _ = self.L
        return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))

    def boundary_signs(self, antiperiodic_t: bool = True):
        """Signs of the forward / backward hops: -1 where a t-hop wraps."""
        fs = torch.ones((4, self.V), dtype=torch.float64)
        bs = torch.ones((4, self.V), dtype=torch.float64)
        if antiperiodic_t:
            t = self.coords[:, 3]
            fs[3, t == self.L[3] - 1] = -1.0
            bs[3, t == 0] = -1.0
        return fs, bs


class Blocking:
    """Domains of extent ``b`` on a geometry: block index, colour, site lists."""

    def __init__(self, geom: Geometry, b):
        self.geom = geom
        self.b = tuple(int(v) for v in b)
        for mu in range(4):
            if self.b[mu] < 1 or geom.L[mu] % self.b[mu]:
                raise ValueError("block extent must divide the lattice extent")
        self.grid = tuple(geom.L[mu] // self.b[mu] for mu in range(4))
        self.coarse = Geometry(self.grid)
        bc = geom.coords // torch.tensor(self.b)
        self.block_of_site = self.coarse.index(bc)
        self.colour_of_block = self.coarse.parity
        self.colour_of_site = self.colour_of_block[self.block_of_site]
        self.n_blocks = self.coarse.V
        self.block_volume = self.b[0] * self.b[1] * self.b[2] * self.b[3]
        # site lists of every block, in increasing fine index
        order = torch.argsort(self.block_of_site, stable=True)
        self.sites = order.reshape(self.n_blocks, self.block_volume)


def index_maps(L, sap_block, agg_block):
    """All the bit-exact index maps the method uses, per lexicographic site.

    Returns a dict of int32 tensors: ``parity``, ``block``, ``colour``,
    ``aggregate`` (fine sites) and ``coarse_parity`` (coarse sites).
    """
    g = Geometry(L)
    s = Blocking(g, sap_block)
    a = Blocking(g, agg_block)
    return {
        "parity": g.parity.to(torch.int32),
        "block": s.block_of_site.to(torch.int32),
        "colour": s.colour_of_site.to(torch.int32),
        "aggregate": a.block_of_site.to(torch.int32),
        "coarse_parity": a.coarse.parity.to(torch.int32),
    }
