"""Wilson-clover Dirac operator D (oracle; test infrastructure).

Paper Sec. 1 names the operator (clover fermions, Sec. 2 follows the
DD-alpha-AMG method for them) and Sec. 3 describes its data: the clover term
is two 6x6 Hermitian blocks per site in the chiral representation, stored
packed as 6 real + 15 complex numbers.  The paper prints no formula for D;
the reading used here (m0 normalisation, Hermitian chiral gamma basis,
clover-leaf field strength) is the standard one:

    (D psi)(x) = (4 + m0) psi(x) + C(x) psi(x)
                 - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x + mu)
                              + (1 + g_mu) U_mu(x - mu)^H psi(x - mu) ]

    C(x) = -(csw / 32) sum_{mu != nu} g_mu g_nu (x) (Q_munu(x) - Q_numu(x))

with Q_munu the sum of the four plaquettes ("clover leaves") in the mu-nu
plane that start and end at x.  C equals csw * (i/4) sigma_munu F_munu summed
over all ordered pairs, with sigma_munu = (i/2)[g_mu, g_nu] and
F = (Q_munu - Q_numu) / 8.  Time-direction hops that cross the lattice edge
carry a factor -1 (antiperiodic in t); the clover leaves are closed loops and
use the plain links.
"""
from __future__ import annotations

import torch

from .lattice import Geometry

C128 = torch.complex128


def gamma_matrices():
    """Hermitian chiral-basis gammas ``[g_x, g_y, g_z, g_t]`` and ``g5``.

    g_k = [[0, -i sigma_k], [i sigma_k, 0]], g_t = [[0, 1], [1, 0]];
    g5 = g_x g_y g_z g_t = diag(1, 1, -1, -1): spins {0, 1} have chirality +,
    spins {2, 3} chirality -.
    """
    s1 = torch.tensor([[0, 1], [1, 0]], dtype=C128)
    s2 = torch.tensor([[0, -1j], [1j, 0]], dtype=C128)
    s3 = torch.tensor([[1, 0], [0, -1]], dtype=C128)
    Z = torch.zeros((2, 2), dtype=C128)
    I2 = torch.eye(2, dtype=C128)

    def blk(a, b, c, d):
        return torch.cat([torch.cat([a, b], 1), torch.cat([c, d], 1)], 0)

    g = [blk(Z, -1j * s, 1j * s, Z) for s in (s1, s2, s3)]
    g.append(blk(Z, I2, I2, Z))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()


def _dag(A):
    return A.conj().transpose(-1, -2)


def clover_leaves(U: torch.Tensor, geom: Geometry, mu: int, nu: int) -> torch.Tensor:
    """Q_munu(x): sum of the four plaquettes in the mu-nu plane at x.

    The four leaves are the oriented closed paths from x whose first two
    steps are (+mu, +nu), (+nu, -mu), (-mu, -nu) and (-nu, +mu).
    """
    f, b = geom.fwd, geom.bwd
    Um, Un = U[:, mu], U[:, nu]
    x_pm = f[mu]                      # x + mu
    x_pn = f[nu]                      # x + nu
    x_mm = b[mu]                      # x - mu
    x_mn = b[nu]                      # x - nu
    x_mm_pn = f[nu][x_mm]             # x - mu + nu
    x_mm_mn = b[nu][x_mm]             # x - mu - nu
    x_mn_pm = f[mu][x_mn]             # x - nu + mu
    leaf1 = Um @ Un[x_pm] @ _dag(Um[x_pn]) @ _dag(Un)
    leaf2 = Un @ _dag(Um[x_mm_pn]) @ _dag(Un[x_mm]) @ Um[x_mm]
    leaf3 = _dag(Um[x_mm]) @ _dag(Un[x_mm_mn]) @ Um[x_mm_mn] @ Un[x_mn]
    leaf4 = _dag(Un[x_mn]) @ Um[x_mn] @ Un[x_mn_pm] @ _dag(Um)
    return leaf1 + leaf2 + leaf3 + leaf4


def clover_term(U: torch.Tensor, geom: Geometry, csw: float) -> torch.Tensor:
    """C(x) as a full 12x12 matrix per site, index ``spin*3 + colour``."""
    V = geom.V
    C = torch.zeros((V, 12, 12), dtype=C128)
    Q = {}
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                Q[mu, nu] = clover_leaves(U, geom, mu, nu)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            gg = GAMMA[mu] @ GAMMA[nu]
            F = Q[mu, nu] - Q[nu, mu]
            C += torch.einsum("st,xab->xsatb", gg, F).reshape(V, 12, 12)
    return -(csw / 32.0) * C


def site_matrix(U: torch.Tensor, geom: Geometry, m0: float, csw: float) -> torch.Tensor:
    """A(x) = (4 + m0) 1 + C(x): the site-diagonal part of D, 12x12 per site."""
    return (4.0 + m0) * torch.eye(12, dtype=C128) + clover_term(U, geom, csw)


def chiral_blocks(A: torch.Tensor) -> torch.Tensor:
    """The two 6x6 diagonal blocks (chirality +, -) of site matrices, ``[V][2][6][6]``."""
    return torch.stack([A[:, 0:6, 0:6], A[:, 6:12, 6:12]], dim=1)


def from_chiral_blocks(B: torch.Tensor) -> torch.Tensor:
    V = B.shape[0]
    A = torch.zeros((V, 12, 12), dtype=C128)
    A[:, 0:6, 0:6] = B[:, 0]
    A[:, 6:12, 6:12] = B[:, 1]
    return A


_UPPER = [(i, j) for i in range(6) for j in range(i + 1, 6)]


def pack_hermitian(B: torch.Tensor) -> torch.Tensor:
    """Pack Hermitian 6x6 matrices into 36 reals: 6 real diagonal entries, then
    the 15 complex strictly-upper entries (row-major) as (re, im) pairs.

    Sec. 3 keeps each Hermitian block in this minimal form (36 reals rather
    than 36 complex numbers).
    """
    out = torch.empty(B.shape[:-2] + (36,), dtype=torch.float64)
    for i in range(6):
        out[..., i] = B[..., i, i].real
    for k, (i, j) in enumerate(_UPPER):
        out[..., 6 + 2 * k] = B[..., i, j].real
        out[..., 7 + 2 * k] = B[..., i, j].imag
    return out


def unpack_hermitian(P: torch.Tensor) -> torch.Tensor:
    B = torch.zeros(P.shape[:-1] + (6, 6), dtype=C128)
    for i in range(6):
        B[..., i, i] = P[..., i].to(C128)
    for k, (i, j) in enumerate(_UPPER):
        v = torch.complex(P[..., 6 + 2 * k], P[..., 7 + 2 * k])
        B[..., i, j] = v
        B[..., j, i] = v.conj()
    return B


class WilsonClover:
    """Wilson-clover operator on one gauge field, with its site matrices.

    Fields are complex128 tensors ``[..., V, 4, 3]``; the gauge field is
    ``[V, 4, 3, 3]``.
    """

    def __init__(self, U, L, m0: float, csw: float, antiperiodic_t: bool = True):
        self.geom = Geometry(L)
        self.U = torch.as_tensor(U).to(C128)
        self.m0 = float(m0)
        self.csw = float(csw)
        fs, bs = self.geom.boundary_signs(antiperiodic_t)
        self.fsign = fs.to(C128)[:, :, None, None]
        self.bsign = bs.to(C128)[:, :, None, None]
        self.A = site_matrix(self.U, self.geom, m0, csw)   # [V][12][12]
        self.Ainv = from_chiral_blocks(torch.linalg.inv(chiral_blocks(self.A)))
        g = self.geom
        self._Ut = [self.U[:, mu].transpose(-1, -2).contiguous() for mu in range(4)]
        self._Udag_bt = [_dag(self.U[g.bwd[mu], mu]).transpose(-1, -2).contiguous()
                         for mu in range(4)]
        one = torch.eye(4, dtype=C128)
        self._pm = [(one - GAMMA[mu], one + GAMMA[mu]) for mu in range(4)]

    def hop(self, psi: torch.Tensor) -> torch.Tensor:
        """sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^H psi(x-mu)],
        with the time-boundary sign.  ``psi`` has shape ``[..., V, 4, 3]``."""
        g = self.geom
        out = torch.zeros_like(psi)
        d = psi.dim()
        for mu in range(4):
            Pm, Pp = self._pm[mu]
            up = psi.index_select(d - 3, g.fwd[mu]) @ self._Ut[mu]
            out += Pm @ (up * self.fsign[mu])
            dn = psi.index_select(d - 3, g.bwd[mu]) @ self._Udag_bt[mu]
            out += Pp @ (dn * self.bsign[mu])
        return out

    def site(self, psi: torch.Tensor, inverse: bool = False) -> torch.Tensor:
        """A(x) psi(x) (or A(x)^-1 psi(x)), A = (4 + m0) + C."""
        M = self.Ainv if inverse else self.A
        sh = psi.shape
        v = psi.reshape(sh[:-2] + (12, 1))
        return (M @ v).reshape(sh)

    def apply(self, psi: torch.Tensor) -> torch.Tensor:
        """D psi."""
        return self.site(psi) - 0.5 * self.hop(psi)

    def packed_clover(self, inverse: bool = False) -> torch.Tensor:
        """The packed chiral blocks of A (or A^-1), ``[V][2][36]``."""
        M = self.Ainv if inverse else self.A
        return pack_hermitian(chiral_blocks(M))

    def dense(self) -> torch.Tensor:
        """D as a dense ``12V x 12V`` matrix (small lattices only)."""
        V = self.geom.V
        n = 12 * V
        out = torch.empty((n, n), dtype=C128)
        step = 384
        for s in range(0, n, step):
            m = min(step, n - s)
            e = torch.zeros((m, n), dtype=C128)
            e[torch.arange(m), s + torch.arange(m)] = 1.0
            out[:, s:s + m] = self.apply(e.reshape(m, V, 4, 3)).reshape(m, n).T
        return out


def gauge_transform(U: torch.Tensor, Omega: torch.Tensor, geom: Geometry) -> torch.Tensor:
    """U_mu(x) -> Omega(x) U_mu(x) Omega(x + mu)^H."""
    out = torch.empty_like(U)
    for mu in range(4):
        out[:, mu] = Omega @ U[:, mu] @ _dag(Omega[geom.fwd[mu]])
    return out
