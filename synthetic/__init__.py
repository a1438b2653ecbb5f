"""Seeded synthetic inputs for the Wilson-clover DD-alpha-AMG hot path.

This module only *draws* inputs: SU(3) gauge links near the unit matrix,
Gaussian complex fields and point sources.  It holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from here without sharing any of the method.

Host exchange layouts (the C-ABI uses the same ones):

* site index ``x + Lx*(y + Ly*(z + Lz*t))`` (x fastest);
* gauge field: complex128 array ``[site][mu][row][col]``, ``mu = 0..3`` is
  ``x, y, z, t``; ``U[x, mu]`` is the link from ``x`` to ``x + mu``; it never
  carries the antiperiodic time boundary sign;
* spinor field: complex128 array ``[site][spin 4][colour 3]``.

The paper measures on a physical-point PACS 96^4 gauge ensemble, which is not
available; these generators stand in for it with near-unit SU(3) links
``U = exp(i * eps * H)``, ``H`` a Gaussian traceless Hermitian 3x3 matrix.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume", "rng", "gauge_field", "gauge_field_sliced", "random_su3", "gaussian_spinors",
    "point_sources", "coarse_stencil", "Philox4x32",
]


def volume(L) -> int:
    L = tuple(int(v) for v in L)
    return L[0] * L[1] * L[2] * L[3]


def rng(seed: int) -> np.random.Generator:
    """NumPy PCG64 generator for a seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _reunitarise(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt the first two rows, third row = conj(row0 x row1).

    The result is unitary with determinant exactly one (to rounding).
    """
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.cross(r0, r1).conj()
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(shape, eps: float, gen: np.random.Generator) -> np.ndarray:
    """SU(3) matrices ``exp(i eps H)`` with ``H`` Gaussian, traceless, Hermitian.

    ``A`` has iid N(0,1) real and imaginary parts, ``H = (A + A^H)/2 - tr/3``;
    the exponential is taken through the eigendecomposition of ``H``, then the
    matrix is reunitarised.
    """
    shape = tuple(shape)
    A = gen.standard_normal(shape + (3, 3)) + 1j * gen.standard_normal(shape + (3, 3))
    H = 0.5 * (A + np.swapaxes(A.conj(), -1, -2))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    w, Q = np.linalg.eigh(H)
    U = (Q * np.exp(1j * eps * w)[..., None, :]) @ np.swapaxes(Q.conj(), -1, -2)
    return _reunitarise(U)


def gauge_field(L, eps: float, seed: int) -> np.ndarray:
    """Near-unit SU(3) gauge field, complex128 ``[V][4][3][3]``."""
    V = volume(L)
    return np.ascontiguousarray(random_su3((V, 4), eps, rng(seed)))


def _slice_links(args):
    n_sites, eps, seed, t = args
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(t)])))
    return random_su3((n_sites, 4), eps, g)


def gauge_field_sliced(L, eps: float, seed: int, workers: int = 0) -> np.ndarray:
    """Near-unit SU(3) gauge field for large lattices, complex128 ``[V][4][3][3]``.

    The same distribution as :func:`gauge_field`, drawn one time slice at a
    time: the links of slice ``t`` come from PCG64 seeded with
    ``SeedSequence([seed, t])``, so the field does not depend on how many
    processes draw it.  ``workers > 1`` draws the slices in a pool of that
    many spawned processes (spawned, so that a process that already uses a
    GPU can call it).
    """
    L = tuple(int(v) for v in L)
    per = L[0] * L[1] * L[2]
    jobs = [(per, eps, seed, t) for t in range(L[3])]
    if workers and workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_slice_links, jobs))
    else:
        parts = [_slice_links(j) for j in jobs]
    return np.ascontiguousarray(np.concatenate(parts, axis=0))


def unit_gauge(L) -> np.ndarray:
    V = volume(L)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_spinors(n: int, L, seed: int) -> np.ndarray:
    """``n`` spinor fields with iid N(0,1) real and imaginary parts, ``[n][V][4][3]``."""
    V = volume(L)
    g = rng(seed)
    return np.ascontiguousarray(
        g.standard_normal((n, V, 4, 3)) + 1j * g.standard_normal((n, V, 4, 3)))


def point_sources(L, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at one site, ``[12][V][4][3]``.

    Source ``k`` is ``delta(x, site) * delta((spin, colour), (k // 3, k % 3))``.
    """
    V = volume(L)
    b = np.zeros((12, V, 4, 3), np.complex128)
    for k in range(12):
        b[k, site, k // 3, k % 3] = 1.0
    return b


def coarse_stencil(NX: int, n2: int, seed: int, diag: float = 4.0, hop: float = 0.15) -> np.ndarray:
    """A 9-point coarse stencil with ``n2 x n2`` complex blocks, complex128
    ``[NX][9][n2][n2]`` (block 0 the self block, 1 + 2 mu / 2 + 2 mu the
    links to X + mu / X - mu): self blocks ``diag * 1`` plus Gaussian entries
    of standard deviation ``hop / sqrt(n2)``, link blocks Gaussian with that
    deviation.  The shape and the diagonal dominance of the coarse operator of
    a massive Wilson-clover D, for exercising coarse solvers on large coarse
    lattices without assembling one."""
    g = rng(seed)
    sd = hop / np.sqrt(n2)
    B = sd * (g.standard_normal((NX, 9, n2, n2)) + 1j * g.standard_normal((NX, 9, n2, n2)))
    B[:, 0] += diag * np.eye(n2)
    return np.ascontiguousarray(B)


class Philox4x32:
    """Philox4x32-10 counter-based generator (Salmon et al., SC'11).

    Written from the published definition: a 128-bit counter and a 64-bit
    key, ten rounds of two 32x32->64 multiplies with the Weyl-sequence key
    schedule.  Used to cross-check the device generator bit for bit.
    """
    M0 = 0xD2511F53
    M1 = 0xCD9E8D57
    W0 = 0x9E3779B9
    W1 = 0xBB67AE85
    MASK = 0xFFFFFFFF

    @classmethod
    def block(cls, ctr, key):
        """Return the 4 output words for counter ``ctr`` (4 ints) and key (2 ints).

        Vectorised over numpy uint64 arrays of equal shape.
        """
        c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in ctr)
        k0, k1 = (np.asarray(k, dtype=np.uint64) for k in key)
        m = np.uint64(cls.MASK)
        for r in range(10):
            p0 = np.uint64(cls.M0) * c0
            p1 = np.uint64(cls.M1) * c2
            hi0, lo0 = p0 >> np.uint64(32), p0 & m
            hi1, lo1 = p1 >> np.uint64(32), p1 & m
            c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & m, lo1, (hi0 ^ c3 ^ k1) & m, lo0
            if r < 9:
                k0 = (k0 + np.uint64(cls.W0)) & m
                k1 = (k1 + np.uint64(cls.W1)) & m
        return c0, c1, c2, c3
