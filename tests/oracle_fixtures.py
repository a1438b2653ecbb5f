"""Shared small lattices and fields for the oracle pin tests (CPU only)."""
from __future__ import annotations

import functools

import numpy as np
import torch

import synthetic as syn
from oracle.dirac import WilsonClover

C128 = torch.complex128


def t(a) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a))


def rel(a, b) -> float:
    a = torch.as_tensor(a)
    b = torch.as_tensor(b)
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


def dot(a, b) -> complex:
    return torch.vdot(a.reshape(-1), b.reshape(-1)).item()


@functools.lru_cache(maxsize=None)
def wilson(L=(4, 4, 4, 4), eps=0.3, seed=0, m0=-0.2, csw=1.0) -> WilsonClover:
    return WilsonClover(t(syn.gauge_field(L, eps, seed)), L, m0, csw)


@functools.lru_cache(maxsize=None)
def dense_D(L=(4, 4, 4, 4), eps=0.3, seed=0, m0=-0.2, csw=1.0) -> torch.Tensor:
    return wilson(L, eps, seed, m0, csw).dense()


def spinors(n, L, seed) -> torch.Tensor:
    return t(syn.gaussian_spinors(n, L, seed))


def colour_rotate(psi, Omega):
    """(Omega psi)(x) = Omega(x) psi(x) on the colour index."""
    return psi @ Omega.transpose(-1, -2)


def dense_P(lam, agg) -> torch.Tensor:
    """Prolongation as a dense matrix: column (X, s*n + i) is the test vector
    lambda_i projected on aggregate X and chirality s (Eq. 1, Eq. 4)."""
    n = lam.shape[0]
    V = lam.shape[1]
    P = torch.zeros((12 * V, agg.NX * 2 * n), dtype=C128)
    for X in range(agg.NX):
        sites = agg.sites[X]
        for s in (0, 1):
            for i in range(n):
                v = torch.zeros((V, 4, 3), dtype=C128)
                v[sites, 2 * s:2 * s + 2] = lam[i, sites, 2 * s:2 * s + 2]
                P[:, X * 2 * n + s * n + i] = v.reshape(-1)
    return P


def dense_block_inverse(blk, D, c) -> torch.Tensor:
    """K_c = sum over the Schwarz blocks B of colour c of I_B D_BB^-1 I_B^T,
    with D_BB the rows and columns of the dense D on the sites of B."""
    K = torch.zeros_like(D)
    for B in range(blk.n_blocks):
        if int(blk.colour_of_block[B]) != c:
            continue
        idx = (blk.sites[B][:, None] * 12 + torch.arange(12)).reshape(-1)
        K[idx[:, None], idx[None, :]] = torch.linalg.inv(D[idx][:, idx])
    return K
