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
