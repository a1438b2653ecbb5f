"""Shared helpers of the GPU tests: seeded workloads, oracle twins, norms."""
from __future__ import annotations

import functools

import numpy as np
import torch

import synthetic as syn
from oracle.dirac import WilsonClover
from oracle.sap import SchwarzSmoother

# per-apply relative error bounds (norm-wise) of the two precisions
TOL64 = 1e-13
TOL32 = 1e-6

# (L, block, eps, m0, csw, n_v, seed): the 4^4 FP64 workload, a mid-size
# lattice that spans several blocks of 4^4 with extent-2 and extent-4 coarse
# directions, and the full 16^4 workload
SMALL = ((4, 4, 4, 4), (2, 2, 2, 2), 0.3, -0.2, 1.0, 8, 0)
MID = ((8, 8, 8, 16), (4, 4, 4, 4), 0.25, -0.3, 1.2, 6, 3)
FULL = ((16, 16, 16, 16), (4, 4, 4, 4), 0.25, -0.3, 1.2, 20, 1)


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def maxrel(a, b) -> float:
    """Largest element-wise deviation over the largest reference element.
    An error confined to a few sites (one block face, one aggregate, the
    hops across the time boundary) is not diluted by the size of the field
    here, as it is in the norm-wise rel()."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def assert_close(a, b, tol, what="", etol=None):
    """Norm-wise relative error below tol and element-wise relative error
    below etol (default tol)."""
    etol = tol if etol is None else etol
    r, m = rel(a, b), maxrel(a, b)
    assert r < tol and m < etol, f"{what} norm-wise {r:.3e} (bound {tol:.1e}), element-wise {m:.3e} (bound {etol:.1e})"
    return r, m


def t(a) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a))


@functools.lru_cache(maxsize=None)
def gauge(L, eps, seed):
    return syn.gauge_field(L, eps, seed)


@functools.lru_cache(maxsize=None)
def oracle_op(L, eps, seed, m0, csw):
    return WilsonClover(t(gauge(L, eps, seed)), L, m0, csw)


def make(cfg, precision, **kw):
    import paper_1811_00355_gb300 as P
    L, b, eps, m0, csw, n_v, seed = cfg
    p = P.default_params(L=L, sap_block=b, n_v=n_v, m0=m0, csw=csw, precision=precision, **kw)
    return P.DDAMG(p, gauge(L, eps, seed))


def smoother(cfg):
    L, b, eps, m0, csw, n_v, seed = cfg
    return SchwarzSmoother(oracle_op(L, eps, seed, m0, csw), b)
