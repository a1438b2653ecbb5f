"""Critical bare mass of a gauge field (oracle; test infrastructure).

The light-mass workload sets m0 just above the critical mass m_c of its
ensemble, found on a small proxy lattice.  The paper does not define m_c
(its ensemble is a physical-point one); the reading here: Q(m0) = g5 D(m0)
is Hermitian and its eigenvalue nearest zero changes sign where D(m0) turns
singular.  With near-unit links and an antiperiodic time direction no
eigenvalue of Q reaches zero on a finite lattice (the lowest modes keep an
imaginary part of about sin(pi / L_t) in D), so there is no sign change to
bisect: m_c is read as the mass where the smallest |eigenvalue| of Q,
which equals the smallest singular value sigma_min of D, is least.

sigma_min(D(m0))^2 is the lowest eigenvalue of D^H D, taken by implicitly
restarted Lanczos (ARPACK through scipy) on the oracle's D; m_c by golden-
section search of sigma_min over an interval that brackets its minimum.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .dirac import WilsonClover


def sigma_min(U, L, m0, csw, tol=1e-8, ncv=40, seed=0):
    """Smallest singular value of the oracle's D(m0) (ARPACK on D^H D)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    op = WilsonClover(U, L, m0, csw)
    n = op.geom.V * 12
    g5 = torch.tensor([1.0, 1.0, -1.0, -1.0], dtype=torch.complex128)[None, :, None]

    def normal(v):
        x = torch.from_numpy(np.ascontiguousarray(v.reshape(op.geom.V, 4, 3)))
        y = op.apply(x)
        z = g5 * op.apply(g5 * y)                   # D^H y = g5 D g5 y
        return z.reshape(-1).numpy()

    A = LinearOperator((n, n), matvec=normal, dtype=np.complex128)
    v0 = np.random.default_rng(seed).standard_normal(n) + 0j
    w = eigsh(A, k=1, which="SA", tol=tol, ncv=ncv, v0=v0, return_eigenvectors=False)
    return math.sqrt(max(float(w[0]), 0.0))


def critical_mass(U, L, csw, lo, hi, xtol=2e-3, **kw):
    """Golden-section search for the m0 in [lo, hi] that minimises
    sigma_min(D(m0)).  Returns (m_c, sigma_min at m_c, evaluations)."""
    r = (math.sqrt(5.0) - 1.0) / 2.0
    evals = []

    def f(m):
        s = sigma_min(U, L, m, csw, **kw)
        evals.append((m, s))
        return s

    a, b = lo, hi
    c, d = b - r * (b - a), a + r * (b - a)
    fc, fd = f(c), f(d)
    while b - a > xtol:
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - r * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + r * (b - a)
            fd = f(d)
    m = 0.5 * (a + b)
    return m, f(m), evals


def main():
    """m_c of a proxy lattice: ``python -m oracle.critical_mass L eps csw seed lo hi``."""
    import json
    import sys
    import synthetic as syn
    Ls, eps, csw, seed, lo, hi = sys.argv[1:7]
    L = tuple(int(v) for v in Ls.split(","))
    U = torch.from_numpy(syn.gauge_field(L, float(eps), int(seed)))
    m, s, evals = critical_mass(U, L, float(csw), float(lo), float(hi), xtol=5e-3, tol=1e-4, ncv=64)
    print(json.dumps({"L": L, "eps": float(eps), "csw": float(csw), "seed": int(seed), "m_c": round(m, 4),
                      "sigma_min": s, "evaluations": [(round(a, 5), b) for a, b in evals]}))


if __name__ == "__main__":
    main()
