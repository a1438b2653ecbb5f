"""The critical-mass reading (host only): sigma_min of D from Lanczos equals
the smallest |eigenvalue| of the Hermitian g5 D formed densely, and on unit
links the search lands on the closed form of the free operator, whose lowest
modes are m0 + 1 - cos(pi/L_t) +- i sin(pi/L_t) (antiperiodic time, zero
spatial momentum)."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.critical_mass import critical_mass, sigma_min
from oracle.dirac import GAMMA5, WilsonClover

L4 = (4, 4, 4, 4)


def test_sigma_min_equals_dense_hermitian_spectrum():
    U = torch.from_numpy(syn.gauge_field(L4, 0.3, 2))
    m0, csw = -0.2, 1.3
    D = WilsonClover(U, L4, m0, csw).dense().numpy()
    g5 = np.tile(np.repeat(np.diag(GAMMA5.numpy()).real, 3), 256)
    Q = g5[:, None] * D
    assert np.allclose(Q, Q.conj().T, atol=1e-13)
    want = np.abs(np.linalg.eigvalsh(Q)).min()
    assert sigma_min(U, L4, m0, csw, tol=1e-10) == pytest.approx(want, rel=1e-7)


def test_free_field_critical_mass():
    U = torch.from_numpy(syn.unit_gauge(L4))
    m, s, evals = critical_mass(U, L4, 1.0, -0.6, 0.0, xtol=2e-3, tol=1e-10)
    assert m == pytest.approx(-(1.0 - math.cos(math.pi / 4)), abs=2e-3)
    assert s == pytest.approx(math.sin(math.pi / 4), rel=1e-5)
    # the searched function really has its least value there
    assert s <= min(v for _, v in evals) + 1e-6
    assert max(v for _, v in evals) > s + 1e-3
