"""The mass-tuning tool's CG on the normal equations and its Lanczos
estimate, on a dense g5-Hermitian stand-in for D (host only)."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

from paper_1811_00355_gb300 import mass_tuning as mt


class _DenseD:
    """D = g5 H (H Hermitian positive definite) on fields [V][4][3]: then
    D^H = g5 D g5, the identity the tool relies on."""

    def __init__(self, V, seed, shift=0.0):
        rng = np.random.default_rng(seed)
        n = 12 * V
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        H = (A + A.conj().T) / 2
        H = H + (np.abs(np.linalg.eigvalsh(H)).max() * 0.5 + 1.0 + shift) * np.eye(n)
        g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
        self.D = g5[:, None] * H
        self.V = V
        self.p = type("P", (), {"csw": 1.0, "m0": 0.0})()

    def apply_D(self, x, precision=None):
        y = self.D @ x.reshape(-1).numpy()
        return torch.from_numpy(y.reshape(self.V, 4, 3))


def test_cg_normal_equations_solves_and_counts():
    d = _DenseD(4, 1)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((4, 4, 3)) + 1j * rng.standard_normal((4, 4, 3))
    its, resid, a, bt, x = mt.cg_normal_equations(d, torch.from_numpy(b), tol=1e-10, max_iter=500)
    assert resid <= 1e-10 and len(a) == its and len(bt) == its - 1
    # the recurrence residual is the true one, and x is D^-1 b
    true = np.linalg.norm(d.D @ x.reshape(-1).numpy() - b.reshape(-1)) / np.linalg.norm(b)
    assert true <= 2e-10
    x_exact = np.linalg.solve(d.D, b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1).numpy() - x_exact) <= 1e-8 * np.linalg.norm(x_exact)


def test_lanczos_extremes_bracket_the_spectrum():
    d = _DenseD(2, 3)
    rng = np.random.default_rng(4)
    b = rng.standard_normal((2, 4, 3)) + 1j * rng.standard_normal((2, 4, 3))
    ev = np.linalg.eigvalsh(d.D.conj().T @ d.D)
    # a few steps: Ritz values inside the spectrum
    _, _, a, bt, _ = mt.cg_normal_equations(d, torch.from_numpy(b), tol=0.0, max_iter=6)
    lo, hi = mt.lanczos_extremes(a, bt)
    assert ev[0] * (1 - 1e-12) <= lo <= hi <= ev[-1] * (1 + 1e-12)
    # the same k steps of Lanczos on D^H D from D^H b, with full
    # reorthogonalisation: CG's coefficients must give its tridiagonal matrix
    k = 10
    A = d.D.conj().T @ d.D
    q = d.D.conj().T @ b.reshape(-1)
    Q = [q / np.linalg.norm(q)]
    al, be = [], []
    for j in range(k):
        w = A @ Q[j]
        al.append(np.vdot(Q[j], w).real)
        for qq in Q:
            w = w - np.vdot(qq, w) * qq
        if j < k - 1:
            be.append(np.linalg.norm(w))
            Q.append(w / be[-1])
    T = np.diag(al) + np.diag(be, 1) + np.diag(be, -1)
    ev_T = np.linalg.eigvalsh(T)
    _, _, a, bt, _ = mt.cg_normal_equations(d, torch.from_numpy(b), tol=0.0, max_iter=k)
    lo, hi = mt.lanczos_extremes(a, bt)
    assert lo == pytest.approx(ev_T[0], rel=1e-9) and hi == pytest.approx(ev_T[-1], rel=1e-9)


def test_predicted_iterations_bound():
    assert mt.predicted_iterations(1.0, 1e-10) == pytest.approx(0.5 * math.log(2e10))
    assert mt.predicted_iterations(4e6, 1e-10) == pytest.approx(1000 * math.log(2e10))


class _ShiftedD:
    """D(m0) = (d + m0) 1 + i K on fields [V][4][3], with K Hermitian and
    mapping chirality + to - (so g5 K g5 = -K): then D^H = g5 D g5, the
    eigenvalues are d + m0 + i kappa (kappa = +-singular values of K's
    chirality block) and the smallest singular value of D is
    sqrt((d + m0)^2 + kappa_min^2), least at m0 = -d."""

    def __init__(self, V, d, kappa, seed):
        rng = np.random.default_rng(seed)
        n = 12 * V
        g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
        plus, minus = np.where(g5 > 0)[0], np.where(g5 < 0)[0]
        h = n // 2
        Q1, _ = np.linalg.qr(rng.standard_normal((h, h)) + 1j * rng.standard_normal((h, h)))
        Q2, _ = np.linalg.qr(rng.standard_normal((h, h)) + 1j * rng.standard_normal((h, h)))
        B = Q1 @ np.diag(np.linspace(kappa, 2.0, h)) @ Q2.conj().T
        self.K = np.zeros((n, n), complex)
        self.K[np.ix_(plus, minus)] = B
        self.K[np.ix_(minus, plus)] = B.conj().T
        self.d, self.V, self.n = d, V, n
        self.p = type("P", (), {"csw": 1.0, "m0": 0.0})()

    def update_mass(self, m0, csw):
        self.p.m0, self.p.csw = m0, csw

    def apply_D(self, x, precision=None):
        v = x.reshape(-1).numpy()
        y = (self.d + self.p.m0) * v + 1j * (self.K @ v)
        return torch.from_numpy(y.reshape(self.V, 4, 3))


def test_dense_stand_in_is_g5_hermitian():
    f = _ShiftedD(2, 0.3, 0.05, 5)
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), 2)
    D = (f.d - 0.1) * np.eye(f.n) + 1j * f.K
    assert np.allclose((g5[:, None] * D) * g5[None, :], D.conj().T)


def test_scan_stops_past_the_most_critical_mass():
    """No mass reaches the target: the scan passes the maximum of the count
    (at m0 = -d) and returns it."""
    f = _ShiftedD(2, 0.3, 0.05, 6)
    rng = np.random.default_rng(7)
    b = torch.from_numpy(rng.standard_normal((2, 4, 3)) + 1j * rng.standard_normal((2, 4, 3)))
    r = mt.scan_mass(f, b, target=1e9, m0_start=0.0, step=0.05, probe_iters=200, probe_tol=1e-12,
                     patience=3, confirm=True, confirm_cap=2000)
    assert not r["target_reached"]
    assert r["m0"] == pytest.approx(-0.3, abs=1e-9)
    preds = [e["predicted"] for e in r["scan"]]
    assert len(preds) == 7 + 3 and max(preds) == preds[6]
    assert r["cg_residual"] <= 1e-10 and not r["capped"]


def test_scan_stops_at_the_first_mass_over_the_target():
    f = _ShiftedD(2, 0.3, 0.01, 8)
    rng = np.random.default_rng(9)
    b = torch.from_numpy(rng.standard_normal((2, 4, 3)) + 1j * rng.standard_normal((2, 4, 3)))
    r = mt.scan_mass(f, b, target=1000, m0_start=0.0, step=0.05, probe_iters=200, probe_tol=1e-12,
                     confirm=False)
    assert r["target_reached"]
    preds = [e["predicted"] for e in r["scan"]]
    assert preds[-1] > 1000 and all(p <= 1000 for p in preds[:-1])
    assert r["m0"] == r["scan"][-1]["m0"]
