"""Pins of the oracle's whole solver on the 4^4 FP64 workload (2^4 blocks and
aggregates, n_v = 8, 3 setup iterations, m0 = -0.2, csw = 1.0, eps = 0.3)."""
from __future__ import annotations

import pytest
import torch

import synthetic as syn
from oracle.coarse import CoarseOperator, coarse_operator
from oracle.solver import Params, TwoLevelMG
from tests.oracle_fixtures import C128, dense_block_inverse, dense_D, dense_P, rel, spinors, t

L = (4, 4, 4, 4)


def _params(**kw):
    base = dict(L=L, sap_block=(2, 2, 2, 2), agg_block=(2, 2, 2, 2), n_v=8,
                m0=-0.2, csw=1.0, setup_iters=3)
    base.update(kw)
    return Params(**base)


@pytest.fixture(scope="module")
def mg4():
    mg = TwoLevelMG(t(syn.gauge_field(L, 0.3, 0)), _params())
    mg.setup(spinors(8, L, 1))
    return mg


def test_setup_invariants(mg4):
    """The setup's output is pinned by what it must satisfy: orthonormal
    projected test vectors and the Galerkin coarse operator."""
    lam = mg4.lam
    agg = mg4.agg
    for X in (0, 5, 15):
        for s in (0, 1):
            B = lam[:, agg.sites[X], 2 * s:2 * s + 2].reshape(lam.shape[0], -1)
            assert rel(B.conj() @ B.T, torch.eye(lam.shape[0], dtype=C128)) < 1e-14
    again = CoarseOperator(coarse_operator(mg4.op, lam, agg), agg.coarse)
    assert rel(again.Dc, mg4.cop.Dc) < 1e-15


def test_solve_matches_dense_lu(mg4):
    D = dense_D(L, 0.3, 0, -0.2, 1.0)
    b = spinors(1, L, 2)[0]
    x, its, ok = mg4.solve(b, 1e-10)
    assert ok
    assert mg4.true_residual(b, x) <= 1e-10
    xd = torch.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    cond = torch.linalg.cond(D).item()
    assert rel(x, xd) <= cond * 1e-10


def test_point_sources_converge(mg4):
    for k in (0, 7, 11):
        b = t(syn.point_sources(L))[k]
        x, its, ok = mg4.solve(b, 1e-10)
        assert ok and mg4.true_residual(b, x) <= 1e-10


def test_setup_improves_convergence(mg4):
    b = spinors(1, L, 3)[0]
    _, its_setup, _ = mg4.solve(b, 1e-10)
    mg0 = TwoLevelMG(t(syn.gauge_field(L, 0.3, 0)), _params(setup_iters=0))
    mg0.setup(spinors(8, L, 1))
    _, its_raw, _ = mg0.solve(b, 1e-10)
    assert its_setup <= its_raw


# Eq. 5 in an exact mode: with the block solves run to convergence (MR on a
# heavier mass) and the coarse system solved to rounding, M is the fixed linear
# map  M = C + S (1 - D C),  C = P D_c^-1 P^H,  S the multiplicative Schwarz
# smoother written with dense block inverses.  Both sides are formed from
# dense matrices that share nothing with the oracle's stencil code.
EXACT = dict(m0=0.3, n_v=4, n_sap=2, mr_iters=200, coarse_tol=1e-14, coarse_maxiter=4000, setup_iters=0)


def _exact_mg(cls=TwoLevelMG):
    mg = cls(t(syn.gauge_field(L, 0.3, 0)), _params(**EXACT))
    mg.set_test_vectors(spinors(EXACT["n_v"], L, 70))
    return mg


def _dense_eq5(mg, r):
    D = dense_D(L, 0.3, 0, EXACT["m0"], 1.0)
    Pd = dense_P(mg.lam, mg.agg)
    C = Pd @ torch.linalg.solve(Pd.conj().T @ D @ Pd, Pd.conj().T)
    K = [dense_block_inverse(mg.sap.blk, D, c) for c in (0, 1)]

    def schwarz(v):
        x = torch.zeros_like(v)
        for _ in range(EXACT["n_sap"]):
            for c in (0, 1):
                x = x + K[c] @ (v - D @ x)
        return x

    rv = r.reshape(-1)
    x1 = C @ rv
    return (x1 + schwarz(rv - D @ x1)).reshape(r.shape)


class _PreSmoothing(TwoLevelMG):
    """Planted mistake: smoothing before the coarse correction."""
    def apply_M(self, r):
        e = self.smoother(r)
        return e + self.coarse_correction(r - self.op.apply(e))


class _NoResidualUpdate(TwoLevelMG):
    """Planted mistake: the smoother applied to r instead of r - D x1."""
    def apply_M(self, r):
        return self.coarse_correction(r) + self.smoother(r)


class _WrongSign(TwoLevelMG):
    """Planted mistake: r + D x1 as the smoother's right-hand side."""
    def apply_M(self, r):
        x1 = self.coarse_correction(r)
        return x1 + self.smoother(r + self.op.apply(x1))


class _CoarseOnly(TwoLevelMG):
    """Planted mistake: the smoother term dropped."""
    def apply_M(self, r):
        return self.coarse_correction(r)


def test_preconditioner_is_eq5_exactly():
    """Eq. 5 with exact block and coarse solves equals the dense formula
    C + S (1 - D C) to rounding."""
    mg = _exact_mg()
    r = spinors(1, L, 71)[0]
    assert rel(mg.apply_M(r), _dense_eq5(mg, r)) < 1e-11


@pytest.mark.parametrize("cls", [_PreSmoothing, _NoResidualUpdate, _WrongSign, _CoarseOnly])
def test_eq5_pin_rejects_planted_mistakes(cls):
    """Each plausible mistake in the preconditioner moves M r far from the
    dense Eq. 5 (so the exact pin above would catch it)."""
    mg = _exact_mg(cls)
    r = spinors(1, L, 71)[0]
    assert rel(mg.apply_M(r), _dense_eq5(mg, r)) > 1e-3


def test_preconditioner_reduces_coarse_residual(mg4):
    """At the method's coarse tolerance the coarse part is removed from the
    residual up to 5e-2 (R (r - D x1) ~ 0), and M is a good approximate inverse."""
    r = spinors(1, L, 4)[0]
    from oracle.coarse import restrict
    x1 = mg4.coarse_correction(r)
    rc = restrict(mg4.lam, mg4.agg, r - mg4.op.apply(x1))
    assert torch.linalg.vector_norm(rc).item() <= 5e-2 * torch.linalg.vector_norm(
        restrict(mg4.lam, mg4.agg, r)).item() * 1.0001
    z = mg4.apply_M(r)
    res = torch.linalg.vector_norm(r - mg4.op.apply(z)).item() / torch.linalg.vector_norm(r).item()
    assert res < 0.5


def test_parameter_validation():
    with pytest.raises(ValueError):
        TwoLevelMG(t(syn.gauge_field(L, 0.3, 0)), _params(sap_block=(3, 2, 2, 2)))
    with pytest.raises(ValueError):
        TwoLevelMG(t(syn.gauge_field(L, 0.3, 0)), _params(agg_block=(4, 2, 2, 2)))
