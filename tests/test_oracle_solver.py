"""Pins of the oracle's whole solver on the 4^4 FP64 workload (2^4 blocks and
aggregates, n_v = 8, 3 setup iterations, m0 = -0.2, csw = 1.0, eps = 0.3)."""
from __future__ import annotations

import pytest
import torch

import synthetic as syn
from oracle.coarse import CoarseOperator, coarse_operator
from oracle.solver import Params, TwoLevelMG
from tests.oracle_fixtures import C128, dense_D, rel, spinors, t

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


def test_preconditioner_is_eq5(mg4):
    """M r = x1 + SAP(r - D x1) with x1 = P D_c^-1 R r: check the coarse part
    is removed from the residual in the coarse space, R (r - D x1) ~ 0 up to the
    coarse tolerance, and that M is a good approximate inverse."""
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
