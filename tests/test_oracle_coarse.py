"""Pins of the oracle's coarse grid: Eq. 1-4 against dense linear algebra."""
from __future__ import annotations

import pytest
import torch

from oracle.coarse import (Aggregation, CoarseOperator, coarse_operator,
                           orthonormalise, prolong, restrict)
from oracle.krylov import gmres
from tests.oracle_fixtures import C128, dense_D, dense_P, dot, rel, spinors, wilson

L = (4, 4, 4, 4)
ARGS = (L, 0.3, 0, -0.2, 1.0)


@pytest.fixture(scope="module")
def setup4():
    op = wilson(*ARGS)
    agg = Aggregation(op.geom, (2, 2, 2, 2))
    lam = orthonormalise(spinors(4, L, 31), agg)
    return op, agg, lam, dense_P(lam, agg)


def test_orthonormal(setup4):
    op, agg, lam, P = setup4
    assert rel(P.conj().T @ P, torch.eye(P.shape[1], dtype=C128)) < 1e-14


def test_orthonormalise_keeps_span():
    """Gram-Schmidt inside (X, s) changes the basis, not the span."""
    op = wilson(*ARGS)
    agg = Aggregation(op.geom, (2, 2, 2, 2))
    raw = spinors(4, L, 32)
    Praw = dense_P(raw, agg)
    Q = dense_P(orthonormalise(raw, agg), agg)
    proj = Q @ (Q.conj().T @ Praw)
    assert rel(proj, Praw) < 1e-13


def test_restrict_prolong_adjoint_and_dense(setup4):
    op, agg, lam, P = setup4
    b = spinors(1, L, 33)[0]
    bc = restrict(lam, agg, b)
    assert rel(bc.reshape(-1), P.conj().T @ b.reshape(-1)) < 1e-14
    y = torch.randn(bc.shape, dtype=torch.float64) + 1j * torch.randn(bc.shape, dtype=torch.float64)
    x = prolong(lam, agg, y)
    assert rel(x.reshape(-1), P @ y.reshape(-1)) < 1e-14
    assert abs(dot(bc, y) - dot(b, x)) < 1e-13 * abs(dot(bc, y))
    assert rel(restrict(lam, agg, prolong(lam, agg, y)), y) < 1e-14  # R P = 1


def test_coarse_operator_is_galerkin(setup4):
    """Eq. 2: D_c = P^H D P, with every coarse extent 2 (forward and backward
    links reach the same aggregate and are kept separate)."""
    op, agg, lam, P = setup4
    D = dense_D(*ARGS)
    Dc = coarse_operator(op, lam, agg)
    cop = CoarseOperator(Dc, agg.coarse)
    assert rel(cop.dense(), P.conj().T @ D @ P) < 1e-13
    # gamma5-hermiticity on the coarse grid
    n = lam.shape[0]
    s = torch.cat([torch.ones(n), -torch.ones(n)]).repeat(agg.NX).to(C128)
    Dd = cop.dense()
    assert rel(s[:, None] * Dd * s[None, :], Dd.conj().T) < 1e-13
    # per direction: backward link of X + mu = Gamma5 (forward link of X)^H Gamma5
    G5 = torch.diag(s[:2 * n])
    for mu in range(4):
        nb = agg.coarse.fwd[mu]
        lhs = Dc[nb, 2 + 2 * mu]
        rhs = G5 @ Dc[:, 1 + 2 * mu].conj().transpose(-1, -2) @ G5
        assert rel(lhs, rhs) < 1e-13


def test_coarse_operator_sampled_aggregates():
    op = wilson((8, 4, 4, 4), 0.3, 5, -0.2, 1.0)
    agg = Aggregation(op.geom, (2, 2, 2, 2))
    lam = orthonormalise(spinors(3, (8, 4, 4, 4), 34), agg)
    full = coarse_operator(op, lam, agg)
    pick = [0, 7, 19]
    part = coarse_operator(op, lam, agg, aggregates=pick)
    assert rel(part[pick], full[pick]) < 1e-15


def test_coarse_operator_4x4_aggregates_larger_coarse_lattice():
    """Galerkin identity with coarse extents 4 and 2 (8x8x4x4 lattice, 2^4 aggregates)."""
    Lr = (8, 4, 4, 8)
    op = wilson(Lr, 0.25, 6, -0.3, 1.2)
    agg = Aggregation(op.geom, (2, 2, 2, 4))
    lam = orthonormalise(spinors(2, Lr, 35), agg)
    cop = CoarseOperator(coarse_operator(op, lam, agg), agg.coarse)
    P = dense_P(lam, agg)
    x = torch.randn(P.shape[1], dtype=torch.float64) + 1j * torch.randn(P.shape[1], dtype=torch.float64)
    fine = op.apply((P @ x).reshape(-1, 4, 3)).reshape(-1)
    expect = P.conj().T @ fine
    got = cop.apply(x.reshape(agg.NX, -1)).reshape(-1)
    assert rel(got, expect) < 1e-13


def test_coarse_even_odd_gmres_tight_equals_dense(setup4):
    op, agg, lam, P = setup4
    cop = CoarseOperator(coarse_operator(op, lam, agg), agg.coarse)
    b = torch.randn(agg.NX, 2 * lam.shape[0], dtype=torch.float64).to(C128)
    x, its = cop.solve(b, 1e-13, 30, 500)
    xd = torch.linalg.solve(cop.dense(), b.reshape(-1)).reshape(b.shape)
    assert rel(x, xd) < 1e-11
    # the loose coarse tolerance of the method stops early, at <= 5e-2 of the Schur residual
    x2, its2 = cop.solve(b, 5e-2, 30, 500)
    assert its2 < its
    res = b.reshape(-1) - cop.dense() @ x2.reshape(-1)
    assert torch.linalg.vector_norm(res).item() < 0.5 * torch.linalg.vector_norm(b).item()


def test_full_space_limit():
    """n_v = 6 |X| (96 for 2^4 aggregates): P is unitary and
    P D_c^-1 P^H b = D^-1 b (brute force through the whole coarse grid)."""
    op = wilson(*ARGS)
    agg = Aggregation(op.geom, (2, 2, 2, 2))
    lam = orthonormalise(spinors(96, L, 36), agg)
    cop = CoarseOperator(coarse_operator(op, lam, agg), agg.coarse)
    b = spinors(1, L, 37)[0]
    bc = restrict(lam, agg, b)
    xc = torch.linalg.solve(cop.dense(), bc.reshape(-1)).reshape(bc.shape)
    x = prolong(lam, agg, xc)
    xd = torch.linalg.solve(dense_D(*ARGS), b.reshape(-1)).reshape(b.shape)
    assert rel(x, xd) < 1e-12


def test_gmres_textbook():
    g = torch.Generator().manual_seed(3)
    n = 60
    A = (torch.eye(n, dtype=C128)
         + 0.3 * torch.complex(torch.randn(n, n, generator=g, dtype=torch.float64),
                               torch.randn(n, n, generator=g, dtype=torch.float64)) / n ** 0.5)
    b = torch.complex(torch.randn(n, generator=g, dtype=torch.float64),
                      torch.randn(n, generator=g, dtype=torch.float64))
    x, its, ok = gmres(lambda v: A @ v, b, 1e-12, 8, 500)
    assert ok and rel(x, torch.linalg.solve(A, b)) < 1e-10
    # without restart GMRES is exact after n steps of a well-defined Arnoldi process
    x, its, ok = gmres(lambda v: A @ v, b, 1e-14, n, n)
    assert rel(x, torch.linalg.solve(A, b)) < 1e-11
    # flexible: a fixed preconditioner M gives the solution of A x = b
    Minv = torch.linalg.inv(A + 0.05 * torch.eye(n, dtype=C128))
    x, its, ok = gmres(lambda v: A @ v, b, 1e-12, 10, 100, precond=lambda v: Minv @ v)
    assert ok and its <= 10 and rel(x, torch.linalg.solve(A, b)) < 1e-10
