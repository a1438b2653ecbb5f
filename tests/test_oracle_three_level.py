"""Pins of the three-level oracle (host only).

Level 2 is built on the coarse operator of an 8^4 lattice with 2^4
aggregates (a 4^4 coarse lattice, 2n components per site); its own
aggregates of 2^4 coarse sites give a 2^4 coarsest lattice.  What fixes the
level-2 pieces independently of their code: orthonormality and adjointness
of R2 and P2, D_cc = P2^H D_c P2 formed densely, G5-hermiticity
(G5 = diag(1_n, -1_n) per coarse site), the full-space limit (P2 unitary:
P2 D_cc^-1 P2^H = D_c^-1), the block solve of the level-2 smoother against
the dense solve of the blocks, the three-level M against the two-level M
when both coarse solves are exact, and the solve itself against the oracle's
D.
"""
from __future__ import annotations

import functools

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.coarse import CoarseOperator
from oracle.solver import Params, TwoLevelMG
from oracle.three_level import (CoarseAggregation, CoarseSchwarz, Level2Params, ThreeLevelMG,
                                coarse_coarse_operator, orthonormalise_c, prolong_c, restrict_c)

L8 = (8, 8, 8, 8)


def _rand(shape, seed):
    g = np.random.default_rng(seed)
    return torch.from_numpy(g.standard_normal(shape) + 1j * g.standard_normal(shape))


@functools.lru_cache(maxsize=None)
def _level1(n1, seed=3):
    """Two-level pieces on 8^4 with random orthonormal fine test vectors."""
    U = torch.from_numpy(syn.gauge_field(L8, 0.25, seed))
    p = Params(L=L8, sap_block=(2, 2, 2, 2), agg_block=(2, 2, 2, 2), n_v=n1, m0=-0.1, csw=1.0)
    mg = TwoLevelMG(U, p)
    mg.set_test_vectors(_rand((n1, 4096, 4, 3), seed + 10))
    return mg


def _dense_P2(lam2, agg2):
    n2 = lam2.shape[0]
    N = agg2.NX * 2 * n2
    E = torch.eye(N, dtype=torch.complex128).reshape(N, agg2.NX, 2 * n2)
    return prolong_c(lam2, agg2, E).reshape(N, -1).T              # [NX 2n1][NX' 2n2]


def _level2(n1, n2, seed=5):
    mg = _level1(n1)
    cop = mg.cop
    agg2 = CoarseAggregation(cop.geom, (2, 2, 2, 2), n1)
    lam2 = orthonormalise_c(_rand((n2, cop.NX, 2 * n1), seed), agg2)
    return mg, cop, agg2, lam2


def _g5(nsites, n):
    return torch.tile(torch.cat([torch.ones(n), -torch.ones(n)]), (nsites,)).to(torch.complex128)


def test_level2_projections_orthonormal_and_adjoint():
    mg, cop, agg2, lam2 = _level2(2, 3)
    P2 = _dense_P2(lam2, agg2)
    assert torch.allclose(P2.conj().T @ P2, torch.eye(P2.shape[1], dtype=torch.complex128), atol=1e-13)
    b = _rand((cop.NX, 4), 7)
    y = _rand((agg2.NX, 6), 8)
    lhs = torch.vdot(restrict_c(lam2, agg2, b).reshape(-1), y.reshape(-1))
    rhs = torch.vdot(b.reshape(-1), prolong_c(lam2, agg2, y).reshape(-1))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # R2 is P2^H
    assert torch.allclose(restrict_c(lam2, agg2, b).reshape(-1), P2.conj().T @ b.reshape(-1), atol=1e-12)


def test_level2_orthonormalisation_holds_for_nearly_dependent_vectors():
    """Vectors that differ by 1e-7 of a common one: one classical
    Gram-Schmidt pass leaves their overlaps at the 1e-9 level, the second
    pass brings P2^H P2 back to the identity."""
    mg = _level1(2)
    agg2 = CoarseAggregation(mg.cop.geom, (2, 2, 2, 2), 2)
    base = _rand((1, mg.cop.NX, 4), 31)
    lam2 = base + 1e-7 * _rand((4, mg.cop.NX, 4), 32)
    P2 = _dense_P2(orthonormalise_c(lam2, agg2), agg2)
    err = torch.linalg.matrix_norm(P2.conj().T @ P2 - torch.eye(P2.shape[1], dtype=torch.complex128))
    assert err < 1e-12


def test_coarse_coarse_operator_is_galerkin_and_gamma5_hermitian():
    mg, cop, agg2, lam2 = _level2(2, 3)
    Dc = cop.dense()
    g5c = _g5(cop.NX, 2)
    assert torch.allclose(g5c[:, None] * Dc * g5c[None, :], Dc.conj().T, atol=1e-13)
    P2 = _dense_P2(lam2, agg2)
    Dcc = CoarseOperator(coarse_coarse_operator(cop, lam2, agg2), agg2.coarse).dense()
    ref = P2.conj().T @ Dc @ P2
    assert torch.linalg.matrix_norm(Dcc - ref) <= 1e-13 * torch.linalg.matrix_norm(ref)
    g5cc = _g5(agg2.NX, 3)
    assert torch.allclose(g5cc[:, None] * Dcc * g5cc[None, :], Dcc.conj().T, atol=1e-13)


def test_level2_full_space_limit():
    """n2 = n1 |X'|: every (X', s) block spans its whole subspace, P2 is
    unitary and the two-grid correction with an exact coarsest solve is
    D_c^-1 itself."""
    n1 = 2
    mg, cop, agg2, lam2 = _level2(n1, n1 * 16)
    P2 = _dense_P2(lam2, agg2)
    I = torch.eye(P2.shape[0], dtype=torch.complex128)
    assert torch.allclose(P2 @ P2.conj().T, I, atol=1e-12)
    Dcc = CoarseOperator(coarse_coarse_operator(cop, lam2, agg2), agg2.coarse).dense()
    b = _rand((cop.NX * 2 * n1,), 9)
    x = P2 @ torch.linalg.solve(Dcc, P2.conj().T @ b)
    assert torch.linalg.vector_norm(cop.dense() @ x - b) <= 1e-11 * torch.linalg.vector_norm(b)


def test_level2_block_solve_converges_to_the_dense_block_solve():
    """With many MR steps the level-2 block solve is the exact solve of D_c
    restricted to the blocks of one colour (links that leave a block cut)."""
    mg, cop, agg2, lam2 = _level2(2, 3)
    sap2 = CoarseSchwarz(cop, (2, 2, 2, 2))
    Dc = cop.dense()
    n2c = 4
    blk = sap2.blk.block_of_site.repeat_interleave(n2c)
    col = sap2.blk.colour_of_site.repeat_interleave(n2c)
    same = blk[:, None] == blk[None, :]
    r = _rand((cop.NX, n2c), 11)
    for c in (0, 1):
        sel = torch.nonzero(col == c)[:, 0]
        DB = (Dc * same)[sel][:, sel]
        want = torch.zeros(cop.NX * n2c, dtype=torch.complex128)
        want[sel] = torch.linalg.solve(DB, r.reshape(-1)[sel])
        got = sap2.block_solve(r, c, 400).reshape(-1)
        assert torch.linalg.vector_norm(got - want) <= 1e-9 * torch.linalg.vector_norm(want)


def test_three_level_M_with_exact_coarse_solves_is_the_two_level_M():
    """Solved to 1e-12, the level-1 coarse system gives the same coarse
    correction whether GMRES or FGMRES with M2 solves it, so the three-level
    M equals the two-level M with an exact coarse solve."""
    n1, n2 = 4, 4
    mg = _level1(n1)
    three = ThreeLevelMG.on(mg, Level2Params(n_v=n2, setup_iters=0))
    three.set_level2_vectors(_rand((n2, mg.cop.NX, 2 * n1), 13))
    r = _rand((4096, 4, 3), 14)
    tol = mg.p.coarse_tol
    mg.p.coarse_tol = 1e-12
    try:
        want = mg.apply_M(r)
    finally:
        mg.p.coarse_tol = tol
    got = three.apply_M(r, tol=1e-12)
    assert torch.linalg.vector_norm(got - want) <= 1e-9 * torch.linalg.vector_norm(want)
    assert three.level1_iters and three.level1_iters[-1] > 0


def test_three_level_solve_reaches_the_tolerance():
    """Full setup (two-level on the fine level, then level 2) and an outer
    solve to 1e-10 by the oracle's D; the solution agrees with the
    two-level one."""
    U = torch.from_numpy(syn.gauge_field(L8, 0.25, 21))
    p = Params(L=L8, sap_block=(2, 2, 2, 2), agg_block=(2, 2, 2, 2), n_v=6, m0=-0.1, csw=1.0,
               setup_iters=2)
    p2 = Level2Params(n_v=6, setup_iters=1)
    mg3 = ThreeLevelMG(U, p, p2)
    mg3.setup(_rand((6, 4096, 4, 3), 22), _rand((6, 256, 12), 23))
    b = _rand((4096, 4, 3), 24)
    x3, its3, ok3 = mg3.solve(b, 1e-10)
    assert ok3 and mg3.true_residual(b, x3) <= 1e-10
    assert mg3.level1_iters and max(mg3.level1_iters) > 0
    x2, its2, ok2 = mg3.two.solve(b, 1e-10)
    assert ok2
    assert torch.linalg.vector_norm(x3 - x2) <= 1e-7 * torch.linalg.vector_norm(x2)
    # the level-2 setup's invariants
    P2 = _dense_P2(mg3.lam2, mg3.agg2)
    assert torch.allclose(P2.conj().T @ P2, torch.eye(P2.shape[1], dtype=torch.complex128), atol=1e-12)


def test_level2_geometry_is_validated():
    mg = _level1(2)
    with pytest.raises(ValueError):
        CoarseSchwarz(mg.cop, (1, 2, 2, 2))          # odd block extent
    with pytest.raises(ValueError):
        CoarseSchwarz(mg.cop, (4, 2, 2, 2))          # one block along x: odd block grid
