"""Pins of the oracle's SAP smoother and even-odd MR block solver.

MR run to convergence must reproduce the dense solve of the block operator
(D with rows and columns restricted to the block), and SAP with converged
block solves must reproduce the textbook multiplicative Schwarz iteration
written with dense matrices.
"""
from __future__ import annotations

import torch

from oracle.sap import SchwarzSmoother
from tests.oracle_fixtures import dense_block_inverse, dense_D, rel, spinors, wilson

L = (4, 4, 4, 4)
ARGS = (L, 0.3, 0, 0.3, 1.0)          # heavier mass: MR converges quickly


def test_mr_converges_to_block_solve():
    op = wilson(*ARGS)
    D = dense_D(*ARGS)
    sm = SchwarzSmoother(op, (2, 2, 2, 2))
    r = spinors(1, L, 21)[0]
    for c in (0, 1):
        e = sm.block_solve(r, c, 200)
        K = dense_block_inverse(sm.blk, D, c)
        expect = (K @ r.reshape(-1)).reshape(r.shape)
        assert rel(e, expect) < 1e-12


def test_mr_few_iterations_reduces_block_residual():
    """Each MR step minimises the Schur residual: with k = 1..4 the block
    residual of the even-odd system decreases monotonically."""
    op = wilson(*ARGS)
    D = dense_D(*ARGS)
    sm = SchwarzSmoother(op, (2, 2, 2, 2))
    r = spinors(1, L, 22)[0]
    mask = sm.mask[0, None]
    prev = None
    for k in range(1, 5):
        e = sm.block_solve(r, 0, k)
        res = mask * (r - (D @ e.reshape(-1)).reshape(r.shape))
        nr = torch.linalg.vector_norm(res).item()
        if prev is not None:
            assert nr < prev
        prev = nr


def test_sap_matches_dense_multiplicative_schwarz():
    op = wilson(*ARGS)
    D = dense_D(*ARGS)
    sm = SchwarzSmoother(op, (2, 2, 2, 2))
    b = spinors(1, L, 23)[0]
    K = [dense_block_inverse(sm.blk, D, c) for c in (0, 1)]
    x = torch.zeros(D.shape[0], dtype=D.dtype)
    bv = b.reshape(-1)
    for _ in range(3):
        for c in (0, 1):
            x = x + K[c] @ (bv - D @ x)
    got = sm.apply(b, 3, 200)
    assert rel(got, x.reshape(b.shape)) < 1e-12


def test_sap_is_linear_for_fixed_iterations_only_in_exact_mode():
    """With converged block solves SAP is a linear map: SAP(a u + v) = a SAP(u) + SAP(v)."""
    op = wilson(*ARGS)
    sm = SchwarzSmoother(op, (2, 2, 2, 2))
    u, v = spinors(2, L, 24)
    a = 0.7 - 0.2j
    lhs = sm.apply(a * u + v, 2, 200)
    rhs = a * sm.apply(u, 2, 200) + sm.apply(v, 2, 200)
    assert rel(lhs, rhs) < 1e-12
