"""The third level on the GPU against the three-level oracle
(oracle/three_level.py), through the C ABI.

8^4 lattice with 2^4 aggregates (a 4^4 coarse lattice of 2 n_v = 8
components per site), level-2 blocks of 2^4 coarse sites (a 2^4 coarsest
lattice), n_v2 = 4.  Both sides start from the same fine test vectors (the
oracle's orthonormalisation) and the same raw level-2 vectors.

Bounds: orthonormal level-2 vectors (FP64 on both sides) 1e-12; D_cc
1e-12 in FP64, 1e-5 in FP32 (it sums Vb x 2 n1 x n1 products of FP32 D_c
entries and vectors); the level-2 smoother 1e-11 / 1e-4 (a few dozen
dependent block products); M2 and the level-1 coarse solve in FP64 only
(the coarsest GMRES to 5e-2 must take the oracle's iteration count, which
FP32 rounding can change by one); whole solves reach the FP64 true residual
1e-10 by the oracle's D in both precisions.
"""
from __future__ import annotations

import functools

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.coarse import Aggregation, CoarseOperator, orthonormalise
from oracle.solver import Params, TwoLevelMG
from oracle.three_level import Level2Params, ThreeLevelMG
from tests.gpu_common import assert_close, gauge, make, oracle_op, rel, t

pytestmark = pytest.mark.gpu

CFG3 = ((8, 8, 8, 8), (2, 2, 2, 2), 0.25, -0.1, 1.0, 4, 3)
N2V = 4
BLOCK2 = (2, 2, 2, 2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1811_00355_gb300 as P
    P.load()
    assert torch.cuda.is_available()


@functools.lru_cache(maxsize=None)
def _fine_vectors():
    L, b, eps, m0, csw, n_v, seed = CFG3
    agg = Aggregation(oracle_op(L, eps, seed, m0, csw).geom, b)
    return orthonormalise(t(syn.gaussian_spinors(n_v, L, 61)), agg)


@functools.lru_cache(maxsize=None)
def _raw_level2():
    L, b, eps, m0, csw, n_v, seed = CFG3
    NX = int(np.prod([L[mu] // b[mu] for mu in range(4)]))
    g = np.random.default_rng(62)
    return g.standard_normal((N2V, NX, 2 * n_v)) + 1j * g.standard_normal((N2V, NX, 2 * n_v))


@functools.lru_cache(maxsize=None)
def _oracle3():
    L, b, eps, m0, csw, n_v, seed = CFG3
    mg = TwoLevelMG(t(gauge(L, eps, seed)), Params(L, b, b, n_v, m0, csw))
    mg.set_test_vectors(_fine_vectors(), orthonormalised=True)
    mg3 = ThreeLevelMG.on(mg, Level2Params(sap_block=BLOCK2, agg_block=BLOCK2, n_v=N2V))
    mg3.set_level2_vectors(t(_raw_level2()))
    return mg3


def _p2(**kw):
    import paper_1811_00355_gb300 as P
    return P.level2_default_params(block=BLOCK2, n_v=N2V, **kw)


def _handle(prec):
    """A GPU handle with the shared fine vectors, D_c and the shared level-2 vectors."""
    s = make(CFG3, prec)
    s.set_test_vectors(np.ascontiguousarray(_fine_vectors().numpy()))
    s.build_coarse()
    s.level2_init(_p2())
    s.level2_set_vectors(_raw_level2())
    return s


def _coarse_field(n, seed):
    L, b, eps, m0, csw, n_v, _ = CFG3
    NX = int(np.prod([L[mu] // b[mu] for mu in range(4)]))
    g = np.random.default_rng(seed)
    return g.standard_normal((n, NX, 2 * n_v)) + 1j * g.standard_normal((n, NX, 2 * n_v))


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_level2_vectors_and_coarse_coarse_operator(prec, tol):
    mg3 = _oracle3()
    s = _handle(prec)
    try:
        assert_close(s.level2_get_vectors(), mg3.lam2.numpy(), 1e-12, "level-2 vectors")
        assert_close(s.level2_get_op(), mg3.cop2.Dc.numpy(), tol, "D_cc")
    finally:
        s.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-4)])
def test_level2_smoother(prec, tol):
    mg3 = _oracle3()
    s = _handle(prec)
    try:
        x = _coarse_field(2, 63)
        s.level2_sap(_coarse_field(2, 73))          # the output buffers hold another result first
        got = s.level2_sap(x)
        for k in range(2):
            ref = mg3.smoother2(t(x[k])).numpy()
            assert_close(got[k], ref, tol, f"S2 field {k}")
    finally:
        s.close()


@functools.lru_cache(maxsize=None)
def _synthetic_dc():
    """A 9-point stencil less diagonal than the D_c of random fine vectors
    (where M2 is nearly exact), so that the FGMRES on D_c takes a dozen
    iterations to 1e-9"""
    L, b, eps, m0, csw, n_v, seed = CFG3
    NX = int(np.prod([L[mu] // b[mu] for mu in range(4)]))
    return syn.coarse_stencil(NX, 2 * n_v, 65, 1.0, 0.21)


def test_level2_preconditioner_and_coarse_solve_fp64():
    """M2 (Eq. 5 on level 2) and the level-1 coarse solve (FGMRES on D_c with
    M2) on a given D_c: the oracle's results and iteration counts."""
    L, b, eps, m0, csw, n_v, seed = CFG3
    mg = TwoLevelMG(t(gauge(L, eps, seed)), Params(L, b, b, n_v, m0, csw))
    mg.set_test_vectors(_fine_vectors(), orthonormalised=True)
    mg.cop = CoarseOperator(torch.from_numpy(_synthetic_dc()), mg.agg.coarse)
    mg3 = ThreeLevelMG.on(mg, Level2Params(sap_block=BLOCK2, agg_block=BLOCK2, n_v=N2V))
    mg3.set_level2_vectors(t(_raw_level2()))
    s = make(CFG3, 0)
    try:
        s.set_coarse_op(_synthetic_dc())
        s.level2_init(_p2())
        s.level2_set_vectors(_raw_level2())
        assert_close(s.level2_get_op(), mg3.cop2.Dc.numpy(), 1e-12, "D_cc of the given D_c")
        x = _coarse_field(2, 64)
        got = s.level2_apply_M2(x)
        for k in range(2):
            assert_close(got[k], mg3.apply_M2(t(x[k])).numpy(), 1e-9, f"M2 field {k}")
        # the method's tolerance (M2 is strong here: one or two iterations)
        # and a tight one that takes the FGMRES through many iterations
        for tol, bound in ((5e-2, 1e-8), (1e-9, 1e-7)):
            xs, its = s.level2_coarse_solve(x, tol)
            for k in range(2):
                xr, ir = mg3.coarse_solve(t(x[k]), tol)
                assert int(its[k]) == ir, (tol, its, ir)
                assert_close(xs[k], xr.numpy(), bound, f"coarse solve {k} to {tol}")
    finally:
        s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_three_level_solves_reach_tolerance(prec):
    """Setup on the GPU (both levels adaptive), three-level solves of point
    sources to the FP64 true residual 1e-10 by the oracle's D, equal to the
    two-level solutions within what the two stopping points allow; a new
    mass rebuilds D_c and D_cc and the three-level solve converges again."""
    L, b, eps, m0, csw, n_v, seed = CFG3
    s = make(CFG3, prec)
    try:
        s.run_setup()
        rhs = np.ascontiguousarray(syn.point_sources(L)[:2])
        x2, _ = s.solve(rhs, 1e-10)
        s.level2_init(_p2())
        s.level2_setup()
        s.set_levels(3)
        x3, info = s.solve(rhs, 1e-10)
        op = oracle_op(L, eps, seed, m0, csw)
        for k in range(rhs.shape[0]):
            assert info[k]["converged"] == 1 and info[k]["coarse_iters"] > 0
            assert rel(op.apply(t(x3[k])).numpy(), rhs[k]) <= 1e-10, info[k]
            assert rel(x3[k], x2[k]) < 1e-6
        print(f"three levels prec {prec}: outer {[i['outer_iters'] for i in info]}, "
              f"level-1 coarse iterations {[i['coarse_iters'] for i in info]}")
        s.update_mass(m0 + 0.05, csw)
        x4, info = s.solve(rhs[:1], 1e-10)
        op = oracle_op(L, eps, seed, m0 + 0.05, csw)
        assert info[0]["converged"] == 1
        assert rel(op.apply(t(x4[0])).numpy(), rhs[0]) <= 1e-10
    finally:
        s.close()


def test_level2_rejects_bad_blocks_and_state():
    import paper_1811_00355_gb300 as P
    s = make(CFG3, 1)
    try:
        with pytest.raises(P.DDAMGError) as e:
            s.level2_init(_p2())                  # no D_c yet
        assert e.value.status == 7
        s.set_test_vectors(np.ascontiguousarray(_fine_vectors().numpy()))
        s.build_coarse()
        with pytest.raises(P.DDAMGError) as e:
            s.level2_init(P.level2_default_params(block=(4, 4, 4, 4), n_v=N2V))   # one block per direction
        assert e.value.status == 1
        with pytest.raises(P.DDAMGError) as e:
            s.set_levels(3)                       # level 2 not set up
        assert e.value.status == 7
    finally:
        s.close()
