"""Parity of every step of the CUDA path with the CPU oracle, through the C ABI.

Per-apply relative (norm-wise) error bounds: FP64 1e-13, FP32 1e-6; index
maps bit-exact; every solution reaches a true FP64 residual <= 1e-10.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.coarse import (Aggregation, CoarseOperator, coarse_operator,
                           orthonormalise, prolong, restrict)
from oracle.dirac import WilsonClover
from oracle.lattice import index_maps
from oracle.solver import Params, TwoLevelMG
from tests.gpu_common import (FULL, MID, SMALL, TOL32, TOL64, assert_close, make, oracle_op, rel,
                              smoother, t)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1811_00355_gb300 as P
    P.load()
    assert torch.cuda.is_available()


def _P():
    import paper_1811_00355_gb300 as P
    return P


@pytest.mark.parametrize("cfg", [SMALL, MID])
def test_index_maps_bit_exact(cfg):
    s = make(cfg, _P().FP64)
    got = s.index_maps()
    ref = index_maps(cfg[0], cfg[1], cfg[1])
    for k in ("parity", "block", "colour", "aggregate", "coarse_parity"):
        assert np.array_equal(got[k], ref[k].numpy()), k


@pytest.mark.parametrize("cfg", [SMALL, MID])
def test_clover_packed_blocks(cfg):
    L, b, eps, m0, csw, n_v, seed = cfg
    s = make(cfg, _P().FP64)
    op = oracle_op(L, eps, seed, m0, csw)
    assert_close(s.get_clover(False), op.packed_clover(False).numpy(), TOL64)
    assert_close(s.get_clover(True), op.packed_clover(True).numpy(), TOL64)


@pytest.mark.parametrize("cfg", [SMALL, MID, FULL])
@pytest.mark.parametrize("prec", [0, 1])
def test_wilson_clover_D(cfg, prec):
    L, b, eps, m0, csw, n_v, seed = cfg
    s = make(cfg, prec)
    op = oracle_op(L, eps, seed, m0, csw)
    x = syn.gaussian_spinors(2, L, 40)
    y = s.apply_D(x, precision=prec)
    ref = op.apply(t(x)).numpy()
    tol = TOL64 if prec == 0 else TOL32
    for k in range(2):
        assert_close(y[k], ref[k], tol)


@pytest.mark.parametrize("cfg", [SMALL, MID, FULL])
@pytest.mark.parametrize("variant", [0, 1])
def test_D_variants_fp32(cfg, variant):
    """Both measured variants of the FP32 D (one thread per site, four threads
    per site) match the oracle; the autotuner records its choice."""
    P = _P()
    L, b, eps, m0, csw, n_v, seed = cfg
    P.pin_variant("D fp32", variant)
    try:
        s = make(cfg, 1)
        op = oracle_op(L, eps, seed, m0, csw)
        x = syn.gaussian_spinors(2, L, 47)
        y = s.apply_D(x, precision=1)
        ref = op.apply(t(x)).numpy()
        for k in range(2):
            assert_close(y[k], ref[k], TOL32)
        s.close()
    finally:
        P.pin_variant("D fp32", -1)


@pytest.mark.parametrize("prec", [0, 1])
def test_clover_and_inverse_apply(prec):
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, prec)
    op = oracle_op(L, eps, seed, m0, csw)
    x = syn.gaussian_spinors(1, L, 41)
    tol = TOL64 if prec == 0 else TOL32
    assert_close(s.apply_clover(x, False, prec), op.site(t(x)).numpy(), tol)
    assert_close(s.apply_clover(x, True, prec), op.site(t(x), inverse=True).numpy(), tol)


@pytest.mark.parametrize("cfg", [SMALL, MID])
@pytest.mark.parametrize("prec", [0, 1])
def test_block_solve(cfg, prec):
    L = cfg[0]
    s = make(cfg, prec)
    sm = smoother(cfg)
    r = syn.gaussian_spinors(1, L, 42)
    for c in (0, 1):
        got = s.block_solve(r, c, prec)
        ref = sm.block_solve(t(r[0]), c, 4).numpy()
        tol = 1e-12 if prec == 0 else 5 * TOL32
        assert_close(got[0], ref, tol)
        # zero on the blocks of the other colour
        other = sm.mask[1 - c, None].numpy().real.astype(bool)[:, 0, 0]
        assert np.abs(got[0][other]).max() == 0.0


@pytest.mark.parametrize("cfg", [SMALL, MID])
@pytest.mark.parametrize("prec", [0, 1])
def test_sap(cfg, prec):
    L = cfg[0]
    s = make(cfg, prec)
    sm = smoother(cfg)
    r = syn.gaussian_spinors(1, L, 43)
    got = s.sap(r, prec)
    ref = sm.apply(t(r[0]), 4, 4).numpy()
    tol = 1e-12 if prec == 0 else 2e-5
    assert_close(got[0], ref, tol)


@pytest.mark.parametrize("variant", [0, 1])
def test_sap_variants_fp32(variant):
    """Both measured variants of the FP32 Schwarz sweep on 4^4 blocks (links
    and clover blocks staged in shared memory, or read from global memory)
    match the oracle's SAP."""
    P = _P()
    P.pin_variant("SAP fp32", variant)
    try:
        s = make(MID, 1)
        r = syn.gaussian_spinors(1, MID[0], 48)
        got = s.sap(r, 1)
        ref = smoother(MID).apply(t(r[0]), 4, 4).numpy()
        assert_close(got[0], ref, 2e-5)
        s.close()
    finally:
        P.pin_variant("SAP fp32", -1)


# FP32 Gram-Schmidt: each coefficient is a sum of 6 |aggregate| products,
# each vector update i of them; for well-conditioned (Gaussian) vectors the
# result carries a few FP32 roundings, 1e-5 with room to spare
@pytest.mark.parametrize("cfg", [SMALL, MID])
@pytest.mark.parametrize("prec,ortho32,tol", [(0, 0, 1e-13), (1, 0, 1e-13), (1, 1, 1e-5)])
def test_orthonormalise(cfg, prec, ortho32, tol):
    """FP64 orthonormalisation (the default, whatever the inner precision)
    and the FP32 one of ortho_fp32 give the oracle's vectors within their
    precision."""
    L, b, eps, m0, csw, n_v, seed = cfg
    s = make(cfg, prec, ortho_fp32=ortho32)
    lam = syn.gaussian_spinors(n_v, L, 44)
    s.set_test_vectors(lam)
    s.orthonormalize()
    op = oracle_op(L, eps, seed, m0, csw)
    ref = orthonormalise(t(lam), Aggregation(op.geom, b)).numpy()
    assert_close(s.get_test_vectors(), ref, tol)


@pytest.mark.parametrize("cfg", [SMALL, MID])
@pytest.mark.parametrize("prec", [0, 1])
def test_restrict_prolong(cfg, prec):
    L, b, eps, m0, csw, n_v, seed = cfg
    s = make(cfg, prec)
    op = oracle_op(L, eps, seed, m0, csw)
    agg = Aggregation(op.geom, b)
    lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 45)), agg)
    s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
    x = syn.gaussian_spinors(2, L, 46)
    tol = TOL64 if prec == 0 else TOL32
    bc = s.restrict(x, prec)
    ref = restrict(lam, agg, t(x)).numpy()
    assert_close(bc, ref, tol)
    y = np.ascontiguousarray(ref)
    got = s.prolong(y, prec)
    assert_close(got, prolong(lam, agg, t(y)).numpy(), tol)


@pytest.mark.parametrize("nrhs", [12, 17])
def test_restrict_prolong_batched_tensor_cores(nrhs):
    """A batch of right-hand sides goes through R and P as complex matrix
    products on the tensor cores (TF32 operands split into hi + lo parts):
    FP32 parity with the oracle element by element, for a full group of
    right-hand sides and a ragged second group, and agreement with the
    one-at-a-time kernels."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    try:
        op = oracle_op(L, eps, seed, m0, csw)
        agg = Aggregation(op.geom, b)
        lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 145)), agg)
        s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
        x = syn.gaussian_spinors(nrhs, L, 146)
        bc = s.restrict(x, 1)
        ref = restrict(lam, agg, t(x)).numpy()
        assert_close(bc, ref, TOL32, "R")
        one = s.restrict(np.ascontiguousarray(x[:1]), 1)
        assert_close(bc[:1], one, TOL32, "R batch vs single")
        y = np.ascontiguousarray(ref)
        got = s.prolong(y, 1)
        assert_close(got, prolong(lam, agg, t(y)).numpy(), TOL32, "P")
        one = s.prolong(np.ascontiguousarray(y[-1:]), 1)
        assert_close(got[-1:], one, TOL32, "P batch vs single")
    finally:
        s.close()


@pytest.fixture(scope="module")
def coarse_pair():
    """GPU handles (FP64 and FP32) sharing orthonormal test vectors with the oracle."""
    out = {}
    L, b, eps, m0, csw, n_v, seed = MID
    op = oracle_op(L, eps, seed, m0, csw)
    agg = Aggregation(op.geom, b)
    lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 47)), agg)
    Dc = coarse_operator(op, lam, agg)
    cop = CoarseOperator(Dc, agg.coarse)
    for prec in (0, 1):
        s = make(MID, prec)
        s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
        s.build_coarse()
        out[prec] = s
    return out, lam, agg, cop


# An entry of D_c sums 6 |X| = 1536 products of test-vector components in
# the working precision; relative to the largest entry its rounding error is
# about sqrt(1536) 2^-24 |largest term| = 2.4e-6 in FP32 (6e-15 in FP64),
# so the element-wise bound of the assembled operator is 1e-5 (1e-12).
ETOL_DC = {0: 1e-12, 1: 1e-5}
# An output component of the coarse stencil sums 9 x 2 n_v products; the
# element-wise bound relative to the largest component is 5e-6 in FP32
# (sqrt(108) 2^-24 = 6e-7 of the largest term at n_v 6, terms up to a few
# times the largest output), 1e-13 in FP64.
ETOL_STENCIL = {0: 1e-13, 1: 5e-6}


@pytest.mark.parametrize("prec", [0, 1])
def test_coarse_operator(coarse_pair, prec):
    handles, lam, agg, cop = coarse_pair
    got = handles[prec].get_coarse_op()
    tol = 1e-12 if prec == 0 else TOL32
    assert_close(got, cop.Dc.numpy(), tol, etol=ETOL_DC[prec])
    for X in (0, 5, agg.NX - 1):
        assert rel(got[X], cop.Dc[X].numpy()) < 10 * tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
def test_coarse_stencil(coarse_pair, prec, variant):
    """All nine blocks (0), or the self and forward blocks with the backward
    ones from G5-hermiticity (1), on an assembled D_c whose coarse extents
    include 2 (x + mu = x - mu)."""
    P = _P()
    handles, lam, agg, cop = coarse_pair
    rng = np.random.default_rng(48)
    x = rng.standard_normal((2, agg.NX, 2 * lam.shape[0])) + 1j * rng.standard_normal((2, agg.NX, 2 * lam.shape[0]))
    P.pin_variant("coarse stencil", variant)
    try:
        got = handles[prec].apply_coarse(x, prec)
    finally:
        P.pin_variant("coarse stencil", -1)
    ref = cop.apply(t(x)).numpy()
    assert_close(got, ref, (TOL64 if prec == 0 else TOL32), etol=ETOL_STENCIL[prec])


@pytest.mark.parametrize("prec", [0, 1])
def test_coarse_stencil_given_operator_uses_all_blocks(prec):
    """A stencil given through ddamg_set_coarse_op (here a random one, not
    G5-hermitian) is applied with all nine blocks even where the G5 variant
    is pinned."""
    P = _P()
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, prec)
    try:
        n2 = 2 * n_v
        Dc = syn.coarse_stencil(s.NX, n2, 9, 1.0, 0.21)
        s.set_coarse_op(Dc)
        geom = Aggregation(oracle_op(L, eps, seed, m0, csw).geom, b).coarse
        cop = CoarseOperator(torch.from_numpy(Dc), geom)
        rng = np.random.default_rng(52)
        x = rng.standard_normal((1, s.NX, n2)) + 1j * rng.standard_normal((1, s.NX, n2))
        P.pin_variant("coarse stencil", 1)
        try:
            got = s.apply_coarse(x, prec)
        finally:
            P.pin_variant("coarse stencil", -1)
        assert_close(got, cop.apply(t(x)).numpy(), (TOL64 if prec == 0 else TOL32), etol=ETOL_STENCIL[prec])
    finally:
        s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_coarse_even_odd_gmres(coarse_pair, prec):
    handles, lam, agg, cop = coarse_pair
    rng = np.random.default_rng(49)
    b = rng.standard_normal((2, agg.NX, 2 * lam.shape[0])) + 1j * rng.standard_normal((2, agg.NX, 2 * lam.shape[0]))
    # loose tolerance of the method: same iteration count as the oracle's
    x, its = handles[prec].coarse_solve(b, 5e-2, prec)
    for k in range(2):
        xr, ir = cop.solve(t(b[k]), 5e-2, 30, 300)
        assert abs(int(its[k]) - ir) <= (0 if prec == 0 else 1)
        if prec == 0:
            assert_close(x[k], xr.numpy(), 1e-11)
    # tight tolerance: the dense solve
    tol = 1e-12 if prec == 0 else 1e-5
    x, its = handles[prec].coarse_solve(b, tol, prec)
    Dd = cop.dense().numpy()
    for k in range(2):
        xd = np.linalg.solve(Dd, b[k].reshape(-1)).reshape(b[k].shape)
        assert_close(x[k], xd, (1e-10 if prec == 0 else 1e-4))


def test_preconditioner_M_fp64():
    L, b, eps, m0, csw, n_v, seed = SMALL
    s = make(SMALL, 0)
    mg = TwoLevelMG(t(syn.gauge_field(L, eps, seed)),
                    Params(L, b, b, n_v, m0, csw, setup_iters=3))
    lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 50)), mg.agg)
    mg.set_test_vectors(lam, orthonormalised=True)
    s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
    s.build_coarse()
    r = syn.gaussian_spinors(1, L, 51)
    got = s.apply_M(r, 0)
    ref = mg.apply_M(t(r[0])).numpy()
    assert_close(got[0], ref, 1e-11)


def test_setup_fp64_matches_oracle():
    """Same initial vectors -> the FP64 setup reproduces the oracle's test
    vectors and coarse operator up to rounding."""
    L, b, eps, m0, csw, n_v, seed = SMALL
    s = make(SMALL, 0, setup_iters=3)
    lam0 = syn.gaussian_spinors(n_v, L, 1)
    s.run_setup(lam0)
    mg = TwoLevelMG(t(syn.gauge_field(L, eps, seed)), Params(L, b, b, n_v, m0, csw, setup_iters=3))
    mg.setup(t(lam0))
    assert_close(s.get_test_vectors(), mg.lam.numpy(), 1e-9)
    assert_close(s.get_coarse_op(), mg.cop.Dc.numpy(), 1e-9)


def test_solve_small_fp64_matches_dense():
    L, b, eps, m0, csw, n_v, seed = SMALL
    s = make(SMALL, 0, setup_iters=3)
    s.run_setup(syn.gaussian_spinors(n_v, L, 1))
    op = oracle_op(L, eps, seed, m0, csw)
    D = op.dense().numpy()
    rhs = syn.gaussian_spinors(2, L, 2)
    x, info = s.solve(rhs, 1e-10)
    cond = np.linalg.cond(D)
    for k in range(2):
        res = rel(op.apply(t(x[k])).numpy(), rhs[k])
        assert res <= 1e-10 and info[k]["converged"] == 1
        xd = np.linalg.solve(D, rhs[k].reshape(-1)).reshape(rhs[k].shape)
        assert rel(x[k], xd) <= cond * 1e-10


def test_solve_full_workload_point_sources():
    """16^4, FP32 smoother / coarse solve, FP64 outer FGMRES: the 12 point
    sources reach a true residual <= 1e-10 checked by the oracle's D."""
    L, b, eps, m0, csw, n_v, seed = FULL
    s = make(FULL, 1)
    s.run_setup()
    op = oracle_op(L, eps, seed, m0, csw)
    rhs = syn.point_sources(L)
    x, info = s.solve(np.ascontiguousarray(rhs), 1e-10)
    for k in range(12):
        res = rel(op.apply(t(x[k])).numpy(), rhs[k])
        assert res <= 1e-10, (k, res, info[k])


@pytest.mark.parametrize("refine", [0.0, 1e-3, 1e-5])
def test_solve_fp32_refinement_modes(refine):
    """FP32 inner solver: with outer_refine > 0 the FGMRES operator products
    are FP32 and cycles restart from the FP64 true residual; with 0 they are
    FP64.  Every mode reaches a true residual <= 1e-10 (oracle's D)."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1, outer_refine=refine)
    s.run_setup()
    op = oracle_op(L, eps, seed, m0, csw)
    rhs = syn.gaussian_spinors(3, L, 31)
    x, info = s.solve(rhs, 1e-10)
    for k in range(3):
        res = rel(op.apply(t(x[k])).numpy(), rhs[k])
        assert res <= 1e-10, (k, res, info[k])
        assert info[k]["converged"] == 1 and info[k]["true_residual"] <= 1e-10
        if refine >= 1e-3:
            assert info[k]["restarts"] >= 2, info[k]
    s.close()


@pytest.mark.parametrize("prec,refine", [(1, 1e-5), (1, 0.0), (0, 0.0)])
def test_solve_batched_matches_one_at_a_time(prec, refine):
    """The lockstep batch gives every right-hand side its own FGMRES: each
    solution reaches the tolerance by the oracle's D, and equals the
    one-at-a-time solution within what the two stopping points allow."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, prec, outer_refine=refine)
    s.run_setup()
    op = oracle_op(L, eps, seed, m0, csw)
    rhs = np.concatenate([syn.gaussian_spinors(3, L, 41), syn.point_sources(L)[:2]])
    xb, ib = s.solve_batched(np.ascontiguousarray(rhs), 1e-10)
    xs, is_ = s.solve(np.ascontiguousarray(rhs), 1e-10)
    for k in range(rhs.shape[0]):
        res = rel(op.apply(t(xb[k])).numpy(), rhs[k])
        assert res <= 1e-10 and ib[k]["converged"] == 1, (k, res, ib[k])
        assert abs(ib[k]["outer_iters"] - is_[k]["outer_iters"]) <= 3, (ib[k], is_[k])
        assert_close(xb[k], xs[k], 1e-6)
    s.close()


def test_update_mass_keeps_vectors_and_rebuilds_operators():
    """ddamg_update_mass (the paper's second mass on one setup): D equals the
    oracle's D at the new (m0, csw), the test vectors are unchanged, D_c is
    P^H D' P with them, and a solve at the new mass reaches 1e-10."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 0)
    s.run_setup()
    lam_before = s.get_test_vectors()
    m1, c1 = m0 + 0.1, csw + 0.2
    s.update_mass(m1, c1)
    op1 = oracle_op(L, eps, seed, m1, c1)
    x = syn.gaussian_spinors(1, L, 60)
    assert_close(s.apply_D(x)[0], op1.apply(t(x[0])).numpy(), TOL64)
    lam = s.get_test_vectors()
    assert np.array_equal(lam, lam_before)
    agg = Aggregation(op1.geom, b)
    Dc = coarse_operator(op1, t(lam), agg)
    assert_close(s.get_coarse_op(), Dc.numpy(), 1e-12)
    xs, info = s.solve(x, 1e-10)
    assert rel(op1.apply(t(xs[0])).numpy(), x[0]) <= 1e-10
    s.close()


def test_saved_setup_loads_into_a_new_handle(tmp_path):
    """A setup written with save_setup and loaded into a fresh handle on the
    same links gives the same D_c and the same solve (the setup is a pure
    function of the test vectors); loaded at another mass it serves that mass
    as the mass update does; a setup of another geometry is refused."""
    P = _P()
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    s.run_setup()
    rhs = syn.gaussian_spinors(1, L, 68)
    x0, info0 = s.solve(rhs, 1e-10)
    Dc0 = s.get_coarse_op()
    path = str(tmp_path / "setup.npz")
    s.save_setup(path)
    s.close()
    s2 = make(MID, 1)
    assert s2.load_setup(path) == (m0, csw)
    assert np.array_equal(s2.get_coarse_op(), Dc0)
    x1, info1 = s2.solve(rhs, 1e-10)
    assert info1[0]["outer_iters"] == info0[0]["outer_iters"]
    assert np.array_equal(x1, x0)
    s2.close()
    s3 = make(MID, 1)
    s3.update_mass(m0 + 0.1, csw)
    s3.load_setup(path)
    op1 = oracle_op(L, eps, seed, m0 + 0.1, csw)
    x2, _ = s3.solve(rhs, 1e-10)
    assert rel(op1.apply(t(x2[0])).numpy(), rhs[0]) <= 1e-10
    s3.close()
    other = make(SMALL, 0)
    with pytest.raises(P.DDAMGError):
        other.load_setup(path)
    other.close()


def test_set_gauge_replaces_links_and_needs_a_new_setup():
    """ddamg_set_gauge: D follows the new links, a solve before the new setup
    is refused, one after it reaches 1e-10, and non-SU(3) links are rejected."""
    P = _P()
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    s.run_setup()
    U2 = syn.gauge_field(L, 0.2, seed + 7)
    s.set_gauge(U2)
    op2 = WilsonClover(t(U2), L, m0, csw)
    x = syn.gaussian_spinors(1, L, 61)
    assert_close(s.apply_D(x, P.FP64)[0], op2.apply(t(x[0])).numpy(), TOL64)
    with pytest.raises(P.DDAMGError) as e:
        s.solve(x, 1e-10)
    assert e.value.status == 7
    s.run_setup()
    xs, info = s.solve(x, 1e-10)
    assert rel(op2.apply(t(xs[0])).numpy(), x[0]) <= 1e-10
    bad = U2.copy()
    bad[0, 0] *= 1.5
    with pytest.raises(P.DDAMGError) as e:
        s.set_gauge(bad)
    assert e.value.status == 1
    s.close()


def test_half_vectors_restrict_prolong_and_coarse_operator():
    """FP16 storage of the test vectors (half_vectors): R, P and D_c against
    the oracle's FP64 vectors within the 2e-2 of half-precision storage."""
    L, b, eps, m0, csw, n_v, seed = MID
    op = oracle_op(L, eps, seed, m0, csw)
    agg = Aggregation(op.geom, b)
    lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 62)), agg)
    s = make(MID, 1, half_vectors=1)
    s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
    s.build_coarse()
    x = syn.gaussian_spinors(2, L, 63)
    got = s.restrict(x, 1)
    ref = restrict(lam, agg, t(x)).numpy()
    assert_close(got, ref, 2e-2)
    xc = np.ascontiguousarray(ref)
    got = s.prolong(xc, 1)
    assert_close(got, prolong(lam, agg, t(xc)).numpy(), 2e-2)
    assert_close(s.get_coarse_op(), coarse_operator(op, lam, agg).numpy(), 2e-2)
    s.close()


def test_half_vectors_solve_reaches_tolerance():
    """With FP16 test vectors the FP64 outer FGMRES still reaches 1e-10."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1, half_vectors=1)
    s.run_setup()
    op = oracle_op(L, eps, seed, m0, csw)
    rhs = syn.gaussian_spinors(2, L, 64)
    x, info = s.solve(rhs, 1e-10)
    for k in range(2):
        assert rel(op.apply(t(x[k])).numpy(), rhs[k]) <= 1e-10, info[k]
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_odd_number_of_test_vectors(prec):
    """n_v = 5 (the paper's even-n restriction is a tiling artefact): D_c and
    the coarse stencil match the oracle, and a solve reaches 1e-10."""
    L, b, eps, m0, csw, _, seed = MID
    n_v = 5
    cfg = (L, b, eps, m0, csw, n_v, seed)
    op = oracle_op(L, eps, seed, m0, csw)
    agg = Aggregation(op.geom, b)
    lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 65)), agg)
    s = make(cfg, prec)
    s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
    s.build_coarse()
    Dc = coarse_operator(op, lam, agg)
    tol = 1e-12 if prec == 0 else TOL32
    assert_close(s.get_coarse_op(), Dc.numpy(), tol, etol=ETOL_DC[prec])
    rng = np.random.default_rng(66)
    x = rng.standard_normal((1, agg.NX, 2 * n_v)) + 1j * rng.standard_normal((1, agg.NX, 2 * n_v))
    got = s.apply_coarse(x, prec)
    ref = CoarseOperator(Dc, agg.coarse).apply(t(x)).numpy()
    assert_close(got, ref, (TOL64 if prec == 0 else TOL32), etol=ETOL_STENCIL[prec])
    s.run_setup()
    rhs = syn.gaussian_spinors(1, L, 67)
    xs, info = s.solve(rhs, 1e-10)
    assert rel(op.apply(t(xs[0])).numpy(), rhs[0]) <= 1e-10
    s.close()


def test_zero_and_empty_right_hand_sides():
    """b = 0 gives x = 0 at once; a call with no right-hand side does nothing."""
    L = MID[0]
    s = make(MID, 1)
    s.run_setup()
    x, info = s.solve(np.zeros((1,) + syn.gaussian_spinors(1, L, 1).shape[1:], np.complex128), 1e-10)
    assert np.all(x == 0) and info[0]["converged"] == 1 and info[0]["outer_iters"] == 0
    empty = np.zeros((0, int(np.prod(L)), 4, 3), np.complex128)
    xe, ie = s.solve(empty, 1e-10)
    assert xe.shape == empty.shape and ie == []
    s.close()


def test_residual_history_and_flop_model():
    """The history of the last solve starts at (0, 1), its cost grows, it has
    one entry per outer iteration plus one per restart, and it ends at the
    FP64 true residual; the model's setup and solve flops are positive."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    s.reset_stats()
    s.run_setup()
    rhs = syn.gaussian_spinors(1, L, 52)
    x, info = s.solve(rhs, 1e-10)
    f, r = s.history()
    assert f[0] == 0.0 and r[0] == 1.0
    assert np.all(np.diff(f) >= 0.0) and f[-1] > 0.0
    assert len(f) == 1 + info[0]["outer_iters"] + info[0]["restarts"]
    assert r[-1] == pytest.approx(info[0]["true_residual"], rel=1e-12)
    st = s.stats()
    assert st["setup_flops"] > 0.0 and st["solve_flops"] > 0.0
    # the solve's cost in the history equals the counter (one right-hand side)
    assert f[-1] * 1e6 * np.prod(L) == pytest.approx(st["solve_flops"], rel=1e-9)
    s.close()


def test_solve_batched_edge_cases():
    """A zero right-hand side in the batch gives x = 0; a batch of one equals
    the single solve; more than 64 is rejected before any device work."""
    P = _P()
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    s.run_setup()
    rhs = syn.gaussian_spinors(2, L, 43)
    rhs[1] = 0
    x, info = s.solve_batched(rhs, 1e-10)
    assert np.all(x[1] == 0) and info[1]["converged"] == 1
    x1, _ = s.solve_batched(np.ascontiguousarray(rhs[:1]), 1e-10)
    xs, _ = s.solve(np.ascontiguousarray(rhs[:1]), 1e-10)
    assert_close(x1[0], xs[0], 1e-12)
    with pytest.raises(P.DDAMGError) as e:
        s.solve_batched(np.zeros((65,) + rhs.shape[1:], np.complex128), 1e-10)
    assert e.value.status == 1
    s.close()


def test_random_vectors_match_philox_definition():
    P = _P()
    s = make(SMALL, 0)
    got = s.random_vectors(1234, 2)
    V = got.shape[1]
    x = np.arange(V, dtype=np.uint64)
    for i in range(2):
        ref = np.empty((V, 24))
        for blk in range(6):
            w = syn.Philox4x32.block((x, np.full(V, i), np.full(V, blk), np.zeros(V)), (1234, 0))
            for pr in range(2):
                u1 = (w[2 * pr].astype(np.float64) + 1.0) * 2.0 ** -32
                u2 = w[2 * pr + 1].astype(np.float64) * 2.0 ** -32
                r = np.sqrt(-2.0 * np.log(u1))
                ref[:, blk * 4 + pr * 2] = r * np.cos(2 * np.pi * u2)
                ref[:, blk * 4 + pr * 2 + 1] = r * np.sin(2 * np.pi * u2)
        assert np.abs(got[i].view(np.float64).reshape(V, 24) - ref).max() < 1e-12


def test_status_codes_on_device():
    P = _P()
    L = SMALL[0]
    s = make(SMALL, 0, setup_iters=1, max_outer_iter=2)
    with pytest.raises(P.DDAMGError) as e:
        s.solve(syn.gaussian_spinors(1, L, 3))
    assert e.value.status == 7          # no setup yet
    s.run_setup(syn.gaussian_spinors(8, L, 1))
    x, info = s.solve(syn.gaussian_spinors(1, L, 3), 1e-12, allow_noconv=True)
    assert info[0]["converged"] == 0 and info[0]["outer_iters"] == 2
    bad = syn.gaussian_spinors(1, L, 3)
    bad[0, 5, 1, 1] = np.nan
    with pytest.raises(P.DDAMGError) as e:
        s.solve(bad)
    assert e.value.status == 5
    with pytest.raises(P.DDAMGError) as e:
        make(SMALL, 0, hbm_budget=1 << 16)
    assert e.value.status == 2
    U = syn.gauge_field(L, 0.3, 0).copy()
    U[3, 2] *= 1.01
    p = P.default_params(L=L, sap_block=(2, 2, 2, 2), n_v=8)
    with pytest.raises(P.DDAMGError) as e:
        P.DDAMG(p, U)
    assert e.value.status == 1


def test_device_pointer_path_and_determinism():
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    s.run_setup()
    rhs = syn.gaussian_spinors(1, L, 60)
    xh, _ = s.solve(rhs, 1e-10)
    xd, _ = s.solve(torch.from_numpy(rhs).cuda(), 1e-10)
    assert np.array_equal(xh, xd.cpu().numpy())
