"""Half-precision storage (BF16 and FP16, FP32 arithmetic) against the FP64
oracle, through the C ABI.

Per-apply bound 2e-2 (norm-wise and element-wise): a stored value carries a
relative rounding error of at most 2^-9 (BF16) or 2^-12 (FP16, spinors
scaled by their site norm into [-1, 1]); one D apply combines rounded
links, clover blocks and spinors in a few dozen FP32 terms per component,
which keeps its error within a few times that (measured on a GB300: BF16
2.4e-3 norm-wise, 4.1e-3 element-wise; FP16 3.0e-4 and 4.1e-4).  The
composite steps stay within the same bound: a block solve (about a dozen
dependent applies on the rounded operators) and a SAP application (eight
sweeps, each also rounding x into storage) contract the rounding errors
rather than adding them (measured: BF16 2.9e-3 / 3.9e-3, FP16 3.6e-4 /
5.8e-4).  Whole solves reach the FP64 true residual 1e-10 through the FP64
outer FGMRES.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.coarse import Aggregation, coarse_operator, orthonormalise, prolong, restrict
from tests.gpu_common import FULL, MID, SMALL, assert_close, make, oracle_op, rel, smoother, t

pytestmark = pytest.mark.gpu

TOL_HALF = 2e-2
# composite steps: (BF16, FP16)
TOL_BLOCK = {2: 2e-2, 3: 2e-2}
TOL_SAP = {2: 2e-2, 3: 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1811_00355_gb300 as P
    P.load()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("cfg", [SMALL, MID, FULL])
@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("variant", [0, 1])
def test_half_storage_D(cfg, prec, variant):
    import paper_1811_00355_gb300 as P
    L, b, eps, m0, csw, n_v, seed = cfg
    name = "D bf16" if prec == 2 else "D fp16"
    P.pin_variant(name, variant)
    s = make(cfg, 1)
    try:
        op = oracle_op(L, eps, seed, m0, csw)
        x = syn.gaussian_spinors(2, L, 140)
        y = s.apply_D(x, precision=prec)
        ref = op.apply(t(x)).numpy()
        errs = [assert_close(y[k], ref[k], TOL_HALF, f"prec {prec}") for k in range(2)]
        print(f"half D prec {prec} L {L}: {errs}")
        # a point source and a zero field: exact zeros stay zero, norms handle tiny sites
        z = np.zeros((1,) + x.shape[1:], np.complex128)
        z[0, 3, 1, 2] = 1e-30
        yz = s.apply_D(z, precision=prec)
        rz = op.apply(t(z)).numpy()
        assert_close(yz[0], rz[0], TOL_HALF, "tiny point source")
    finally:
        s.close()
        P.pin_variant(name, -1)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("variant", [0, 1])
def test_half_storage_block_solve_and_sap(prec, variant):
    """Both forms of the half-storage Schwarz sweep: the staged block
    operators widened to FP32 in shared memory (0) or kept in the half type
    (1)."""
    import paper_1811_00355_gb300 as P
    L = MID[0]
    name = "SAP bf16" if prec == 2 else "SAP fp16"
    P.pin_variant(name, variant)
    s = make(MID, prec)
    try:
        sm = smoother(MID)
        r = syn.gaussian_spinors(1, L, 141)
        for c in (0, 1):
            got = s.block_solve(r, c, prec)
            ref = sm.block_solve(t(r[0]), c, 4).numpy()
            e = assert_close(got[0], ref, TOL_BLOCK[prec], f"block colour {c}")
            print(f"half block solve prec {prec} colour {c}: {e}")
            other = sm.mask[1 - c, None].numpy().real.astype(bool)[:, 0, 0]
            assert np.abs(got[0][other]).max() == 0.0
        got = s.sap(r, prec)
        ref = sm.apply(t(r[0]), 4, 4).numpy()
        e = assert_close(got[0], ref, TOL_SAP[prec], "SAP")
        print(f"half SAP prec {prec} variant {variant}: {e}")
    finally:
        s.close()
        P.pin_variant(name, -1)


@pytest.mark.parametrize("prec", [2, 3])
def test_half_test_vectors_restrict_prolong_coarse_operator(prec):
    L, b, eps, m0, csw, n_v, seed = MID
    op = oracle_op(L, eps, seed, m0, csw)
    agg = Aggregation(op.geom, b)
    lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 142)), agg)
    s = make(MID, prec)
    try:
        s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
        s.build_coarse()
        x = syn.gaussian_spinors(2, L, 143)
        got = s.restrict(x, prec)
        ref = restrict(lam, agg, t(x)).numpy()
        assert_close(got, ref, TOL_HALF, "R")
        xc = np.ascontiguousarray(ref)
        got = s.prolong(xc, prec)
        assert_close(got, prolong(lam, agg, t(xc)).numpy(), TOL_HALF, "P")
        assert_close(s.get_coarse_op(), coarse_operator(op, lam, agg).numpy(), TOL_HALF, "D_c")
    finally:
        s.close()


@pytest.mark.parametrize("prec", [2, 3])
def test_half_storage_solves_reach_tolerance(prec):
    """Single and batched solves with the half-storage smoother reach the FP64
    true residual 1e-10 by the oracle's D, and the batch equals the
    one-at-a-time solutions within what the two stopping points allow."""
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, prec)
    try:
        s.run_setup()
        op = oracle_op(L, eps, seed, m0, csw)
        rhs = np.concatenate([syn.gaussian_spinors(2, L, 144), syn.point_sources(L)[:2]])
        xs, info = s.solve(np.ascontiguousarray(rhs), 1e-10)
        xb, ib = s.solve_batched(np.ascontiguousarray(rhs), 1e-10)
        for k in range(rhs.shape[0]):
            for x, i in ((xs[k], info[k]), (xb[k], ib[k])):
                res = rel(op.apply(t(x)).numpy(), rhs[k])
                assert res <= 1e-10 and i["converged"] == 1, (k, res, i)
            assert_close(xb[k], xs[k], 1e-6)
        print(f"half solve prec {prec}: outer iterations {[i['outer_iters'] for i in info]}, "
              f"batched {[i['outer_iters'] for i in ib]}")
    finally:
        s.close()


@pytest.mark.parametrize("prec", [1, 3])
def test_trim_releases_setup_memory_and_keeps_the_solver(prec):
    """After ddamg_trim (the FP64 test vectors and the setup's temporaries
    released) the solves give the same solutions, a mass update still
    rebuilds D_c from the kept inner-precision vectors, calls that read the
    FP64 test vectors report DDAMG_ESTATE, and a new setup allocates them
    again."""
    import paper_1811_00355_gb300 as P
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, prec)
    try:
        s.run_setup()
        rhs = np.ascontiguousarray(syn.point_sources(L)[:2])
        x0, _ = s.solve(rhs, 1e-10)
        s.trim()
        x1, info = s.solve(rhs, 1e-10)
        for k in range(rhs.shape[0]):
            assert info[k]["converged"] == 1
            assert_close(x1[k], x0[k], 1e-12)
        with pytest.raises(P.DDAMGError) as e:
            s.get_test_vectors()
        assert e.value.status == 7
        op = oracle_op(L, eps, seed, m0 + 0.05, csw)
        s.update_mass(m0 + 0.05, csw)
        x2, info = s.solve(rhs, 1e-10)
        for k in range(rhs.shape[0]):
            assert rel(op.apply(t(x2[k])).numpy(), rhs[k]) <= 1e-10 and info[k]["converged"] == 1
        s.update_mass(m0, csw)
        s.run_setup()
        assert s.get_test_vectors().shape[0] == n_v
    finally:
        s.close()
