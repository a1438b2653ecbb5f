"""The coarse even-odd GMRES (Sec. 2) in every launch configuration the
library chooses, against the oracle's coarse solver on the same operator.

The plan (right-hand sides in lockstep, sites per CTA, Krylov slices in
shared or global memory, resident D_c blocks, blocks streamed through the
shared-memory ring) depends on the size of the
coarse lattice, n_v, the restart length and the batch.  The workloads of the
solver reach all of them: a few dozen coarse sites keep one even site per CTA
with its blocks resident, a 4^3 x 8 coarse lattice needs two sites per CTA, an
8^3 x 16 one (the 32^3 x 64 workload has 8^3 x 16 aggregates) about thirty,
and there wide batches spill the Krylov slices to global scratch.  The
operator is a seeded synthetic 9-point stencil with 2n x 2n blocks
(synthetic.coarse_stencil), given to both sides, so that large coarse
lattices are checked without assembling D_c from fine test vectors.

Checks per right-hand side: at the method's tolerance 5e-2 the iteration
counts equal the oracle's (FP64) or differ by at most one (FP32), and the
FP64 solution equals the oracle's to 1e-11; after a fixed number of
iterations (max_iter 6, a tolerance never reached) both sides return the
same Krylov iterate, compared element by element.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.coarse import CoarseOperator
from oracle.lattice import Geometry
from tests.gpu_common import assert_close

pytestmark = pytest.mark.gpu

# the synthetic operator: about 11 iterations to 5e-2 and 100 to 1e-10
DIAG, HOP = 1.0, 0.21
FIXED_ITERS = 6
# FP32 Krylov iterate after FIXED_ITERS iterations: each iteration is one
# Schur-complement apply (three block products, each within 1e-6 relative)
# and one Gram-Schmidt step; the iterate's error grows with the condition of
# the small Hessenberg least-squares problem, bounded here by 1e-4
TOL_FIXED32 = 1e-4

# (fine lattice, blocks, n_v, precision, nrhs, restart, expected plan features)
CASES = [
    ((8, 8, 8, 16), (4, 4, 4, 4), 6, 1, 2, 30, dict(resident_blocks=1, sites_per_cta=1)),
    ((8, 8, 8, 16), (2, 2, 2, 2), 4, 0, 1, 30, dict(sites_per_cta=2, krylov_in_shared=1)),
    ((8, 8, 8, 16), (2, 2, 2, 2), 4, 1, 12, 8, dict(rhs_per_pass=12, sites_per_cta=2)),
    ((8, 8, 8, 16), (2, 2, 2, 2), 4, 1, 5, 30, dict(rhs_per_pass=4)),
    ((16, 16, 16, 32), (2, 2, 2, 2), 4, 1, 1, 30, dict(rhs_per_pass=1, krylov_in_shared=1)),
    ((16, 16, 16, 32), (2, 2, 2, 2), 4, 1, 8, 30, dict(rhs_per_pass=8, krylov_in_shared=0)),
    ((16, 16, 16, 32), (2, 2, 2, 2), 4, 0, 4, 30, dict(rhs_per_pass=4, krylov_in_shared=0)),
    ((16, 16, 16, 32), (2, 2, 2, 2), 4, 0, 1, 8, dict(rhs_per_pass=1, krylov_in_shared=1)),
    ((16, 16, 16, 32), (2, 2, 2, 2), 8, 1, 2, 30, dict(rhs_per_pass=2)),
    ((16, 16, 16, 32), (2, 2, 2, 2), 4, 1, 12, 30, dict(rhs_per_pass=12, krylov_in_shared=0)),
    # n_v 16: 32 x 32 blocks, streamed through the shared-memory block ring
    ((8, 8, 8, 16), (2, 2, 2, 2), 16, 1, 1, 30, dict(rhs_per_pass=1, block_ring=1, krylov_in_shared=1)),
    ((8, 8, 8, 16), (2, 2, 2, 2), 16, 1, 4, 30, dict(rhs_per_pass=4, block_ring=1, sites_per_cta=2)),
    ((8, 8, 8, 16), (2, 2, 2, 2), 16, 1, 8, 30, dict(rhs_per_pass=8, block_ring=1, krylov_in_shared=0)),
    ((8, 8, 8, 16), (2, 2, 2, 2), 16, 1, 12, 30, dict(rhs_per_pass=12, block_ring=1)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_1811_00355_gb300 as P
    P.load()
    assert torch.cuda.is_available()


def _handle(L, b, n_v, prec, restart, max_iter):
    import paper_1811_00355_gb300 as P
    p = P.default_params(L=L, sap_block=b, n_v=n_v, precision=prec, coarse_restart=restart,
                         coarse_max_iter=max_iter)
    return P.DDAMG(p, syn.unit_gauge(L))


@pytest.mark.parametrize("L,b,n_v,prec,nrhs,restart,want", CASES)
def test_coarse_gmres_plan_matches_oracle(L, b, n_v, prec, nrhs, restart, want):
    cL = tuple(L[mu] // b[mu] for mu in range(4))
    geom = Geometry(cL)
    n2 = 2 * n_v
    Dc = syn.coarse_stencil(geom.V, n2, 5, DIAG, HOP)
    cop = CoarseOperator(torch.from_numpy(Dc), geom)
    gen = np.random.default_rng(80 + nrhs)
    bc = gen.standard_normal((nrhs, geom.V, n2)) + 1j * gen.standard_normal((nrhs, geom.V, n2))

    # the method's tolerance
    s = _handle(L, b, n_v, prec, restart, 300)
    try:
        s.set_coarse_op(Dc)
        plan = s.coarse_plan(nrhs)
        for k, v in want.items():
            assert plan[k] == v, (k, plan)
        x, its = s.coarse_solve(bc, 5e-2, prec)
        for r in range(nrhs):
            xr, ir = cop.solve(torch.from_numpy(bc[r]), 5e-2, restart, 300)
            assert abs(int(its[r]) - ir) <= (0 if prec == 0 else 1), (r, its, ir, plan)
            if prec == 0:
                assert_close(x[r], xr.numpy(), 1e-11, f"rhs {r}")
    finally:
        s.close()

    # a fixed number of iterations: the same Krylov iterate
    s = _handle(L, b, n_v, prec, restart, FIXED_ITERS)
    try:
        s.set_coarse_op(Dc)
        x, its = s.coarse_solve(bc, 1e-30, prec)
        assert np.all(its == FIXED_ITERS), its
        for r in range(nrhs):
            xr, ir = cop.solve(torch.from_numpy(bc[r]), 1e-30, restart, FIXED_ITERS)
            assert ir == FIXED_ITERS
            assert_close(x[r], xr.numpy(), 1e-11 if prec == 0 else TOL_FIXED32, f"rhs {r}")
    finally:
        s.close()


def test_plans_cover_every_kind():
    """The cases above reach the resident, the several-sites-per-CTA and the
    global-scratch configurations, and every lockstep width."""
    seen = set()
    widths = set()
    rings = set()
    for L, b, n_v, prec, nrhs, restart, _ in CASES:
        s = _handle(L, b, n_v, prec, restart, 300)
        try:
            p = s.coarse_plan(nrhs)
        finally:
            s.close()
        seen.add(("resident" if p["resident_blocks"] else "per1" if p["sites_per_cta"] == 1 else "per>1",
                  "smem" if p["krylov_in_shared"] else "global"))
        widths.add(p["rhs_per_pass"])
        rings.add((p["block_ring"], p["krylov_in_shared"]))
    assert ("resident", "smem") in seen and ("per>1", "smem") in seen
    assert (1, 1) in rings and (1, 0) in rings and (0, 0) in rings
    assert any(k[1] == "global" for k in seen)
    assert widths == {1, 2, 4, 8, 12}


def test_bounded_waits_time_out_and_the_handle_recovers():
    """With the wait limit at zero polls, the SAP kernel's wait for its staged
    block and the coarse grid barrier give up at once: the calls return
    DDAMG_ETIMEOUT (no fault, no hang, every wait bounded); with the default
    limits restored the same handle computes what the oracle computes."""
    import paper_1811_00355_gb300 as P
    from tests.gpu_common import MID, make, smoother
    L = MID[0]
    s = make(MID, P.FP32)
    try:
        r = syn.gaussian_spinors(1, L, 90)
        s.set_coarse_op(syn.coarse_stencil(s.NX, 2 * s.n_v, 6, DIAG, HOP))
        gen = np.random.default_rng(91)
        bc = gen.standard_normal((1, s.NX, 2 * s.n_v)) + 1j * gen.standard_normal((1, s.NX, 2 * s.n_v))
        s.set_wait_limit(0)
        with pytest.raises(P.DDAMGError) as e:
            s.sap(r, P.FP32)
        assert e.value.status == 6
        with pytest.raises(P.DDAMGError) as e:
            s.coarse_solve(bc, 5e-2, P.FP32)
        assert e.value.status == 6
        s.set_wait_limit(-1)
        got = s.sap(r, P.FP32)
        ref = smoother(MID).apply(torch.from_numpy(r[0]), 4, 4).numpy()
        assert_close(got[0], ref, 2e-5)
        x, its = s.coarse_solve(bc, 5e-2, P.FP32)
        assert its[0] > 0 and np.all(np.isfinite(x))
    finally:
        s.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_ring_block_products_on_cuda_and_tensor_cores(variant):
    """Eight right-hand sides through the block ring: the block products on
    the CUDA cores (0) and on the tensor cores (1, 3xTF32) both return the
    oracle's Krylov iterate after a fixed number of iterations."""
    import paper_1811_00355_gb300 as P
    L, b, n_v, nrhs = (8, 8, 8, 16), (2, 2, 2, 2), 16, 8
    cL = tuple(L[mu] // b[mu] for mu in range(4))
    geom = Geometry(cL)
    n2 = 2 * n_v
    Dc = syn.coarse_stencil(geom.V, n2, 7, DIAG, HOP)
    cop = CoarseOperator(torch.from_numpy(Dc), geom)
    gen = np.random.default_rng(95)
    bc = gen.standard_normal((nrhs, geom.V, n2)) + 1j * gen.standard_normal((nrhs, geom.V, n2))
    P.pin_variant("coarse product", variant)
    s = _handle(L, b, n_v, P.FP32, 30, FIXED_ITERS)
    try:
        s.set_coarse_op(Dc)
        plan = s.coarse_plan(nrhs)
        assert plan["block_ring"] == 1 and plan["rhs_per_pass"] == 8, plan
        x, its = s.coarse_solve(bc, 1e-30, P.FP32)
        assert np.all(its == FIXED_ITERS), its
        for r in range(nrhs):
            xr, _ = cop.solve(torch.from_numpy(bc[r]), 1e-30, 30, FIXED_ITERS)
            assert_close(x[r], xr.numpy(), TOL_FIXED32, f"variant {variant} rhs {r}")
    finally:
        s.close()
        P.pin_variant("coarse product", -1)
