"""Continuous batching through the C ABI: the resumable lockstep batch
(ddamg_batch_*) admits right-hand sides between FGMRES restart cycles, and
the serving loop (ddamg_server_*) refills freed slots with requests that
arrive while others run and serves two gauge configurations at the same
time on their own streams.  Every result reaches its own tolerance by the
oracle's D and equals the same right-hand side solved alone within what the
two stopping points allow (1e-5)."""
from __future__ import annotations

import time

import numpy as np
import pytest

import synthetic as syn
from tests.gpu_common import MID, assert_close, make, oracle_op, rel, t

pytestmark = pytest.mark.gpu

OTHER = ((8, 8, 8, 8), (4, 4, 4, 4), 0.3, -0.25, 1.0, 8, 5)


def _op(cfg):
    L, b, eps, m0, csw, n_v, seed = cfg
    return oracle_op(L, eps, seed, m0, csw)


def _alone(cfg, rhs, tol):
    s = make(cfg, 1)
    try:
        s.run_setup()
        x, _ = s.solve_batched(np.ascontiguousarray(rhs), tol)
    finally:
        s.close()
    return x


def test_batch_run_admits_between_cycles():
    """Two right-hand sides start; after two restart cycles a third enters a
    free slot; each finishes to its own tolerance and is taken out."""
    L = MID[0]
    s = make(MID, 1)
    try:
        s.run_setup()
        rhs = syn.gaussian_spinors(3, L, 120)
        tols = [1e-10, 1e-8, 1e-10]
        s.batch_begin(4)
        assert [s.batch_slot(k) for k in range(4)] == [0, 0, 0, 0]
        s.batch_admit(0, np.ascontiguousarray(rhs[0]), tols[0])
        s.batch_admit(2, np.ascontiguousarray(rhs[1]), tols[1])
        assert s.batch_cycle() == 2
        s.batch_cycle()
        assert s.batch_slot(1) == 0
        s.batch_admit(1, np.ascontiguousarray(rhs[2]), tols[2])     # mid-batch admission
        assert s.batch_slot(1) == 1
        got = {}
        for _ in range(200):
            running = s.batch_cycle()
            for k, j in ((0, 0), (2, 1), (1, 2)):
                if j not in got and s.batch_slot(k) == 2:
                    got[j] = s.batch_take(k)
            if running == 0 and len(got) == 3:
                break
        assert len(got) == 3
        op = _op(MID)
        for j in range(3):
            x, info = got[j]
            assert info["converged"] == 1
            assert rel(op.apply(t(x)).numpy(), rhs[j]) <= tols[j]
            assert_close(x, _alone(MID, rhs[j:j + 1], tols[j])[0], 1e-5)
    finally:
        s.close()


def _params(cfg):
    import paper_1811_00355_gb300 as P
    L, b, eps, m0, csw, n_v, seed = cfg
    return P.default_params(L=L, sap_block=b, n_v=n_v, m0=m0, csw=csw, precision=P.FP32)


def test_server_admits_mid_batch_and_serves_configs_together():
    """A long request runs; a short one of the same configuration submitted
    after it started joins its batch and finishes first; a request of a
    second configuration runs at the same time on another worker; all
    results equal their solo solves."""
    import paper_1811_00355_gb300 as P
    srv = P.Server(max_batch=8, workers=2)
    try:
        c0 = srv.add_config(_params(MID), syn.gauge_field(MID[0], MID[2], MID[6]))
        c1 = srv.add_config(_params(OTHER), syn.gauge_field(OTHER[0], OTHER[2], OTHER[6]))
        # set both configurations up first (resident afterwards)
        for c, cfg in ((c0, MID), (c1, OTHER)):
            srv.wait(srv.submit(c, syn.gaussian_spinors(1, cfg[0], 7), 1e-6))
        long_rhs = syn.gaussian_spinors(3, MID[0], 121)
        short_rhs = syn.gaussian_spinors(1, MID[0], 122)
        other_rhs = syn.gaussian_spinors(4, OTHER[0], 123)
        t0 = time.perf_counter()
        i_long = srv.submit(c0, long_rhs, 1e-12)
        i_other = srv.submit(c1, other_rhs, 1e-12)
        time.sleep(0.05)
        i_short = srv.submit(c0, short_rhs, 1e-6)
        x_short, inf_short, ri_short = srv.wait(i_short)
        t_short = time.perf_counter() - t0
        x_long, inf_long, ri_long = srv.wait(i_long)
        t_long = time.perf_counter() - t0
        x_other, inf_other, ri_other = srv.wait(i_other)
        # the short request shared the long one's batch and finished first
        assert ri_short["batch_requests"] >= 2, ri_short
        assert t_short < t_long
        # the two configurations ran at the same time: each was admitted
        # before the other finished
        s_long = ri_long["queue_seconds"]
        s_other = ri_other["queue_seconds"]
        assert s_other < ri_long["latency_seconds"] and s_long < ri_other["latency_seconds"]
        for cfg, rhs, x, tol in ((MID, long_rhs, x_long, 1e-12), (MID, short_rhs, x_short, 1e-6),
                                 (OTHER, other_rhs, x_other, 1e-12)):
            op = _op(cfg)
            for k in range(rhs.shape[0]):
                assert rel(op.apply(t(x[k])).numpy(), rhs[k]) <= tol
            assert_close(x, _alone(cfg, rhs, tol), 1e-5)
    finally:
        srv.close()
