"""Serving loop (ddamg_server_*): requests for two resident gauge
configurations submitted while others run are batched together, every result
reaches its tolerance by the oracle's D and equals the same request solved
alone, and a device-memory budget that holds one configuration at a time
releases and re-creates setups without changing results."""
from __future__ import annotations

import pytest

import synthetic as syn
from tests.gpu_common import MID, assert_close, make, oracle_op, rel, t

pytestmark = pytest.mark.gpu

OTHER = ((8, 8, 8, 8), (4, 4, 4, 4), 0.3, -0.25, 1.0, 8, 5)


def _params(cfg):
    import paper_1811_00355_gb300 as P
    L, b, eps, m0, csw, n_v, seed = cfg
    return P.default_params(L=L, sap_block=b, n_v=n_v, m0=m0, csw=csw, precision=P.FP32)


def _requests():
    reqs = []
    for k, (ci, n, tol) in enumerate([(0, 3, 1e-10), (1, 2, 1e-8), (0, 1, 1e-8), (1, 4, 1e-10),
                                      (0, 2, 1e-10), (1, 1, 1e-10)]):
        L = (MID if ci == 0 else OTHER)[0]
        reqs.append((ci, syn.gaussian_spinors(n, L, 100 + k), tol))
    return reqs


def _alone(cfg, rhs, tol):
    s = make(cfg, 1)
    s.run_setup()
    x, _ = s.solve_batched(rhs, tol)
    s.close()
    return x


def _check(results, reqs):
    ops = [oracle_op(*[MID[0], MID[2], MID[6], MID[3], MID[4]]),
           oracle_op(*[OTHER[0], OTHER[2], OTHER[6], OTHER[3], OTHER[4]])]
    for (ci, rhs, tol), (x, info, ri) in zip(reqs, results):
        assert ri["status"] == 0
        for k in range(rhs.shape[0]):
            res = rel(ops[ci].apply(t(x[k])).numpy(), rhs[k])
            assert res <= tol, (ci, k, res)
            assert info[k]["converged"] == 1
        alone = _alone(MID if ci == 0 else OTHER, rhs, tol)
        assert_close(x, alone, 1e-5)


def test_server_batches_requests_and_matches_alone():
    import paper_1811_00355_gb300 as P
    srv = P.Server(max_batch=12)
    try:
        c0 = srv.add_config(_params(MID), syn.gauge_field(MID[0], MID[2], MID[6]))
        c1 = srv.add_config(_params(OTHER), syn.gauge_field(OTHER[0], OTHER[2], OTHER[6]))
        assert (c0, c1) == (0, 1)
        reqs = _requests()
        ids = [srv.submit(ci, rhs, tol) for ci, rhs, tol in reqs]
        results = [srv.wait(i) for i in ids]
        # the first request starts alone (setup); later ones of a config share batches
        assert max(ri["batch_requests"] for _, _, ri in results) >= 2
        for (_, _, ri) in results:
            assert ri["latency_seconds"] >= ri["queue_seconds"] >= 0.0
        _check(results, reqs)
    finally:
        srv.close()


def test_server_budget_releases_idle_configs():
    import paper_1811_00355_gb300 as P
    # the footprint of the larger configuration after a batched solve
    s = make(MID, 1)
    s.run_setup()
    s.solve_batched(syn.gaussian_spinors(4, MID[0], 1), 1e-8)
    big = s.stats()["device_bytes"]
    s.close()
    srv = P.Server(hbm_budget=int(1.05 * big), max_batch=4)
    try:
        srv.add_config(_params(MID), syn.gauge_field(MID[0], MID[2], MID[6]))
        srv.add_config(_params(OTHER), syn.gauge_field(OTHER[0], OTHER[2], OTHER[6]))
        reqs = _requests()[:4]
        results = []
        for ci, rhs, tol in reqs:                       # one at a time: configs alternate
            results.append(srv.wait(srv.submit(ci, rhs, tol)))
            assert srv.device_bytes() <= int(1.05 * big)
        assert all(ri["setup_run"] == 1 for _, _, ri in results)
        _check(results, reqs)
    finally:
        srv.close()
