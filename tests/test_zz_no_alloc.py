"""The coarse solve that allocates no device memory.

Some callers cannot allocate device memory at solve time, for instance a
serving loop that must not take cudaMalloc's implicit synchronisation, or a
thread that works inside a memory budget reserved in advance.  For them
ddamg_coarse_solve_noalloc runs the coarse GMRES kernel out of a fixed array
the library reserves in device memory.  This file checks, through the C ABI,
that it returns what ddamg_coarse_solve returns on the same inputs, on two
calls in a row, and that no call grows the handle's device memory or the
device's memory in use (beyond the fixed array itself, which the CUDA driver
may only load at the first call on a device).
It is collected last so that a run stopping at the first failure has already
run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.coarse import Aggregation, orthonormalise
from tests.gpu_common import MID, TOL32, TOL64, assert_close, make, oracle_op, t

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_coarse_solve_matches_coarse_solve(prec):
    import paper_1811_00355_gb300 as P
    P.load()
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, prec)
    try:
        agg = Aggregation(oracle_op(L, eps, seed, m0, csw).geom, b)
        lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 70)), agg)
        s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
        s.build_coarse()
        tol = TOL64 if prec == 0 else TOL32
        rng = np.random.default_rng(71)
        for call in range(2):
            shape = (2, agg.NX, 2 * n_v)
            bc = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
            ref, its_ref = s.coarse_solve(np.ascontiguousarray(bc), 5e-2, prec)
            dev_in = torch.from_numpy(bc).cuda()
            torch.cuda.synchronize()
            held = s.stats()["device_bytes"]
            free_before = torch.cuda.mem_get_info()[0]
            got, its = s.coarse_solve_noalloc(dev_in, 5e-2)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            # the primary check: the handle allocated nothing
            assert s.stats()["device_bytes"] == held
            # a loose secondary bound on the device-wide free memory (other
            # processes on the GPU could move it): the first call on a device
            # may load the fixed 16 MiB array (module loading is lazy), and
            # no call allocates anything near a spinor field's size beyond that
            slack = (16 << 20) + ((16 << 20) if call == 0 else 0)
            assert free_after >= free_before - slack
            assert np.array_equal(its, its_ref), call
            assert_close(got.cpu().numpy(), ref, tol, call)
    finally:
        s.close()


def test_noalloc_rejects_oversized_requests():
    import paper_1811_00355_gb300 as P
    P.load()
    L, b, eps, m0, csw, n_v, seed = MID
    s = make(MID, 1)
    try:
        agg = Aggregation(oracle_op(L, eps, seed, m0, csw).geom, b)
        lam = orthonormalise(t(syn.gaussian_spinors(n_v, L, 72)), agg)
        s.set_test_vectors(np.ascontiguousarray(lam.numpy()))
        s.build_coarse()
        big = torch.zeros((4096, agg.NX, 2 * n_v), dtype=torch.complex128, device="cuda")
        with pytest.raises(P.DDAMGError) as e:
            s.coarse_solve_noalloc(big, 5e-2)
        assert e.value.status == 1 and "scratch" in str(e.value)
    finally:
        s.close()
