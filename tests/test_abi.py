"""Host-only checks of the C ABI: the library builds, loads and exports every
function include/ddamg.h declares; parameter validation happens before any
device work (so it is checkable without a GPU)."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ddamg.h")


@pytest.fixture(scope="session")
def lib():
    from paper_1811_00355_gb300 import build as b
    b.build()
    import paper_1811_00355_gb300 as P
    return P.load()


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"DDAMG_API[^;(]*?\b(ddamg_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared()
    for must in ("ddamg_setup", "ddamg_solve", "ddamg_apply_D", "ddamg_update_mass",
                 "ddamg_last_error", "ddamg_destroy", "ddamg_restrict", "ddamg_prolong",
                 "ddamg_build_coarse", "ddamg_coarse_solve", "ddamg_sap", "ddamg_apply_M"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1811_00355_gb300._ddamg import LIB_PATH, SIGNATURES
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ddamg_\w+)", out))
    for name in declared():
        assert name in exported, name
        assert hasattr(lib, name)
        assert name in SIGNATURES, f"binding misses {name}"


def test_struct_sizes_match_header(lib):
    """Compile a tiny C program against the header and compare struct sizes
    with the ctypes mirrors."""
    from paper_1811_00355_gb300._ddamg import CoarsePlan, Level2Params, Params, RequestInfo, SolveInfo, Stats
    src = ('#include "ddamg.h"\n#include <stdio.h>\nint main(void){printf("%zu %zu %zu %zu %zu %zu\\n",'
           ' sizeof(ddamg_params), sizeof(ddamg_solve_info), sizeof(ddamg_stats),'
           ' sizeof(ddamg_request_info), sizeof(ddamg_coarse_plan), sizeof(ddamg_level2_params));return 0;}\n')
    tmp = os.path.join(ROOT, "paper_1811_00355_gb300", "_build")
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, "sizes.c")
    exe = os.path.join(tmp, "sizes")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [C.sizeof(Params), C.sizeof(SolveInfo), C.sizeof(Stats), C.sizeof(RequestInfo),
                     C.sizeof(CoarsePlan), C.sizeof(Level2Params)]


def _create(lib, **kw):
    import paper_1811_00355_gb300 as P
    p = P.default_params(**kw)
    h = C.c_void_p()
    U = np.zeros((int(np.prod(list(p.L))), 4, 3, 3), np.complex128)
    st = lib.ddamg_create(C.byref(p), C.c_void_p(U.ctypes.data), 0, None, C.byref(h))
    return st, lib.ddamg_last_error(None).decode()


@pytest.mark.parametrize("kw, words", [
    (dict(L=(4, 4, 4, 5)), "even"),
    (dict(L=(8, 8, 8, 8), sap_block=(3, 2, 2, 2)), "even"),
    (dict(L=(12, 8, 8, 8), sap_block=(4, 4, 4, 4)), "number of Schwarz blocks"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), agg_block=(4, 4, 4, 4)), "aggregates"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), n_v=0), "n_v"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), coarse_restart=65), "coarse_restart"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), precision=7), "precision"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), m0=float("nan")), "finite"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), precision=0, ortho_fp32=1), "ortho_fp32"),
    (dict(L=(8, 8, 8, 8), sap_block=(2, 2, 2, 2), precision=1, ortho_fp32=2), "ortho_fp32"),
])
def test_invalid_parameters_rejected_before_device_work(lib, kw, words):
    st, msg = _create(lib, **kw)
    assert st == 1 and words in msg


def test_status_strings(lib):
    lib.ddamg_status_string.restype = C.c_char_p
    assert lib.ddamg_status_string(4) == b"DDAMG_ENOCONV"
    assert lib.ddamg_status_string(6) == b"DDAMG_ETIMEOUT"


def test_null_handle_calls_are_rejected(lib):
    assert lib.ddamg_solve(None, 1, None, None, 0, 1e-10, None) == 1
    assert lib.ddamg_apply_D(None, 0, 1, None, None, 0) == 1
    lib.ddamg_destroy(None)


def test_level2_calls_reject_missing_handles_and_buffers(lib):
    """The third level's entry points validate before any device work, and
    its default parameters are the oracle's level-2 defaults."""
    import paper_1811_00355_gb300 as P
    from oracle.three_level import Level2Params as OracleLevel2
    p = P.level2_default_params()
    o = OracleLevel2()
    assert tuple(p.block) == o.sap_block == o.agg_block
    assert (p.n_v, p.setup_iters, p.n_sap, p.mr_iters) == (o.n_v, o.setup_iters, o.n_sap, o.mr_iters)
    assert (p.coarsest_tol, p.coarsest_restart, p.coarsest_max_iter, p.restart) == \
        (o.coarsest_tol, o.coarsest_restart, o.coarsest_maxiter, o.restart)
    assert lib.ddamg_level2_default_params(None) == 1
    assert lib.ddamg_level2_init(None, C.byref(p)) == 1
    assert lib.ddamg_level2_setup(None, None) == 1
    assert lib.ddamg_level2_set_vectors(None, None) == 1
    assert lib.ddamg_level2_get_vectors(None, None) == 1
    assert lib.ddamg_level2_get_op(None, None) == 1
    assert lib.ddamg_level2_sap(None, 1, None, None) == 1
    assert lib.ddamg_level2_apply_M2(None, 1, None, None) == 1
    assert lib.ddamg_level2_coarse_solve(None, 1, None, None, 1e-2, None) == 1
    assert lib.ddamg_set_levels(None, 3) == 1


def test_server_rejects_invalid_arguments_before_device_work(lib):
    """The serving API validates its arguments before touching the GPU."""
    h = C.c_void_p()
    assert lib.ddamg_server_create(0, 0, None, C.byref(h)) == 1          # max_batch < 1
    assert lib.ddamg_server_create(0, 65, None, C.byref(h)) == 1         # max_batch > 64
    assert lib.ddamg_server_create(0, 12, None, None) == 1
    assert lib.ddamg_server_wait(None, 1, None) == 1
    assert lib.ddamg_server_submit(None, 0, 1, None, None, 1e-10, None, None) == 1


class _StubHandle:
    """The part of a DDAMG handle that save_setup / load_setup use, with
    the device calls replaced by host arrays (no GPU needed)."""

    def __init__(self, P, L, n_v):
        self._SETUP_KEYS = P.DDAMG._SETUP_KEYS
        self.p = P.default_params(L=L, sap_block=(2, 2, 2, 2), n_v=n_v, m0=-0.2, csw=1.1)
        self.V = int(np.prod(L))
        self.vectors = None
        self.built = False
        rng = np.random.default_rng(1)
        self._mine = rng.standard_normal((n_v, self.V, 4, 3)) + 1j * rng.standard_normal((n_v, self.V, 4, 3))

    def get_test_vectors(self):
        return self._mine

    def set_test_vectors(self, v):
        self.vectors = v

    def build_coarse(self):
        self.built = True


def test_setup_file_round_trip_and_geometry_check(lib, tmp_path):
    """save_setup writes the vectors with geometry and mass; load_setup gives
    them back unchanged with that mass, and refuses another geometry before
    any device call."""
    import paper_1811_00355_gb300 as P
    a = _StubHandle(P, (4, 4, 4, 4), 3)
    path = str(tmp_path / "s.npz")
    P.DDAMG.save_setup(a, path)
    b = _StubHandle(P, (4, 4, 4, 4), 3)
    b.p.m0 = 0.1
    assert P.DDAMG.load_setup(b, path) == (-0.2, 1.1)
    assert b.built and np.array_equal(b.vectors, a._mine)
    for L, n_v in (((4, 4, 4, 8), 3), ((4, 4, 4, 4), 4)):
        c = _StubHandle(P, L, n_v)
        with pytest.raises(P.DDAMGError):
            P.DDAMG.load_setup(c, path)
        assert c.vectors is None and not c.built
