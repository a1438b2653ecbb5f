"""ctypes binding of the C ABI in ``include/ddamg.h`` (argument marshalling only).

Every computation runs in ``libddamg.so``; this module converts NumPy host
arrays or torch CUDA tensors to pointers, calls the library and raises on a
non-zero status.  Field layouts are the host exchange layouts of the header:
spinors ``complex128 [nrhs][V][4][3]``, gauge ``complex128 [V][4][3][3]``,
coarse vectors ``complex128 [nrhs][NX][2 n_v]``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddamg.so")

FP64 = 0
FP32 = 1
BF16 = 2
FP16 = 3

STATUS = {0: "DDAMG_OK", 1: "DDAMG_EINVAL", 2: "DDAMG_ENOMEM", 3: "DDAMG_ECUDA",
          4: "DDAMG_ENOCONV", 5: "DDAMG_ENUMERIC", 6: "DDAMG_ETIMEOUT", 7: "DDAMG_ESTATE"}


class DDAMGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_int * 4), ("sap_block", C.c_int * 4), ("agg_block", C.c_int * 4),
        ("n_v", C.c_int), ("m0", C.c_double), ("csw", C.c_double),
        ("setup_iters", C.c_int), ("n_sap", C.c_int), ("mr_iters", C.c_int),
        ("coarse_tol", C.c_double), ("coarse_restart", C.c_int), ("coarse_max_iter", C.c_int),
        ("precision", C.c_int), ("outer_restart", C.c_int), ("max_outer_iter", C.c_int),
        ("seed", C.c_uint64), ("hbm_budget", C.c_size_t), ("outer_refine", C.c_double),
        ("half_vectors", C.c_int),
        ("ortho_fp32", C.c_int),
    ]


class Level2Params(C.Structure):
    _fields_ = [
        ("block", C.c_int * 4), ("n_v", C.c_int), ("setup_iters", C.c_int), ("n_sap", C.c_int),
        ("mr_iters", C.c_int), ("coarsest_tol", C.c_double), ("coarsest_restart", C.c_int),
        ("coarsest_max_iter", C.c_int), ("restart", C.c_int), ("seed", C.c_uint64),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int), ("restarts", C.c_int), ("coarse_iters", C.c_int),
        ("precond_calls", C.c_int), ("true_residual", C.c_double), ("converged", C.c_int),
        ("seconds", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [
        ("kernel_launches", C.c_uint64), ("dslash_launches", C.c_uint64), ("dslash_ms", C.c_double),
        ("sap_launches", C.c_uint64), ("sap_ms", C.c_double),
        ("coarse_launches", C.c_uint64), ("coarse_ms", C.c_double), ("device_bytes", C.c_size_t),
        ("coarse_apply_launches", C.c_uint64), ("coarse_apply_ms", C.c_double),
        ("reorth_passes", C.c_uint64), ("setup_flops", C.c_double), ("solve_flops", C.c_double),
        ("restrict_launches", C.c_uint64), ("restrict_ms", C.c_double),
        ("prolong_launches", C.c_uint64), ("prolong_ms", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RequestInfo(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("batch_rhs", C.c_int), ("batch_requests", C.c_int), ("setup_run", C.c_int),
        ("queue_seconds", C.c_double), ("latency_seconds", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CoarsePlan(C.Structure):
    _fields_ = [
        ("rhs_per_pass", C.c_int), ("ctas", C.c_int), ("sites_per_cta", C.c_int),
        ("krylov_in_shared", C.c_int), ("resident_blocks", C.c_int), ("block_ring", C.c_int),
        ("shared_bytes", C.c_size_t), ("scratch_bytes", C.c_size_t),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("kernel", C.c_char * 32), ("problem", C.c_char * 96), ("variants", C.c_int), ("best", C.c_int),
                ("us", C.c_float * 4)]

    def as_dict(self):
        n = self.variants
        return {"kernel": self.kernel.decode(), "problem": self.problem.decode(), "best": self.best,
                "us": [round(float(v), 2) for v in self.us[:n]]}


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_H = C.c_void_p

SIGNATURES = {
    "ddamg_default_params": (None, [C.POINTER(Params)]),
    "ddamg_status_string": (C.c_char_p, [_I]),
    "ddamg_create": (_I, [C.POINTER(Params), _P, _I, _P, C.POINTER(_H)]),
    "ddamg_setup": (_I, [C.POINTER(Params), _P, _I, _P, C.POINTER(_H)]),
    "ddamg_run_setup": (_I, [_H, _P, _I]),
    "ddamg_set_gauge": (_I, [_H, _P, _I]),
    "ddamg_update_mass": (_I, [_H, _D, _D]),
    "ddamg_solve": (_I, [_H, _I, _P, _P, _I, _D, C.POINTER(SolveInfo)]),
    "ddamg_solve_batched": (_I, [_H, _I, _P, _P, _I, _D, C.POINTER(SolveInfo)]),
    "ddamg_apply_D": (_I, [_H, _I, _I, _P, _P, _I]),
    "ddamg_apply_clover": (_I, [_H, _I, _I, _I, _P, _P, _I]),
    "ddamg_get_clover": (_I, [_H, _I, _P]),
    "ddamg_block_solve": (_I, [_H, _I, _I, _I, _P, _P, _I]),
    "ddamg_sap": (_I, [_H, _I, _I, _P, _P, _I]),
    "ddamg_set_test_vectors": (_I, [_H, _P, _I]),
    "ddamg_get_test_vectors": (_I, [_H, _P]),
    "ddamg_orthonormalize": (_I, [_H]),
    "ddamg_build_coarse": (_I, [_H]),
    "ddamg_get_coarse_op": (_I, [_H, _P]),
    "ddamg_restrict": (_I, [_H, _I, _I, _P, _P, _I]),
    "ddamg_prolong": (_I, [_H, _I, _I, _P, _P, _I]),
    "ddamg_apply_coarse": (_I, [_H, _I, _I, _P, _P, _I]),
    "ddamg_coarse_solve": (_I, [_H, _I, _I, _P, _P, _I, _D, _P]),
    "ddamg_coarse_solve_noalloc": (_I, [_H, _I, _P, _P, _D, _P]),
    "ddamg_apply_M": (_I, [_H, _I, _I, _P, _P, _I]),
    "ddamg_set_coarse_op": (_I, [_H, _P, _I]),
    "ddamg_batch_begin": (_I, [_H, _I]),
    "ddamg_batch_admit": (_I, [_H, _I, _P, _I, _D]),
    "ddamg_batch_cycle": (_I, [_H, C.POINTER(_I)]),
    "ddamg_batch_slot": (_I, [_H, _I, C.POINTER(_I)]),
    "ddamg_batch_take": (_I, [_H, _I, _P, _I, C.POINTER(SolveInfo)]),
    "ddamg_get_coarse_plan": (_I, [_H, _I, C.POINTER(CoarsePlan)]),
    "ddamg_trim": (_I, [_H]),
    "ddamg_set_graphs": (_I, [_H, _I]),
    "ddamg_set_wait_limit": (_I, [_H, C.c_int64]),
    "ddamg_tuning_count": (_I, []),
    "ddamg_get_tuning": (_I, [_I, C.POINTER(Tuning)]),
    "ddamg_pin_variant": (_I, [C.c_char_p, _I]),
    "ddamg_get_index_maps": (_I, [_H, _P, _P, _P, _P, _P]),
    "ddamg_get_stats": (_I, [_H, C.POINTER(Stats)]),
    "ddamg_reset_stats": (_I, [_H]),
    "ddamg_enable_kernel_timing": (_I, [_H, _I]),
    "ddamg_random_vectors": (_I, [_H, C.c_uint64, _I, _P]),
    "ddamg_get_history": (_I, [_H, _I, _P, _P, C.POINTER(_I)]),
    "ddamg_last_error": (C.c_char_p, [_H]),
    "ddamg_server_create": (_I, [C.c_size_t, _I, _P, C.POINTER(_H)]),
    "ddamg_server_create2": (_I, [C.c_size_t, _I, _I, _P, C.POINTER(_H)]),
    "ddamg_server_add_config": (_I, [_H, C.POINTER(Params), _P, C.POINTER(_I)]),
    "ddamg_server_submit": (_I, [_H, _I, _I, _P, _P, _D, _P, C.POINTER(C.c_uint64)]),
    "ddamg_server_wait": (_I, [_H, C.c_uint64, C.POINTER(RequestInfo)]),
    "ddamg_server_device_bytes": (_I, [_H, C.POINTER(C.c_size_t)]),
    "ddamg_server_last_error": (C.c_char_p, [_H]),
    "ddamg_server_destroy": (None, [_H]),
    "ddamg_level2_default_params": (_I, [C.POINTER(Level2Params)]),
    "ddamg_level2_init": (_I, [_H, C.POINTER(Level2Params)]),
    "ddamg_level2_setup": (_I, [_H, _P]),
    "ddamg_level2_set_vectors": (_I, [_H, _P]),
    "ddamg_level2_get_vectors": (_I, [_H, _P]),
    "ddamg_level2_get_op": (_I, [_H, _P]),
    "ddamg_level2_sap": (_I, [_H, _I, _P, _P]),
    "ddamg_level2_apply_M2": (_I, [_H, _I, _P, _P]),
    "ddamg_level2_coarse_solve": (_I, [_H, _I, _P, _P, _D, _P]),
    "ddamg_set_levels": (_I, [_H, _I]),
    "ddamg_destroy": (None, [_H]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libddamg.so is missing at {path}: build it with "
                           "paper_1811_00355_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def tuning():
    """The autotuner's measured choices so far (kernel, problem, times, choice)."""
    lib = load()
    out = []
    for i in range(lib.ddamg_tuning_count()):
        t = Tuning()
        if lib.ddamg_get_tuning(i, C.byref(t)) == 0:
            out.append(t.as_dict())
    return out


def pin_variant(kernel: str, variant: int) -> None:
    """Fix the variant of a kernel with measured variants (variant < 0: measure)."""
    load().ddamg_pin_variant(kernel.encode(), int(variant))


def level2_default_params(**kw) -> Level2Params:
    """Third-level parameters (ddamg_level2_default_params, then the given fields)."""
    p = Level2Params()
    load().ddamg_level2_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "block":
            p.block[:] = list(v)
        else:
            setattr(p, k, v)
    return p


def default_params(**kw) -> Params:
    p = Params()
    load().ddamg_default_params(C.byref(p))
    for k, v in kw.items():
        if k in ("L", "sap_block", "agg_block"):
            getattr(p, k)[:] = list(v)
        else:
            setattr(p, k, v)
    if "sap_block" in kw and "agg_block" not in kw:
        p.agg_block[:] = list(kw["sap_block"])
    return p


# ---------------------------------------------------------------------------
def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _ptr(a):
    """(pointer, on_device) of a contiguous complex128/float64/int32 buffer."""
    if _is_torch_cuda(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), 1
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("host arrays must be C-contiguous numpy arrays")
    return C.c_void_p(a.ctypes.data), 0


def _like(a, shape, dtype=np.complex128):
    if _is_torch_cuda(a):
        import torch
        tdt = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device=a.device)
    return np.empty(shape, dtype)


class DDAMG:
    """One gauge field with its clover term, test vectors and coarse operator."""

    def __init__(self, params: Params, gauge, stream=None):
        self.lib = load()
        self.p = params
        self.V = int(np.prod(list(params.L)))
        self.n_v = params.n_v
        self.NX = self.V // int(np.prod(list(params.sap_block)))
        h = _H()
        gp, dev = _ptr(gauge)
        st = C.c_void_p(stream) if stream else None
        self._check(self.lib.ddamg_create(C.byref(params), gp, dev, st, C.byref(h)), None)
        self.h = h

    # -- plumbing ----------------------------------------------------------------
    def _check(self, status, h="self"):
        if status != 0:
            hh = self.h if h == "self" else h
            msg = self.lib.ddamg_last_error(hh).decode()
            raise DDAMGError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ddamg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _fine_out(self, a, n):
        return _like(a, (n, self.V, 4, 3))

    def _nrhs(self, a):
        return a.shape[0] if len(a.shape) == 4 else 1

    # -- setup and solve ---------------------------------------------------------
    def run_setup(self, init=None):
        if init is None:
            self._check(self.lib.ddamg_run_setup(self.h, None, 0))
        else:
            p, dev = _ptr(init)
            self._check(self.lib.ddamg_run_setup(self.h, p, dev))

    def set_gauge(self, gauge):
        p, dev = _ptr(gauge)
        self._check(self.lib.ddamg_set_gauge(self.h, p, dev))

    def update_mass(self, m0, csw):
        self._check(self.lib.ddamg_update_mass(self.h, m0, csw))
        self.p.m0, self.p.csw = m0, csw

    # the geometry a saved setup must match to be loaded
    _SETUP_KEYS = ("L", "sap_block", "agg_block", "n_v")

    def save_setup(self, path):
        """Write the setup's test vectors (orthonormal per aggregate and
        chirality, FP64) with the geometry and mass they belong to to an .npz
        file.  The links are not saved: they are the caller's input."""
        meta = {k: np.array(list(getattr(self.p, k)) if k != "n_v" else [self.p.n_v], np.int64)
                for k in self._SETUP_KEYS}
        np.savez(path, vectors=self.get_test_vectors(), m0=self.p.m0, csw=self.p.csw, **meta)

    def load_setup(self, path):
        """Install test vectors written by save_setup in this handle and
        assemble D_c from them with the handle's own links and mass (a saved
        setup serves another mass as the mass update does).  The geometry
        must match.  Returns the (m0, csw) the vectors were saved at."""
        z = np.load(path)
        for k in self._SETUP_KEYS:
            want = list(getattr(self.p, k)) if k != "n_v" else [self.p.n_v]
            if list(z[k]) != want:
                raise DDAMGError(1, "saved setup has %s=%s, this handle %s" % (k, list(z[k]), want))
        self.set_test_vectors(np.ascontiguousarray(z["vectors"]))
        self.build_coarse()
        return float(z["m0"]), float(z["csw"])

    def solve(self, rhs, tol=1e-10, allow_noconv=False, out=None):
        n = self._nrhs(rhs)
        x = self._fine_out(rhs, n).reshape(rhs.shape) if out is None else out
        info = (SolveInfo * n)()
        pi, dev = _ptr(rhs)
        po, _ = _ptr(x)
        st = self.lib.ddamg_solve(self.h, n, pi, po, dev, tol, info)
        if not (allow_noconv and st == 4):
            self._check(st)
        return x, [i.as_dict() for i in info]

    def solve_batched(self, rhs, tol=1e-10, allow_noconv=False, out=None):
        n = self._nrhs(rhs)
        x = self._fine_out(rhs, n).reshape(rhs.shape) if out is None else out
        info = (SolveInfo * n)()
        pi, dev = _ptr(rhs)
        po, _ = _ptr(x)
        st = self.lib.ddamg_solve_batched(self.h, n, pi, po, dev, tol, info)
        if not (allow_noconv and st == 4):
            self._check(st)
        return x, [i.as_dict() for i in info]

    # -- the batch as a resumable run ---------------------------------------------------
    def batch_begin(self, slots):
        self._check(self.lib.ddamg_batch_begin(self.h, slots))

    def batch_admit(self, slot, rhs, tol=1e-10):
        p, dev = _ptr(rhs)
        self._check(self.lib.ddamg_batch_admit(self.h, slot, p, dev, tol))

    def batch_cycle(self):
        """One restart cycle; returns the number of slots still running."""
        n = _I()
        self._check(self.lib.ddamg_batch_cycle(self.h, C.byref(n)))
        return n.value

    def batch_slot(self, slot):
        """0 free, 1 running, 2 finished."""
        st = _I()
        self._check(self.lib.ddamg_batch_slot(self.h, slot, C.byref(st)))
        return st.value

    def batch_take(self, slot, out=None, allow_noconv=False):
        x = np.empty((self.V, 4, 3), np.complex128) if out is None else out
        info = SolveInfo()
        p, dev = _ptr(x)
        st = self.lib.ddamg_batch_take(self.h, slot, p, dev, C.byref(info))
        if not (allow_noconv and st == 4):
            self._check(st)
        return x, info.as_dict()

    # -- single steps ----------------------------------------------------------------
    def _fine_op(self, fn, x, *args):
        n = self._nrhs(x)
        out = self._fine_out(x, n).reshape(x.shape)
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(fn(self.h, *args[:-1], n, pi, po, dev) if args else fn(self.h, n, pi, po, dev))
        return out

    def apply_D(self, x, precision=FP64):
        n = self._nrhs(x)
        out = self._fine_out(x, n).reshape(x.shape)
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_apply_D(self.h, precision, n, pi, po, dev))
        return out

    def apply_clover(self, x, inverse=False, precision=FP64):
        n = self._nrhs(x)
        out = self._fine_out(x, n).reshape(x.shape)
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_apply_clover(self.h, precision, int(inverse), n, pi, po, dev))
        return out

    def get_clover(self, inverse=False):
        out = np.empty((self.V, 2, 36))
        self._check(self.lib.ddamg_get_clover(self.h, int(inverse), C.c_void_p(out.ctypes.data)))
        return out

    def block_solve(self, x, colour, precision=FP64):
        n = self._nrhs(x)
        out = self._fine_out(x, n).reshape(x.shape)
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_block_solve(self.h, precision, colour, n, pi, po, dev))
        return out

    def sap(self, x, precision=FP64):
        n = self._nrhs(x)
        out = self._fine_out(x, n).reshape(x.shape)
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_sap(self.h, precision, n, pi, po, dev))
        return out

    def set_test_vectors(self, vecs):
        p, dev = _ptr(vecs)
        self._check(self.lib.ddamg_set_test_vectors(self.h, p, dev))

    def get_test_vectors(self):
        out = np.empty((self.n_v, self.V, 4, 3), np.complex128)
        self._check(self.lib.ddamg_get_test_vectors(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def orthonormalize(self):
        self._check(self.lib.ddamg_orthonormalize(self.h))

    def build_coarse(self):
        self._check(self.lib.ddamg_build_coarse(self.h))

    def get_coarse_op(self):
        n2 = 2 * self.n_v
        out = np.empty((self.NX, 9, n2, n2), np.complex128)
        self._check(self.lib.ddamg_get_coarse_op(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def set_coarse_op(self, dc):
        """Install a coarse operator ``[NX][9][2n][2n]`` (host or device) and
        invert its self blocks."""
        p, dev = _ptr(dc)
        self._check(self.lib.ddamg_set_coarse_op(self.h, p, dev))

    def trim(self):
        """Release the setup's temporaries and, for an inner precision other
        than FP64, the FP64 copy of the test vectors (ddamg_trim)."""
        self._check(self.lib.ddamg_trim(self.h))

    def set_graphs(self, on=True):
        """Outer iterations through CUDA graphs (default) or kernel by kernel."""
        self._check(self.lib.ddamg_set_graphs(self.h, int(bool(on))))

    def coarse_plan(self, nrhs=1):
        """Launch configuration of the coarse GMRES for nrhs right-hand sides."""
        c = CoarsePlan()
        self._check(self.lib.ddamg_get_coarse_plan(self.h, nrhs, C.byref(c)))
        return c.as_dict()

    def set_wait_limit(self, polls=-1):
        """Polls of the device-side bounded waits before they give up
        (0: at the first unsuccessful poll; negative: the defaults)."""
        self._check(self.lib.ddamg_set_wait_limit(self.h, polls))

    def restrict(self, x, precision=FP64):
        n = self._nrhs(x)
        out = _like(x, (n, self.NX, 2 * self.n_v))
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_restrict(self.h, precision, n, pi, po, dev))
        return out if len(x.shape) == 4 else out[0]

    def prolong(self, xc, precision=FP64):
        n = xc.shape[0] if len(xc.shape) == 3 else 1
        out = _like(xc, (n, self.V, 4, 3))
        pi, dev = _ptr(xc)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_prolong(self.h, precision, n, pi, po, dev))
        return out if len(xc.shape) == 3 else out[0]

    def apply_coarse(self, xc, precision):
        n = xc.shape[0] if len(xc.shape) == 3 else 1
        out = _like(xc, tuple(xc.shape))
        pi, dev = _ptr(xc)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_apply_coarse(self.h, precision, n, pi, po, dev))
        return out

    def coarse_solve(self, bc, tol, precision):
        n = bc.shape[0] if len(bc.shape) == 3 else 1
        out = _like(bc, tuple(bc.shape))
        its = np.zeros(n, np.int32)
        pi, dev = _ptr(bc)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_coarse_solve(self.h, precision, n, pi, po, dev, tol,
                                                C.c_void_p(its.ctypes.data)))
        return out, its

    def coarse_solve_noalloc(self, bc, tol):
        """Coarse solve out of the library's fixed device array (device tensors only)."""
        if not _is_torch_cuda(bc):
            raise ValueError("ddamg_coarse_solve_noalloc takes device buffers")
        n = bc.shape[0] if len(bc.shape) == 3 else 1
        out = _like(bc, tuple(bc.shape))
        its = np.zeros(n, np.int32)
        self._check(self.lib.ddamg_coarse_solve_noalloc(self.h, n, C.c_void_p(bc.data_ptr()),
                                                        C.c_void_p(out.data_ptr()), tol,
                                                        C.c_void_p(its.ctypes.data)))
        return out, its

    # ---- third level (host numpy arrays of complex128) ------------------------
    def level2_init(self, p2: "Level2Params"):
        """Lay out level 2 on this handle's D_c (ddamg_level2_init)."""
        self._check(self.lib.ddamg_level2_init(self.h, C.byref(p2)))
        self.n_v2 = int(p2.n_v)
        self.NX2 = self.NX // int(np.prod(list(p2.block)))

    def level2_setup(self, vecs=None):
        """Adaptive setup on D_c from host vectors [n_v2][NX][2 n_v] (None: seeded)."""
        if vecs is None:
            self._check(self.lib.ddamg_level2_setup(self.h, None))
        else:
            v = np.ascontiguousarray(vecs, np.complex128)
            self._check(self.lib.ddamg_level2_setup(self.h, C.c_void_p(v.ctypes.data)))

    def level2_set_vectors(self, vecs):
        v = np.ascontiguousarray(vecs, np.complex128)
        self._check(self.lib.ddamg_level2_set_vectors(self.h, C.c_void_p(v.ctypes.data)))

    def level2_get_vectors(self):
        out = np.empty((self.n_v2, self.NX, 2 * self.n_v), np.complex128)
        self._check(self.lib.ddamg_level2_get_vectors(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def level2_get_op(self):
        m2 = 2 * self.n_v2
        out = np.empty((self.NX2, 9, m2, m2), np.complex128)
        self._check(self.lib.ddamg_level2_get_op(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def _level2_fields(self, fn, x, *extra):
        x = np.ascontiguousarray(x, np.complex128)
        n = x.shape[0] if x.ndim == 3 else 1
        out = np.empty(x.shape, np.complex128)
        self._check(fn(self.h, n, C.c_void_p(x.ctypes.data), C.c_void_p(out.ctypes.data), *extra))
        return out

    def level2_sap(self, x):
        return self._level2_fields(self.lib.ddamg_level2_sap, x)

    def level2_apply_M2(self, x):
        return self._level2_fields(self.lib.ddamg_level2_apply_M2, x)

    def level2_coarse_solve(self, b, tol):
        n = b.shape[0] if b.ndim == 3 else 1
        its = np.zeros(n, np.int32)
        out = self._level2_fields(self.lib.ddamg_level2_coarse_solve, b, tol, C.c_void_p(its.ctypes.data))
        return out, its

    def set_levels(self, levels: int):
        self._check(self.lib.ddamg_set_levels(self.h, int(levels)))

    def apply_M(self, x, precision):
        n = self._nrhs(x)
        out = self._fine_out(x, n).reshape(x.shape)
        pi, dev = _ptr(x)
        po, _ = _ptr(out)
        self._check(self.lib.ddamg_apply_M(self.h, precision, n, pi, po, dev))
        return out

    def index_maps(self):
        V, NX = self.V, self.NX
        arrs = {k: np.empty(V, np.int32) for k in ("parity", "block", "colour", "aggregate")}
        arrs["coarse_parity"] = np.empty(NX, np.int32)
        self._check(self.lib.ddamg_get_index_maps(
            self.h, *(C.c_void_p(arrs[k].ctypes.data)
                      for k in ("parity", "block", "colour", "aggregate", "coarse_parity"))))
        return arrs

    def random_vectors(self, seed, n):
        out = np.empty((n, self.V, 4, 3), np.complex128)
        self._check(self.lib.ddamg_random_vectors(self.h, seed, n, C.c_void_p(out.ctypes.data)))
        return out

    def stats(self):
        s = Stats()
        self._check(self.lib.ddamg_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def history(self):
        """(MFLOP/site, relative residual) after every outer iteration of the
        last right-hand side of solve()."""
        n = _I()
        self._check(self.lib.ddamg_get_history(self.h, 0, None, None, C.byref(n)))
        f = np.empty(n.value)
        r = np.empty(n.value)
        self._check(self.lib.ddamg_get_history(self.h, n.value, C.c_void_p(f.ctypes.data),
                                               C.c_void_p(r.ctypes.data), C.byref(n)))
        return f, r

    def reset_stats(self):
        self._check(self.lib.ddamg_reset_stats(self.h))

    def enable_kernel_timing(self, on=True):
        self._check(self.lib.ddamg_enable_kernel_timing(self.h, int(on)))


class Server:
    """Continuous-batching request loop over resident gauge configurations
    (ddamg_server_*): submit returns at once, wait blocks for one request;
    `workers` configurations are served at the same time, each on its own
    stream unless `stream` is given."""

    def __init__(self, hbm_budget=0, max_batch=12, stream=None, workers=2):
        self.lib = load()
        h = _H()
        st = C.c_void_p(stream) if stream else None
        status = self.lib.ddamg_server_create2(hbm_budget, max_batch, workers, st, C.byref(h))
        if status != 0:
            raise DDAMGError(status, self.lib.ddamg_status_string(status).decode())
        self.h = h
        self.V = {}
        self._live = {}

    def _check(self, status):
        if status != 0:
            msg = self.lib.ddamg_server_last_error(self.h) if self.h else b""
            raise DDAMGError(status, (msg or self.lib.ddamg_status_string(status)).decode())

    def add_config(self, params: Params, gauge) -> int:
        gauge = np.ascontiguousarray(gauge, dtype=np.complex128)
        cid = _I()
        self._check(self.lib.ddamg_server_add_config(self.h, C.byref(params), C.c_void_p(gauge.ctypes.data),
                                                     C.byref(cid)))
        self.V[cid.value] = int(np.prod(list(params.L)))
        return cid.value

    def submit(self, config_id, rhs, tol=1e-10) -> int:
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        n = rhs.shape[0] if rhs.ndim == 4 else 1
        x = np.empty_like(rhs)
        info = (SolveInfo * n)()
        rid = C.c_uint64()
        self._check(self.lib.ddamg_server_submit(self.h, config_id, n, C.c_void_p(rhs.ctypes.data),
                                                 C.c_void_p(x.ctypes.data), tol, C.cast(info, C.c_void_p),
                                                 C.byref(rid)))
        self._live[rid.value] = (rhs, x, info)     # buffers stay alive until wait
        return rid.value

    def wait(self, request_id, allow_noconv=False):
        ri = RequestInfo()
        status = self.lib.ddamg_server_wait(self.h, request_id, C.byref(ri))
        rhs, x, info = self._live.pop(request_id)
        if not (allow_noconv and status == 4):
            self._check(status)
        return x, [i.as_dict() for i in info], ri.as_dict()

    def device_bytes(self) -> int:
        b = C.c_size_t()
        self._check(self.lib.ddamg_server_device_bytes(self.h, C.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.ddamg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
