"""Host-side behaviour of bench.py that needs no GPU: the 32^3 x 64 workload
runs in a child process whose failure is reported in the JSON line instead
of ending the benchmark, and the stencil lattice option is validated."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the no-device path")
def test_large_workload_failure_is_reported_not_raised():
    import bench
    out = bench.large_batched()
    assert set(out) == {"error"} and "exit 1" in out["error"] and "no CUDA device" in out["error"]


def test_stencil_lattice_option_is_validated():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--stencils-only",
                        "--stencil-lattice", "12,8,8,8"], capture_output=True, text=True, cwd=ROOT)
    assert r.returncode != 0 and "multiples of 8" in (r.stderr + r.stdout)
