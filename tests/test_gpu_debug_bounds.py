"""GPU: the range-checked build (libmd_debug.so, -DMD_DEBUG_BOUNDS) through the parity suites.

compute-sanitizer is not available here, so the library has its own range checks: in the
debug build every index into the shared-memory rows and pair tables, the binomial tables, the
work tables and the tensor-core kernel's tables, tiles and head slices is checked, an index
out of range is recorded and replaced by a safe one, and the call that launched the kernel
returns MD_EINTERNAL.  This test runs the parity tests that reach every kernel family (every
level forced onto the tensor cores with every head size and product width, the popcount
kernels with every filter mode and row width, edge shapes, batches, the allocation-free scan)
in a child process bound to the debug build: each comparison with the oracle must hold and no
call may report a failed check.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_range_checked_build_passes_parity_suites():
    from paper_1911_08963_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, MD_LIBRARY=lib)
    probe = subprocess.run([sys.executable, "-c", "from paper_1911_08963_gb300 import binding as B; "
                            "print(B.md_debug_bounds())"], cwd=ROOT, env=env, capture_output=True, text=True)
    assert probe.returncode == 0 and probe.stdout.strip() == "(True, 0)", probe.stdout + probe.stderr
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_tensor.py", "tests/test_gpu_parity.py", "tests/test_gpu_batch.py", "tests/test_zz_no_alloc.py",
           "-k", "forced_tensor_levels or forced_tensor_product_words or random_codes or textbook or edge_shapes "
                 "or small_chunks or wide_rows or scan_range_matches or batch_matches or batch_heavy or noalloc"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
