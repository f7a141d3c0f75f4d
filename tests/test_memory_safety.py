"""Memory safety of the kernels on the CPU: the host-check library, built with
AddressSanitizer and with poisoned guard bands between the simulation's
workspace arrays, runs every derivative shape and every simulation call
(tests/asan_driver.py) in a subprocess that preloads libasan.  An access
outside an input, an output, a shared-memory block or a workspace array
aborts that process with a sanitizer report."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT


def _libasan():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    except OSError:
        return None
    return p if p and os.path.isabs(p) and os.path.exists(p) else None


@pytest.mark.slow
def test_kernel_sequences_under_address_sanitizer():
    asan = _libasan()
    if asan is None:
        pytest.skip("libasan not available")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import build
    lib = build.build_hostcheck_asan()
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "asan_driver.py"), lib], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
    assert "all sequences ran" in r.stdout
