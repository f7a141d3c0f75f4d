"""Host-side failure injection of the C ABI (no GPU involved): an armed entry
point returns the requested status before it does anything, after the given
number of calls have passed, for the given number of calls; rules come from
fc_inject_failure or from the FCNS_INJECT environment variable."""
import ctypes
import os
import subprocess
import sys

import pytest

from conftest import ROOT


@pytest.fixture()
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_01392_gb300 import api as a
    a.clear_injected()
    yield a
    a.clear_injected()


def test_skip_then_count(api):
    api.inject_failure("fc_setup", "FC_ERR_NOMEM", skip=1, count=1)
    api.Plan(5, 25, 33).close()                       # let through
    with pytest.raises(api.FcError) as e:
        api.Plan(5, 25, 33)
    assert e.value.name == "FC_ERR_NOMEM" and "injected failure" in str(e.value)
    api.Plan(5, 25, 33).close()                       # rule used up


def test_wildcard_until_cleared(api):
    api.inject_failure("*", "FC_ERR_TIMEOUT", count=-1)
    for _ in range(3):
        with pytest.raises(api.FcError) as e:
            api.Plan(5, 25, 33)
        assert e.value.name == "FC_ERR_TIMEOUT"
    # the injected status comes before any argument check (nothing is touched)
    assert api._lib.rk_step(None, ctypes.c_double(1e-3), None) == api.STATUS["FC_ERR_TIMEOUT"]
    assert api._lib.ns_batch_step(None, None, None) == api.STATUS["FC_ERR_TIMEOUT"]
    api.clear_injected()
    assert api._lib.rk_step(None, ctypes.c_double(1e-3), None) == api.STATUS["FC_ERR_ARG"]
    api.Plan(5, 25, 33).close()


def test_rules_on_other_entries_do_not_fire(api):
    api.inject_failure("rk_step", "FC_ERR_CUDA", count=-1)
    api.Plan(5, 25, 33).close()
    assert api._lib.rk_step(None, ctypes.c_double(1e-3), None) == api.STATUS["FC_ERR_CUDA"]
    f = ctypes.c_longlong()
    # fc_count_nonfinite is not armed: its own argument check answers
    assert api._lib.fc_count_nonfinite(0, None, -1, ctypes.byref(f), None) == api.STATUS["FC_ERR_ARG"]


def test_bad_rules_rejected(api):
    for args in (("fc_setup", 0, 0, 1), ("fc_setup", 3, -1, 1), ("fc_setup", 3, 0, 0), ("fc_setup", 9, 0, 1)):
        assert api._lib.fc_inject_failure(args[0].encode(), *args[1:]) == api.STATUS["FC_ERR_ARG"]
    api.Plan(5, 25, 33).close()


def test_environment_rules():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2002_01392_gb300 import api\n"
            "out = []\n"
            "for _ in range(4):\n"
            "    try:\n"
            "        api.Plan(5, 25, 33).close(); out.append('ok')\n"
            "    except api.FcError as e:\n"
            "        out.append(e.name)\n"
            "print(','.join(out))\n") % ROOT
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, FCNS_INJECT="ns_create:FC_ERR_NOMEM:0:1,fc_setup:FC_ERR_CUDA:1:2")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().splitlines()[-1] == "ok,FC_ERR_CUDA,FC_ERR_CUDA,ok"
