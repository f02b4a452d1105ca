"""The checked build (libfdas_checked.so: device bounds checks written as error
records, canary guards around every workspace buffer, a check after each
launch group).

A child process loads the checked build (FDAS_CHECKED=1) and runs the cases
of tests/checked_cases.py; this process runs the same cases on the ordinary
build.  Every output must be the same bytes (the checks change no result and
none of them fails on valid work), and the checked build's fault injections
must be reported as FDAS_ERR_BOUNDS naming the damaged buffer or the failed
check, with the plan usable afterwards.  Nothing here faults the GPU: the
canary fault writes one byte inside a guard (inside the allocation), and the
bounds fault lowers the limits so that checks fail while the accesses they
skip were in bounds.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import checked_cases as CC

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def capi():
    if os.environ.get("FDAS_CHECKED") == "1":
        pytest.skip("this process already runs the checked build")
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    return c


@pytest.fixture(scope="module")
def checked(capi, tmp_path_factory):
    path = str(tmp_path_factory.mktemp("checked") / "run")
    env = dict(os.environ, FDAS_CHECKED="1")
    env.pop("FDAS_FAULT", None)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), path], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    with open(path + ".json") as f:
        faults = json.load(f)
    return dict(np.load(path + ".npz")), faults


def test_ordinary_build_is_not_checked(capi):
    assert not capi.fdas_checked_build()
    assert "checked" not in capi.fdas_version()


def test_checked_build_gives_the_same_bytes(capi, checked):
    outs, _ = checked
    ref = CC.run_cases(capi, torch)
    assert set(outs) == set(ref)
    for name in sorted(ref):
        assert outs[name].tobytes() == ref[name].tobytes(), name


def test_canary_fault_is_reported_with_its_buffer(capi, checked):
    _, faults = checked
    st, msg = faults["canary"]
    assert st == capi.FDAS_ERR_BOUNDS, msg
    assert "canary of workspace buffer plane[0]" in msg and "the correlation of series 0" in msg
    # the byte written is the first one after the plane: offset = its size
    size = int(msg.split("plane[0] (")[1].split(" bytes")[0])
    assert msg.rstrip().endswith(f"overwritten at byte offset {size}"), msg
    assert faults["canary_then_clean"]


def test_canary_fault_inside_a_graph_is_found_after_its_launch(capi, checked):
    _, faults = checked
    st, msg = faults["canary_graph"]
    assert st == capi.FDAS_ERR_BOUNDS and "after the candidate ordering" in msg, msg
    assert "canary of workspace buffer plane[0]" in msg
    assert faults["canary_graph_then_clean"]


def test_bounds_fault_is_reported_with_its_site(capi, checked):
    _, faults = checked
    for key in ("bounds", "bounds_async"):
        st, msg = faults[key]
        assert st == capi.FDAS_ERR_BOUNDS, (key, msg)
        assert "failed device bounds check" in msg and "against a limit of" in msg, msg
    # the first failure is in the correlation of the first series
    assert "after the correlation of series 0" in faults["bounds"][1]
    assert faults["bounds_then_clean"]
