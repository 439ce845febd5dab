"""The memory checks (a stand-in for a memory checker, which this pool does not
run): every decoder kernel, run on the checked build of the library, must store
into none of its shared-memory redzones; every kernel, on both builds, must
leave the sentinels around its outputs untouched; and the checked build must
give the default build's results bit for bit (its redzones move the layouts
but change no arithmetic).

The checked build runs in a child process (POLARBP_LIBRARY names it), the
default build in this one; both run the cases of tests/checked_cases.py."""
import os
import subprocess
import sys

import numpy as np
import pytest

import checked_cases as C

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = [name for name, _, _ in C.cases()]


@pytest.fixture(scope="module")
def checked(tmp_path_factory):
    from paper_1505_04979_gb300 import build
    lib = build.build(checked=True)
    out = str(tmp_path_factory.mktemp("checked") / "checked.npz")
    env = dict(os.environ, POLARBP_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), out], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return C.load(out)


@pytest.fixture(scope="module")
def default():
    return C.run()


def test_child_ran_the_checked_build(checked):
    _, meta = checked
    assert meta["_version"].endswith("checked"), meta["_version"]


@pytest.mark.parametrize("name", NAMES)
def test_no_redzone_store_and_no_store_past_an_output(checked, default, name):
    arrays, meta = checked
    m = meta[name]
    assert m["status"] == 0, f"{name}: status {m['status']}: {m['message']}"
    assert m["guards_intact"], f"{name}: a sentinel next to an output changed (checked build)"
    out, intact, rc, msg = default[name]
    assert rc == 0, f"{name}: status {rc}: {msg}"
    assert intact, f"{name}: a sentinel next to an output changed (default build)"
    # the checked build computes the same results
    for k, v in out.items():
        np.testing.assert_array_equal(arrays[f"{name}/{k}"], v, err_msg=f"{name}/{k}")
