"""The debug-bounds build (index checks in the mixed forms' kernels, compiled
with PIC_DEBUG_BOUNDS) runs every mixed kernel family without a failed check
and gives results bit-identical to the normal build's; its device-side check
records an index outside its range and passes one inside.

The two libraries are loaded by separate processes (pic.lib() takes one per
process), each running tests/debug_bounds_runs.py."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RUNS = os.path.join(ROOT, "tests", "debug_bounds_runs.py")

pytestmark = pytest.mark.gpu


def _run(out, debug):
    env = dict(os.environ)
    env.pop("PIC_DEBUG_BOUNDS", None)
    if debug:
        env["PIC_DEBUG_BOUNDS"] = "1"
    r = subprocess.run([sys.executable, RUNS, out], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    with np.load(out) as f:
        return {k: f[k] for k in f.files}


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    from paper_2411_09605_gb300 import build
    build.build()
    build.build(debug_bounds=True)
    d = tmp_path_factory.mktemp("debug_bounds")
    return _run(str(d / "normal.npz"), False), _run(str(d / "debug.npz"), True)


def test_debug_build_loaded(results):
    normal, debug = results
    assert "debug-bounds" in str(debug["version"])
    assert "debug-bounds" not in str(normal["version"])


def test_device_check_flags_out_of_range(results):
    _, debug = results
    # (3, 10) and (0, 1) pass; (10, 10) and (-1, 10) are recorded
    assert debug["probe"].tolist() == [0, 1, 1, 0]


def test_no_check_fails_and_results_match(results):
    """A failed check would have raised PIC_ERR_BOUNDS in the runs (every step
    reads the flags); the checks change no result.  Markers (in id order),
    fields and fallback counts are compared bit for bit.  The total energy is
    compared to 1e-12: the sorts place the markers of a cell in the order their
    warps' atomics come, which decides the blocks over which the kinetic
    energy's float-pair partial sums run, so it may differ in its last bits
    from one run to the next in the same build."""
    normal, debug = results
    keys = [k for k in normal if k not in ("probe", "version")]
    assert set(keys) == {k for k in debug if k not in ("probe", "version")}
    assert len(keys) > 100
    for k in keys:
        assert normal[k].shape == debug[k].shape, k
        if k.endswith("/te"):
            rel = np.abs(normal[k] - debug[k]).max() / np.abs(normal[k]).max()
            assert rel <= 1e-12, (k, rel)
        else:
            assert np.array_equal(normal[k], debug[k]), k
    # the runs moved markers and made fields (not an all-zero comparison)
    assert np.abs(normal["em2d/o2/sort1/B"]).max() > 0
    assert np.abs(normal["es1d/o2/sort1/E"]).max() > 0
