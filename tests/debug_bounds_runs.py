"""Short runs of every mixed-form kernel family, stepped through the library
that pic.lib() loads (the normal build, or the debug-bounds build when the
environment sets PIC_DEBUG_BOUNDS=1), saved to an .npz file.

Run as ``python tests/debug_bounds_runs.py OUT.npz``; the GPU test compares
the files of the two builds.  Every run is seeded and small (several tiles
and blocks, ragged marker counts); together they form every index the checks
of the debug build cover: the shapes of both orders, unsorted markers, the
sort kernels (sort period > 1), sort on write (period 1 in 1D, every period
in 2D), the filtered form, the batches of both block sizes and the 1D
spectral solvers' mixed form.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2411_09605_gb300 import pic  # noqa: E402
from paper_2411_09605_gb300 import workloads as W  # noqa: E402

MIXED = pic.PIC_PREC_MIXED


def _es1d(out, tag, prob, steps, **kw):
    sim = pic.Simulation(prob, precision=MIXED, **kw)
    fb, te = sim.step(steps)
    x, v = sim.particles()
    out[tag + "/x"], out[tag + "/v"], out[tag + "/E"] = x, v, sim.field()
    out[tag + "/fb"], out[tag + "/te"] = fb, te
    sim.close()


def _em2d(out, tag, prob, steps, **kw):
    sim = pic.Simulation2D(prob, precision=MIXED, **kw)
    fb, te = sim.step(steps)
    x, v = sim.particles()
    E, B = sim.fields()
    out[tag + "/x"], out[tag + "/v"], out[tag + "/E"], out[tag + "/B"] = x, v, E, B
    out[tag + "/fb"], out[tag + "/te"] = fb, te
    sim.close()


def _em1d(out, tag, prob, steps, solver):
    sim = pic.Simulation1D2V(prob, solver=solver, precision=MIXED)
    fb, te = sim.step(steps)
    y, vx, vy = sim.particles()
    E, B = sim.fields()
    out[tag + "/y"], out[tag + "/vx"], out[tag + "/vy"] = y, vx, vy
    out[tag + "/E"], out[tag + "/B"], out[tag + "/fb"], out[tag + "/te"] = E, B, fb, te
    sim.close()


def _batch(out, tag, probs, steps):
    b = pic.Batch(probs)
    fb, te = b.step(steps)
    out[tag + "/fb"], out[tag + "/te"] = fb, te
    for r in range(len(probs)):
        x, v = b.particles(r)
        out[f"{tag}/{r}/x"], out[f"{tag}/{r}/v"], out[f"{tag}/{r}/E"] = x, v, b.field(r)
    b.close()


def run_all() -> dict:
    out = {}
    for order in (1, 2):
        prob = W.landau(n=50_001, nc=64, order=order, seed=order)
        for sp in (0, 1, 4):
            _es1d(out, f"es1d/o{order}/sort{sp}", prob, 12, sort_period=sp)
        _es1d(out, f"es1d/o{order}/esec1", prob, 12, scheme=pic.PIC_SCHEME_ESEC1)
        _es1d(out, f"es1d/o{order}/filter2", prob, 12, binomial_passes=2)
    ts = W.two_stream(n=40_003, nc=512, order=2, seed=3)
    _es1d(out, "es1d/two_stream/sort1", ts, 12, sort_period=1)
    for order in (1, 2):
        prob = W.weibel(nx=32, ny=24, ppc=20, order=order, seed=order)
        for sp in (0, 1, 3):
            _em2d(out, f"em2d/o{order}/sort{sp}", prob, 8, sort_period=sp)
    p12 = W.weibel_1d2v(n=32, ppc=400, seed=5)
    _em1d(out, "em1d/psatd", p12, 10, pic.PIC_SOLVER_PSATD)
    _em1d(out, "em1d/cn", p12, 10, pic.PIC_SOLVER_CN_SPECTRAL)
    # batches: all runs <= 2^15 markers (256-thread blocks), then larger runs
    small = W.ensemble(nruns=6, seed=7, n_min=2e3, n_max=2e4, nc_min=32, nc_max=256)
    _batch(out, "batch/small", small, 8)
    large = W.ensemble(nruns=3, seed=8, n_min=5e4, n_max=1.2e5, nc_min=64, nc_max=512)
    _batch(out, "batch/large", large, 8)
    # the device-side check itself (debug build): passes in range, records outside
    version = pic.pic_version()
    probes = ((3, 10), (10, 10), (-1, 10), (0, 1))
    if "debug-bounds" in version:
        out["probe"] = np.array([pic.pic_debug_bounds(i, n) for i, n in probes])
    else:
        out["probe"] = np.full(len(probes), -1)
    out["version"] = np.array(version)
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_all())
