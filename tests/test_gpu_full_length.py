"""The configurations at their full length on the GPU.

* Two-stream, 2^23 markers, 512 cells, quadratic shapes, 2000 steps (through
  saturation), mixed and FP64 forms: every step in which no marker falls back
  changes TE by round-off only (Eq. exp_econs_simple); the fallbacks of the
  saturated phase (Gamma's radicand negative near v = 0) are of the same order
  in both forms.
* Weibel 2D3V, 128 x 128 cells, 1,048,576 markers, 4000 steps (t = 141),
  mixed and FP64 forms: the same per-step energy property, and the instability
  turns part of the anisotropic thermal energy into magnetic energy (W_B grows
  from the markers' noise to well above it)."""
import numpy as np
import pytest

from paper_2411_09605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _run_1d(prob, precision, steps):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, precision=precision)
    try:
        te0 = sim.energy()[3]
        fbs, tes = [], []
        for _ in range(steps // 500):
            fb, te = sim.step(500)
            fbs.append(fb)
            tes.append(te)
    finally:
        sim.close()
    return te0, np.concatenate(fbs), np.concatenate(tes)


def _per_step(te0, fb, te):
    d = np.abs(np.diff(np.concatenate([[te0], te]))) / te0
    return d[fb == 0]


def test_two_stream_full_size_2000_steps():
    prob = W.two_stream(seed=0)
    res = {}
    for precision in (0, 1):
        te0, fb, te = _run_1d(prob, precision, 2000)
        clean = _per_step(te0, fb, te)
        assert (fb[:150] == 0).all()                   # linear phase: no fallback
        # round-off per step; the mixed form's saturated phase has many markers
        # on the FP32 branch of Gamma (|t| >= 2^-8, relative error 2^-24 of t)
        assert np.max(clean) <= (1e-13 if precision == 0 else 2e-13), (precision, np.max(clean))
        res[precision] = fb.sum()
    # the same physics in both forms: fallback counts of the same order
    assert 0.5 <= res[1] / max(res[0], 1) <= 2.0, res


@pytest.mark.parametrize("precision", [0, 1])
def test_weibel_2d_4000_steps(precision):
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(seed=0)
    sim = pic.Simulation2D(prob, precision=precision)
    try:
        te0 = sim.energy()[3]
        fbs, tes, wb = [], [], []
        for _ in range(8):
            fb, te = sim.step(500)
            fbs.append(fb)
            tes.append(te)
            wb.append(sim.energy()[2])
    finally:
        sim.close()
    fb, te = np.concatenate(fbs), np.concatenate(tes)
    clean = _per_step(te0, fb, te)
    assert np.max(clean) <= 1e-13, np.max(clean)
    if fb.sum() == 0:
        assert np.max(np.abs(te - te0)) / te0 <= 1e-11
    # W_B after 500 steps (t = 18) is still near the noise; the instability
    # (growth rate of order 0.1 here) lifts it by orders of magnitude by t = 141
    assert wb[-1] > 100 * wb[0], wb
