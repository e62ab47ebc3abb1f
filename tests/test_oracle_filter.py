"""Pins of the energy-conserving scheme with binomial filtering inside it
(Ampere uses F j, the gathers read F E; F the 1-2-1 filter, p passes).

  * energy is conserved to round-off per step (F is symmetric, so
    sum E (F j) = sum (F E) j), for 1 and 2 passes, ESEC1 and ESEC2;
  * one marker, one ESEC1 step from E = 0, computed by hand: the tent
    deposit of v at x + dt/2 v filtered by the stencil, the Ampere update, the
    gather of the filtered E^{n+1/2}, v^dag and Gamma;
  * the Nyquist mode of E never grows (the filter's purpose in Sec. 5);
  * p = 0 is the unfiltered scheme bit for bit;
  * the Landau damping rate."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W


def _species(prob):
    return [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None if s.w is None else s.w.copy(),
                      s.w0) for s in prob.species]


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_energy_conserved_with_the_filter(passes, scheme, order):
    prob = W.two_stream(n=64 * 100, nc=64, order=order, seed=5, dt=0.05)
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=order, dt=prob.dt, scheme=scheme,
                       passes=passes)
    sp = _species(prob)
    E = O.std_field(cfg, sp, passes)
    te, we, nfb = O.es1d_run(cfg, sp, E, 200)
    d = np.abs(np.diff(te)) / te[0]
    assert np.all(d[nfb == 0] <= 2e-14), d.max()
    if nfb.sum() == 0:
        assert np.max(np.abs(te - te[0])) / te[0] <= 1e-12
    assert we.max() > 10 * we[0]          # the instability does grow


def test_one_marker_by_hand():
    nc, L, dt, x0, v0, w = 8, 4.0, 0.3, 1.1, 0.7, 0.25
    h = L / nc
    cfg = O.ES1DConfig(nc=nc, L=L, order=1, dt=dt, scheme=1, passes=1)
    sp = [O.Species(-1.0, 1.0, np.array([x0]), np.array([v0]), np.array([w]), 0.0)]
    E = np.zeros(nc)
    O.es1d_step(cfg, sp, E)

    def tent(x):
        i, f = int(x // h), x / h - int(x // h)
        s = np.zeros(nc)
        s[i % nc] += 1 - f
        s[(i + 1) % nc] += f
        return s

    def filt(a):
        return 0.25 * (np.roll(a, 1) + 2 * a + np.roll(a, -1))

    # E* = E^n = 0, so v* = v0; x^{n+1/2} = x0 + dt/2 v0
    xh = x0 + 0.5 * dt * v0
    J = filt(-1.0 * w * v0 * tent(xh) / h)
    En = -dt * (J - J.mean())
    Ep = np.dot(filt(0.5 * En), tent(xh))
    vd = v0 + dt * (-1.0) * Ep
    R = v0 * v0 + 2 * v0 * (vd - v0)
    vnew = vd * math.sqrt(R) / abs(vd)
    assert np.max(np.abs(E - En)) <= 1e-15
    assert abs(sp[0].v[0] - vnew) <= 1e-15
    assert abs(sp[0].x[0] - (x0 + dt * v0)) <= 1e-15


def test_nyquist_mode_of_E_never_grows():
    prob = W.landau(n=3000, nc=32, alpha=0.2, seed=12)
    for passes, expect_zero in ((1, True), (0, False)):
        cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=1, dt=prob.dt, passes=passes)
        sp = _species(prob)
        E = np.zeros(prob.nc)
        ny = []
        for _ in range(30):
            O.es1d_step(cfg, sp, E)
            ny.append(abs(np.dot(E, np.cos(np.pi * np.arange(prob.nc)))))
        if expect_zero:
            assert max(ny) <= 1e-14 * np.max(np.abs(E)) * prob.nc
        else:
            assert max(ny) > 1e-8


def test_zero_passes_is_the_unfiltered_scheme():
    prob = W.landau(n=2000, nc=32, seed=13)
    outs = []
    for cfg in (O.ES1DConfig(nc=32, L=prob.L, passes=0), O.ES1DConfig(nc=32, L=prob.L)):
        sp = _species(prob)
        E = O.poisson_e0_1d(cfg, sp)
        O.es1d_run(cfg, sp, E, 20)
        outs.append((sp[0].x.copy(), sp[0].v.copy(), E.copy()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.slow
def test_landau_damping_rate_with_the_filter():
    from scipy.special import wofz

    def eps(w, k=0.5):
        z = w / (math.sqrt(2) * k)
        return 1 + (1 + z * 1j * math.sqrt(math.pi) * wofz(z)) / k ** 2
    root = 1.4 - 0.15j
    for _ in range(60):
        f = eps(root)
        root = root - f / ((eps(root + 1e-7) - f) / 1e-7)
    prob = W.landau(n=512 * 256, nc=64, lattice_nv=256, steps=160)
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, passes=1)
    sp = _species(prob)
    E = O.std_field(cfg, sp, 1)
    te, we, nfb = O.es1d_run(cfg, sp, E, prob.steps)
    t = np.arange(len(we)) * prob.dt
    pk = [i for i in range(1, len(we) - 1) if we[i] > we[i - 1] and we[i] >= we[i + 1]
          and 1.0 <= t[i] <= 16.0]
    gamma = -np.polyfit(t[pk], np.log(we[pk]), 1)[0] / 2
    assert abs(gamma + root.imag) < 0.05 * abs(root.imag), gamma
    assert nfb.sum() == 0 and np.max(np.abs(te - te[0])) / te[0] < 1e-12
