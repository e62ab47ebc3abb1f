"""Pins of the oracle's standard-PIC comparator (Sec. 5: Vlasov-Poisson with
the leapfrog push and binomially filtered charge density).

  * the 1-2-1 filter multiplies Fourier mode k by cos^2(pi k / nc), and the
    field of the filtered charge is the unfiltered field times that factor;
  * one marker's field: its spectral derivative (numpy) is the filtered tent
    charge minus its mean;
  * cold plasma oscillation at the leapfrog frequency (2/dt) asin(omega_p dt/2),
    not at omega_p: the time discretisation shows;
  * the linear Landau damping rate (the exact kinetic root);
  * leapfrog time reversibility (the kick at x^n, then the drift);
  * on one problem, its energy error is many orders above the
    energy-conserving scheme's."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W


def _cfg(prob, order=None):
    return O.ES1DConfig(nc=prob.nc, L=prob.L, order=order or prob.order, dt=prob.dt, scheme=2)


def _species(prob):
    return [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None if s.w is None else s.w.copy(),
                      s.w0) for s in prob.species]


def test_binomial_filter_transfer_function():
    rng = np.random.default_rng(1)
    nc = 16
    a = rng.standard_normal(nc)
    ratio = np.fft.fft(O.binomial_filter(a)) / np.fft.fft(a)
    expect = np.cos(np.pi * np.arange(nc) / nc) ** 2
    assert np.max(np.abs(ratio - expect)) <= 1e-13
    assert abs(np.fft.fft(O.binomial_filter(a))[nc // 2]) <= 1e-13


def test_field_of_filtered_charge():
    prob = W.landau(n=3000, nc=32, seed=2)
    cfg = _cfg(prob)
    sp = _species(prob)
    e0, e1 = O.std_field(cfg, sp, 0), O.std_field(cfg, sp, 1)
    k = np.arange(prob.nc)
    gain = np.cos(np.pi * k / prob.nc) ** 2
    f0, f1 = np.fft.fft(e0), np.fft.fft(e1)
    assert np.max(np.abs(f1 - gain * f0)) <= 1e-12 * np.max(np.abs(f0))


@pytest.mark.parametrize("passes", [0, 1, 2])
def test_single_marker_field(passes):
    """One electron (q = -1, weight w) at x0: tent charge on nodes i, i+1 of
    (1 - f, f) q w / h, filtered `passes` times; E' (numpy spectral
    derivative, Nyquist mode 0) equals that charge minus its mean."""
    nc, L, x0, w = 16, 5.0, 1.37, 0.3
    h = L / nc
    cfg = O.ES1DConfig(nc=nc, L=L, order=1, dt=0.1)
    sp = [O.Species(-1.0, 1.0, np.array([x0]), np.array([0.0]), np.array([w]), 0.0)]
    E = O.std_field(cfg, sp, passes)
    i, f = int(x0 // h), x0 / h - int(x0 // h)
    rho = np.zeros(nc)
    rho[i], rho[(i + 1) % nc] = -w * (1 - f) / h, -w * f / h
    for _ in range(passes):
        rho = 0.25 * (np.roll(rho, 1) + 2 * rho + np.roll(rho, -1))
    kk = 2 * np.pi * np.fft.fftfreq(nc, d=h)
    kk[nc // 2] = 0.0
    dE = np.real(np.fft.ifft(1j * kk * np.fft.fft(E)))
    target = rho - rho.mean()
    # the Nyquist component of the target has no field; compare without it
    tf = np.fft.fft(target)
    tf[nc // 2] = 0.0
    assert np.max(np.abs(dE - np.real(np.fft.ifft(tf)))) <= 1e-12 * np.max(np.abs(target))


def _cold_frequency(dt, steps):
    prob = W.cold_oscillation(n=16384, nc=128, amp=1e-4, dt=dt)
    cfg = _cfg(prob)
    sp = _species(prob)
    E = O.std_start(cfg, sp, 1)
    xh = np.arange(prob.nc) * (prob.L / prob.nc)
    amp = []
    for _ in range(steps):
        amp.append(np.dot(E, np.sin(xh)))
        O.std_step(cfg, sp, E, 1)
    amp = np.array(amp)
    t = np.arange(len(amp)) * dt
    zc = [t[i] - amp[i] * (t[i + 1] - t[i]) / (amp[i + 1] - amp[i])
          for i in range(len(amp) - 1) if amp[i] * amp[i + 1] < 0]
    return 2 * np.pi / (2 * np.mean(np.diff(zc)))


def test_cold_plasma_oscillates_at_the_leapfrog_frequency():
    """Leapfrog maps a harmonic oscillator of frequency 1 to one of frequency
    (2/dt) asin(dt/2): 1.0472 at dt = 1, 0.3% from it here (shape and filter
    factors of the 128-cell grid), and far from 1."""
    dt = 1.0
    w = _cold_frequency(dt, 300)
    expect = 2.0 / dt * math.asin(dt / 2)
    assert abs(w - expect) <= 3e-3 * expect, (w, expect)
    assert w - 1.0 > 0.03


@pytest.mark.slow
def test_landau_damping_rate():
    from scipy.special import wofz

    def eps(w, k=0.5):
        z = w / (math.sqrt(2) * k)
        return 1 + (1 + z * 1j * math.sqrt(math.pi) * wofz(z)) / k ** 2
    root = 1.4 - 0.15j
    for _ in range(60):
        f = eps(root)
        root = root - f / ((eps(root + 1e-7) - f) / 1e-7)
    prob = W.landau(n=512 * 256, nc=64, lattice_nv=256, steps=160)
    cfg = _cfg(prob)
    sp = _species(prob)
    E = O.std_start(cfg, sp, 1)
    te, we = O.std_run(cfg, sp, E, prob.steps, 1)
    t = np.arange(len(we)) * prob.dt
    pk = [i for i in range(1, len(we) - 1) if we[i] > we[i - 1] and we[i] >= we[i + 1]
          and 1.0 <= t[i] <= 16.0]
    gamma = -np.polyfit(t[pk], np.log(we[pk]), 1)[0] / 2
    assert abs(gamma + root.imag) < 0.05 * abs(root.imag), gamma


def test_leapfrog_is_time_reversible():
    """From (x^N, v^{N-1/2}, E^N), reversing v^{N+1/2} = v^{N-1/2} + dt (q/m) E^N_p
    and stepping N more times returns x^0 and -v^{1/2} (reversed step j ends at
    x^{N-j} with -v^{N-j+1/2}): the kick uses the field of the current
    positions, then the drift uses the new velocity."""
    prob = W.landau(n=4000, nc=32, alpha=0.2, seed=8, dt=0.2)
    cfg = _cfg(prob)
    sp = _species(prob)
    x0 = sp[0].x.copy()
    E = O.std_start(cfg, sp, 1)
    O.std_step(cfg, sp, E, 1)
    vm = sp[0].v.copy()                       # v^{1/2}
    for _ in range(19):
        O.std_step(cfg, sp, E, 1)
    a = O.gather_1d(cfg.order, cfg.nc, cfg.L, sp[0].x, E)
    sp[0].v[:] = -(sp[0].v + cfg.dt * (sp[0].q / sp[0].m) * a)
    for _ in range(20):
        O.std_step(cfg, sp, E, 1)
    dx = (sp[0].x - x0 + prob.L / 2) % prob.L - prob.L / 2
    assert np.max(np.abs(dx)) <= 1e-11 * prob.L
    assert np.max(np.abs(sp[0].v + vm)) <= 1e-11 * np.max(np.abs(vm))


def test_standard_pic_versus_the_energy_conserving_scheme():
    """The comparison of Sec. 5 on one problem: the standard scheme's energy
    error is many orders above the energy-conserving scheme's."""
    prob = W.two_stream(n=64 * 200, nc=64, seed=3, dt=0.05)
    cfg = _cfg(prob)
    sp = _species(prob)
    E = O.std_start(cfg, sp, 1)
    te_std, _ = O.std_run(cfg, sp, E, 300, 1)
    sp2 = _species(prob)
    E2 = O.poisson_e0_1d(cfg, sp2)
    te_ec, _, nfb = O.es1d_run(cfg, sp2, E2, 300)
    err_std = np.max(np.abs(te_std - te_std[0])) / te_std[0]
    err_ec = np.max(np.abs(te_ec - te_ec[0])) / te_ec[0]
    assert nfb.sum() == 0
    assert err_ec < 1e-12 and err_std > 1e4 * err_ec, (err_std, err_ec)
