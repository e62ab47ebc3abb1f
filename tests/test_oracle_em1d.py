"""Pins of the oracle's 1D2V electromagnetic schemes with the pseudospectral
field solve: EMEC(LI), Eq. (EMbasic), and EMEC(PSATD), Eq. (EM_PSATD).

None of these re-derives the oracle's own formulas:
  * the spectral derivative against analytic derivatives of band-limited
    fields, and its matrix (built here with numpy's FFT) antisymmetric;
  * vacuum standing waves: PSATD exact (cos(k c t)), Crank-Nicolson with its
    known phase 2 atan(k c tau / 2) per step;
  * PSATD with a fixed current against a fine Runge-Kutta integration of the
    ODE system Eq. (PSATDconstruction), including the time average <E>;
  * the Crank-Nicolson relations as residuals with an independently built
    derivative matrix;
  * test particles (negligible weight): the exact discrete gyration in a
    uniform Bz and uniform acceleration in a uniform E;
  * energy conservation per step (Eq. EM_econs, Eq. PSATDecons), and its
    loss without the Gamma correction;
  * Gamma - 1 = O(dt^3) without the half step and O(dt^4) with it;
  * the linear Weibel growth rate against the root of the kinetic dispersion
    relation for the bi-Maxwellian of Sec. 5."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W


def _dmatrix(n, L):
    """d/dy as a dense matrix from numpy's FFT (Nyquist mode of an even n -> 0)."""
    kk = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    if n % 2 == 0:
        kk[n // 2] = 0.0
    return np.real(np.fft.ifft(1j * kk[:, None] * np.fft.fft(np.eye(n), axis=0), axis=0))


@pytest.mark.parametrize("n", [15, 16])
def test_spectral_derivative(n):
    L = 3.7
    y = np.arange(n) * L / n
    rng = np.random.default_rng(n)
    f = np.zeros(n)
    df = np.zeros(n)
    for m in range(0, (n - 1) // 2 + 1):
        k = 2 * np.pi * m / L
        a, b = rng.standard_normal(2)
        f += a * np.cos(k * y) + b * np.sin(k * y)
        df += -a * k * np.sin(k * y) + b * k * np.cos(k * y)
    assert np.max(np.abs(O.spectral_deriv(n, L, f) - df)) <= 1e-12 * np.max(np.abs(df))
    if n % 2 == 0:
        # the Nyquist mode has no real derivative on the grid: it maps to 0
        assert np.max(np.abs(O.spectral_deriv(n, L, np.cos(np.pi * np.arange(n))))) <= 1e-13
    D = np.stack([O.spectral_deriv(n, L, e) for e in np.eye(n)], axis=1)
    assert np.max(np.abs(D + D.T)) <= 1e-13 * np.max(np.abs(D))
    assert np.max(np.abs(D - _dmatrix(n, L))) <= 1e-12 * np.max(np.abs(D))


@pytest.mark.parametrize("kind", [1, 2])
def test_vacuum_standing_wave(kind):
    """Ex = cos(ky), Bz = 0, no current.  The vacuum solution is
    Ex = cos(k c t) cos(ky), Bz = -sin(k c t) sin(ky) / c: PSATD follows it
    exactly; Crank-Nicolson turns the mode by 2 atan(k c tau / 2) per step
    instead of k c tau."""
    n, L, c, tau, m, steps = 16, 2 * np.pi, 0.7, 0.37, 3, 50
    cfg = O.EM1DConfig(n=n, L=L, c=c)
    y = np.arange(n) * L / n
    k = 2 * np.pi * m / L
    E = np.stack([np.cos(k * y), np.zeros(n)])
    B = np.zeros(n)
    j = np.zeros((2, n))
    for _ in range(steps):
        E, B, _ = O.em1d_field_advance(cfg, kind, tau, E, B, j)
    phase = k * c * tau * steps if kind == 2 else 2 * np.arctan(k * c * tau / 2) * steps
    assert np.max(np.abs(E[0] - np.cos(phase) * np.cos(k * y))) <= 1e-12
    assert np.max(np.abs(B + np.sin(phase) / c * np.sin(k * y))) <= 1e-12
    assert np.max(np.abs(E[1])) == 0.0


def test_psatd_is_the_exact_solution_with_fixed_current():
    """Fine RK4 of dEx/dt = c^2 D Bz - jx, dEy/dt = -jy, dBz/dt = D Ex, with the
    integral of E carried along, against PSATD(tau) and its <E>."""
    n, L, c, tau = 8, 2.3, 1.3, 0.6
    rng = np.random.default_rng(2)
    E, B, j = rng.standard_normal((2, n)), rng.standard_normal(n), rng.standard_normal((2, n))
    D = _dmatrix(n, L)

    def rhs(s):
        ex, ey, bz = s[0], s[1], s[2]
        return np.stack([c * c * D @ bz - j[0], -j[1], D @ ex, ex, ey])

    s = np.stack([E[0], E[1], B, np.zeros(n), np.zeros(n)])
    m = 4000
    h = tau / m
    for _ in range(m):
        k1 = rhs(s)
        k2 = rhs(s + 0.5 * h * k1)
        k3 = rhs(s + 0.5 * h * k2)
        k4 = rhs(s + h * k3)
        s = s + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    cfg = O.EM1DConfig(n=n, L=L, c=c)
    Eo, Bo, Ea = O.em1d_field_advance(cfg, 2, tau, E, B, j)
    scale = np.max(np.abs(s[:3]))
    assert np.max(np.abs(Eo - s[:2])) <= 1e-11 * scale
    assert np.max(np.abs(Bo - s[2])) <= 1e-11 * scale
    assert np.max(np.abs(Ea - s[3:] / tau)) <= 1e-11 * scale


def test_crank_nicolson_and_explicit_relations():
    n, L, c, tau = 12, 4.1, 0.9, 0.45
    rng = np.random.default_rng(3)
    E, B, j = rng.standard_normal((2, n)), rng.standard_normal(n), rng.standard_normal((2, n))
    D = _dmatrix(n, L)
    cfg = O.EM1DConfig(n=n, L=L, c=c)
    Eo, Bo, Ea = O.em1d_field_advance(cfg, 1, tau, E, B, j)
    Bh = 0.5 * (B + Bo)
    Eh = 0.5 * (E + Eo)
    assert np.max(np.abs(Eo[0] - E[0] - tau * (c * c * D @ Bh - j[0]))) <= 1e-13
    assert np.max(np.abs(Eo[1] - E[1] + tau * j[1])) <= 1e-13
    assert np.max(np.abs(Bo - B - tau * D @ Eh[0])) <= 1e-13
    assert np.max(np.abs(Ea - Eh)) <= 1e-15
    Ee, Be, _ = O.em1d_field_advance(cfg, 0, tau, E, B, j)
    assert np.max(np.abs(Ee[0] - E[0] - tau * (c * c * D @ B - j[0]))) <= 1e-13
    assert np.max(np.abs(Be - B - tau * D @ E[0])) <= 1e-13


def _test_particles(y, vx, vy):
    # weight 1e-30: the particles' own current changes the fields by ~1e-30
    return [O.Species1D2V(-1.0, 1.0, np.array(y, float), np.array(vx, float),
                          np.array(vy, float), None, 1e-30)]


@pytest.mark.parametrize("solver", [O.CN, O.PSATD])
@pytest.mark.parametrize("scheme", [1, 2])
def test_test_particle_gyration(solver, scheme):
    """Uniform Bz (the k = 0 mode, constant under both solvers), E = 0:
    z = vx + i vy turns by -2 atan(qm B dt/2) per step (dz/dt = -i qm B z),
    Gamma = 1, and y advances by dt Im of the mid-step velocity (z_n + z_{n+1})/2."""
    n, L, dt, Bz, steps = 16, 2 * np.pi, 0.1, 0.8, 40
    cfg = O.EM1DConfig(n=n, L=L, order=2, dt=dt, c=1.0, solver=solver, scheme=scheme)
    z0 = np.array([0.3 + 0.1j, -0.2 + 0.45j])
    sp = _test_particles([1.0, 4.0], z0.real, z0.imag)
    E, B = np.zeros((2, n)), np.full(n, Bz)
    for _ in range(steps):
        assert O.em1d_step(cfg, sp, E, B) == [0]
    qm = -1.0
    phi = -2 * np.arctan(qm * Bz * dt / 2)
    zs = z0[None, :] * np.exp(1j * phi * np.arange(steps + 1))[:, None]
    mid = 0.5 * (zs[:-1] + zs[1:])
    y = (np.array([1.0, 4.0]) + dt * mid.imag.sum(axis=0)) % L
    assert np.max(np.abs(sp[0].vx + 1j * sp[0].vy - zs[-1])) <= 1e-13
    assert np.max(np.abs(sp[0].y - y)) <= 1e-12


@pytest.mark.parametrize("solver", [O.CN, O.PSATD])
def test_test_particle_uniform_acceleration(solver):
    """Uniform E (k = 0 mode), B = 0: v_n = v_0 + n dt qm E exactly and y is
    the uniformly accelerated motion."""
    n, L, dt, steps = 16, 2 * np.pi, 0.05, 60
    cfg = O.EM1DConfig(n=n, L=L, order=1, dt=dt, c=1.0, solver=solver)
    sp = _test_particles([0.5], [0.1], [0.2])
    Ex, Ey = 0.3, -0.15
    E, B = np.stack([np.full(n, Ex), np.full(n, Ey)]), np.zeros(n)
    for _ in range(steps):
        O.em1d_step(cfg, sp, E, B)
    t = steps * dt
    qm = -1.0
    assert abs(sp[0].vx[0] - (0.1 + qm * Ex * t)) <= 1e-13
    assert abs(sp[0].vy[0] - (0.2 + qm * Ey * t)) <= 1e-13
    assert abs(sp[0].y[0] - (0.5 + 0.2 * t + 0.5 * qm * Ey * t * t) % L) <= 1e-12


def _small_weibel(order, seed=1):
    return W.weibel_1d2v(n=16, ppc=64, k0=0.5, b=0.02, order=order, seed=seed)


@pytest.mark.parametrize("solver", [O.CN, O.PSATD])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_energy_is_conserved(solver, scheme, order):
    p = _small_weibel(order)
    s = p.species[0]
    cfg = O.EM1DConfig(n=p.n, L=p.L, order=order, dt=0.2, c=p.c, solver=solver, scheme=scheme)
    sp = [O.Species1D2V(s.q, s.m, s.y.copy(), s.vx.copy(), s.vy.copy(), None, s.w0)]
    E, B = p.E0.copy(), p.B0.copy()
    te, we, wb, fb = O.em1d_run(cfg, sp, E, B, 150)
    d = np.abs(np.diff(te)) / te[0]
    assert np.all(d[fb == 0] <= 2e-14), d.max()
    if fb.sum() == 0:
        assert np.max(np.abs(te - te[0])) / te[0] <= 1e-12
    assert wb.max() > 2 * wb[0]      # the fields do change


def test_energy_drifts_without_the_correction():
    p = _small_weibel(1)
    s = p.species[0]
    cfg = O.EM1DConfig(n=p.n, L=p.L, order=1, dt=0.2, c=p.c, solver=O.CN, gamma_on=False)
    sp = [O.Species1D2V(s.q, s.m, s.y.copy(), s.vx.copy(), s.vy.copy(), None, s.w0)]
    te, _, _, _ = O.em1d_run(cfg, sp, p.E0.copy(), p.B0.copy(), 150)
    assert np.max(np.abs(te - te[0])) / te[0] > 1e-9


@pytest.mark.parametrize("solver", [O.CN, O.PSATD])
def test_gamma_order(solver):
    """RMS of Gamma - 1 over markers faster than 0.3 after one step from a
    fixed state with smooth fields: slope 3 in dt without the half step, 4
    with it (Appendix A)."""
    rng = np.random.default_rng(3)
    n, L, N = 16, 2 * np.pi, 400
    y0, vx0, vy0 = rng.uniform(0, L, N), 0.5 * rng.standard_normal(N), 0.5 * rng.standard_normal(N)
    nodes = np.arange(n) * L / n
    E0 = np.stack([0.3 * np.cos(nodes) + 0.1 * np.sin(2 * nodes), 0.2 * np.sin(nodes)])
    B0 = 0.5 + 0.3 * np.cos(nodes + 0.4)
    fast = np.hypot(vx0, vy0) > 0.3
    for scheme, slope in ((1, 3.0), (2, 4.0)):
        res = []
        for dt in (0.04, 0.02, 0.01):
            out = []
            for g in (True, False):
                cfg = O.EM1DConfig(n=n, L=L, order=2, dt=dt, solver=solver, scheme=scheme,
                                   gamma_on=g)
                sp = [O.Species1D2V(-1.0, 1.0, y0.copy(), vx0.copy(), vy0.copy(), None, L / N)]
                O.em1d_step(cfg, sp, E0.copy(), B0.copy())
                out.append(np.stack([sp[0].vx, sp[0].vy]))
            rel = np.linalg.norm(out[0] - out[1], axis=0) / np.linalg.norm(out[1], axis=0)
            res.append(np.sqrt(np.mean(rel[fast] ** 2)))
        res = np.array(res)
        slopes = np.log2(res[:-1] / res[1:])
        assert np.all(np.abs(slopes - slope) <= 0.1), (scheme, slopes)


def _weibel_root(k, beta=0.01, v0=0.3, c=1.0):
    """Purely growing root gamma of w^2 - c^2 k^2 - 1 + (<vx^2>/s^2)(1 + zeta Z(zeta))
    = 0, zeta = w / (sqrt(2) k s), s^2 = beta/2, for w = i gamma:
    zeta Z(zeta) = -sqrt(pi) y erfcx(y) with y = gamma / (sqrt(2) k s)."""
    from scipy.optimize import brentq
    from scipy.special import erfcx
    s2 = beta / 2
    a = (v0 ** 2 + s2) / s2
    sk = np.sqrt(2 * s2) * k

    def D(g):
        y = g / sk
        return -g * g - c * c * k * k - 1.0 + a * (1.0 - np.sqrt(np.pi) * y * erfcx(y))
    return brentq(D, 1e-6, 2.0)


@pytest.mark.parametrize("solver", [O.CN, O.PSATD])
def test_weibel_growth_rate(solver):
    """The Weibel setup of Sec. 5 (beta 0.01, two beams +-0.3, 32 cells, 3200
    markers per cell, dt 0.1, c 1) in a box L = pi (k0 = 2), where the seeded
    mode is the only fast-growing one; velocities in symmetric fours so that
    particle noise does not seed (Ex, Bz).  The growth of the k0 mode of Bz
    over t in [20, 40] matches the kinetic root 0.1843 within 2%."""
    pytest.importorskip("scipy")
    k0 = 2.0
    p = W.weibel_1d2v(n=32, ppc=3200, k0=k0, b=1e-5, mirrored=True, seed=1)
    s = p.species[0]
    cfg = O.EM1DConfig(n=p.n, L=p.L, order=1, dt=p.dt, c=p.c, solver=solver)
    sp = [O.Species1D2V(s.q, s.m, s.y.copy(), s.vx.copy(), s.vy.copy(), None, s.w0)]
    E, B = p.E0.copy(), p.B0.copy()
    amp = []
    for k in range(401):
        amp.append(2 * np.abs(np.fft.rfft(B)[1]) / p.n)
        if k < 400:
            O.em1d_step(cfg, sp, E, B)
    t = np.arange(401) * p.dt
    g = np.polyfit(t[200:401], np.log(amp[200:401]), 1)[0]
    theory = _weibel_root(k0)
    assert abs(theory - 0.18432) < 1e-4
    assert abs(g - theory) <= 0.02 * theory, (g, theory)
