"""Parity of the CUDA 2D3V leapfrog / Yee path (Sec. 4.1, Eq. EMleapfrog) with the
oracle, through the C ABI.

Bar (FP64 arithmetic): after 10 steps, positions / L, velocities / max|v| and the
fields E, B (2-norm relative) within 1e-11; fallback counts identical; the
energy with W_B^n = (c^2/2)|h| sum B^{n+1/2} . B^{n-1/2} conserved to 1e-12 over
the run when no particle falls back."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _oracle(prob, scheme, steps, E0, B0):
    cfg = O.EM2DConfig(nx=prob.nx, ny=prob.ny, Lx=prob.Lx, Ly=prob.Ly, order=prob.order,
                       dt=prob.dt, c=prob.c, scheme=scheme)
    sp = [O.Species2D(s.q, s.m, s.x.copy(), s.y.copy(), s.vx.copy(), s.vy.copy(), s.vz.copy(),
                      None if s.w is None else s.w.copy(), s.w0) for s in prob.species]
    E, B = E0.copy(), B0.copy()
    te, nfb = [], []
    for _ in range(steps):
        nfb.append(sum(O.em2d_step(cfg, sp, E, B)))
        ke, we, wb = O.em2d_energy(cfg, sp, E, B)
        te.append(sum(ke) + we + wb)
    return sp, E, B, np.array(nfb), np.array(te)


def _gpu(prob, scheme, steps, E0, B0):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation2D(prob, scheme=scheme, E0=E0, B0=B0)
    try:
        fb, te = sim.step(steps)
        out = [sim.particles(s) for s in range(len(prob.species))]
        E, B = sim.fields()
        energy = sim.energy()
    finally:
        sim.close()
    return out, E, B, fb, te, energy


def _fields(prob, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    shape = (3, prob.ny, prob.nx)
    return (np.ascontiguousarray(amp * rng.standard_normal(shape)),
            np.ascontiguousarray(amp * rng.standard_normal(shape)))


def _check(prob, scheme, steps=10, seed=0):
    E0, B0 = _fields(prob, seed)
    sp, Eo, Bo, nfb_o, te_o = _oracle(prob, scheme, steps, E0, B0)
    parts, Eg, Bg, nfb_g, te_g, energy = _gpu(prob, scheme, steps, E0, B0)
    vmax = max(max(np.abs(s.vx).max(), np.abs(s.vy).max(), np.abs(s.vz).max()) for s in sp)
    for s, (x, v) in zip(sp, parts):
        for ref, got, L in ((s.x, x[0], prob.Lx), (s.y, x[1], prob.Ly)):
            d = np.abs(ref - got) % L
            assert np.max(np.minimum(d, L - d)) / L <= TOL
        for ref, got in ((s.vx, v[0]), (s.vy, v[1]), (s.vz, v[2])):
            assert np.max(np.abs(ref - got)) / vmax <= TOL
    assert np.linalg.norm(Eo - Eg) / np.linalg.norm(Eo) <= TOL
    assert np.linalg.norm(Bo - Bg) / np.linalg.norm(Bo) <= TOL
    assert np.array_equal(nfb_o, nfb_g)
    assert np.max(np.abs(te_o - te_g)) <= 1e-12 * te_o[0]
    assert abs(energy[3] - te_g[-1]) <= 1e-12 * te_o[0]
    return te_g, nfb_g


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_weibel_parity(scheme, order):
    prob = W.weibel(nx=32, ny=24, ppc=8, L=6.4, order=order, vth_par=0.1, seed=1)
    prob.Ly = 4.8
    prob.species[0].y *= 0.75
    _check(prob, scheme)


def test_two_species_weighted_parity():
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.2, seed=2)
    ions = W.weibel(nx=16, ny=16, ppc=4, L=3.2, vth_par=0.02, seed=3).species[0]
    ions.q, ions.m = 1.0, 25.0
    ions.w = np.full(len(ions.x), ions.w0) * (1.0 + 0.1 * np.cos(ions.x))
    prob.species.append(ions)
    _check(prob, 2)


def test_weibel_full_size_sampled():
    """The 128 x 128, 64-per-cell Weibel workload (1,048,576 markers), 3 steps,
    against the oracle on the same markers."""
    prob = W.weibel(seed=4)
    _check(prob, 2, steps=3)


def test_em_energy_conservation_long():
    prob = W.weibel(nx=32, ny=32, ppc=16, L=6.4, vth_par=0.1, seed=5)
    E0, B0 = _fields(prob, 6)
    _, _, _, fb, te, _ = _gpu(prob, 2, 300, E0, B0)
    assert fb.sum() == 0
    assert np.max(np.abs(te - te[0])) / te[0] <= 1e-12


def test_uniform_b_rotation():
    """E = 0, uniform Bz, one zero-weight marker: symmetric Boris rotation by
    -2 atan((q/m) B dt / 2) per step and |v| conserved (Sec. 2.2.1)."""
    import math
    prob = W.weibel(nx=8, ny=8, ppc=1, L=4.0, seed=7)
    s = prob.species[0]
    s.x, s.y = np.array([1.1]), np.array([2.3])
    s.vx, s.vy, s.vz = np.array([0.3]), np.array([-0.4]), np.array([0.25])
    s.w0 = 0.0
    prob.dt = 0.1
    B0 = np.zeros((3, 8, 8))
    B0[2] = 1.7
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation2D(prob, E0=np.zeros((3, 8, 8)), B0=B0)
    try:
        sim.step(50)
        x, v = sim.particles(0)
    finally:
        sim.close()
    th = -2.0 * math.atan(-1.0 * 1.7 * 0.1 / 2) * 50
    ref = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]) @ np.array([0.3, -0.4])
    assert np.max(np.abs(v[:2, 0] - ref)) <= 1e-13
    assert abs(np.sum(v[:, 0] ** 2) - (0.3 ** 2 + 0.4 ** 2 + 0.25 ** 2)) <= 1e-15
