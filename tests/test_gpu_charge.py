"""GPU parity and properties of the charge-conserving option of the 2D3V Yee
path (Sec. 3.5, Eq. detbal), through the C ABI.

Bar (FP64 arithmetic): after 10 steps of hot markers that cross grid lines,
positions / L, velocities / max|v| and E, B (2-norm relative) within 1e-11 of
the oracle; the Gauss's-law residual div_h E - rho of the GPU's state (rho
with the bilinear shape, computed by the oracle from the GPU's markers) kept
at its initial value to 1e-12 of max|rho| over 60 steps in which every marker
changes cell; energy to 1e-12."""
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


def _hot(seed, nx=32, ny=24, ppc=8, L=6.4, vth=0.4):
    prob = W.weibel(nx=nx, ny=ny, ppc=ppc, L=L, vth_par=vth, t_ratio=2.0, seed=seed)
    prob.Ly = L * ny / nx
    prob.species[0].y *= ny / nx
    return prob


def _fields(prob, seed, amp=1e-2):
    rng = np.random.default_rng(seed)
    shape = (3, prob.ny, prob.nx)
    return (np.ascontiguousarray(amp * rng.standard_normal(shape)),
            np.ascontiguousarray(amp * rng.standard_normal(shape)))


def _cfg(prob, scheme):
    return O.EM2DConfig(nx=prob.nx, ny=prob.ny, Lx=prob.Lx, Ly=prob.Ly, order=1, dt=prob.dt,
                        c=prob.c, scheme=scheme, charge_conserving=True)


def _species(prob, x=None, v=None):
    s = prob.species[0]
    if x is None:
        x, v = np.stack([s.x, s.y]), np.stack([s.vx, s.vy, s.vz])
    return [O.Species2D(s.q, s.m, x[0].copy(), x[1].copy(), v[0].copy(), v[1].copy(),
                        v[2].copy(), None, s.w0)]


@pytest.mark.parametrize("scheme", [1, 2])
def test_charge_conserving_parity(scheme):
    from paper_2411_09605_gb300 import pic
    prob = _hot(seed=1)
    E0, B0 = _fields(prob, 2)
    cfg = _cfg(prob, scheme)
    sp = _species(prob)
    Eo, Bo = E0.copy(), B0.copy()
    nfb_o = [sum(O.em2d_step(cfg, sp, Eo, Bo)) for _ in range(10)]
    sim = pic.Simulation2D(prob, scheme=scheme, E0=E0, B0=B0, charge_conserving=True)
    try:
        fb, te = sim.step(10)
        x, v = sim.particles(0)
        Eg, Bg = sim.fields()
    finally:
        sim.close()
    s = sp[0]
    for ref, got, L in ((s.x, x[0], prob.Lx), (s.y, x[1], prob.Ly)):
        d = np.abs(ref - got) % L
        assert np.max(np.minimum(d, L - d)) / L <= TOL
    vmax = max(np.abs(s.vx).max(), np.abs(s.vy).max(), np.abs(s.vz).max())
    for ref, got in ((s.vx, v[0]), (s.vy, v[1]), (s.vz, v[2])):
        assert np.max(np.abs(ref - got)) / vmax <= TOL
    assert np.linalg.norm(Eo - Eg) / np.linalg.norm(Eo) <= TOL
    assert np.linalg.norm(Bo - Bg) / np.linalg.norm(Bo) <= TOL
    assert np.array_equal(np.array(nfb_o), fb)


def test_gauss_law_kept_on_the_gpu():
    """div_h E - rho of the GPU's own states (196,608 markers, 128 x 96 cells)."""
    from paper_2411_09605_gb300 import pic
    prob = _hot(seed=3, nx=128, ny=96, ppc=16, L=12.8)
    E0, B0 = _fields(prob, 4)
    cfg = _cfg(prob, 2)
    sim = pic.Simulation2D(prob, E0=E0, B0=B0, charge_conserving=True)
    try:
        x0, v0 = sim.particles(0)
        rho0, r0 = O.em2d_gauss_residual(cfg, _species(prob, x0, v0), E0)
        h = prob.Lx / prob.nx
        cell0 = np.floor(x0 / h)
        crossed = np.zeros(x0.shape[1], bool)
        worst = 0.0
        for _ in range(6):
            fb, te = sim.step(10)
            x, v = sim.particles(0)
            E, _ = sim.fields()
            _, r = O.em2d_gauss_residual(cfg, _species(prob, x, v), E)
            worst = max(worst, np.max(np.abs(r - r0)) / np.max(np.abs(rho0)))
            crossed |= np.any(np.floor(x / h) != cell0, axis=0)
            assert fb.sum() == 0
    finally:
        sim.close()
    assert crossed.mean() > 0.9
    assert worst <= 1e-12, worst


def test_charge_conserving_energy():
    from paper_2411_09605_gb300 import pic
    prob = _hot(seed=5)
    E0, B0 = _fields(prob, 6)
    sim = pic.Simulation2D(prob, E0=E0, B0=B0, charge_conserving=True)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(200)
    finally:
        sim.close()
    assert fb.sum() == 0
    assert np.max(np.abs(te - te0)) / te0 <= 1e-12


def test_charge_conserving_restrictions():
    from paper_2411_09605_gb300 import pic
    prob = _hot(seed=7, nx=16, ny=16, ppc=2, L=3.2)
    for kw in ({"precision": 1}, ):
        with pytest.raises(pic.PicError) as ei:
            pic.Simulation2D(prob, charge_conserving=True, **kw)
        assert ei.value.code == -7
    prob.order = 2
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation2D(prob, charge_conserving=True)
    assert ei.value.code == -7
    one = W.landau(n=1000, nc=32, seed=1)
    s = one.species[0]
    cfg = pic.make_config(32, one.L, one.dt, charge_conserving=1)
    with pytest.raises(pic.PicError) as ei:
        pic.pic_init(cfg, [dict(q=s.q, m=s.m, x=s.x, v=s.v, w=None, w0=s.w0)])
    assert ei.value.code == -7
