"""Empty marker sets: the degenerate case of every solver.  With no markers
the electromagnetic fields evolve in vacuum (the oracle's step with an empty
species is the reference, 1e-12), the electrostatic field stays as it is
(there is no current), and the energy is the field energy, conserved."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _empty_2d(prob):
    s = prob.species[0]
    z = np.zeros(0)
    s.x, s.y, s.vx, s.vy, s.vz = z, z.copy(), z.copy(), z.copy(), z.copy()
    return prob


@pytest.mark.parametrize("precision,cc", [(0, False), (1, False), (0, True)])
def test_yee_vacuum(precision, cc):
    from paper_2411_09605_gb300 import pic
    prob = _empty_2d(W.weibel(nx=16, ny=16, ppc=1, L=3.2, seed=1))
    rng = np.random.default_rng(2)
    E0 = np.ascontiguousarray(rng.standard_normal((3, 16, 16)))
    B0 = np.ascontiguousarray(rng.standard_normal((3, 16, 16)))
    cfg = O.EM2DConfig(nx=16, ny=16, Lx=prob.Lx, Ly=prob.Ly, order=1, dt=prob.dt, c=prob.c,
                       scheme=2, charge_conserving=cc)
    sp = [O.Species2D(-1.0, 1.0, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0),
                      np.zeros(0), None, prob.species[0].w0)]
    Eo, Bo = E0.copy(), B0.copy()
    for _ in range(20):
        O.em2d_step(cfg, sp, Eo, Bo)
    sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=precision, charge_conserving=cc)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(20)
        E, B = sim.fields()
    finally:
        sim.close()
    assert np.max(np.abs(E - Eo)) <= 1e-12 * np.max(np.abs(Eo))
    assert np.max(np.abs(B - Bo)) <= 1e-12 * np.max(np.abs(Bo))
    assert fb.sum() == 0 and np.max(np.abs(te - te0)) <= 1e-12 * te0


@pytest.mark.parametrize("solver", ["cn", "psatd"])
def test_spectral_vacuum(solver):
    from paper_2411_09605_gb300 import pic
    prob = W.weibel_1d2v(n=32, ppc=1, steps=10)
    s = prob.species[0]
    s.y, s.vx, s.vy = np.zeros(0), np.zeros(0), np.zeros(0)
    code = pic.PIC_SOLVER_CN_SPECTRAL if solver == "cn" else pic.PIC_SOLVER_PSATD
    sim = pic.Simulation1D2V(prob, solver=code)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(20)
    finally:
        sim.close()
    assert te0 > 0 and fb.sum() == 0
    assert np.max(np.abs(te - te0)) <= 1e-12 * te0


@pytest.mark.parametrize("precision", [0, 1])
def test_electrostatic_without_markers(precision):
    from paper_2411_09605_gb300 import pic
    prob = W.landau(n=1, nc=32, seed=3)
    s = prob.species[0]
    s.x, s.v = np.zeros(0), np.zeros(0)
    E0 = np.ascontiguousarray(np.sin(2 * np.pi * np.arange(32) / 32))
    sim = pic.Simulation(prob, E0=E0, precision=precision)
    try:
        fb, te = sim.step(5)
        E = sim.field()
    finally:
        sim.close()
    assert np.array_equal(E, E0) and fb.sum() == 0
    assert np.max(np.abs(te - te[0])) == 0.0
