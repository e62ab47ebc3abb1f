"""The mixed-precision form of the 1D2V spectral path (Crank-Nicolson and
PSATD, Secs. 3.4 and 4.3) against the FP64 oracle, through the C ABI.

The markers carry y as 32-bit fixed point (dx = L / 2^32), (vx, vy) as float
pairs and v* as integers (one unit is dv); shape weights are integers of 2^-23
and gather #1 runs in FP32, while the fields and their spectral solve stay
FP64.  The bars are the 1D1V mixed form's, derived from the same quanta
(tests/parity_util.mixed_bars, with dx and dv from pic_mixed_resolution): per
marker, the position within 1e-6 h + 4 steps dx and the velocity within
4 steps dv (1 + kick / |v|), the kick taking E and v x B; E and Bz within 3e-6
(they integrate the weight quanta of every deposit); fallback counts equal
(the R < 0 test is FP64); energy conserved to the FP64 bound,
max_n |TE^n - TE^0| / TE^0 <= 1e-11 without fallbacks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W
from tests.parity_util import mixed_bars

pytestmark = pytest.mark.gpu
TOL_F = 3e-6
MIXED = 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _solver(s):
    from paper_2411_09605_gb300 import pic
    return pic.PIC_SOLVER_CN_SPECTRAL if s == O.CN else pic.PIC_SOLVER_PSATD


def _oracle_run(prob, solver, scheme, nsteps):
    cfg = O.EM1DConfig(n=prob.n, L=prob.L, order=prob.order, dt=prob.dt, c=prob.c,
                       solver=solver, scheme=scheme)
    s = prob.species[0]
    sp = [O.Species1D2V(s.q, s.m, s.y.copy(), s.vx.copy(), s.vy.copy(), None, s.w0)]
    E, B = prob.E0.copy(), prob.B0.copy()
    te, _, _, fb = O.em1d_run(cfg, sp, E, B, nsteps)
    return sp[0], E, B, te, fb


def _gpu_run(prob, solver, scheme, nsteps, precision=MIXED):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation1D2V(prob, solver=_solver(solver), scheme=scheme, precision=precision)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(nsteps)
        y, vx, vy = sim.particles(0)
        E, B = sim.fields()
        energy = sim.energy()
        res = pic.pic_mixed_resolution(sim.h) if precision == MIXED else None
    finally:
        sim.close()
    return y, vx, vy, E, B, te, fb, te0, energy, res


def _diff(prob, ref, got):
    yr, vxr, vyr, Er, Br = ref
    yg, vxg, vyg, Eg, Bg = got
    dy = (yg - yr + prob.L / 2) % prob.L - prob.L / 2
    vmax = max(np.max(np.abs(vxr)), np.max(np.abs(vyr)))
    slow = np.hypot(vxr, vyr) < 0.01 * vmax
    dv = np.maximum(np.abs(vxg - vxr), np.abs(vyg - vyr))
    return {"y": np.max(np.abs(dy)) / prob.L,
            "v": np.max(dv[~slow], initial=0.0) / vmax,
            "v_slow": np.max(dv[slow], initial=0.0) / vmax,
            "E": np.linalg.norm(Eg - Er) / np.linalg.norm(Er),
            "B": np.linalg.norm(Bg - Br) / np.linalg.norm(Br)}


def _bars_vs(prob, ref, got, res, steps):
    """mixed_bars of got against ref, both (y, vx, vy, E, B)."""
    yr, vxr, vyr, Er, Br = ref
    yg, vxg, vyg = got[:3]
    dx, dv, _ = res
    sp = prob.species[0]
    vmax = max(np.max(np.abs(vxr)), np.max(np.abs(vyr)))
    Emax = max(np.max(np.abs(prob.E0)), np.max(np.abs(Er)))
    Bmax = max(np.max(np.abs(prob.B0)), np.max(np.abs(Br)))
    dy = (yg - yr + prob.L / 2) % prob.L - prob.L / 2
    b = mixed_bars(np.stack([vxr, vyr]), np.stack([vxg, vyg]), dy, prob.L / prob.n, dx, dv,
                   prob.dt, sp.q / sp.m, Emax + vmax * Bmax, steps)
    assert b["x"] <= 1.0 and b["v"] <= 1.0, b


def _check(prob, solver, scheme, steps=10):
    s, E, B, te_o, fb_o = _oracle_run(prob, solver, scheme, steps)
    y, vx, vy, Eg, Bg, te, fb, te0, energy, res = _gpu_run(prob, solver, scheme, steps)
    d = _diff(prob, (s.y, s.vx, s.vy, E, B), (y, vx, vy, Eg, Bg))
    _bars_vs(prob, (s.y, s.vx, s.vy, E, B), (y, vx, vy), res, steps)
    assert d["E"] <= TOL_F and d["B"] <= TOL_F, d
    assert np.array_equal(np.asarray(fb_o), fb), (fb_o, fb)
    if fb.sum() == 0:
        assert np.max(np.abs(te - te0)) / te0 <= 1e-11
    assert abs(energy[3] - te[-1]) <= 1e-12 * te0
    return d


@pytest.mark.parametrize("solver", [O.CN, O.PSATD])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_parity_mixed(solver, scheme, order):
    prob = W.weibel_1d2v(n=32, ppc=401, k0=0.5, b=0.02, order=order, seed=3)
    _check(prob, solver, scheme)


@pytest.mark.parametrize("drop", [1, 2, 3])
def test_ragged_marker_count_mixed(drop):
    """Marker counts that are not a multiple of four: the last group of four
    holds one to three markers and the padding (the passes move four markers a
    thread, and pass C stages them in shared memory), against the oracle."""
    prob = W.weibel_1d2v(n=32, ppc=401, k0=0.5, b=0.02, order=2, seed=9 + drop)
    s = prob.species[0]
    keep = len(s.y) - drop
    s.y, s.vx, s.vy = s.y[:keep], s.vx[:keep], s.vy[:keep]
    for solver in (O.CN, O.PSATD):
        _check(prob, solver, 2, steps=6)


@pytest.mark.parametrize("n", [4, 1024])
def test_grid_size_limits_mixed(n):
    prob = W.weibel_1d2v(n=n, ppc=max(8, 4096 // n), k0=0.5, b=0.02, order=2, seed=5)
    for solver in (O.CN, O.PSATD):
        _check(prob, solver, 2, steps=6)


def test_paper_weibel_size_mixed():
    """Sec. 5's Weibel run (32 cells, 3200 markers per cell): 10 steps against
    the oracle, then 1000 steps with the energy held to the FP64 bound."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel_1d2v(seed=0)
    _check(prob, O.PSATD, 2)
    for solver in (O.CN, O.PSATD):
        sim = pic.Simulation1D2V(prob, solver=_solver(solver), precision=MIXED)
        try:
            te0 = sim.energy()[3]
            fb, te = sim.step(1000)
        finally:
            sim.close()
        d = np.abs(np.diff(np.concatenate([[te0], te]))) / te0
        assert np.all(d[fb == 0] <= 1e-13), d.max()
        if fb.sum() == 0:
            assert np.max(np.abs(te - te0)) / te0 <= 1e-11


def test_large_run_follows_fp64_form():
    """2^22 markers, 5 steps: the mixed form against the FP64 form on the GPU."""
    prob = W.weibel_1d2v(n=32, ppc=(1 << 22) // 32, seed=6)
    a = _gpu_run(prob, O.PSATD, 2, 5, precision=0)
    b = _gpu_run(prob, O.PSATD, 2, 5)
    _bars_vs(prob, a[:5], b[:5], b[9], 5)
    d = _diff(prob, a[:5], b[:5])
    assert d["E"] <= TOL_F and d["B"] <= TOL_F, d
    assert b[6].sum() == 0 and np.max(np.abs(b[5] - b[7])) / b[7] <= 1e-11


def test_weibel_growth_rate_mixed():
    """The k0 = 2 box with symmetric velocity fours: the k0 mode of Bz grows at
    the kinetic root 0.1843 within 2% over t in [20, 40]."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel_1d2v(n=32, ppc=3200, k0=2.0, b=1e-5, mirrored=True, seed=1)
    sim = pic.Simulation1D2V(prob, solver=pic.PIC_SOLVER_PSATD, precision=MIXED)
    amp = []
    try:
        for k in range(41):
            amp.append(2 * np.abs(np.fft.rfft(sim.fields()[1])[1]) / prob.n)
            if k < 40:
                sim.step(10)
    finally:
        sim.close()
    t = np.arange(41) * 10 * prob.dt
    g = np.polyfit(t[20:], np.log(amp[20:]), 1)[0]
    assert abs(g - 0.18432) <= 0.02 * 0.18432, g


def test_state_changes_mixed():
    """pic_set_particles and pic_set_fields restart from the given state; the
    run continues as the oracle does from it."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel_1d2v(n=32, ppc=64, k0=0.5, b=0.02, order=2, seed=7)
    other = W.weibel_1d2v(n=32, ppc=64, k0=0.5, b=0.02, order=2, seed=8)
    sim = pic.Simulation1D2V(prob, solver=pic.PIC_SOLVER_PSATD, precision=MIXED)
    try:
        sim.step(3)
        s = other.species[0]
        pic.pic_set_particles(sim.h, 0, np.ascontiguousarray(s.y),
                              np.ascontiguousarray(np.stack([s.vx, s.vy])))
        pic.pic_set_fields(sim.h, np.ascontiguousarray(other.E0), np.ascontiguousarray(other.B0))
        sim.step(5)
        y, vx, vy = sim.particles(0)
        E, B = sim.fields()
        res = pic.pic_mixed_resolution(sim.h)
    finally:
        sim.close()
    r, Er, Br, _, _ = _oracle_run(other, O.PSATD, 2, 5)
    _bars_vs(other, (r.y, r.vx, r.vy, Er, Br), (y, vx, vy, E, B), res, 5)
    d = _diff(other, (r.y, r.vx, r.vy, Er, Br), (y, vx, vy, E, B))
    assert d["E"] <= TOL_F and d["B"] <= TOL_F, d


def test_input_errors_mixed():
    """Positions outside [0, L), non-finite velocities and speeds beyond the
    fixed-point range come back as status codes, at pic_init and through
    pic_set_particles."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel_1d2v(n=32, ppc=16, k0=0.5, b=0.02, seed=31)
    s = prob.species[0]
    bad = W.weibel_1d2v(n=32, ppc=16, k0=0.5, b=0.02, seed=31)
    bad.species[0].y = bad.species[0].y.copy()
    bad.species[0].y[3] = -1e-9
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation1D2V(bad, precision=MIXED)
    assert ei.value.code == -6
    sim = pic.Simulation1D2V(prob, precision=MIXED)
    try:
        y = np.ascontiguousarray(s.y)
        for v, code in ((np.stack([s.vx, np.full_like(s.vy, np.inf)]), -4),
                        (np.stack([s.vx, s.vy]) * 1000.0, -6)):
            with pytest.raises(pic.PicError) as ei:
                pic.pic_set_particles(sim.h, 0, y, np.ascontiguousarray(v))
            assert ei.value.code == code
    finally:
        sim.close()
