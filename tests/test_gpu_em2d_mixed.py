"""Parity of the mixed-precision form of the 2D3V Yee path (Sec. 4.1, Eq.
EMleapfrog) with the FP64 oracle and with the FP64 form, through the C ABI.

The mixed form stores positions as 32-bit fixed point (dx = L / 2^32), v* as
an integer (one unit is dv = 1 / cxk, cxk = 2^kv dt 2^31 / L), shape weights
as integers of 2^-23 per axis and runs gather #1 (E*, B at x*) in FP32, so it
follows the oracle to its quanta, not to 1e-11.  Bars (tests/parity_util.
mixed_bars, dx and dv from pic_mixed_resolution): per marker, the position
within 1e-6 h + 4 steps dx and the velocity within 4 steps dv (1 + kick / |v|),
the kick taking E and v x B; E and B (2-norm relative) within 3e-6, since they
integrate the weight quanta of every deposit; fallback counts equal (the
R < 0 test is FP64).  Energy is conserved to the FP64 bound: runs without
imaginary-Gamma fallbacks stay within max_n |TE^n - TE^0| / TE^0 <= 1e-11."""
import math

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


def _fields(prob, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    shape = (3, prob.ny, prob.nx)
    return (np.ascontiguousarray(amp * rng.standard_normal(shape)),
            np.ascontiguousarray(amp * rng.standard_normal(shape)))


def _oracle(prob, scheme, steps, E0, B0):
    cfg = O.EM2DConfig(nx=prob.nx, ny=prob.ny, Lx=prob.Lx, Ly=prob.Ly, order=prob.order,
                       dt=prob.dt, c=prob.c, scheme=scheme)
    sp = [O.Species2D(s.q, s.m, s.x.copy(), s.y.copy(), s.vx.copy(), s.vy.copy(), s.vz.copy(),
                      None, s.w0) for s in prob.species]
    E, B = E0.copy(), B0.copy()
    nfb = []
    for _ in range(steps):
        nfb.append(sum(O.em2d_step(cfg, sp, E, B)))
    s = sp[0]
    return np.stack([s.x, s.y]), np.stack([s.vx, s.vy, s.vz]), E, B, np.array(nfb)


def _gpu(prob, scheme, steps, E0, B0, precision=MIXED):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation2D(prob, scheme=scheme, E0=E0, B0=B0, precision=precision)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(steps)
        x, v = sim.particles(0)
        E, B = sim.fields()
        energy = sim.energy()
        res = pic.pic_mixed_resolution(sim.h) if precision == MIXED else None
    finally:
        sim.close()
    return x, v, E, B, fb, te, te0, energy, res


def _bars(prob, ref, got, E0, B0, res, steps):
    (xr, vr, Er, Br), (xg, vg) = ref, got
    dx, dv, _ = res
    s = prob.species[0]
    vmax = np.max(np.abs(vr))
    Emax = max(np.max(np.abs(E0)), np.max(np.abs(Er)))
    Bmax = max(np.max(np.abs(B0)), np.max(np.abs(Br)))
    d = np.abs(xr - xg) % prob.Lx
    b = mixed_bars(vr, vg, np.minimum(d, prob.Lx - d), [prob.Lx / prob.nx, prob.Ly / prob.ny],
                   dx, dv, prob.dt, s.q / s.m, Emax + math.sqrt(3) * vmax * Bmax, steps)
    assert b["x"] <= 1.0 and b["v"] <= 1.0, b


def _diff(prob, ref, got):
    (xr, vr, Er, Br), (xg, vg, Eg, Bg) = ref, got
    d = np.abs(xr - xg) % prob.Lx
    vmax = np.max(np.abs(vr))
    slow = np.sqrt(np.sum(vr ** 2, axis=0)) < 0.01 * vmax
    dv = np.max(np.abs(vr - vg), axis=0)
    return {"x": np.max(np.minimum(d, prob.Lx - d)) / prob.Lx,
            "v": np.max(dv[~slow], initial=0.0) / vmax,
            "v_slow": np.max(dv[slow], initial=0.0) / vmax,
            "E": np.linalg.norm(Er - Eg) / np.linalg.norm(Er),
            "B": np.linalg.norm(Br - Bg) / np.linalg.norm(Br)}


def _check(prob, scheme, steps=10, seed=0):
    E0, B0 = _fields(prob, seed)
    xr, vr, Er, Br, nfb_o = _oracle(prob, scheme, steps, E0, B0)
    xg, vg, Eg, Bg, fb, te, te0, energy, res = _gpu(prob, scheme, steps, E0, B0)
    _bars(prob, (xr, vr, Er, Br), (xg, vg), E0, B0, res, steps)
    d = _diff(prob, (xr, vr, Er, Br), (xg, vg, Eg, Bg))
    assert d["E"] <= TOL_F and d["B"] <= TOL_F, d
    assert np.array_equal(nfb_o, fb), (nfb_o, fb)
    if fb.sum() == 0:
        assert np.max(np.abs(te - te0)) / te0 <= 1e-11
    assert abs(energy[3] - te[-1]) <= 1e-12 * te0
    return d


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_weibel_parity_mixed(scheme, order):
    prob = W.weibel(nx=32, ny=24, ppc=8, L=6.4, order=order, vth_par=0.1, seed=1)
    _check(prob, scheme)


def test_ragged_marker_count_mixed():
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.2, seed=2)
    s = prob.species[0]
    keep = 16 * 16 * 8 - 77
    s.x, s.y, s.vx, s.vy, s.vz = s.x[:keep], s.y[:keep], s.vx[:keep], s.vy[:keep], s.vz[:keep]
    _check(prob, 2, seed=3)


def test_weibel_full_size_mixed():
    """The 128 x 128, 64-per-cell Weibel workload (1,048,576 markers), 3 steps,
    against the oracle on the same markers."""
    _check(W.weibel(seed=4), 2, steps=3, seed=5)


def test_mixed_follows_fp64_form_full_size():
    """The mixed form against the FP64 form on the GPU, same workload, 5 steps."""
    prob = W.weibel(seed=6)
    E0, B0 = _fields(prob, 7)
    a = _gpu(prob, 2, 5, E0, B0, precision=0)
    b = _gpu(prob, 2, 5, E0, B0)
    _bars(prob, a[:4], b[:2], E0, B0, b[8], 5)
    d = _diff(prob, a[:4], b[:4])
    assert d["E"] <= TOL_F and d["B"] <= TOL_F, d
    assert np.max(np.abs(a[5] - b[5])) / a[6] <= 1e-6


@pytest.mark.parametrize("order", [1, 2])
def test_mixed_energy_conservation_long(order):
    prob = W.weibel(nx=32, ny=32, ppc=16, L=6.4, vth_par=0.1, order=order, seed=8)
    E0, B0 = _fields(prob, 9)
    _, _, _, _, fb, te, te0, _, _ = _gpu(prob, 2, 300, E0, B0)
    assert fb.sum() == 0
    assert np.max(np.abs(te - te0)) / te0 <= 1e-11


def test_mixed_uniform_b_rotation():
    """E = 0, uniform Bz, one zero-weight marker: the rotation angle of the
    exact scheme, -2 atan((q/m) B dt / 2) per step, to the FP32 rounding of
    gather #1, and |v| kept to the float pairs' precision (B does no work)."""
    prob = W.weibel(nx=8, ny=8, ppc=1, L=4.0, seed=10)
    s = prob.species[0]
    s.x, s.y = np.array([1.1]), np.array([2.3])
    s.vx, s.vy, s.vz = np.array([0.3]), np.array([-0.4]), np.array([0.25])
    s.w0 = 0.0
    prob.dt = 0.1
    B0 = np.zeros((3, 8, 8))
    B0[2] = 1.7
    x, v, *_ = _gpu(prob, 2, 50, np.zeros((3, 8, 8)), B0)
    th = -2.0 * math.atan(-1.0 * 1.7 * 0.1 / 2) * 50
    ref = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]) @ np.array([0.3, -0.4])
    assert np.max(np.abs(v[:2, 0] - ref)) <= 2e-6
    assert abs(np.sum(v[:, 0] ** 2) / (0.3 ** 2 + 0.4 ** 2 + 0.25 ** 2) - 1.0) <= 1e-13


def test_mixed_state_changes():
    """pic_set_fields keeps the markers; pic_set_particles replaces them; both
    continue like an oracle started from the new state."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.1, seed=11)
    other = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.1, seed=12)
    E0, B0 = _fields(prob, 13)
    sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED)
    try:
        sim.step(3)
        s = other.species[0]
        pic.pic_set_particles(sim.h, 0, np.ascontiguousarray(np.stack([s.x, s.y])),
                              np.ascontiguousarray(np.stack([s.vx, s.vy, s.vz])))
        pic.pic_set_fields(sim.h, E0, B0)
        sim.step(5)
        xg, vg = sim.particles(0)
        Eg, Bg = sim.fields()
        res = pic.pic_mixed_resolution(sim.h)
    finally:
        sim.close()
    xr, vr, Er, Br, _ = _oracle(other, 2, 5, E0, B0)
    _bars(other, (xr, vr, Er, Br), (xg, vg), E0, B0, res, 5)
    d = _diff(other, (xr, vr, Er, Br), (xg, vg, Eg, Bg))
    assert d["E"] <= TOL_F and d["B"] <= TOL_F, d


def test_mixed_restrictions():
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=4, L=3.2, seed=14)
    prob.Ly = 2.4
    prob.species[0].y *= 0.75
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation2D(prob, precision=MIXED)
    assert ei.value.code == -7
    prob = W.weibel(nx=16, ny=16, ppc=4, L=3.2, seed=15)
    prob.species.append(W.weibel(nx=16, ny=16, ppc=2, L=3.2, seed=16).species[0])
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation2D(prob, precision=MIXED)
    assert ei.value.code == -7


def test_input_errors_mixed():
    """Positions outside [0, L), non-finite velocities and speeds beyond the
    fixed-point range come back as status codes, at pic_init and through
    pic_set_particles."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=4, L=3.2, vth_par=0.1, seed=30)
    s = prob.species[0]
    bad = W.weibel(nx=16, ny=16, ppc=4, L=3.2, vth_par=0.1, seed=30)
    bad.species[0].x = bad.species[0].x.copy()
    bad.species[0].x[5] = prob.Lx
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation2D(bad, precision=MIXED)
    assert ei.value.code == -6
    sim = pic.Simulation2D(prob, precision=MIXED)
    try:
        x = np.ascontiguousarray(np.stack([s.x, s.y]))
        for v, code in ((np.stack([s.vx, s.vy, s.vz]) * np.array([[1.0], [1.0], [np.nan]]), -4),
                        (np.stack([s.vx, s.vy, s.vz]) * 1000.0, -6)):
            with pytest.raises(pic.PicError) as ei:
                pic.pic_set_particles(sim.h, 0, x, np.ascontiguousarray(v))
            assert ei.value.code == code
    finally:
        sim.close()


@pytest.mark.parametrize("order,scheme,period", [(1, 2, 1), (1, 1, 3), (2, 2, 2), (2, 2, 5)])
def test_quarter_cell_sort_does_not_change_the_physics(order, scheme, period):
    """The markers written in quarter-cell order by pass E every `period`
    steps, each thread's run of consecutive markers in one quarter cell summed
    in registers and the runs over the warp's lanes before the atomics: the
    currents are exact integer sums, so the run equals the unsorted one bit
    for bit (markers compared through their ids), over 12 steps."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=32, ny=32, ppc=16, L=6.4, vth_par=0.1, order=order, seed=21)
    E0, B0 = _fields(prob, 22)
    res = []
    for sp in (0, period):
        sim = pic.Simulation2D(prob, scheme=scheme, E0=E0, B0=B0, precision=MIXED,
                               sort_period=sp)
        try:
            fb, te = sim.step(12)
            x, v = sim.particles(0)
            E, B = sim.fields()
        finally:
            sim.close()
        res.append((x, v, E, B, fb, te))
    a, b = res
    for u, w in zip(a[:5], b[:5]):
        assert np.array_equal(u, w)
    assert np.max(np.abs(a[5] - b[5])) <= 1e-14 * abs(a[5][0])


def test_quarter_cell_order_after_a_sort():
    """Right after a sort the slots run in quarter-cell order and the ids are a
    permutation (bit-exact integer work)."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.05, seed=23)
    sim = pic.Simulation2D(prob, precision=MIXED, sort_period=4)
    n = prob.n_markers
    try:
        sim.step(4)   # pass E of the 4th step writes the markers in the order of x^4
        x, v = np.zeros((2, n)), np.zeros((3, n))
        pic.pic_get_particles(sim.h, 0, x, v)
        ids = np.zeros(n, dtype=np.int64)
        pic.pic_get_ids(sim.h, 0, ids)
    finally:
        sim.close()
    assert np.array_equal(np.sort(ids), np.arange(n))
    q = np.floor(2 * x[0] / (prob.Lx / 16)).astype(int) + 32 * np.floor(2 * x[1] / (prob.Ly / 16)).astype(int)
    assert np.mean(np.diff(q) >= 0) > 0.999


def test_sorted_mixed_against_oracle():
    """The sorted mode at the mixed bars against the oracle (orders 1 and 2)."""
    for order in (1, 2):
        prob = W.weibel(nx=32, ny=32, ppc=8, L=6.4, order=order, vth_par=0.1, seed=24)
        E0, B0 = _fields(prob, 25)
        xr, vr, Er, Br, nfb_o = _oracle(prob, 2, 10, E0, B0)
        from paper_2411_09605_gb300 import pic
        sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED, sort_period=2)
        try:
            fb, te = sim.step(10)
            xg, vg = sim.particles(0)
            Eg, Bg = sim.fields()
            res = pic.pic_mixed_resolution(sim.h)
        finally:
            sim.close()
        _bars(prob, (xr, vr, Er, Br), (xg, vg), E0, B0, res, 10)
        d = _diff(prob, (xr, vr, Er, Br), (xg, vg, Eg, Bg))
        assert d["E"] <= TOL_F and d["B"] <= TOL_F, d
        assert np.array_equal(nfb_o, fb)


def _truncated(prob, n):
    import dataclasses
    s = prob.species[0]
    part = dataclasses.replace(s, x=s.x[:n].copy(), y=s.y[:n].copy(), vx=s.vx[:n].copy(),
                               vy=s.vy[:n].copy(), vz=s.vz[:n].copy())
    return dataclasses.replace(prob, species=[part])


@pytest.mark.parametrize("n", [1, 5, 1037, 2047])
def test_sorted_mode_ragged_counts(n):
    """Marker counts that fill no warp, block or run of four evenly: the sorted
    mode's partial last runs and lanes without markers still give the unsorted
    run bit for bit (sorts every step and every third step)."""
    from paper_2411_09605_gb300 import pic
    prob = _truncated(W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.1, seed=31), n)
    E0, B0 = _fields(prob, 32)
    res = {}
    for sp in (0, 1, 3):
        sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED, sort_period=sp)
        try:
            fb, te = sim.step(7)
            x, v = sim.particles(0)
            E, B = sim.fields()
        finally:
            sim.close()
        res[sp] = (x, v, E, B, fb, te)
    for sp in (1, 3):
        for u, w in zip(res[0][:5], res[sp][:5]):
            assert np.array_equal(u, w), sp
        assert np.max(np.abs(res[0][5] - res[sp][5])) <= 1e-14 * abs(res[0][5][0])


def test_sorted_mode_without_ids():
    """skip_ids: the sort moves the markers without their ids (pic_get_ids then
    fails); fields, fallback counts and the set of marker states are the
    unsorted run's bit for bit."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.1, seed=33)
    E0, B0 = _fields(prob, 34)
    n = prob.n_markers
    out = []
    for sp, skip in ((0, False), (2, True)):
        sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED, sort_period=sp,
                               skip_ids=skip)
        try:
            fb, te = sim.step(6)
            x, v = np.zeros((2, n)), np.zeros((3, n))
            pic.pic_get_particles(sim.h, 0, x, v)
            E, B = sim.fields()
            if skip:
                with pytest.raises(pic.PicError):
                    pic.pic_get_ids(sim.h, 0, np.zeros(n, dtype=np.int64))
        finally:
            sim.close()
        rows = np.concatenate([x, v])
        out.append((rows[:, np.lexsort(rows[::-1])], E, B, fb))
    for u, w in zip(*out):
        assert np.array_equal(u, w)


def test_async_steps_with_energy_calls_between():
    """The mixed form reduces each step's total energy in the next step's first
    kernel (the last one when the stats are read): asynchronous steps with
    pic_energy calls in between (which use partials of their own) give the same
    per-step TE and fallbacks as one synchronous run: bit for bit on unsorted
    markers; to the float-pair kinetic sums' round-off when sorting, whose order
    within a quarter cell is not fixed."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.1, seed=35)
    E0, B0 = _fields(prob, 36)
    for sp in (0, 2):
        sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED, sort_period=sp)
        try:
            fb_ref, te_ref = sim.step(7)
        finally:
            sim.close()
        sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED, sort_period=sp)
        try:
            pic.pic_step_async(sim.h, 3)
            e_mid = sim.energy()
            pic.pic_step_async(sim.h, 1)
            sim.energy()
            pic.pic_step_async(sim.h, 3)
            fb, te = pic.pic_read_stats(sim.h)
        finally:
            sim.close()
        assert np.array_equal(fb, fb_ref), sp
        if sp == 0:
            assert np.array_equal(te, te_ref)
        else:
            assert np.max(np.abs(te - te_ref)) <= 1e-14 * abs(te_ref[0])
        # pic_energy recomputes TE from the state: step 3's, to round-off
        assert abs(e_mid[3] - te_ref[2]) <= 1e-13 * abs(te_ref[2])


def test_state_change_in_a_sorted_run():
    """pic_set_particles between steps of a sorted run (the markers arrive in
    the caller's order, the ids restart from it): the run goes on as the
    unsorted run given the same states does, bit for bit."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel(nx=16, ny=16, ppc=8, L=3.2, vth_par=0.1, seed=37)
    E0, B0 = _fields(prob, 38)
    rng = np.random.default_rng(39)
    res = []
    for sp in (0, 3):
        sim = pic.Simulation2D(prob, E0=E0, B0=B0, precision=MIXED, sort_period=sp)
        try:
            sim.step(4)
            x, v = sim.particles(0)
            # a new state in a fixed order (the same for both runs): shuffled and kicked
            order = rng.permutation(x.shape[1]) if not res else res[0][0]
            x2 = np.ascontiguousarray(x[:, order])
            v2 = np.ascontiguousarray(1.01 * v[:, order])
            pic.pic_set_particles(sim.h, 0, x2, v2)
            fb, te = sim.step(5)
            xa, va = sim.particles(0)
            E, B = sim.fields()
        finally:
            sim.close()
        res.append((order, xa, va, E, B, fb, te))
    for u, w in zip(res[0][1:6], res[1][1:6]):
        assert np.array_equal(u, w)
    assert np.max(np.abs(res[0][6] - res[1][6])) <= 1e-14 * abs(res[0][6][0])
