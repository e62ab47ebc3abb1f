"""GPU parity of the energy-conserving 1D scheme with binomial filtering inside
it (binomial_passes > 0: Ampere uses F j, the gathers F E), against the
oracle, and its energy conservation, in the FP64 form (to 1e-11) and in the
mixed form (to its quanta, tests/parity_util.mixed_bars).  The initial field
is Gauss's law of the filtered charge on both sides."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W
from tests.parity_util import compare, mixed_bars, periodic_dist

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _oracle(prob, scheme, passes, steps):
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=scheme,
                       passes=passes)
    sp = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None if s.w is None else s.w.copy(), s.w0)
          for s in prob.species]
    E = O.std_field(cfg, sp, passes)
    E0 = E.copy()
    te, we, nfb = O.es1d_run(cfg, sp, E, steps)
    return dict(x=[s.x for s in sp], v=[s.v for s in sp], E=E, nfb=nfb, te=te, E0=E0)


def _gpu(prob, scheme, passes, steps):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, scheme=scheme, binomial_passes=passes)
    try:
        E0 = sim.field()
        te0 = sim.energy()[3]
        fb, te = sim.step(steps)
        xs, vs = [], []
        for s in range(len(prob.species)):
            x, v = sim.particles(s)
            xs.append(x)
            vs.append(v)
        E = sim.field()
    finally:
        sim.close()
    return dict(x=xs, v=vs, E=E, nfb=fb, te=np.concatenate([[te0], te]), E0=E0)


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_filtered_parity(order, scheme, passes):
    prob = W.two_stream(n=40_009, nc=128, order=order, seed=order + 2 * scheme + 5 * passes)
    ref = _oracle(prob, scheme, passes, 10)
    got = _gpu(prob, scheme, passes, 10)
    assert np.linalg.norm(got["E0"] - ref["E0"]) <= TOL * np.linalg.norm(ref["E0"])
    d = compare(prob, ref, got)
    assert d["x"] <= TOL and d["v"] <= TOL and d["E"] <= TOL, d
    assert np.array_equal(got["nfb"], ref["nfb"])
    assert np.max(np.abs(got["te"] - ref["te"])) <= TOL * ref["te"][0]


def test_filtered_energy_over_a_long_run():
    from paper_2411_09605_gb300 import pic
    prob = W.two_stream(n=1 << 20, nc=512, seed=3)
    sim = pic.Simulation(prob, binomial_passes=1)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(400)
    finally:
        sim.close()
    d = np.abs(np.diff(np.concatenate([[te0], te]))) / te0
    assert np.all(d[fb == 0] <= 1e-13)
    if fb.sum() == 0:
        assert np.max(np.abs(te - te0)) / te0 <= 1e-11


def test_filter_declined_where_not_built():
    from paper_2411_09605_gb300 import pic
    prob = W.landau(n=1000, seed=1)
    sim = pic.Simulation(prob, binomial_passes=1)
    try:
        with pytest.raises(pic.PicError) as ei:
            pic.pic_grad_forward(sim.h, 2, 1)
        assert ei.value.code == -7
    finally:
        sim.close()


def _mixed(prob, scheme, passes, steps, E0=None, sort_period=0):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, scheme=scheme, precision=1, binomial_passes=passes, E0=E0,
                         sort_period=sort_period)
    try:
        E_init = sim.field()
        te0 = sim.energy()[3]
        fb, te = sim.step(steps)
        x, v = sim.particles(0)
        E = sim.field()
        res = pic.pic_mixed_resolution(sim.h)
    finally:
        sim.close()
    return dict(x=[x], v=[v], E=E, nfb=fb, te=np.concatenate([[te0], te]), E0=E_init,
                resolution=res)


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_filtered_mixed_parity(order, scheme, passes):
    """The mixed form with the filter against the oracle's filtered scheme from
    the same initial field: markers within the mixed bars, E within 3e-6,
    fallback counts equal; TE kept to round-off on steps without fallbacks."""
    prob = W.two_stream(n=40_009, nc=128, order=order, seed=order + 2 * scheme + 5 * passes)
    ref = _oracle(prob, scheme, passes, 10)
    got = _mixed(prob, scheme, passes, 10, E0=ref["E0"])
    dx, dv, _ = got["resolution"]
    s = prob.species[0]
    Emax = max(np.max(np.abs(ref["E0"])), np.max(np.abs(ref["E"])))
    b = mixed_bars(ref["v"][0], got["v"][0], periodic_dist(ref["x"][0], got["x"][0], prob.L),
                   prob.L / prob.nc, dx, dv, prob.dt, s.q / s.m, Emax, 10)
    assert b["x"] <= 1.0 and b["v"] <= 1.0, b
    assert compare(prob, ref, got)["E"] <= 3e-6
    assert np.array_equal(got["nfb"], ref["nfb"])
    d = np.abs(np.diff(got["te"])) / got["te"][0]
    assert np.all(d[got["nfb"] == 0] <= 1e-13), d


def test_filtered_mixed_initial_field():
    """Without E0 the mixed form solves Gauss's law of the filtered charge of
    its own quantised weights: the oracle's filtered field to the weights'
    2^-23."""
    prob = W.two_stream(n=40_009, nc=128, order=2, seed=11)
    for passes in (1, 3):
        ref = _oracle(prob, 2, passes, 0)
        got = _mixed(prob, 2, passes, 1)
        assert np.linalg.norm(got["E0"] - ref["E0"]) <= 1e-6 * np.linalg.norm(ref["E0"])


def test_filtered_mixed_energy_long_and_sorted():
    """1e6 markers, 300 steps with two filter passes: per-step TE changes on
    steps without fallbacks at round-off; the cell-sorted modes give the
    unsorted run bit for bit (exact integer currents)."""
    prob = W.two_stream(n=1 << 20, nc=512, seed=13)
    res = {}
    for sp in (0, 1, 4):
        got = _mixed(prob, 2, 2, 300 if sp == 0 else 20, sort_period=sp)
        res[sp] = got
    d = np.abs(np.diff(res[0]["te"])) / res[0]["te"][0]
    assert np.all(d[res[0]["nfb"] == 0] <= 1e-13), np.max(d)
    short = _mixed(prob, 2, 2, 20)
    for sp in (1, 4):
        for key in ("x", "v"):
            assert np.array_equal(short[key][0], res[sp][key][0]), (sp, key)
        assert np.array_equal(short["E"], res[sp]["E"]) and np.array_equal(short["nfb"], res[sp]["nfb"])
