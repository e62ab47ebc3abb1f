"""GPU parity of the energy-conserving FP64 1D scheme with binomial filtering
inside it (binomial_passes > 0: Ampere uses F j, the gathers F E), against the
oracle, and its energy conservation.  The initial field is Gauss's law of the
filtered charge on both sides."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W
from tests.parity_util import compare

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
