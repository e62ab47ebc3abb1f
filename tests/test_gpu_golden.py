"""The GPU path, through the C ABI, at the parameters the paper prints for its
tests (Sec. 5), against the outcomes it reports there; both are read from
tests/golden/paper_tests.txt.  Sec. 5.1 and 5.2 are restated in 1D1V with the
paper's box, cells, markers per cell, thermal spread and time step (what
carries over to 1D is explained in test_golden_paper.py); Sec. 5.3 runs at
the paper's size.  Both forms of each solver."""
import numpy as np
import pytest

from paper_2411_09605_gb300 import workloads as W
from tests.parity_util import paper_values

pytestmark = pytest.mark.gpu
P = paper_values()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _run(prob, steps, **kw):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, **kw)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(steps)
    finally:
        sim.close()
    return np.max(np.abs(te - te0)) / te0, fb


def _landau_paper(seed):
    cells = int(P["landau.cells"])
    return W.landau(n=cells * int(P["landau.ppc"]), nc=cells, k=2 * np.pi / P["landau.L"],
                    alpha=P["landau.alpha"], vth=P["landau.vth"], dt=P["landau.dt"], seed=seed)


@pytest.mark.parametrize("precision", [0, 1])
def test_landau_at_paper_parameters(precision):
    """Sec. 5.1 at its printed parameters, 500 steps (t = 50): no imaginary Gamma
    for ESEC2 at this time step, and the energy within the abstract's 1e-12
    (FP64 form) or within 1e-11 (mixed form).
    In 1D a velocity passes through zero far more often than |v| does in 2D, so
    the FP64 oracle itself sees a rare ESEC2 fallback on some seeds (0 to 4 in
    500 steps over seeds 1..20; 0 on seed 1, which the FP64 form follows
    exactly).  Past the first steps the mixed form's trajectory departs from
    the FP64 one (the run is chaotic), so its count is held to the oracle's
    range over seeds 1..5 instead of to the seed's own count."""
    from tests.parity_util import oracle_run
    prob = _landau_paper(1)
    err, fb = _run(prob, 500, precision=precision)
    if precision == 0:
        assert fb.sum() == P["landau.esec2_fallbacks"]
    else:
        counts = [int(oracle_run(_landau_paper(sd), 2, 500)["nfb"].sum()) for sd in range(1, 6)]
        assert fb.sum() <= max(counts), (fb.sum(), counts)
    assert err <= (P["energy_error_order"] if precision == 0 else 10 * P["energy_error_order"])


def test_two_stream_against_standard_pic():
    """Sec. 5.2 at its printed parameters, 600 steps (past saturation): the
    energy error of ESEC2 (FP64 form) at least the printed 8 orders of
    magnitude below the standard scheme's."""
    from paper_2411_09605_gb300 import pic
    cells = int(P["two_stream.cells"])
    prob = W.two_stream(n=cells * int(P["two_stream.ppc"]), nc=cells,
                        k=2 * np.pi / P["two_stream.L"], v0=P["two_stream.vb"],
                        vth=P["two_stream.vth"], alpha=P["two_stream.alpha"],
                        dt=P["two_stream.dt"], order=1, seed=1)
    err_ec, _ = _run(prob, 600)
    sim = pic.Simulation(prob, solver=pic.PIC_SOLVER_STANDARD_LEAPFROG, binomial_passes=1)
    try:
        _, te_std = sim.step(600)
    finally:
        sim.close()
    err_std = np.max(np.abs(te_std - te_std[0])) / te_std[0]
    assert err_ec * 10 ** P["two_stream.esec2_orders_below_standard"] <= err_std, (err_ec, err_std)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("solver", ["cn", "psatd"])
def test_weibel_at_paper_parameters(solver, precision):
    """Sec. 5.3 at its printed parameters and size (102,400 markers), 300
    steps: the printed 11 digits of energy, imaginary Gamma extremely rare."""
    from paper_2411_09605_gb300 import pic
    prob = W.weibel_1d2v(n=int(P["weibel.cells"]), ppc=int(P["weibel.ppc"]), k0=P["weibel.k0"],
                         beta=P["weibel.beta"], delta=P["weibel.delta"], v01=P["weibel.v01"],
                         v02=P["weibel.v02"], b=P["weibel.b"], dt=P["weibel.dt"],
                         c=P["weibel.c"], seed=2)
    assert len(prob.species[0].y) == P["weibel.markers"]
    code = pic.PIC_SOLVER_CN_SPECTRAL if solver == "cn" else pic.PIC_SOLVER_PSATD
    sim = pic.Simulation1D2V(prob, solver=code, precision=precision)
    try:
        te0 = sim.energy()[3]
        fb, te = sim.step(300)
    finally:
        sim.close()
    assert np.max(np.abs(te - te0)) / te0 <= 10.0 ** -P["weibel.energy_digits"]
    assert fb.sum() <= 1e-5 * P["weibel.markers"] * 300
