"""ESEC1 in one launch per step (mixed 1D1V form, unsorted markers): the update
of step n fused with the push and deposit of step n+1 (Eq. naivetranslation
has no j^{n,*}, so no grid quantity lies between them).  It must give the
two-launch form's markers, field and fallback counts bit for bit, across
calls, restarts (pic_set_particles / pic_set_fields) and the asynchronous
interface, and meet the oracle at the mixed bars.  The per-step energies agree
to 1e-12: the fused pass runs 768-thread blocks and the two-launch form
1024-thread ones, so the float-pair partial sums of the kinetic energy run
over different markers (each a float-pair sum of about 2^-46 relative error
per term); two runs of one form give the same bits."""


def _same_energies(a, b):
    return np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
import numpy as np
import pytest

from paper_2411_09605_gb300 import workloads as W
from tests.parity_util import compare, gpu_run, mixed_bars, oracle_run, periodic_dist

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _run(prob, separate, chunks, restart_at=None):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, scheme=1, precision=1, separate_passes=separate)
    fbs, tes = [], []
    try:
        for k, n in enumerate(chunks):
            if restart_at is not None and k == restart_at:
                x, v = sim.particles(0)
                E = sim.field()
                pic.pic_set_particles(sim.h, 0, x, v)
                pic.pic_set_fields(sim.h, E)
            fb, te = sim.step(n)
            fbs.append(fb)
            tes.append(te)
        x, v = sim.particles(0)
        E = sim.field()
        energy = sim.energy()
        launches = pic.pic_launch_count(sim.h)
    finally:
        sim.close()
    return x, v, E, np.concatenate(fbs), np.concatenate(tes), energy, launches


@pytest.mark.parametrize("order,nc", [(1, 64), (2, 512), (2, 2048)])
def test_fused_equals_two_launches(order, nc):
    prob = W.landau(n=50_003, nc=nc, order=order, seed=30, dt=0.2)
    a = _run(prob, True, [7, 5, 1])
    b = _run(prob, False, [7, 5, 1])
    for u, w in zip(a[:4], b[:4]):
        assert np.array_equal(u, w)
    assert _same_energies(a[4], b[4])          # per-step energies
    assert a[3].sum() > 0                      # ESEC1 at dt = 0.2 falls back on some markers
    # one launch per step (plus one pass C after each start) against two
    assert b[6] < a[6]


def test_fused_marker_bound_of_both_block_sizes():
    """At 9,806,432 markers on 152 SMs a tile copy of a 768-thread block takes
    22 trips of 96 markers (2112), more than a 1024-thread block's 16 trips of
    128 (2048): the handle's bound covers both block sizes (one more bit in
    the counters' split), and the fused and two-launch forms still agree."""
    import torch
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the marker count is chosen for 152 SMs")
    prob = W.two_stream(n=9_806_432, nc=512, order=2, seed=33)
    a = _run(prob, True, [2, 1])
    b = _run(prob, False, [2, 1])
    for u, w in zip(a[:4], b[:4]):
        assert np.array_equal(u, w)
    assert _same_energies(a[4], b[4])


def test_fused_restart_and_async():
    """A restart drops the pending push of the next step and redoes it; the
    asynchronous interface reads the same stats."""
    from paper_2411_09605_gb300 import pic
    prob = W.two_stream(n=70_001, nc=256, order=2, seed=31)
    a = _run(prob, True, [4, 6], restart_at=1)
    b = _run(prob, False, [4, 6], restart_at=1)
    for u, w in zip(a[:4], b[:4]):
        assert np.array_equal(u, w)
    assert _same_energies(a[4], b[4])
    sim = pic.Simulation(prob, scheme=1, precision=1)
    try:
        pic.pic_step_async(sim.h, 3)
        pic.pic_step_async(sim.h, 7)
        fb, te = pic.pic_read_stats(sim.h)
        x, v = sim.particles(0)
    finally:
        sim.close()
    assert np.array_equal(te, b[4]) and np.array_equal(fb, a[3])


@pytest.mark.parametrize("prob_fn", [lambda: W.landau(n=20_000, order=1, seed=1),
                                     lambda: W.two_stream(n=3 * (1 << 15) + 77, nc=512, seed=2)])
def test_fused_esec1_against_oracle(prob_fn):
    prob = prob_fn()
    ref = oracle_run(prob, 1, 10)
    got = gpu_run(prob, 1, 10, precision=1)
    dx, dv, _ = got["resolution"]
    s = prob.species[0]
    Emax = max(np.max(np.abs(ref["E0"])), np.max(np.abs(ref["E"])))
    b = mixed_bars(ref["v"][0], got["v"][0], periodic_dist(ref["x"][0], got["x"][0], prob.L),
                   prob.L / prob.nc, dx, dv, prob.dt, s.q / s.m, Emax, 10)
    assert b["x"] <= 1.0 and b["v"] <= 1.0, b
    assert compare(prob, ref, got)["E"] <= 3e-6
    assert np.array_equal(ref["nfb"], got["nfb"])
