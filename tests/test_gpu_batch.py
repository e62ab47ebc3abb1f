"""Batched runs (one launch per pass for many independent problems).

A run stepped in a batch must follow exactly the path it follows alone: the
markers, the field and the fallback counts are bit-identical (the current is an
exact integer sum and every per-marker operation is the same), and the total
energies agree to round-off (the kinetic partial sums are blocked differently).
One run is also held to the oracle at the mixed form's bar."""
import numpy as np
import pytest

from paper_2411_09605_gb300 import workloads as W
from tests.parity_util import compare, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _problems():
    return [W.landau(n=12_345, nc=32, seed=1), W.two_stream(n=70_001, nc=512, seed=2),
            W.landau(n=200_003, nc=100, order=2, seed=3), W.two_stream(n=4096, nc=37, seed=4),
            W.landau(n=1, nc=16, seed=5), W.two_stream(n=333_333, nc=256, order=1, seed=6)]


def _alone(prob, steps):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, precision=pic.PIC_PREC_MIXED)
    try:
        fb, te = sim.step(steps)
        x, v = sim.particles(0)
        E = sim.field()
    finally:
        sim.close()
    return x, v, E, fb, te


def _batched(problems, steps, graphs=False, chunks=1):
    from paper_2411_09605_gb300 import pic
    b = pic.Batch(problems, graphs=graphs)
    try:
        fbs, tes = [], []
        for _ in range(chunks):
            fb, te = b.step(steps // chunks)
            fbs.append(fb)
            tes.append(te)
        out = [(*b.particles(r), b.field(r)) for r in range(len(problems))]
        info = pic.pic_batch_info(b.b)
    finally:
        b.close()
    return out, np.concatenate(fbs, axis=1), np.concatenate(tes, axis=1), info


def test_batch_equals_runs_alone():
    probs = _problems()
    steps = 8
    got, fb, te, (nruns, nblocks, launches) = _batched(probs, steps)
    assert nruns == len(probs) and nblocks >= len(probs)
    assert launches == 2 * steps + 2
    for r, p in enumerate(probs):
        x, v, E, fb1, te1 = _alone(p, steps)
        assert np.array_equal(got[r][0], x), r
        assert np.array_equal(got[r][1], v), r
        assert np.array_equal(got[r][2], E), r
        assert np.array_equal(fb[r], fb1), r
        assert np.max(np.abs(te[r] - te1)) <= 1e-14 * abs(te1[0]), r


def test_batch_graphs_replay_the_same_steps():
    probs = _problems()[:4]
    a, fa, ta, _ = _batched(probs, 12, graphs=False, chunks=3)
    b, fb, tb, _ = _batched(probs, 12, graphs=True, chunks=3)
    for r in range(len(probs)):
        for k in range(3):
            assert np.array_equal(a[r][k], b[r][k])
    assert np.array_equal(fa, fb)
    assert np.array_equal(ta, tb)


def test_batched_run_follows_the_oracle():
    prob = W.two_stream(n=50_000, nc=128, seed=7)
    got, _, _, _ = _batched([prob, W.landau(n=20_000, seed=8)], 10)
    ref = oracle_run(prob, 2, 10)
    d = compare(prob, ref, {"x": [got[0][0]], "v": [got[0][1]], "E": got[0][2]})
    assert d["x"] <= 1e-6 and d["v"] <= 1e-6 and d["E"] <= 3e-6, d


def test_autotune_keeps_the_runs_exact():
    """Tuning runs real steps with three work lists (4, 8 and 16 trips per
    block), switching between them; the runs and their per-step energies must be
    those of the runs stepped alone."""
    from paper_2411_09605_gb300 import pic
    probs = _problems()[:3]
    b = pic.Batch(probs)
    try:
        trips = pic.pic_batch_autotune(b.b, 2)
        assert trips in (4, 8, 16)
        fb, te = b.step(3)        # reads the 6 tuning steps and 3 more
        assert fb.shape == (3, 9)
        out = [(*b.particles(r), b.field(r)) for r in range(len(probs))]
    finally:
        b.close()
    for r, p in enumerate(probs):
        x, v, E, fb1, te1 = _alone(p, 9)
        assert np.array_equal(out[r][0], x) and np.array_equal(out[r][1], v), r
        assert np.array_equal(out[r][2], E), r
        assert np.array_equal(fb[r], fb1), r
        assert np.max(np.abs(te[r] - te1)) <= 1e-14 * abs(te1[0]), r


def _small_problems():
    """Runs of at most 2^15 markers: the batch runs 256-thread blocks."""
    return [W.landau(n=1_000, nc=32, seed=11), W.two_stream(n=32_768, nc=64, seed=12),
            W.landau(n=5_003, nc=47, order=2, seed=13), W.two_stream(n=1, nc=16, seed=14),
            W.landau(n=17_777, nc=512, seed=15), W.two_stream(n=2_048, nc=33, order=1, seed=16)]


def test_small_run_batch_equals_runs_alone():
    """The 256-thread layout of batches of small runs (8 tile copies, a copy
    taking at most 2048 markers a launch as in the 1024-thread layout): the
    runs follow their single-run paths bit for bit, with graph replay and with
    every trip target of the autotuner."""
    from paper_2411_09605_gb300 import pic
    probs = _small_problems()
    steps = 8
    got, fb, te, (nruns, nblocks, launches) = _batched(probs, steps)
    assert nruns == len(probs) and nblocks >= len(probs)
    alone = [_alone(p, steps) for p in probs]
    for r in range(len(probs)):
        x, v, E, fb1, te1 = alone[r]
        assert np.array_equal(got[r][0], x), r
        assert np.array_equal(got[r][1], v), r
        assert np.array_equal(got[r][2], E), r
        assert np.array_equal(fb[r], fb1), r
        assert np.max(np.abs(te[r] - te1)) <= 1e-14 * abs(te1[0]), r
    g, fg, tg, _ = _batched(probs, 8, graphs=True, chunks=2)
    for r in range(len(probs)):
        for k in range(3):
            assert np.array_equal(g[r][k], got[r][k]), r
    b = pic.Batch(probs)
    try:
        assert pic.pic_batch_autotune(b.b, 2) in (4, 8, 16)
        fb8, _ = b.step(2)
        out = [(*b.particles(r), b.field(r)) for r in range(len(probs))]
    finally:
        b.close()
    for r, p in enumerate(probs):
        x, v, E, fb1, _ = _alone(p, 8)
        assert np.array_equal(out[r][0], x) and np.array_equal(out[r][2], E), r
        assert np.array_equal(fb8[r], fb1), r


def test_small_run_batch_follows_the_oracle():
    prob = W.two_stream(n=20_000, nc=128, seed=17)
    got, _, _, _ = _batched([prob, W.landau(n=3_000, seed=18)], 10)
    ref = oracle_run(prob, 2, 10)
    d = compare(prob, ref, {"x": [got[0][0]], "v": [got[0][1]], "E": got[0][2]})
    assert d["x"] <= 1e-6 and d["v"] <= 1e-6 and d["E"] <= 3e-6, d
