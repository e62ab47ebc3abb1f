"""pic_es1d_step_noalloc, the entry point for callers that may not allocate
device memory (for example a framework that owns the whole device heap through
its own pool), must give the same result as the ordinary handle-based
pic_step on the same inputs.  Two calls in a row are checked, since every call
shares the library's one static scratch array and must clear what it reuses.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2411_09605_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _handle_run(prob, scheme, E0, steps):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, scheme=scheme, E0=E0)
    try:
        fb, te = sim.step(steps)
        x, v = sim.particles(0)
        E = sim.field()
    finally:
        sim.close()
    return x, v, E, fb, te


@pytest.mark.parametrize("scheme,order", [(2, 2), (1, 1), (2, 1)])
def test_noalloc_matches_pic_step(scheme, order):
    import torch
    from paper_2411_09605_gb300 import pic
    prob = W.two_stream(n=3 * (1 << 14) + 5, nc=256, order=order, seed=21)
    s = prob.species[0]
    # the initial field both paths start from: the handle's own Poisson solve
    sim = pic.Simulation(prob, scheme=scheme)
    E0 = sim.field()
    sim.close()

    dev = torch.device("cuda", 0)
    x = torch.from_numpy(s.x.copy()).to(dev)
    v = torch.from_numpy(s.v.copy()).to(dev)
    E = torch.from_numpy(E0.copy()).to(dev)
    cfg = pic.make_config(prob.nc, prob.L, prob.dt, order, scheme)
    done = 0
    for nsteps in (4, 7):           # two calls in a row on the shared scratch
        fb = np.zeros(nsteps, dtype=np.int64)
        te = np.zeros(nsteps)
        torch.cuda.synchronize()
        pic.pic_es1d_step_noalloc(cfg, s.q, s.m, s.w0, len(s.x), x, v, E, nsteps, fb, te)
        done += nsteps
        xr, vr, Er, fbr, ter = _handle_run(prob, scheme, E0, done)
        d = np.abs(x.cpu().numpy() - xr) % prob.L
        dx = np.max(np.minimum(d, prob.L - d)) / prob.L
        dv = np.max(np.abs(v.cpu().numpy() - vr)) / np.max(np.abs(vr))
        dE = np.linalg.norm(E.cpu().numpy() - Er) / np.linalg.norm(Er)
        assert dx <= TOL and dv <= TOL and dE <= TOL, (nsteps, dx, dv, dE)
        assert np.array_equal(fb, fbr[-nsteps:])
        assert np.max(np.abs(te - ter[-nsteps:])) <= 1e-12 * abs(ter[0])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2411_09605_gb300 import pic
    dev = torch.device("cuda", 0)
    x = torch.full((8,), 0.5, dtype=torch.float64, device=dev)
    v = torch.zeros(8, dtype=torch.float64, device=dev)
    big = pic.make_config(8193, 1.0, 0.1)
    with pytest.raises(pic.PicError) as ei:
        pic.pic_es1d_step_noalloc(big, -1.0, 1.0, 0.1, 8, x, v,
                                  torch.zeros(8193, dtype=torch.float64, device=dev), 1)
    assert ei.value.code == -1 and "8192" in str(ei.value)
    cfg = pic.make_config(16, 1.0, 0.1)
    E = torch.zeros(16, dtype=torch.float64, device=dev)
    with pytest.raises(pic.PicError) as ei:
        pic.pic_es1d_step_noalloc(cfg, -1.0, 1.0, 0.1, 8, x, v, E, 1025)
    assert ei.value.code == -1 and "1024" in str(ei.value)
    # host arrays are refused: the entry point only works on device memory
    with pytest.raises(pic.PicError) as ei:
        pic.pic_es1d_step_noalloc(cfg, -1.0, 1.0, 0.1, 8, np.full(8, 0.5), np.zeros(8),
                                  np.zeros(16), 1)
    assert ei.value.code == -1


def test_noalloc_bad_input_leaves_buffers_untouched():
    """A position outside [0, L) or a non-finite velocity or field is reported before
    any step runs, so the caller's x, v and E come back exactly as passed."""
    import torch
    from paper_2411_09605_gb300 import pic
    dev = torch.device("cuda", 0)
    prob = W.two_stream(n=1000, nc=64, seed=22)
    s = prob.species[0]
    cfg = pic.make_config(prob.nc, prob.L, prob.dt, prob.order, 2)
    E0 = np.linspace(-0.1, 0.1, prob.nc)
    cases = [("x", 17, prob.L, -6), ("x", 3, -1e-12, -6), ("v", 5, np.inf, -4),
             ("E", 9, np.nan, -4)]
    for which, idx, bad, code in cases:
        xs, vs, Es = s.x.copy(), s.v.copy(), E0.copy()
        {"x": xs, "v": vs, "E": Es}[which][idx] = bad
        x = torch.from_numpy(xs).to(dev)
        v = torch.from_numpy(vs).to(dev)
        E = torch.from_numpy(Es).to(dev)
        with pytest.raises(pic.PicError) as ei:
            pic.pic_es1d_step_noalloc(cfg, s.q, s.m, s.w0, len(xs), x, v, E, 3)
        assert ei.value.code == code, (which, ei.value)
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), xs, equal_nan=True)
        assert np.array_equal(v.cpu().numpy(), vs, equal_nan=True)
        assert np.array_equal(E.cpu().numpy(), Es, equal_nan=True)
