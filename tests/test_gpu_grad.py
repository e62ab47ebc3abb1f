"""Reverse mode of the FP64 1D form on the GPU (pic_grad_forward/backward).

The GPU adjoints are held to the oracle's reverse mode (itself pinned by
central differences, tests/test_oracle_grad.py) on the same inputs and
adjoint seeds: the two forward runs agree to FP64 round-off, so the
adjoints agree to about 1e-10 relative (norm-wise) over a few steps.  The
checkpoint interval must not change the result, the handle must be left at
the state after the forward steps, the derivatives by the bump-on-tail
parameters (the seed amplitude alpha through the weights, the beam velocity
v_b through the beam markers) must match central differences of the GPU
forward, and the torch wrapper must return the same gradients."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09605_gb300 import build
    build.build()


def _small(seed, order=2, n=3000, nc=32):
    rng = np.random.default_rng(seed)
    L = 2 * np.pi
    x = rng.uniform(0, L, n)
    v = rng.standard_normal(n) + np.where(np.arange(n) % 2, 1.5, -1.5)
    w = (L / n) * (1.0 + 0.2 * rng.uniform(-1, 1, n))
    E0 = 0.05 * rng.standard_normal(nc)
    E0 -= E0.mean()
    return W.Problem1D("grad", L, nc, order, 0.1, 0, [W.Markers1D(-1.0, 1.0, x, v, w, 0.0)]), E0


def _gpu_grad(prob, scheme, E0, nsteps, every, Ebar, xbar, vbar):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, scheme=scheme, E0=E0)
    try:
        pic.pic_grad_forward(sim.h, nsteps, every)
        xf, vf = sim.particles(0)
        Ef = sim.field()
        n, nc = len(xf), len(Ef)
        out = [np.zeros(nc), np.zeros(n), np.zeros(n), np.zeros(n)]
        pic.pic_grad_backward(sim.h, Ebar, xbar, vbar, *out)
        xa, va = sim.particles(0)
        Ea = sim.field()
    finally:
        sim.close()
    return out, (xf, vf, Ef), (xa, va, Ea)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_gpu_adjoint_matches_oracle(scheme, order):
    prob, E0 = _small(10 * scheme + order, order)
    s = prob.species[0]
    nsteps = 9
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=order, dt=prob.dt, scheme=scheme)
    spf = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), s.w.copy(), 0.0)]
    Ef = E0.copy()
    O.es1d_run(cfg, spf, Ef, nsteps)
    rng = np.random.default_rng(5)
    h = prob.L / prob.nc
    Ebar, xbar, vbar = h * Ef, rng.standard_normal(len(s.x)), rng.standard_normal(len(s.x))
    Eb, xb, vb, wb = O.es1d_grad(cfg, [O.Species(s.q, s.m, s.x, s.v, s.w, 0.0)], E0, nsteps,
                                 Ebar, [xbar], [vbar])
    (gE, gx, gv, gw), (xf, vf, Ef_gpu), (xa, va, Ea) = _gpu_grad(prob, scheme, E0, nsteps, 4,
                                                                  Ebar, xbar, vbar)
    assert _rel(Ef_gpu, Ef) <= 1e-11
    assert _rel(gE, Eb) <= TOL, _rel(gE, Eb)
    assert _rel(gx, xb[0]) <= TOL, _rel(gx, xb[0])
    assert _rel(gv, vb[0]) <= TOL, _rel(gv, vb[0])
    assert _rel(gw, wb[0]) <= TOL, _rel(gw, wb[0])
    # the handle is back at the state after the forward steps
    assert np.array_equal(xa, xf) and np.array_equal(va, vf) and np.array_equal(Ea, Ef_gpu)


def test_checkpoint_interval_does_not_change_the_gradient():
    prob, E0 = _small(3)
    n = prob.n_markers
    rng = np.random.default_rng(8)
    seeds = (0.1 * rng.standard_normal(prob.nc), rng.standard_normal(n), rng.standard_normal(n))
    ref, _, _ = _gpu_grad(prob, 2, E0, 12, 12, *seeds)
    for every in (1, 5):
        got, _, _ = _gpu_grad(prob, 2, E0, 12, every, *seeds)
        for a, b in zip(got, ref):
            assert _rel(a, b) <= 1e-12


def test_bump_on_tail_parameter_derivatives():
    """L = W_E after 12 steps of a weighted bump-on-tail problem whose initial
    field is Gauss's law of its charge; dL/dalpha = sum_p wbar_p (L/N) cos(k x_p)
    + E0_bar . dE0/dalpha and dL/dv_b = sum over beam markers of vbar_p, against
    central differences of the GPU forward."""
    from paper_2411_09605_gb300 import pic
    n, nc, k, nsteps = 1 << 14, 64, 0.3, 12

    def run(alpha, vb):
        prob = W.bump_on_tail(n=n, nc=nc, k=k, alpha=alpha, vb=vb, dt=0.05, seed=4)
        sim = pic.Simulation(prob)
        try:
            pic.pic_grad_forward(sim.h, nsteps, 5)
            fb, _ = pic.pic_read_stats(sim.h)
            E = sim.field()
            h = prob.L / nc
            out = [np.zeros(nc), np.zeros(n), np.zeros(n), np.zeros(n)]
            pic.pic_grad_backward(sim.h, h * E, None, None, *out)
        finally:
            sim.close()
        # a marker switching between Gamma and its fallback makes the objective
        # jump; the comparison needs runs without fallbacks
        assert fb.sum() == 0
        return 0.5 * h * np.sum(E * E), out, prob

    a0, vb0 = 0.04, 4.5
    L0, (gE, gx, gv, gw), prob = run(a0, vb0)
    s = prob.species[0]
    rng = np.random.default_rng(4)          # the generator's draws, to mark the beam markers
    rng.random(n)
    beam = rng.random(n) < 0.1
    # alpha also moves the initial field (Gauss's law from the weighted charge,
    # linear in the weights): add E0_bar . dE0/dalpha
    cfg = O.ES1DConfig(nc=nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=2)
    dE0 = O.poisson_e0_1d(cfg, [O.Species(s.q, s.m, s.x, s.v, (prob.L / n) * np.cos(k * s.x),
                                          0.0)])
    d_alpha = np.sum(gw * (prob.L / n) * np.cos(k * s.x)) + np.dot(gE, dE0)
    d_vb = np.sum(gv[beam])
    for param, ad in (("alpha", d_alpha), ("vb", d_vb)):
        eps = 1e-6
        lp = run(a0 + eps, vb0)[0] if param == "alpha" else run(a0, vb0 + eps)[0]
        lm = run(a0 - eps, vb0)[0] if param == "alpha" else run(a0, vb0 - eps)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - ad) <= 1e-5 * abs(fd) + 1e-14 * L0, (param, fd, ad)


def test_torch_wrapper_gives_the_same_gradients():
    torch = pytest.importorskip("torch")
    from paper_2411_09605_gb300 import pic
    prob, E0 = _small(6)
    s = prob.species[0]
    sim = pic.Simulation(prob, E0=E0)
    try:
        x0 = torch.tensor(s.x, requires_grad=True)
        v0 = torch.tensor(s.v, requires_grad=True)
        e0 = torch.tensor(E0, requires_grad=True)
        w = torch.tensor(s.w, requires_grad=True)
        x, v, E = pic.differentiable_steps(sim.h, 7, x0, v0, e0, w, checkpoint_every=3)
        loss = 0.5 * (prob.L / prob.nc) * (E * E).sum() + (v * v).sum()
        gx, gv, gE, gw = torch.autograd.grad(loss, (x0, v0, e0, w))
    finally:
        sim.close()
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=2)
    spf = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), s.w.copy(), 0.0)]
    Ef = E0.copy()
    O.es1d_run(cfg, spf, Ef, 7)
    Eb, xb, vb, wb = O.es1d_grad(cfg, [O.Species(s.q, s.m, s.x, s.v, s.w, 0.0)], E0, 7,
                                 (prob.L / prob.nc) * Ef, [np.zeros(len(s.x))],
                                 [2.0 * spf[0].v])
    assert _rel(gE.numpy(), Eb) <= TOL
    assert _rel(gx.numpy(), xb[0]) <= TOL
    assert _rel(gv.numpy(), vb[0]) <= TOL
    assert _rel(gw.numpy(), wb[0]) <= TOL
