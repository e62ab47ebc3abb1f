"""Pins of the oracle's reverse mode (orc_es1d_grad) by central differences of
the oracle's own forward run: for random directions (dx, dv, dw, dE) in the
initial state, <gradient, direction> must equal
(L(state + eps dir) - L(state - eps dir)) / (2 eps) for the objective
L = W_E(final) + sum_p (a_p x_p + b_p v_p)(final) with random a, b.  A dropped
term, a wrong sign or a transposed gather/deposit in the reverse pass breaks
the agreement by far more than the O(eps^2) truncation."""
import numpy as np
import pytest

from oracle import oracle as O


def _problem(order, seed, n=48, nc=16, weighted=True, vscale=1.0):
    rng = np.random.default_rng(seed)
    L = 2 * np.pi
    x = rng.uniform(0, L, n)
    v = vscale * (rng.standard_normal(n) + np.where(np.arange(n) % 2, 1.5, -1.5))
    w = (L / n) * (1.0 + 0.2 * rng.uniform(-1, 1, n)) if weighted else None
    E0 = 0.05 * rng.standard_normal(nc)
    E0 -= E0.mean()
    return L, x, v, w, E0


def _objective(cfg, L, x, v, w, E0, a, b, nsteps, w0):
    sp = [O.Species(-1.0, 1.0, x.copy(), v.copy(), None if w is None else w.copy(), w0)]
    E = E0.copy()
    O.es1d_run(cfg, sp, E, nsteps)
    h = L / cfg.nc
    xf = sp[0].x.copy()
    # the periodic wrap makes x^N jump by L where a marker crosses the boundary:
    # measure the final positions relative to the unperturbed run's
    return 0.5 * h * np.sum(E * E) + np.sum(a * xf) + np.sum(b * sp[0].v), xf


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("order", [1, 2])
def test_gradient_matches_central_differences(scheme, order):
    L, x, v, w, E0 = _problem(order, seed=10 * scheme + order)
    nc, n, nsteps = len(E0), len(x), 6
    cfg = O.ES1DConfig(nc=nc, L=L, order=order, dt=0.1, scheme=scheme)
    rng = np.random.default_rng(99)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    # gradient by reverse mode
    sp = [O.Species(-1.0, 1.0, x.copy(), v.copy(), w.copy(), 0.0)]
    Ef = E0.copy()
    spf = [O.Species(-1.0, 1.0, x.copy(), v.copy(), w.copy(), 0.0)]
    O.es1d_run(cfg, spf, Ef, nsteps)
    h = L / nc
    Eb, xb, vb, wb = O.es1d_grad(cfg, sp, E0, nsteps, h * Ef, [a], [b])
    assert np.array_equal(sp[0].x, x) and np.array_equal(sp[0].v, v)  # state unchanged
    base, xf0 = _objective(cfg, L, x, v, w, E0, a, b, nsteps, 0.0)
    for k in range(4):
        d = np.random.default_rng(1000 + k)
        dx, dv = d.standard_normal(n), d.standard_normal(n)
        dw, dE = d.standard_normal(n) * (L / n), d.standard_normal(nc) * 0.05
        eps = 1e-6
        lp, xp = _objective(cfg, L, x + eps * dx, v + eps * dv, w + eps * dw, E0 + eps * dE,
                            a, b, nsteps, 0.0)
        lm, xm = _objective(cfg, L, x - eps * dx, v - eps * dv, w - eps * dw, E0 - eps * dE,
                            a, b, nsteps, 0.0)
        # undo boundary crossings of the perturbed runs in the position term
        lp -= np.sum(a * (xp - xf0 - L * np.round((xp - xf0) / L)) - a * (xp - xf0))
        lm -= np.sum(a * (xm - xf0 - L * np.round((xm - xf0) / L)) - a * (xm - xf0))
        fd = (lp - lm) / (2 * eps)
        ad = np.dot(xb[0], dx) + np.dot(vb[0], dv) + np.dot(wb[0], dw) + np.dot(Eb, dE)
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (k, fd, ad)


def test_uniform_weight_gradient_is_the_sum_over_markers():
    L, x, v, _, E0 = _problem(2, seed=3, weighted=False)
    nc, n = len(E0), len(x)
    w0 = L / n
    cfg = O.ES1DConfig(nc=nc, L=L, order=2, dt=0.1, scheme=2)
    spf = [O.Species(-1.0, 1.0, x.copy(), v.copy(), None, w0)]
    Ef = E0.copy()
    O.es1d_run(cfg, spf, Ef, 5)
    h = L / nc
    zero = np.zeros(n)
    _, _, _, wb_u = O.es1d_grad(cfg, [O.Species(-1.0, 1.0, x, v, None, w0)], E0, 5, h * Ef,
                                [zero], [zero])
    _, _, _, wb_w = O.es1d_grad(cfg, [O.Species(-1.0, 1.0, x, v, np.full(n, w0), 0.0)], E0, 5,
                                h * Ef, [zero], [zero])
    assert wb_u[0].shape == (1,)
    assert abs(wb_u[0][0] - wb_w[0].sum()) <= 1e-12 * abs(wb_w[0].sum())


def test_fallback_branch_gradient():
    """Slow markers in a strong field take the imaginary-Gamma fallback; the
    reverse pass must then differentiate v^{n+1} = v^dag."""
    L, x, v, w, E0 = _problem(2, seed=5, vscale=0.05)
    E0 = 3.0 * E0 / np.max(np.abs(E0))
    nc, n, nsteps = len(E0), len(x), 4
    cfg = O.ES1DConfig(nc=nc, L=L, order=2, dt=0.4, scheme=2)
    spf = [O.Species(-1.0, 1.0, x.copy(), v.copy(), w.copy(), 0.0)]
    Ef = E0.copy()
    _, _, nfb = O.es1d_run(cfg, spf, Ef, nsteps)
    assert nfb.sum() > 0
    rng = np.random.default_rng(7)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    h = L / nc
    Eb, xb, vb, wb = O.es1d_grad(cfg, [O.Species(-1.0, 1.0, x, v, w, 0.0)], E0, nsteps, h * Ef,
                                 [a], [b])
    base, xf0 = _objective(cfg, L, x, v, w, E0, a, b, nsteps, 0.0)
    d = np.random.default_rng(11)
    dv = d.standard_normal(n)
    eps = 1e-7
    lp, _ = _objective(cfg, L, x, v + eps * dv, w, E0, a, b, nsteps, 0.0)
    lm, _ = _objective(cfg, L, x, v - eps * dv, w, E0, a, b, nsteps, 0.0)
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - np.dot(vb[0], dv)) <= 1e-5 * max(1.0, abs(fd)), (fd, np.dot(vb[0], dv))
