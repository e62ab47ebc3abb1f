"""Helpers that run one workload through the oracle and through the C ABI and
compare them (used by the -m gpu parity tests and by smoke())."""
from __future__ import annotations

import os

import numpy as np

from oracle import oracle as O

GOLDEN_PAPER = os.path.join(os.path.dirname(__file__), "golden", "paper_tests.txt")


def paper_values(path: str = GOLDEN_PAPER) -> dict:
    """The values of tests/golden/paper_tests.txt (key = value, '#' comments):
    the parameters and outcomes the paper prints for its tests."""
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, val = (t.strip() for t in line.split("=", 1))
                vals[key] = float(val)
    return vals


def oracle_run(prob, scheme=2, steps=10, remove_mean=True, gamma_on=True, E0=None):
    cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=scheme,
                       remove_mean=remove_mean, gamma_on=gamma_on)
    sp = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None if s.w is None else s.w.copy(), s.w0)
          for s in prob.species]
    E = O.poisson_e0_1d(cfg, sp) if E0 is None else E0.copy()
    E_init = E.copy()
    te, we, nfb = O.es1d_run(cfg, sp, E, steps)
    return dict(x=[s.x for s in sp], v=[s.v for s in sp], E=E, nfb=nfb, te=te, E0=E_init)


def gpu_run(prob, scheme=2, steps=10, precision=0, remove_mean=True, gamma_on=True, E0=None,
            sort_period=0):
    from paper_2411_09605_gb300 import pic
    sim = pic.Simulation(prob, scheme=scheme, precision=precision, E0=E0,
                         sort_period=sort_period, remove_mean=remove_mean, gamma_on=gamma_on)
    try:
        E_init = sim.field()
        ke0, we0, wb0, te0 = sim.energy()
        fb, te = sim.step(steps) if steps else (np.zeros(0, np.int64), np.zeros(0))
        xs, vs = [], []
        for s in range(len(prob.species)):
            x, v = sim.particles(s)
            xs.append(x)
            vs.append(v)
        E = sim.field()
        ke, we, wb, te_now = sim.energy()
        res = pic.pic_mixed_resolution(sim.h) if precision == 1 else None
    finally:
        sim.close()
    return dict(x=xs, v=vs, E=E, nfb=fb, te=np.concatenate([[te0], te]), E0=E_init,
                te_now=te_now, resolution=res)


def periodic_dist(a, b, L):
    d = np.abs(a - b) % L
    return np.minimum(d, L - d)


def compare(prob, ref, got):
    """Scale-normalised maximum differences (x over L, v over max|v|, E in 2-norm)."""
    out = {}
    out["x"] = max(np.max(periodic_dist(r, g, prob.L), initial=0.0) / prob.L
                   for r, g in zip(ref["x"], got["x"]))
    vmax = max(np.max(np.abs(r), initial=0.0) for r in ref["v"]) or 1.0
    out["v"] = max(np.max(np.abs(r - g), initial=0.0) for r, g in zip(ref["v"], got["v"])) / vmax
    En = np.linalg.norm(ref["E"]) or 1.0
    out["E"] = np.linalg.norm(ref["E"] - got["E"]) / En
    return out


def mixed_bars(ref_v, got_v, pos_err, h, dx, dv, dt, qm, Emax, steps):
    """The mixed forms against the FP64 oracle after `steps` steps, in units of
    their own quanta (pic_mixed_resolution: dx = L / 2^32 the position step,
    dv the velocity of one unit of the integer v*).  Returns the ratios
    error / bar (each must be <= 1):

    positions: 1e-6 h (the gathers' FP32 weights and tables, relative 2^-23)
      plus 4 dx per step (x^{n+1/2} and x^{n+1} are rounded to dx, and the
      rounded v* moves a marker by up to one dx more per step);
    velocities, marker by marker: 4 dv per step times (1 + kick / |v|), kick =
      dt |q/m| max|E|.  Each step rounds v* to one unit (+-dv/2) and the
      fixed-point position perturbs the gathered kick; through Gamma
      (Eq. opt_solution) a change of v* moves v^{n+1} by about
      |v^dag - v^n| / |v^dag| times itself, the 1 / |v| growth of slow markers.

    ref_v, got_v: [K][N] velocity components; pos_err: [D][N] periodic
    position differences; h: cell size (per axis, the smallest is used)."""
    ref_v = np.atleast_2d(ref_v)
    got_v = np.atleast_2d(got_v)
    speed = np.sqrt(np.sum(ref_v ** 2, axis=0))
    kick = dt * abs(qm) * Emax
    vbar = 4.0 * steps * dv * (1.0 + kick / np.maximum(speed, 1e-300))
    verr = np.max(np.abs(got_v - ref_v), axis=0)
    xbar = 1e-6 * np.min(np.atleast_1d(h)) + 4.0 * steps * dx
    xerr = np.max(np.abs(np.atleast_2d(pos_err)), axis=0)
    return {"x": float(np.max(xerr, initial=0.0) / xbar),
            "v": float(np.max(verr / vbar, initial=0.0)),
            "x_over_h": float(np.max(xerr, initial=0.0) / np.min(np.atleast_1d(h)))}
