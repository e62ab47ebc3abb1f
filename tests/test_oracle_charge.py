"""Pins of the oracle's charge-conserving option of the 2D3V Yee scheme
(Sec. 3.5, Eq. detbal): the current and field take degree 0 on a component's
half-node axes and degree 1 on its integer-node axes, and the deposit of
j^{*,n+1/2} and the gather of E^{n+1/2} run over the pieces of the path
x^n -> x^{n+1} cut at the grid lines.

Expected values come from: the box B0 and the tent as the box convolved with
itself (quadrature here); the discrete continuity equation, which with the Yee
update and div curl = 0 keeps div_h E - rho at its initial value (Sec. 3.5),
while the point-shape deposit does not; the energy identity (same pieces and
shapes in deposit and gather); and one marker crossing one grid line, with the
two pieces' currents computed here by hand.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W


def test_box_shape_and_tent_as_box_convolution():
    rng = np.random.default_rng(0)
    nc = 8
    for xi in list(rng.random(50) * nc) + [0.0, 0.49999, 0.5, 7.5, 7.99]:
        idx, wt = O.shape_weights(0, xi, nc)
        assert len(idx) == 1 and wt[0] == 1.0
        assert idx[0] == int(np.floor(xi + 0.5)) % nc
        # tent weight at node i = measure of s in [-1/2, 1/2] whose box node is i
        m = 4000
        s = (np.arange(m) + 0.5) / m - 0.5
        counts = np.zeros(nc)
        for z in xi + s:
            counts[O.shape_weights(0, z, nc)[0][0]] += 1.0 / m
        ti, tw = O.shape_weights(1, xi, nc)
        ref = np.zeros(nc)
        ref[ti] += tw
        assert np.max(np.abs(counts - ref)) <= 1.0 / m + 1e-12


def _hot(seed, nx=16, ny=12, ppc=6, L=3.2, vth=0.4):
    prob = W.weibel(nx=nx, ny=ny, ppc=ppc, L=L, vth_par=vth, t_ratio=2.0, seed=seed)
    prob.Ly = L * ny / nx
    prob.species[0].y *= ny / nx
    return prob


def _species(prob):
    return [O.Species2D(s.q, s.m, s.x.copy(), s.y.copy(), s.vx.copy(), s.vy.copy(), s.vz.copy(),
                        None if s.w is None else s.w.copy(), s.w0) for s in prob.species]


def _run(prob, cc, scheme, steps, seed=1):
    cfg = O.EM2DConfig(nx=prob.nx, ny=prob.ny, Lx=prob.Lx, Ly=prob.Ly, order=1, dt=prob.dt,
                       c=prob.c, scheme=scheme, charge_conserving=cc)
    rng = np.random.default_rng(seed)
    E = np.ascontiguousarray(1e-2 * rng.standard_normal((3, prob.ny, prob.nx)))
    B = np.ascontiguousarray(1e-2 * rng.standard_normal((3, prob.ny, prob.nx)))
    sp = _species(prob)
    rho0, r0 = O.em2d_gauss_residual(cfg, sp, E)
    cells0 = np.floor(sp[0].x / (prob.Lx / prob.nx)) + 1000 * np.floor(sp[0].y / (prob.Ly / prob.ny))
    dr, te, nfb, crossed = [], [], [], np.zeros(len(sp[0].x), bool)
    for _ in range(steps):
        nfb.append(sum(O.em2d_step(cfg, sp, E, B)))
        _, r = O.em2d_gauss_residual(cfg, sp, E)
        dr.append(np.max(np.abs(r - r0)))
        ke, we, wb = O.em2d_energy(cfg, sp, E, B)
        te.append(sum(ke) + we + wb)
        cells = np.floor(sp[0].x / (prob.Lx / prob.nx)) + 1000 * np.floor(sp[0].y / (prob.Ly / prob.ny))
        crossed |= cells != cells0
    return np.array(dr) / np.max(np.abs(rho0)), np.array(te), np.array(nfb), crossed


@pytest.mark.parametrize("scheme", [1, 2])
def test_gauss_law_residual_is_kept(scheme):
    prob = _hot(seed=3)
    dr, te, nfb, crossed = _run(prob, True, scheme, 40)
    assert crossed.mean() > 0.5                 # most markers changed cell
    assert dr.max() <= 1e-12, dr.max()


def test_point_shape_deposit_breaks_gauss_law():
    prob = _hot(seed=3)
    dr, _, _, _ = _run(prob, False, 2, 10)
    assert dr.max() > 1e-4, dr.max()


@pytest.mark.parametrize("scheme", [1, 2])
def test_energy_conserved_with_charge_conservation(scheme):
    prob = _hot(seed=4)
    _, te, nfb, _ = _run(prob, True, scheme, 40)
    d = np.abs(np.diff(np.concatenate([[te[0]], te]))) / te[0]
    assert nfb.sum() == 0 or scheme == 1
    ok = nfb == 0
    assert np.all(d[ok] <= 1e-13), d.max()


def test_one_marker_crossing_by_hand():
    """E = B = 0, ESEC1 (v* = v^n), h = 1, dt = 1: the marker goes from
    (0.7, 1.4) to (1.3, 1.5), crossing x = 1 at the path's midpoint.  Two pieces
    of fraction 1/2 with midpoints (0.85, 1.425) and (1.15, 1.475)."""
    nx = ny = 4
    q, w, v = -1.0, 0.3, np.array([0.6, 0.1, 0.2])
    cfg = O.EM2DConfig(nx=nx, ny=ny, Lx=4.0, Ly=4.0, order=1, dt=1.0, c=1.0, scheme=1,
                       charge_conserving=True)
    sp = [O.Species2D(q, 1.0, np.array([0.7]), np.array([1.4]), v[:1].copy(), v[1:2].copy(),
                      v[2:].copy(), None, w)]
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    O.em2d_step(cfg, sp, E, B)
    J = np.zeros((3, ny, nx))
    for tau, (mx, my) in ((0.5, (0.85, 1.425)), (0.5, (1.15, 1.475))):
        ix, fx = int(np.floor(mx)), mx - np.floor(mx)
        iy, fy = int(np.floor(my)), my - np.floor(my)
        tx = {ix: 1 - fx, ix + 1: fx}           # tent on integer nodes
        ty = {iy: 1 - fy, iy + 1: fy}
        for j, wy in ty.items():                # Jx: box in x (half node ix + 1/2), tent in y
            J[0, j % ny, ix % nx] += q * w * v[0] * tau * wy
        for i, wx in tx.items():                # Jy: tent in x, box in y (half node iy + 1/2)
            J[1, iy % ny, i % nx] += q * w * v[1] * tau * wx
        for i, wx in tx.items():                # Jz: tent x tent
            for j, wy in ty.items():
                J[2, j % ny, i % nx] += q * w * v[2] * tau * wx * wy
    assert np.max(np.abs(E - (-1.0 * J))) <= 1e-15
    assert abs(sp[0].x[0] - 1.3) <= 1e-15 and abs(sp[0].y[0] - 1.5) <= 1e-15


def test_no_crossing_is_the_point_deposit_at_the_midpoint():
    """A path inside one cell is one piece: the current is the mixed-degree
    shape at x^{n+1/2}, i.e. Jx is the box of the cell times the tent in y."""
    cfg = O.EM2DConfig(nx=4, ny=4, Lx=4.0, Ly=4.0, order=1, dt=1.0, c=1.0, scheme=1,
                       charge_conserving=True)
    sp = [O.Species2D(1.0, 1.0, np.array([2.2]), np.array([3.1]), np.array([0.5]),
                      np.array([0.6]), np.array([0.0]), None, 1.0)]
    E = np.zeros((3, 4, 4))
    B = np.zeros((3, 4, 4))
    O.em2d_step(cfg, sp, E, B)
    # midpoint (2.45, 3.4): Jx at half node (2 + 1/2) in x, tent weights 0.6 / 0.4 at y = 3, 0
    assert abs(E[0, 3, 2] - (-0.5 * 0.6)) <= 1e-15 and abs(E[0, 0, 2] - (-0.5 * 0.4)) <= 1e-15
    assert np.count_nonzero(E[0]) == 2
