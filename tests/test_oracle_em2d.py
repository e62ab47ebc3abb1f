"""Pins of the oracle's 2D3V electromagnetic scheme with the leapfrog / Yee field step
(Sec. 4.1, Eq. EMleapfrog).

Expected values come from: the discrete curl identity Eq. (curlIdentity) and
div curl = 0 on the Yee lattice; the Yee vacuum dispersion relation
sin(w dt/2) / (c dt) = sqrt(sum_d sin^2(k_d h_d/2) / h_d^2); the symmetric Boris
rotation that the push reduces to when E = 0 (Sec. 3.2: the magnetic field does
no work, v* = v^{n+1/2}); the implicit relation that defines v*; and the energy
identity with W_B^n = (c^2/2)|h| sum B^{n+1/2} . B^{n-1/2} (Sec. 4.1).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09605_gb300 import workloads as W


def _rand_field(rng, ny, nx):
    return np.ascontiguousarray(rng.standard_normal((3, ny, nx)))


def test_curl_identity():
    rng = np.random.default_rng(0)
    nx, ny, hx, hy = 12, 9, 0.3, 0.7
    E = _rand_field(rng, ny, nx)
    B = _rand_field(rng, ny, nx)
    lhs = np.sum(E * O.yee_curl_b(nx, ny, hx, hy, B))
    rhs = np.sum(B * O.yee_curl_e(nx, ny, hx, hy, E))
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(E * O.yee_curl_b(nx, ny, hx, hy, B)))


def test_div_curl_vanishes():
    rng = np.random.default_rng(1)
    nx, ny, hx, hy = 10, 14, 0.4, 0.25
    E = _rand_field(rng, ny, nx)
    cE = O.yee_curl_e(nx, ny, hx, hy, E)
    # divergence at the Bz locations (cell centres): Bx at (i, j+1/2), By at (i+1/2, j)
    div = (np.roll(cE[0], -1, axis=1) - cE[0]) / hx + (np.roll(cE[1], -1, axis=0) - cE[1]) / hy
    assert np.max(np.abs(div)) < 1e-12 * np.max(np.abs(cE))
    # and the E-locations divergence of curl B at the nodes
    B = _rand_field(rng, ny, nx)
    cB = O.yee_curl_b(nx, ny, hx, hy, B)
    div2 = (cB[0] - np.roll(cB[0], 1, axis=1)) / hx + (cB[1] - np.roll(cB[1], 1, axis=0)) / hy
    assert np.max(np.abs(div2)) < 1e-12 * np.max(np.abs(cB))


def _empty_species():
    z = np.zeros(0)
    return [O.Species2D(-1.0, 1.0, z.copy(), z.copy(), z.copy(), z.copy(), z.copy(), None, 0.0)]


@pytest.mark.parametrize("mx", [1, 3, 7])
def test_yee_vacuum_dispersion(mx):
    """One leapfrog step maps a plane wave (Ez, By) along x by a 2x2 matrix with
    eigenvalues exp(+-i w dt), sin(w dt/2) = c dt sin(k hx/2)/hx."""
    nx, ny, L, c, dt = 32, 4, 6.0, 1.3, 0.05
    hx, hy = L / nx, L / ny
    k = 2 * np.pi * mx / L
    xi = np.arange(nx) * hx
    cfg = O.EM2DConfig(nx=nx, ny=ny, Lx=L, Ly=L, dt=dt, c=c, order=1)
    ez_shape = np.cos(k * xi)                # Ez at nodes
    by_shape = np.sin(k * (xi + 0.5 * hx))   # By at (i+1/2, j)
    M = np.zeros((2, 2))
    for col in range(2):
        E = np.zeros((3, ny, nx))
        B = np.zeros((3, ny, nx))
        if col == 0:
            E[2] = ez_shape[None, :]
        else:
            B[1] = by_shape[None, :]
        O.em2d_step(cfg, _empty_species(), E, B)
        M[0, col] = np.dot(E[2, 0], ez_shape) / np.dot(ez_shape, ez_shape)
        M[1, col] = np.dot(B[1, 0], by_shape) / np.dot(by_shape, by_shape)
        # the step maps the mode onto itself
        assert np.max(np.abs(E[2] - M[0, col] * ez_shape[None, :])) < 1e-13
    ev = np.linalg.eigvals(M)
    assert np.allclose(np.abs(ev), 1.0, atol=1e-13)
    w_num = np.max(np.abs(np.angle(ev))) / dt
    w_th = 2.0 / dt * math.asin(c * dt * math.sin(k * hx / 2) / hx)
    assert abs(w_num - w_th) < 1e-11 * w_th


@pytest.mark.parametrize("scheme", [1, 2])
def test_uniform_b_push_is_boris_rotation(scheme):
    """E = 0, uniform B: |v| is conserved exactly and v rotates by
    -2 atan((q/m) B dt/2) per step (symmetric Boris, Sec. 2.2.1 / Sec. 3.2)."""
    nx = ny = 8
    L, dt, B0, q, m = 4.0, 0.1, 1.7, -1.0, 1.0
    cfg = O.EM2DConfig(nx=nx, ny=ny, Lx=L, Ly=L, dt=dt, c=1.0, order=1, scheme=scheme)
    v0 = np.array([0.3, -0.4, 0.25])
    x0, y0 = 1.1, 2.3
    sp = [O.Species2D(q, m, np.array([x0]), np.array([y0]), np.array([v0[0]]),
                      np.array([v0[1]]), np.array([v0[2]]), None, 0.0)]
    E = np.zeros((3, ny, nx))
    B = np.zeros((3, ny, nx))
    B[2] = B0
    theta = -2.0 * math.atan(q / m * B0 * dt / 2)
    nsteps = 50
    vs = [v0[:2].copy()]
    for n in range(1, nsteps + 1):
        nfb = O.em2d_step(cfg, sp, E, B)
        assert nfb == [0]
        ang = n * theta
        rot = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
        vs.append(rot @ v0[:2])
        v = np.array([sp[0].vx[0], sp[0].vy[0], sp[0].vz[0]])
        assert abs(np.dot(v, v) - np.dot(v0, v0)) < 1e-15
        assert np.max(np.abs(v[:2] - vs[-1])) < 1e-13
        assert abs(sp[0].vz[0] - v0[2]) < 1e-15
    # positions advance with v* = (v^n + v^{n+1})/2
    xs = x0 + dt * sum(0.5 * (vs[i] + vs[i + 1])[0] for i in range(nsteps))
    ys = y0 + dt * sum(0.5 * (vs[i] + vs[i + 1])[1] for i in range(nsteps))
    assert abs(sp[0].x[0] - xs % L) < 1e-12
    assert abs(sp[0].y[0] - ys % L) < 1e-12


def test_vstar_solves_implicit_relation():
    rng = np.random.default_rng(2)
    for _ in range(20):
        u = rng.standard_normal(3)
        t = rng.standard_normal(3)
        vs = O.vstar_solve(u, t)
        assert np.max(np.abs(vs - np.cross(vs, t) - u)) < 1e-14 * (1 + np.abs(u).max())


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("scheme", [1, 2])
def test_em_energy_identity(order, scheme):
    prob = W.weibel(nx=16, ny=16, ppc=16, L=3.2, order=order, vth_par=0.2, seed=3)
    s = prob.species[0]
    sp = [O.Species2D(s.q, s.m, s.x.copy(), s.y.copy(), s.vx.copy(), s.vy.copy(), s.vz.copy(),
                      None, s.w0)]
    cfg = O.EM2DConfig(nx=prob.nx, ny=prob.ny, Lx=prob.Lx, Ly=prob.Ly, order=order, dt=prob.dt,
                       c=prob.c, scheme=scheme)
    rng = np.random.default_rng(4)
    E = np.ascontiguousarray(1e-3 * rng.standard_normal((3, prob.ny, prob.nx)))
    B = np.ascontiguousarray(1e-3 * rng.standard_normal((3, prob.ny, prob.nx)))
    te = []
    for _ in range(40):
        ke, we, wb = O.em2d_energy(cfg, sp, E, B)
        te.append(sum(ke) + we + wb)
        nfb = O.em2d_step(cfg, sp, E, B)
        assert nfb == [0]
    te = np.array(te)
    assert np.max(np.abs(te - te[0])) / te[0] < 1e-13
