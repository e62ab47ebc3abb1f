"""Pins of the oracle's shape functions, deposition and interpolation (Sec. 2.2).

Each check comes from the definition of the B-spline shapes, not from the
oracle's own formulas: partition of unity, exact reproduction of linear
functions, symmetry, the quadratic B-spline as the tent convolved with the
unit box (computed here by numerical quadrature), and the adjoint relation
between deposition and interpolation that Eq. (exp_econs_simple) uses.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O


def _tent(z):
    return max(0.0, 1.0 - abs(z))


def _quad_bspline(z):
    # B-spline of degree 2 = tent (degree 1) convolved with the unit box [-1/2, 1/2]
    val, _ = quad(lambda s: _tent(z - s), -0.5, 0.5, points=[z - 1, z, z + 1], epsabs=1e-14,
                  epsrel=1e-14)
    return val


@pytest.mark.parametrize("order", [1, 2])
def test_partition_of_unity_and_linear_reproduction(order):
    rng = np.random.default_rng(1)
    nc = 16
    for xi in list(rng.random(200) * nc) + [0.0, 0.5, 1.0, 15.999999, 7.5]:
        idx, wt = O.shape_weights(order, xi, nc)
        assert len(idx) == order + 1
        assert np.all(wt >= 0.0)
        assert abs(wt.sum() - 1.0) < 1e-15
        # first moment: sum_k S_k x_k = xi (node positions unwrapped near xi)
        nodes = idx.astype(float)
        nodes = nodes + nc * np.round((xi - nodes) / nc)
        assert abs(np.dot(wt, nodes) - xi) < 1e-13


@pytest.mark.parametrize("order", [1, 2])
def test_weights_match_bspline_definition(order):
    rng = np.random.default_rng(2)
    nc = 8
    for xi in rng.random(40) * nc:
        idx, wt = O.shape_weights(order, xi, nc)
        for k, w in zip(idx, wt):
            node = k + nc * np.round((xi - k) / nc)
            ref = _tent(xi - node) if order == 1 else _quad_bspline(xi - node)
            assert abs(w - ref) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_symmetry(order):
    # S(x_p - x_h) = S(x_h - x_p): a particle at node i + d and one at i - d carry
    # mirrored weights
    nc = 10
    for d in [0.1, 0.25, 0.3333, 0.49]:
        i1, w1 = O.shape_weights(order, 5 + d, nc)
        i2, w2 = O.shape_weights(order, 5 - d, nc)
        m1 = {int(k): w for k, w in zip(i1, w1)}
        m2 = {int(k): w for k, w in zip(i2, w2)}
        for k, w in m1.items():
            assert abs(m2.get(10 - k, 0.0) - w) < 1e-15


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_gather_adjoint(order):
    """<E, D(c)>_h h = <G(E), c>_p: the pairing behind Eq. (brokenEcons)."""
    rng = np.random.default_rng(3)
    nc, L = 32, 7.0
    h = L / nc
    x = rng.random(1000) * L
    c = rng.standard_normal(1000)
    E = rng.standard_normal(nc)
    J = O.deposit_1d(order, nc, L, x, c)
    Ep = O.gather_1d(order, nc, L, x, E)
    lhs = h * np.dot(E, J)
    rhs = np.dot(Ep, c)
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(Ep * c))


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_total_charge_and_periodic_wrap(order):
    rng = np.random.default_rng(4)
    nc, L = 12, 3.0
    h = L / nc
    x = rng.random(500) * L
    x[:5] = [0.0, L - 1e-12, h * 3, 0.5 * h, L - 0.5 * h]
    q = rng.random(500)
    J = O.deposit_1d(order, nc, L, x, q)
    assert abs(h * J.sum() - q.sum()) < 1e-12
