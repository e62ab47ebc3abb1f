"""Pins of the oracle's 1D charge diagnostics (orc_es1d_charge_diag): the charge
density, its totals and the residual of Gauss's law dE/dx = rho - <rho> (Sec. 2.1)
on the Fourier modes the spectral derivative represents.

None of these re-types the oracle's formula: the residual is checked against
numpy's FFT, a single field mode against its closed-form derivative, the field
of the (separately pinned) Poisson solve against a zero residual, and the
totals against the markers' charge."""
import numpy as np
import pytest

from oracle import oracle as O


def _species(rng, n, L, q=-1.0, weighted=False):
    x = rng.uniform(0.0, L, n)
    v = rng.standard_normal(n)
    w = rng.uniform(0.5, 1.5, n) * L / n if weighted else None
    return O.Species(q, 1.0, x, v, w, L / n)


def _numpy_residual(E, rho, L):
    nc = len(E)
    M = (nc - 1) // 2
    Ek, Rk = np.fft.fft(E), np.fft.fft(rho)
    R, P = np.zeros(nc, complex), np.zeros(nc, complex)
    for m in range(1, M + 1):
        kappa = 2 * np.pi * m / L
        R[m] = 1j * kappa * Ek[m] - Rk[m]
        R[nc - m] = np.conj(R[m])
        P[m], P[nc - m] = Rk[m], np.conj(Rk[m])
    return np.fft.ifft(R).real, np.fft.ifft(P).real


@pytest.mark.parametrize("nc,order", [(64, 1), (37, 2), (128, 2)])
def test_residual_against_numpy_fft(nc, order):
    rng = np.random.default_rng(nc)
    L = 7.3
    cfg = O.ES1DConfig(nc=nc, L=L, order=order)
    sp = [_species(rng, 500, L), _species(rng, 300, L, q=2.0, weighted=True)]
    E = rng.standard_normal(nc)
    d = O.es1d_charge_diag(cfg, sp, E)
    rho = np.zeros(nc)
    for s in sp:
        w = s.w if s.w is not None else np.full(len(s.x), s.w0)
        O.deposit_1d(order, nc, L, s.x, s.q * w, rho)
    r, rt = _numpy_residual(E, rho, L)
    h = L / nc
    scale = np.max(np.abs(r))
    assert np.max(np.abs(d["r"] - r)) <= 1e-13 * scale
    assert np.max(np.abs(d["rhot"] - rt)) <= 1e-13 * np.max(np.abs(rt))
    assert d["gauss_l2"] == pytest.approx(np.sqrt(h * np.sum(r * r)), rel=1e-13)
    assert d["rho_l2"] == pytest.approx(np.sqrt(h * np.sum(rt * rt)), rel=1e-13)


def test_single_mode_closed_form():
    """E = A sin(kappa_3 x) and no markers: r = dE/dx = A kappa_3 cos(kappa_3 x),
    ||r|| = A kappa_3 sqrt(L / 2); an E on the Nyquist mode or a constant E leaves
    no residual (neither mode is represented)."""
    nc, L, A = 64, 5.0, 0.7
    cfg = O.ES1DConfig(nc=nc, L=L, order=1)
    empty = [O.Species(-1.0, 1.0, np.zeros(0), np.zeros(0), None, 1.0)]
    xj = np.arange(nc) * L / nc
    k3 = 2 * np.pi * 3 / L
    d = O.es1d_charge_diag(cfg, empty, A * np.sin(k3 * xj))
    assert np.max(np.abs(d["r"] - A * k3 * np.cos(k3 * xj))) <= 1e-13 * A * k3
    assert d["gauss_l2"] == pytest.approx(A * k3 * np.sqrt(L / 2), rel=1e-13)
    assert d["rho_l2"] == 0.0 and d["Q_grid"] == 0.0 and d["Q_markers"] == 0.0
    nyq = np.cos(np.pi * np.arange(nc)) + 3.0
    assert O.es1d_charge_diag(cfg, empty, nyq)["gauss_l2"] <= 1e-13


@pytest.mark.parametrize("nc,order", [(64, 1), (512, 2), (45, 2)])
def test_poisson_field_satisfies_gauss(nc, order):
    """The field of the spectral Poisson solve (pinned in test_oracle_es1d.py)
    leaves a residual at round-off; the opposite sign of D would leave twice
    ||rho||."""
    rng = np.random.default_rng(3 + nc)
    L = 4 * np.pi
    cfg = O.ES1DConfig(nc=nc, L=L, order=order)
    sp = [_species(rng, 4000, L)]
    E = O.poisson_e0_1d(cfg, sp)
    d = O.es1d_charge_diag(cfg, sp, E)
    assert d["rho_l2"] > 0
    assert d["gauss_l2"] <= 1e-13 * d["rho_l2"]
    d2 = O.es1d_charge_diag(cfg, sp, -E)
    assert d2["gauss_l2"] == pytest.approx(2 * d2["rho_l2"], rel=1e-12)


def test_charge_totals():
    """Q_grid = h sum rho equals sum q w (the shapes are a partition of unity)."""
    rng = np.random.default_rng(9)
    L = 3.0
    for order in (1, 2):
        cfg = O.ES1DConfig(nc=50, L=L, order=order)
        sp = [_species(rng, 1000, L), _species(rng, 700, L, q=3.0, weighted=True)]
        d = O.es1d_charge_diag(cfg, sp, np.zeros(50))
        qm = sp[0].q * sp[0].w0 * 1000 + sp[1].q * np.sum(sp[1].w)
        assert d["Q_markers"] == pytest.approx(qm, rel=1e-14)
        assert d["Q_grid"] == pytest.approx(qm, rel=1e-13)


def test_point_deposit_breaks_gauss_over_time():
    """With point shapes and collocated E, J (the Ampere form), continuity is not
    kept discretely (Sec. 3.5 needs charge-conserving shapes), so the residual of
    a Landau run that starts from the Poisson field grows from round-off."""
    rng = np.random.default_rng(5)
    L = 4 * np.pi
    cfg = O.ES1DConfig(nc=64, L=L, order=1, dt=0.1, scheme=2)
    x = rng.uniform(0, L, 20000)
    sp = [O.Species(-1.0, 1.0, x, rng.standard_normal(20000), None, L / 20000)]
    E = O.poisson_e0_1d(cfg, sp)
    g0 = O.es1d_charge_diag(cfg, sp, E)
    O.es1d_run(cfg, sp, E, 10)
    g1 = O.es1d_charge_diag(cfg, sp, E)
    assert g0["gauss_l2"] <= 1e-13 * g0["rho_l2"]
    assert g1["gauss_l2"] >= 1e-3 * g1["rho_l2"]
    assert g1["Q_grid"] == pytest.approx(g0["Q_grid"], rel=1e-13)
