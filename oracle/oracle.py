"""ctypes front end of the plain FP64 CPU oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library under
``paper_2411_09605_gb300`` never does.  It shares no code with the CUDA path.

Every function works on numpy float64 arrays in place (positions and
velocities of each species, the grid fields), mirroring the C functions one to
one; the C source states, next to each function, which part of the paper it
restates and what pins it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no FMA contraction, one thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """The same source with -fopenmp: orc_es1d_step's particle loops run on all
    host cores (per-thread private current sums).  Used only to time the CPU
    baseline; the tests check against the single-threaded build."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_OMP_PATH)) or (
        os.path.getmtime(_OMP_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _OMP_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


def lib_omp():
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = C.CDLL(build_omp())
        _declare(_lib_omp)
    return _lib_omp


def omp_threads() -> int:
    """Threads the OpenMP build runs with (its omp_get_max_threads())."""
    f = lib_omp().omp_get_max_threads
    f.restype = C.c_int
    return int(f())


_dp = C.POINTER(C.c_double)
_lp = C.POINTER(C.c_long)


class _EsCfg(C.Structure):
    _fields_ = [("nc", C.c_long), ("L", C.c_double), ("order", C.c_int), ("dt", C.c_double),
                ("scheme", C.c_int), ("remove_mean", C.c_int), ("gamma_on", C.c_int),
                ("passes", C.c_int)]


class _Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_long), ("x", _dp), ("v", _dp),
                ("w", _dp), ("w0", C.c_double)]


class _EmCfg(C.Structure):
    _fields_ = [("nx", C.c_long), ("ny", C.c_long), ("Lx", C.c_double), ("Ly", C.c_double),
                ("order", C.c_int), ("dt", C.c_double), ("c", C.c_double), ("scheme", C.c_int),
                ("gamma_on", C.c_int), ("charge_conserving", C.c_int)]


class _Species2d(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_long), ("x", _dp), ("y", _dp),
                ("vx", _dp), ("vy", _dp), ("vz", _dp), ("w", _dp), ("w0", C.c_double)]


class _Em1Cfg(C.Structure):
    _fields_ = [("n", C.c_long), ("L", C.c_double), ("order", C.c_int), ("dt", C.c_double),
                ("c", C.c_double), ("solver", C.c_int), ("scheme", C.c_int), ("gamma_on", C.c_int)]


class _Species1d2v(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_long), ("y", _dp), ("vx", _dp),
                ("vy", _dp), ("w", _dp), ("w0", C.c_double)]


def _declare(L):
    L.orc_shape_weights.argtypes = [C.c_int, C.c_double, C.c_long, _lp, _dp]
    L.orc_shape_weights.restype = C.c_int
    L.orc_deposit_1d.argtypes = [C.c_int, C.c_long, C.c_double, C.c_long, _dp, _dp, _dp]
    L.orc_gather_1d.argtypes = [C.c_int, C.c_long, C.c_double, C.c_long, _dp, _dp, _dp]
    L.orc_es1d_step.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp, _lp,
                                C.POINTER(_dp)]
    L.orc_es1d_step.restype = C.c_int
    L.orc_es1d_step_radicand.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp,
                                         _lp, C.POINTER(_dp), C.POINTER(_dp)]
    L.orc_es1d_step_radicand.restype = C.c_int
    L.orc_es1d_charge_diag.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp,
                                       _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_es1d_energy.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp, _dp, _dp]
    L.orc_es1d_run.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp, C.c_long,
                               _dp, _dp, _lp]
    L.orc_es1d_run.restype = C.c_int
    L.orc_poisson_e0_1d.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp]
    L.orc_es1d_grad.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, _dp, C.c_long,
                                _dp, C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp)]
    L.orc_yee_curl_e.argtypes = [C.c_long, C.c_long, C.c_double, C.c_double] + [_dp] * 6
    L.orc_yee_curl_b.argtypes = [C.c_long, C.c_long, C.c_double, C.c_double] + [_dp] * 6
    L.orc_vstar_solve.argtypes = [_dp, _dp, _dp]
    L.orc_em2d_step.argtypes = [C.POINTER(_EmCfg), C.POINTER(_Species2d), C.c_int, _dp, _dp, _lp]
    L.orc_em2d_step.restype = C.c_int
    L.orc_em2d_energy.argtypes = [C.POINTER(_EmCfg), C.POINTER(_Species2d), C.c_int, _dp, _dp,
                                  _dp, _dp, _dp]
    L.orc_em2d_gauss_residual.argtypes = [C.POINTER(_EmCfg), C.POINTER(_Species2d), C.c_int,
                                          _dp, _dp, _dp]
    L.orc_binomial_filter.argtypes = [C.c_long, _dp, _dp]
    L.orc_std_field.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, C.c_int, _dp]
    L.orc_std_start.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, C.c_int, _dp]
    L.orc_std_step.argtypes = [C.POINTER(_EsCfg), C.POINTER(_Species), C.c_int, C.c_int, _dp, _dp,
                               _dp]
    L.orc_std_step.restype = C.c_int
    L.orc_spectral_deriv.argtypes = [C.c_long, C.c_double, _dp, _dp]
    L.orc_em1d_field_advance.argtypes = [C.POINTER(_Em1Cfg), C.c_int, C.c_double, _dp, _dp, _dp,
                                         _dp, _dp, _dp]
    L.orc_em1d_step.argtypes = [C.POINTER(_Em1Cfg), C.POINTER(_Species1d2v), C.c_int, _dp, _dp,
                                _lp]
    L.orc_em1d_step.restype = C.c_int
    L.orc_em1d_energy.argtypes = [C.POINTER(_Em1Cfg), C.POINTER(_Species1d2v), C.c_int, _dp, _dp,
                                  _dp, _dp, _dp]


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return C.cast(None, _dp)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


# ----------------------------------------------------------------------------- 1D


@dataclass
class ES1DConfig:
    nc: int
    L: float
    order: int = 1
    dt: float = 0.1
    scheme: int = 2
    remove_mean: bool = True
    gamma_on: bool = True
    passes: int = 0          # binomial filter passes inside the scheme

    def _c(self):
        return _EsCfg(self.nc, self.L, self.order, self.dt, self.scheme, int(self.remove_mean),
                      int(self.gamma_on), int(self.passes))


@dataclass
class Species:
    """Markers of one species; x and v are float64 arrays updated in place."""
    q: float
    m: float
    x: np.ndarray
    v: np.ndarray
    w: Optional[np.ndarray] = None
    w0: float = 0.0

    def _c(self):
        return _Species(self.q, self.m, len(self.x), _ptr(self.x), _ptr(self.v), _ptr(self.w),
                        self.w0)


def _sp_array(species: Sequence[Species]):
    arr = (_Species * len(species))()
    for i, s in enumerate(species):
        arr[i] = s._c()
    return arr


def shape_weights(order: int, xi: float, nc: int):
    idx = (C.c_long * 3)()
    wt = (C.c_double * 3)()
    k = lib().orc_shape_weights(order, xi, nc, idx, wt)
    return np.array(idx[:k], dtype=np.int64), np.array(wt[:k])


def deposit_1d(order, nc, L, x, c, J=None):
    J = np.zeros(nc) if J is None else J
    lib().orc_deposit_1d(order, nc, L, len(x), _ptr(x), _ptr(c), _ptr(J))
    return J


def gather_1d(order, nc, L, x, E):
    Ep = np.zeros(len(x))
    lib().orc_gather_1d(order, nc, L, len(x), _ptr(x), _ptr(E), _ptr(Ep))
    return Ep


def es1d_step(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray, want_gamma=False,
              threaded: bool = False):
    """One step; returns (fallback counts per species, Gamma arrays or None).
    threaded=True runs the OpenMP build (CPU-baseline timing only)."""
    sp = _sp_array(species)
    nfb = (C.c_long * len(species))()
    gam = None
    gptr = C.cast(None, C.POINTER(_dp))
    if want_gamma:
        gam = [np.zeros(len(s.x)) for s in species]
        garr = (_dp * len(species))(*[_ptr(g) for g in gam])
        gptr = C.cast(garr, C.POINTER(_dp))
    L = lib_omp() if threaded else lib()
    rc = L.orc_es1d_step(C.byref(cfg._c()), sp, len(species), _ptr(E), nfb, gptr)
    assert rc == 0
    return list(nfb), gam


def es1d_step_radicand(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray):
    """One step; returns (fallback counts per species, R / |v^dag|^2 per marker of
    each species: negative where Gamma would be imaginary)."""
    sp = _sp_array(species)
    nfb = (C.c_long * len(species))()
    rad = [np.zeros(len(s.x)) for s in species]
    rarr = (_dp * len(species))(*[_ptr(g) for g in rad])
    rc = lib().orc_es1d_step_radicand(C.byref(cfg._c()), sp, len(species), _ptr(E), nfb,
                                      C.cast(None, C.POINTER(_dp)), C.cast(rarr, C.POINTER(_dp)))
    assert rc == 0
    return list(nfb), rad


def es1d_energy(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray):
    """Returns (KE per species, W_E)."""
    sp = _sp_array(species)
    ke = (C.c_double * len(species))()
    we = C.c_double()
    lib().orc_es1d_energy(C.byref(cfg._c()), sp, len(species), _ptr(E), ke, C.byref(we))
    return list(ke), we.value


def es1d_run(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray, nsteps: int):
    """Runs nsteps; returns (TE[nsteps+1], W_E[nsteps+1], fallbacks[nsteps])."""
    sp = _sp_array(species)
    te = np.zeros(nsteps + 1)
    we = np.zeros(nsteps + 1)
    nfb = np.zeros(nsteps, dtype=np.int64)
    rc = lib().orc_es1d_run(C.byref(cfg._c()), sp, len(species), _ptr(E), nsteps, _ptr(te),
                            _ptr(we), nfb.ctypes.data_as(_lp))
    assert rc == 0
    return te, we, nfb


def es1d_grad(cfg: ES1DConfig, species: Sequence[Species], E0: np.ndarray, nsteps: int,
              Ebar: np.ndarray, xbar: Sequence[np.ndarray], vbar: Sequence[np.ndarray]):
    """Reverse mode of nsteps steps from the state (species, E0), which is left
    unchanged.  Ebar, xbar, vbar: adjoints of the final field and markers.
    Returns (Ebar, xbar, vbar, wbar) of the initial state (wbar[s] per marker, or
    one entry for a uniform w0)."""
    sp = _sp_array(species)
    Eb = np.ascontiguousarray(Ebar, dtype=np.float64).copy()
    xb = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in xbar]
    vb = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in vbar]
    wb = [np.zeros(len(s.x) if s.w is not None else 1) for s in species]
    arr = lambda lst: (_dp * len(lst))(*[_ptr(a) for a in lst])  # noqa: E731
    rc = lib().orc_es1d_grad(C.byref(cfg._c()), sp, len(species), _ptr(np.ascontiguousarray(E0)),
                             nsteps, _ptr(Eb), arr(xb), arr(vb), arr(wb))
    assert rc == 0
    return Eb, xb, vb, wb


def es1d_charge_diag(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray):
    """Charge diagnostics of the state: dict with Q_markers, Q_grid, gauss_l2,
    rho_l2 and the real-space residual r and filtered charge rhot ([nc])."""
    nc = cfg.nc
    qm, qg, g, pl = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    r, rt = np.zeros(nc), np.zeros(nc)
    lib().orc_es1d_charge_diag(C.byref(cfg._c()), _sp_array(species), len(species),
                               _ptr(np.ascontiguousarray(E, dtype=np.float64)), C.byref(qm),
                               C.byref(qg), C.byref(g), C.byref(pl), _ptr(r), _ptr(rt))
    return dict(Q_markers=qm.value, Q_grid=qg.value, gauss_l2=g.value, rho_l2=pl.value, r=r,
                rhot=rt)


def poisson_e0_1d(cfg: ES1DConfig, species: Sequence[Species]):
    E = np.zeros(cfg.nc)
    lib().orc_poisson_e0_1d(C.byref(cfg._c()), _sp_array(species), len(species), _ptr(E))
    return E


# ----------------------------------------------------------------------------- standard PIC


def binomial_filter(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros_like(a)
    lib().orc_binomial_filter(len(a), _ptr(a), _ptr(out))
    return out


def std_field(cfg: ES1DConfig, species: Sequence[Species], passes: int = 1) -> np.ndarray:
    E = np.zeros(cfg.nc)
    lib().orc_std_field(C.byref(cfg._c()), _sp_array(species), len(species), passes, _ptr(E))
    return E


def std_start(cfg: ES1DConfig, species: Sequence[Species], passes: int = 1) -> np.ndarray:
    """E^0 of x^0; turns each species' v^0 into v^{-1/2} in place."""
    E = np.zeros(cfg.nc)
    lib().orc_std_start(C.byref(cfg._c()), _sp_array(species), len(species), passes, _ptr(E))
    return E


def std_step(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray, passes: int = 1):
    """One leapfrog step in place; returns (KE per species, W_E) at the start time."""
    ke = (C.c_double * len(species))()
    we = C.c_double()
    rc = lib().orc_std_step(C.byref(cfg._c()), _sp_array(species), len(species), passes, _ptr(E),
                            ke, C.byref(we))
    assert rc == 0
    return list(ke), we.value


def std_run(cfg: ES1DConfig, species: Sequence[Species], E: np.ndarray, nsteps: int,
            passes: int = 1):
    """nsteps leapfrog steps from a started state; TE[n] and W_E[n] of times 0..nsteps-1."""
    te, we = np.zeros(nsteps), np.zeros(nsteps)
    for k in range(nsteps):
        ke, we[k] = std_step(cfg, species, E, passes)
        te[k] = sum(ke) + we[k]
    return te, we


# ----------------------------------------------------------------------------- 2D3V


@dataclass
class EM2DConfig:
    nx: int
    ny: int
    Lx: float
    Ly: float
    order: int = 1
    dt: float = 0.05
    c: float = 1.0
    scheme: int = 2
    gamma_on: bool = True
    charge_conserving: bool = False    # Sec. 3.5: mixed-degree shapes, path pieces

    def _c(self):
        return _EmCfg(self.nx, self.ny, self.Lx, self.Ly, self.order, self.dt, self.c,
                      self.scheme, int(self.gamma_on), int(self.charge_conserving))


@dataclass
class Species2D:
    q: float
    m: float
    x: np.ndarray
    y: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    w: Optional[np.ndarray] = None
    w0: float = 0.0

    def _c(self):
        return _Species2d(self.q, self.m, len(self.x), _ptr(self.x), _ptr(self.y), _ptr(self.vx),
                          _ptr(self.vy), _ptr(self.vz), _ptr(self.w), self.w0)


def _sp2_array(species):
    arr = (_Species2d * len(species))()
    for i, s in enumerate(species):
        arr[i] = s._c()
    return arr


def yee_curl_e(nx, ny, hx, hy, E):
    """E: [3, ny, nx] -> curl at the B locations, [3, ny, nx]."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    out = np.zeros_like(E)
    lib().orc_yee_curl_e(nx, ny, hx, hy, _ptr(E[0]), _ptr(E[1]), _ptr(E[2]), _ptr(out[0]),
                         _ptr(out[1]), _ptr(out[2]))
    return out


def yee_curl_b(nx, ny, hx, hy, B):
    B = np.ascontiguousarray(B, dtype=np.float64)
    out = np.zeros_like(B)
    lib().orc_yee_curl_b(nx, ny, hx, hy, _ptr(B[0]), _ptr(B[1]), _ptr(B[2]), _ptr(out[0]),
                         _ptr(out[1]), _ptr(out[2]))
    return out


def vstar_solve(u, t):
    u = np.ascontiguousarray(u, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_vstar_solve(_ptr(u), _ptr(t), _ptr(out))
    return out


def em2d_step(cfg: EM2DConfig, species: Sequence[Species2D], E: np.ndarray, B: np.ndarray):
    """E, B: float64 [3, ny, nx] (B holds B^{n-1/2}); updated in place."""
    assert E.flags.c_contiguous and B.flags.c_contiguous
    nfb = (C.c_long * len(species))()
    rc = lib().orc_em2d_step(C.byref(cfg._c()), _sp2_array(species), len(species), _ptr(E),
                             _ptr(B), nfb)
    assert rc == 0
    return list(nfb)


def em2d_gauss_residual(cfg: EM2DConfig, species: Sequence[Species2D], E):
    """(rho, div_h E - rho) on the nodes, each [ny, nx]; rho with the bilinear shape."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    rho = np.zeros((cfg.ny, cfg.nx))
    r = np.zeros((cfg.ny, cfg.nx))
    lib().orc_em2d_gauss_residual(C.byref(cfg._c()), _sp2_array(species), len(species), _ptr(E),
                                  _ptr(rho), _ptr(r))
    return rho, r


def em2d_energy(cfg: EM2DConfig, species: Sequence[Species2D], E, B):
    """Returns (KE per species, W_E, W_B)."""
    ke = (C.c_double * len(species))()
    we, wb = C.c_double(), C.c_double()
    lib().orc_em2d_energy(C.byref(cfg._c()), _sp2_array(species), len(species), _ptr(E), _ptr(B),
                          ke, C.byref(we), C.byref(wb))
    return list(ke), we.value, wb.value


# ----------------------------------------------------------------------------- 1D2V spectral EM

CN, PSATD = 1, 2


@dataclass
class EM1DConfig:
    """1D2V geometry of the Weibel test: coordinate y, velocities (vx, vy),
    fields E = (Ex, Ey) [2, n] and Bz [n]; solver CN (Eq. EMbasic) or PSATD
    (Eq. EM_PSATD)."""
    n: int
    L: float
    order: int = 1
    dt: float = 0.1
    c: float = 1.0
    solver: int = CN
    scheme: int = 2
    gamma_on: bool = True

    def _c(self):
        return _Em1Cfg(self.n, self.L, self.order, self.dt, self.c, self.solver, self.scheme,
                       int(self.gamma_on))


@dataclass
class Species1D2V:
    q: float
    m: float
    y: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    w: Optional[np.ndarray] = None
    w0: float = 0.0

    def _c(self):
        return _Species1d2v(self.q, self.m, len(self.y), _ptr(self.y), _ptr(self.vx),
                            _ptr(self.vy), _ptr(self.w), self.w0)


def _sp12_array(species):
    arr = (_Species1d2v * len(species))()
    for i, s in enumerate(species):
        arr[i] = s._c()
    return arr


def spectral_deriv(n: int, L: float, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(n)
    lib().orc_spectral_deriv(n, L, _ptr(f), _ptr(out))
    return out


def em1d_field_advance(cfg: EM1DConfig, kind: int, tau: float, E, B, j):
    """kind 0 explicit Euler, 1 Crank-Nicolson, 2 PSATD, over tau with j fixed.
    Returns (E', B', Eavg)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    j = np.ascontiguousarray(j, dtype=np.float64)
    Eo, Bo, Ea = np.zeros_like(E), np.zeros_like(B), np.zeros_like(E)
    lib().orc_em1d_field_advance(C.byref(cfg._c()), kind, tau, _ptr(E), _ptr(B), _ptr(j),
                                 _ptr(Eo), _ptr(Bo), _ptr(Ea))
    return Eo, Bo, Ea


def em1d_step(cfg: EM1DConfig, species: Sequence[Species1D2V], E: np.ndarray, B: np.ndarray):
    """E [2, n], B [n] float64, updated in place with the species."""
    assert E.flags.c_contiguous and B.flags.c_contiguous
    nfb = (C.c_long * len(species))()
    rc = lib().orc_em1d_step(C.byref(cfg._c()), _sp12_array(species), len(species), _ptr(E),
                             _ptr(B), nfb)
    assert rc == 0
    return list(nfb)


def em1d_energy(cfg: EM1DConfig, species: Sequence[Species1D2V], E, B):
    """Returns (KE per species, W_E, W_B)."""
    ke = (C.c_double * len(species))()
    we, wb = C.c_double(), C.c_double()
    lib().orc_em1d_energy(C.byref(cfg._c()), _sp12_array(species), len(species), _ptr(E), _ptr(B),
                          ke, C.byref(we), C.byref(wb))
    return list(ke), we.value, wb.value


def em1d_run(cfg: EM1DConfig, species: Sequence[Species1D2V], E, B, nsteps: int):
    """Runs nsteps; returns (TE[nsteps+1], W_E[nsteps+1], W_B[nsteps+1], fallbacks[nsteps])."""
    te, we, wb = np.zeros(nsteps + 1), np.zeros(nsteps + 1), np.zeros(nsteps + 1)
    fb = np.zeros(nsteps, dtype=np.int64)
    for k in range(nsteps + 1):
        ke, we[k], wb[k] = em1d_energy(cfg, species, E, B)
        te[k] = sum(ke) + we[k] + wb[k]
        if k < nsteps:
            fb[k] = sum(em1d_step(cfg, species, E, B))
    return te, we, wb, fb
