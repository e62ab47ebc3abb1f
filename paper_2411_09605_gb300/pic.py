"""Thin ctypes binding of the C ABI in include/pic.h (argument marshalling only).

Every function here forwards to the function of the same name in libpic.so;
all arithmetic of the method runs in the library's CUDA kernels.  The library
must have been built (``paper_2411_09605_gb300.build.build()``); importing this
module without it raises, there is no fallback.  With PIC_DEBUG_BOUNDS=1 in the
environment the debug-bounds build libpic_debug.so is loaded instead
(``build(debug_bounds=True)``).

Arrays may be numpy float64 arrays (host) or, with ``ptr_on_device=1`` in the
config, torch CUDA tensors (their ``data_ptr()`` is passed through).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "libpic_debug.so")

PIC_OK = 0
ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_OOM", -4: "PIC_ERR_NONFINITE",
          -5: "PIC_ERR_TIMEOUT", -6: "PIC_ERR_BOUNDS", -7: "PIC_ERR_UNSUPPORTED"}
PIC_SOLVER_AMPERE_ES, PIC_SOLVER_YEE_LEAPFROG, PIC_SOLVER_CN_SPECTRAL, PIC_SOLVER_PSATD = 0, 1, 2, 3
PIC_SOLVER_STANDARD_LEAPFROG = 4
PIC_SCHEME_ESEC1, PIC_SCHEME_ESEC2 = 1, 2
PIC_PREC_FP64, PIC_PREC_MIXED = 0, 1

# every function declared in include/pic.h
EXPORTS = ["pic_init", "pic_step", "pic_step_async", "pic_read_stats", "pic_launch_count",
           "pic_set_profiling", "pic_profile",
           "pic_energy", "pic_get_particles", "pic_get_ids",
           "pic_set_particles", "pic_get_fields", "pic_set_fields", "pic_step_count", "pic_free",
           "pic_last_error", "pic_version", "pic_es1d_step_noalloc",
           "pic_batch_init", "pic_batch_step", "pic_batch_set_graph", "pic_batch_read_stats",
           "pic_batch_run", "pic_batch_info", "pic_batch_free", "pic_batch_autotune",
           "pic_grad_forward", "pic_grad_backward", "pic_mixed_resolution", "pic_charge",
           "pic_debug_bounds"]


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class pic_grid(C.Structure):
    _fields_ = [("dim_x", C.c_int), ("dim_v", C.c_int), ("n", C.c_int64 * 2),
                ("L", C.c_double * 2)]


class pic_species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_int64), ("x", C.c_void_p),
                ("v", C.c_void_p), ("w", C.c_void_p), ("w0", C.c_double)]


class pic_config(C.Structure):
    _fields_ = [("grid", pic_grid), ("shape_order", C.c_int), ("dt", C.c_double),
                ("c", C.c_double), ("solver", C.c_int), ("scheme", C.c_int),
                ("precision", C.c_int), ("sort_period", C.c_int), ("remove_mean", C.c_int),
                ("gamma_on", C.c_int), ("ptr_on_device", C.c_int), ("cuda_stream", C.c_void_p),
                ("skip_ids", C.c_int), ("binomial_passes", C.c_int),
                ("charge_conserving", C.c_int), ("gamma_fp64", C.c_int),
                ("separate_passes", C.c_int)]


_lib = None


def lib() -> C.CDLL:
    """Loads libpic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        debug = os.environ.get("PIC_DEBUG_BOUNDS") == "1"
        path = DEBUG_LIB_PATH if debug else LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "paper_2411_09605_gb300.build.build("
                              f"{'debug_bounds=True' if debug else ''}) (needs nvcc)")
        L = C.CDLL(path)
        vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.c_void_p
        L.pic_init.argtypes = [C.POINTER(pic_config), C.POINTER(pic_species), C.c_int, dp, dp,
                               C.POINTER(vp)]
        L.pic_step.argtypes = [vp, C.c_int, vp, vp]
        L.pic_step_async.argtypes = [vp, C.c_int]
        L.pic_read_stats.argtypes = [vp, C.c_int, vp, vp, C.POINTER(C.c_int)]
        L.pic_launch_count.argtypes = [vp, i64p]
        L.pic_set_profiling.argtypes = [vp, C.c_int]
        L.pic_profile.argtypes = [vp, C.c_int, i64p, C.POINTER(C.c_double)]
        L.pic_energy.argtypes = [vp, vp, vp, vp, vp]
        L.pic_get_particles.argtypes = [vp, C.c_int, vp, vp]
        L.pic_get_ids.argtypes = [vp, C.c_int, vp]
        L.pic_set_particles.argtypes = [vp, C.c_int, vp, vp]
        L.pic_get_fields.argtypes = [vp, vp, vp]
        L.pic_set_fields.argtypes = [vp, vp, vp]
        L.pic_step_count.argtypes = [vp, i64p]
        L.pic_mixed_resolution.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                           C.POINTER(C.c_int)]
        dblp = C.POINTER(C.c_double)
        L.pic_charge.argtypes = [vp, dblp, dblp, dblp, dblp, vp]
        L.pic_es1d_step_noalloc.argtypes = [C.POINTER(pic_config), C.c_double, C.c_double,
                                             C.c_double, C.c_int64, vp, vp, vp, C.c_int, vp, vp]
        L.pic_grad_forward.argtypes = [vp, C.c_int, C.c_int]
        L.pic_grad_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.pic_debug_bounds.argtypes = [C.c_int64, C.c_int64, C.POINTER(C.c_int)]
        L.pic_free.argtypes = [vp]
        L.pic_free.restype = None
        L.pic_batch_init.argtypes = [C.POINTER(pic_config), C.POINTER(pic_species), C.c_int,
                                     C.POINTER(vp)]
        L.pic_batch_step.argtypes = [vp, C.c_int]
        L.pic_batch_set_graph.argtypes = [vp, C.c_int]
        L.pic_batch_read_stats.argtypes = [vp, C.c_int, vp, vp, C.POINTER(C.c_int)]
        L.pic_batch_run.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.pic_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), i64p]
        L.pic_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.pic_batch_free.argtypes = [vp]
        L.pic_batch_free.restype = None
        L.pic_last_error.restype = C.c_char_p
        L.pic_version.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("pic_free", "pic_last_error", "pic_version", "pic_batch_free"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != PIC_OK:
        raise PicError(rc, lib().pic_last_error().decode())


def _addr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "arrays must be contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def make_config(nc, L, dt, order=1, scheme=PIC_SCHEME_ESEC2, precision=PIC_PREC_FP64,
                solver=PIC_SOLVER_AMPERE_ES, dim_x=1, dim_v=1, ny=0, Ly=0.0, c=1.0,
                sort_period=0, remove_mean=1, gamma_on=1, ptr_on_device=0, stream=None,
                skip_ids=0, binomial_passes=0, charge_conserving=0, gamma_fp64=0,
                separate_passes=0):
    g = pic_grid(dim_x, dim_v, (C.c_int64 * 2)(nc, ny), (C.c_double * 2)(L, Ly))
    return pic_config(g, order, dt, c, solver, scheme, precision, sort_period, int(remove_mean),
                      int(gamma_on), int(ptr_on_device), stream, int(skip_ids),
                      int(binomial_passes), int(charge_conserving), int(gamma_fp64),
                      int(separate_passes))


def pic_init(cfg: pic_config, species: Sequence[dict], E0=None, B0=None) -> int:
    """species: dicts with q, m, x, v, w (or None), w0.  Returns the handle."""
    arr = (pic_species * len(species))()
    keep = []
    for i, s in enumerate(species):
        n = s["n"] if "n" in s else (s["x"].shape[-1] if s["x"] is not None else 0)
        arr[i] = pic_species(s["q"], s["m"], n, _addr(s["x"]), _addr(s["v"]),
                             _addr(s.get("w")), s.get("w0", 0.0))
        keep.append(s)
    h = C.c_void_p()
    _check(lib().pic_init(C.byref(cfg), arr, len(species), _addr(E0), _addr(B0), C.byref(h)))
    return h.value


def pic_step(h: int, nsteps: int, nfallback_per_step=None, te_per_step=None):
    _check(lib().pic_step(h, nsteps, _addr(nfallback_per_step), _addr(te_per_step)))


def pic_step_async(h: int, nsteps: int):
    _check(lib().pic_step_async(h, nsteps))


def pic_read_stats(h: int, capacity: int = 1024):
    """Returns (fallbacks, total energies) of the steps pending since the last read."""
    fb = np.zeros(capacity, dtype=np.int64)
    te = np.zeros(capacity)
    n = C.c_int()
    _check(lib().pic_read_stats(h, capacity, fb.ctypes.data, te.ctypes.data, C.byref(n)))
    return fb[:n.value], te[:n.value]


def pic_launch_count(h: int) -> int:
    n = C.c_int64()
    _check(lib().pic_launch_count(h, C.byref(n)))
    return n.value


def pic_set_profiling(h: int, on: bool):
    _check(lib().pic_set_profiling(h, int(on)))


def pic_profile(h: int, kind: int):
    """(launches, total device ms) of one kernel kind since profiling was enabled."""
    n = C.c_int64()
    ms = C.c_double()
    _check(lib().pic_profile(h, kind, C.byref(n), C.byref(ms)))
    return n.value, ms.value


def pic_energy(h: int, nspecies: int):
    ke = np.zeros(nspecies)
    we, wb, te = C.c_double(), C.c_double(), C.c_double()
    _check(lib().pic_energy(h, ke.ctypes.data, C.addressof(we), C.addressof(wb),
                            C.addressof(te)))
    return ke, we.value, wb.value, te.value


def pic_get_particles(h: int, s: int, x, v):
    _check(lib().pic_get_particles(h, s, _addr(x), _addr(v)))


def pic_get_ids(h: int, s: int, ids):
    _check(lib().pic_get_ids(h, s, _addr(ids)))


def pic_set_particles(h: int, s: int, x, v):
    _check(lib().pic_set_particles(h, s, _addr(x), _addr(v)))


def pic_get_fields(h: int, E, B=None):
    _check(lib().pic_get_fields(h, _addr(E), _addr(B)))


def pic_set_fields(h: int, E, B=None):
    _check(lib().pic_set_fields(h, _addr(E), _addr(B)))


def pic_charge(h: int, residual=None):
    """Charge diagnostics (see pic.h): dict with Q_markers, Q_grid, gauss_l2,
    rho_l2; residual (optional array of the grid's nodes) receives r."""
    q, g, l2, p2 = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(lib().pic_charge(h, C.byref(q), C.byref(g), C.byref(l2), C.byref(p2),
                            _addr(residual)))
    return dict(Q_markers=q.value, Q_grid=g.value, gauss_l2=l2.value, rho_l2=p2.value)


def pic_mixed_resolution(h: int):
    """(dx, dv, deposit_bits) of a mixed-form handle (see pic.h)."""
    dx, dv, T = C.c_double(), C.c_double(), C.c_int()
    _check(lib().pic_mixed_resolution(h, C.byref(dx), C.byref(dv), C.byref(T)))
    return dx.value, dv.value, T.value


def pic_step_count(h: int) -> int:
    n = C.c_int64()
    _check(lib().pic_step_count(h, C.byref(n)))
    return n.value


def pic_free(h: int):
    lib().pic_free(h)


def pic_es1d_step_noalloc(cfg: pic_config, q: float, m: float, w0: float, n: int, x, v, E,
                          nsteps: int, nfallback_per_step=None, te_per_step=None):
    """Steps caller-owned device arrays without any device allocation (see pic.h)."""
    _check(lib().pic_es1d_step_noalloc(C.byref(cfg), q, m, w0, n, _addr(x), _addr(v), _addr(E),
                                       nsteps, _addr(nfallback_per_step), _addr(te_per_step)))


def pic_version() -> str:
    return lib().pic_version().decode()


def pic_debug_bounds(index: int, extent: int) -> int:
    """One device-side index check of the debug-bounds build: 1 if it flagged
    index outside [0, extent), 0 if it passed."""
    flagged = C.c_int()
    _check(lib().pic_debug_bounds(index, extent, C.byref(flagged)))
    return flagged.value


class Simulation:
    """Convenience owner of one handle built from a ``workloads.Problem1D``."""

    def __init__(self, prob, scheme=PIC_SCHEME_ESEC2, precision=PIC_PREC_FP64, E0=None,
                 sort_period=0, remove_mean=True, gamma_on=True, stream=None,
                 solver=PIC_SOLVER_AMPERE_ES, binomial_passes=0, gamma_fp64=False,
                 separate_passes=False):
        """solver PIC_SOLVER_STANDARD_LEAPFROG selects the standard-PIC comparator
        (its particles() then returns v^{n-1/2})."""
        self.prob = prob
        self.cfg = make_config(prob.nc, prob.L, prob.dt, prob.order, scheme, precision,
                               sort_period=sort_period, remove_mean=remove_mean,
                               gamma_on=gamma_on, stream=stream, solver=solver,
                               binomial_passes=binomial_passes, gamma_fp64=gamma_fp64,
                               separate_passes=separate_passes)
        self.species = [dict(q=s.q, m=s.m, x=np.ascontiguousarray(s.x, dtype=np.float64),
                             v=np.ascontiguousarray(s.v, dtype=np.float64),
                             w=None if s.w is None else np.ascontiguousarray(s.w, np.float64),
                             w0=s.w0) for s in prob.species]
        self.h = pic_init(self.cfg, self.species, E0)

    def step(self, nsteps: int):
        fb = np.zeros(nsteps, dtype=np.int64)
        te = np.zeros(nsteps)
        pic_step(self.h, nsteps, fb, te)
        return fb, te

    def particles(self, s: int = 0):
        n = len(self.species[s]["x"])
        x, v = np.zeros(n), np.zeros(n)
        pic_get_particles(self.h, s, x, v)
        ids = np.zeros(n, dtype=np.int64)
        pic_get_ids(self.h, s, ids)
        xo, vo = np.zeros(n), np.zeros(n)
        xo[ids], vo[ids] = x, v
        return xo, vo

    def field(self):
        E = np.zeros(self.prob.nc)
        pic_get_fields(self.h, E)
        return E

    def energy(self):
        return pic_energy(self.h, len(self.species))

    def close(self):
        if self.h:
            pic_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation2D:
    """Owner of one Yee-solver handle built from a ``workloads.Problem2D``."""

    def __init__(self, prob, scheme=PIC_SCHEME_ESEC2, E0=None, B0=None, gamma_on=True,
                 precision=PIC_PREC_FP64, charge_conserving=False, sort_period=0,
                 skip_ids=False):
        self.prob = prob
        self.cfg = make_config(prob.nx, prob.Lx, prob.dt, prob.order, scheme, precision,
                               solver=PIC_SOLVER_YEE_LEAPFROG, dim_x=2, dim_v=3, ny=prob.ny,
                               Ly=prob.Ly, c=prob.c, gamma_on=gamma_on,
                               charge_conserving=charge_conserving, sort_period=sort_period,
                               skip_ids=int(skip_ids))
        self.species = []
        for s in prob.species:
            x = np.ascontiguousarray(np.stack([s.x, s.y]), dtype=np.float64)
            v = np.ascontiguousarray(np.stack([s.vx, s.vy, s.vz]), dtype=np.float64)
            self.species.append(dict(q=s.q, m=s.m, x=x, v=v, n=len(s.x),
                                     w=None if s.w is None else np.ascontiguousarray(s.w),
                                     w0=s.w0))
        self.h = pic_init(self.cfg, self.species,
                          None if E0 is None else np.ascontiguousarray(E0, dtype=np.float64),
                          None if B0 is None else np.ascontiguousarray(B0, dtype=np.float64))

    def step(self, nsteps: int):
        fb = np.zeros(nsteps, dtype=np.int64)
        te = np.zeros(nsteps)
        pic_step(self.h, nsteps, fb, te)
        return fb, te

    def particles(self, s: int = 0):
        """(x [2, n], v [3, n]) of species s in the order the markers were given."""
        n = self.species[s]["n"]
        x, v = np.zeros((2, n)), np.zeros((3, n))
        pic_get_particles(self.h, s, x, v)
        ids = np.zeros(n, dtype=np.int64)
        pic_get_ids(self.h, s, ids)
        xo, vo = np.zeros_like(x), np.zeros_like(v)
        xo[:, ids], vo[:, ids] = x, v
        return xo, vo

    def fields(self):
        shape = (3, self.prob.ny, self.prob.nx)
        E, B = np.zeros(shape), np.zeros(shape)
        pic_get_fields(self.h, E, B)
        return E, B

    def energy(self):
        return pic_energy(self.h, len(self.species))

    def close(self):
        if self.h:
            pic_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation1D2V:
    """Owner of one spectral-solver handle (Crank-Nicolson or PSATD) built from
    a ``workloads.Problem1D2V``."""

    def __init__(self, prob, solver=PIC_SOLVER_PSATD, scheme=PIC_SCHEME_ESEC2, E0=None, B0=None,
                 gamma_on=True, stream=None, precision=PIC_PREC_FP64):
        self.prob = prob
        self.cfg = make_config(prob.n, prob.L, prob.dt, prob.order, scheme, precision,
                               solver=solver, dim_x=1, dim_v=2, c=prob.c, gamma_on=gamma_on,
                               stream=stream)
        self.species = []
        for s in prob.species:
            self.species.append(dict(q=s.q, m=s.m, x=np.ascontiguousarray(s.y, dtype=np.float64),
                                     v=np.ascontiguousarray(np.stack([s.vx, s.vy]),
                                                            dtype=np.float64),
                                     n=len(s.y),
                                     w=None if s.w is None else np.ascontiguousarray(s.w),
                                     w0=s.w0))
        E0 = prob.E0 if E0 is None else E0
        B0 = prob.B0 if B0 is None else B0
        self.h = pic_init(self.cfg, self.species, np.ascontiguousarray(E0, dtype=np.float64),
                          np.ascontiguousarray(B0, dtype=np.float64))

    def step(self, nsteps: int):
        fb = np.zeros(nsteps, dtype=np.int64)
        te = np.zeros(nsteps)
        pic_step(self.h, nsteps, fb, te)
        return fb, te

    def particles(self, s: int = 0):
        """(y, vx, vy) of species s."""
        n = self.species[s]["n"]
        y, v = np.zeros(n), np.zeros((2, n))
        pic_get_particles(self.h, s, y, v)
        return y, v[0], v[1]

    def fields(self):
        """(E [2, n], Bz [n])."""
        E, B = np.zeros((2, self.prob.n)), np.zeros(self.prob.n)
        pic_get_fields(self.h, E, B)
        return E, B

    def energy(self):
        return pic_energy(self.h, len(self.species))

    def close(self):
        if self.h:
            pic_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches


def pic_batch_init(cfgs: Sequence[pic_config], species: Sequence[dict]) -> int:
    """Run r from cfgs[r] and the single species dict species[r]; returns the batch."""
    n = len(cfgs)
    ca = (pic_config * n)(*cfgs)
    sa = (pic_species * n)()
    for i, s in enumerate(species):
        sa[i] = pic_species(s["q"], s["m"], s["x"].shape[-1], _addr(s["x"]), _addr(s["v"]),
                            _addr(s.get("w")), s.get("w0", 0.0))
    b = C.c_void_p()
    _check(lib().pic_batch_init(ca, sa, n, C.byref(b)))
    return b.value


def pic_batch_step(b: int, nsteps: int):
    _check(lib().pic_batch_step(b, nsteps))


def pic_batch_set_graph(b: int, on: bool):
    _check(lib().pic_batch_set_graph(b, int(on)))


def pic_batch_read_stats(b: int, nruns: int, capacity: int = 1024):
    """(fallbacks [runs, steps], total energies [runs, steps]) since the last read."""
    fb = np.zeros((nruns, capacity), dtype=np.int64)
    te = np.zeros((nruns, capacity))
    n = C.c_int()
    _check(lib().pic_batch_read_stats(b, capacity, fb.ctypes.data, te.ctypes.data, C.byref(n)))
    return fb[:, :n.value], te[:, :n.value]


def pic_batch_run(b: int, run: int) -> int:
    h = C.c_void_p()
    _check(lib().pic_batch_run(b, run, C.byref(h)))
    return h.value


def pic_batch_info(b: int):
    nr, nb, nl = C.c_int(), C.c_int(), C.c_int64()
    _check(lib().pic_batch_info(b, C.byref(nr), C.byref(nb), C.byref(nl)))
    return nr.value, nb.value, nl.value


def pic_batch_autotune(b: int, steps_per_trial: int) -> int:
    """Times each work list for steps_per_trial real steps and keeps the fastest;
    returns its trips per block."""
    t = C.c_int()
    _check(lib().pic_batch_autotune(b, steps_per_trial, C.byref(t)))
    return t.value


def pic_batch_free(b: int):
    lib().pic_batch_free(b)


class Batch:
    """Independent 1D problems (workloads.Problem1D, one species each) stepped
    together in the mixed form."""

    def __init__(self, problems, scheme=PIC_SCHEME_ESEC2, graphs=False, stream=None):
        """stream: a cudaStream_t (int) for every run, or None for a stream the batch
        creates."""
        self.problems = problems
        cfgs = [make_config(p.nc, p.L, p.dt, p.order, scheme, PIC_PREC_MIXED, stream=stream)
                for p in problems]
        sp = [dict(q=p.species[0].q, m=p.species[0].m, x=p.species[0].x, v=p.species[0].v,
                   w=None, w0=p.species[0].w0) for p in problems]
        self.b = pic_batch_init(cfgs, sp)
        if graphs:
            pic_batch_set_graph(self.b, True)

    def step(self, nsteps: int):
        """Steps every run; returns (fallbacks, total energies), each [runs, steps]."""
        fbs, tes = [], []
        done = 0
        while done < nsteps:
            k = min(1024, nsteps - done)
            pic_batch_step(self.b, k)
            fb, te = pic_batch_read_stats(self.b, len(self.problems))
            fbs.append(fb)
            tes.append(te)
            done += k
        return np.concatenate(fbs, axis=1), np.concatenate(tes, axis=1)

    def run(self, r: int) -> int:
        return pic_batch_run(self.b, r)

    def particles(self, r: int):
        n = self.problems[r].n_markers
        x, v = np.zeros(n), np.zeros(n)
        pic_get_particles(self.run(r), 0, x, v)
        return x, v

    def field(self, r: int):
        E = np.zeros(self.problems[r].nc)
        pic_get_fields(self.run(r), E)
        return E

    def close(self):
        if self.b:
            pic_batch_free(self.b)
            self.b = None


# ------------------------------------------------------------------ gradients


def pic_grad_forward(h: int, nsteps: int, checkpoint_every: int = 50):
    _check(lib().pic_grad_forward(h, nsteps, checkpoint_every))


def pic_grad_backward(h: int, Ebar=None, xbar=None, vbar=None, Ebar0=None, xbar0=None,
                      vbar0=None, wbar0=None):
    """Adjoints of the state before the forward steps into the given arrays."""
    _check(lib().pic_grad_backward(h, _addr(Ebar), _addr(xbar), _addr(vbar), _addr(Ebar0),
                                   _addr(xbar0), _addr(vbar0), _addr(wbar0)))


def differentiable_steps(h: int, nsteps: int, x0, v0, E0, w=None, checkpoint_every: int = 50):
    """Steps the FP64 1D handle h (one species) nsteps steps from (x0, v0, E0)
    and returns (x, v, E) after them as torch tensors whose gradients flow back
    to x0, v0, E0 and w through pic_grad_backward.  w, when given, must be the
    marker weights h was created with (the steps use those); its gradient is
    returned all the same.  Inputs are float64 tensors on the CPU or the GPU."""
    import torch

    class _Steps(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x0, v0, E0, w):
            ctx.dev, ctx.n, ctx.nc = x0.device, x0.numel(), E0.numel()
            xs, vs, Es = (t.detach().contiguous().to(torch.float64) for t in (x0, v0, E0))
            if ctx.dev.type == "cuda":
                torch.cuda.synchronize(ctx.dev)
            pic_set_particles(h, 0, xs, vs)
            pic_set_fields(h, Es)
            pic_grad_forward(h, nsteps, checkpoint_every)
            x, v, E = torch.empty_like(xs), torch.empty_like(vs), torch.empty_like(Es)
            pic_get_particles(h, 0, x, v)
            pic_get_fields(h, E)
            return x, v, E

        @staticmethod
        def backward(ctx, gx, gv, gE):
            gx, gv, gE = (None if t is None else t.detach().contiguous().to(torch.float64)
                          for t in (gx, gv, gE))
            xb0 = torch.zeros(ctx.n, dtype=torch.float64, device=ctx.dev)
            vb0, wb0 = torch.zeros_like(xb0), torch.zeros_like(xb0)
            Eb0 = torch.zeros(ctx.nc, dtype=torch.float64, device=ctx.dev)
            if ctx.dev.type == "cuda":
                torch.cuda.synchronize(ctx.dev)
            pic_grad_backward(h, gE, gx, gv, Eb0, xb0, vb0, wb0)
            return xb0, vb0, Eb0, wb0

    if w is None:
        w = torch.zeros(x0.numel(), dtype=torch.float64, device=x0.device)
    return _Steps.apply(x0, v0, E0, w)
