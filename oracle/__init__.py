"""FP64 CPU oracle of the coupled electroconvection step (arXiv:1812.05711).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_1812_05711_gb300``) never imports it
and shares no code with it.

The arithmetic lives in ``ehd_oracle.c`` (plain C, double precision, one
thread).  This module only compiles it with gcc and marshals numpy arrays
through ctypes.  Functions and the passages they follow:

* :func:`setup`            -- Eq. 26 groups -> lattice units, Eqs. 16-17 rates
* :func:`hydrostatic`      -- Eqs. 27-28 constants from the wall conditions
* :func:`dft` / :func:`fft` -- Eq. 19
* :func:`thomas`           -- tridiagonal solve used per wavenumber (Eq. 18)
* :func:`poisson`          -- Sec. IV.3 (Eqs. 18-25)
* :func:`poisson_oddext`   -- Sec. IV.3 literally (Eqs. 19-25, odd extension)
* :func:`init_state`       -- Eqs. 27-29
* :func:`step`             -- Eqs. 5-17 and Table I
* :func:`fields`           -- Eqs. 5-7 and E = -grad phi
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ehd_oracle.c")
_HDR = os.path.join(_HERE, "ehd_oracle.h")
_LIB = os.path.join(_HERE, "libehd_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libehd_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

NDIAG = 6  # mass, charge, q_in, q_out, kinetic energy, max|u_y|
FIELDS = ("rho", "ux", "uy", "rho_c", "phi", "Ex", "Ey")


class Params(ctypes.Structure):
    _fields_ = [
        ("Nx", ctypes.c_int), ("Ny", ctypes.c_int),
        ("T", ctypes.c_double), ("C", ctypes.c_double),
        ("M", ctypes.c_double), ("Fe", ctypes.c_double),
        ("Lambda", ctypes.c_double), ("Lambda_g", ctypes.c_double),
        ("u_ion", ctypes.c_double),
        ("wall_mode", ctypes.c_int), ("x_symbol", ctypes.c_int),
        ("ex_spectral", ctypes.c_int), ("dc_printed", ctypes.c_int),
        ("periodic_y", ctypes.c_int), ("no_poisson", ctypes.c_int),
        ("no_force", ctypes.c_int),
        ("ext_E", ctypes.c_double * 2), ("ext_F", ctypes.c_double * 2),
        ("rho_ref", ctypes.c_double), ("dphi0", ctypes.c_double),
        ("phi0", ctypes.c_double), ("H", ctypes.c_double),
        ("mu_b", ctypes.c_double), ("eps", ctypes.c_double),
        ("nu", ctypes.c_double), ("rho0", ctypes.c_double),
        ("Dc", ctypes.c_double),
        ("tau_p", ctypes.c_double), ("tau_m", ctypes.c_double),
        ("taug_p", ctypes.c_double), ("taug_m", ctypes.c_double),
        ("rho_a", ctypes.c_double), ("y_a", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: (list(getattr(self, name)) if name in ("ext_E", "ext_F")
                       else getattr(self, name)) for name, _ in self._fields_}


def _compile(out: str, extra, force: bool) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", *extra,
             "-shared", "-o", tmp, _SRC, "-lm"], cwd=_HERE)
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ehd_oracle.c into libehd_oracle.so next to it (gcc, -O2), and
    the same source with -fopenmp into libehd_oracle_omp.so (used only to
    time the oracle on all host cores; if the compiler has no OpenMP, that
    build is skipped)."""
    with _lock:
        _compile(_LIB, [], force)
        try:
            _compile(_LIB_OMP, ["-fopenmp"], force)
        except (subprocess.CalledProcessError, OSError):
            pass
    return _LIB


def use_threads(n: int | None = None) -> int:
    """Switch this process's oracle calls to the -fopenmp build with n
    threads (all host cores when None).  Rows, wavenumbers and nodes are
    shared among threads; the states it computes are bitwise those of the
    one-thread build (only the diagnostic sums are reordered).  Returns the
    thread count, or 0 if no OpenMP build is available.  For timing only."""
    global _lib, _lib_omp
    build()
    if not os.path.exists(_LIB_OMP):
        return 0
    with _lock:
        if _lib_omp is None:
            _lib_omp = ctypes.CDLL(_LIB_OMP)
        L = _lib_omp
    _declare(L)
    L.orc_threads.argtypes = [ctypes.c_int]
    L.orc_threads.restype = ctypes.c_int
    got = L.orc_threads(int(n) if n else (os.cpu_count() or 1))
    _lib = L
    return got


def use_one_thread():
    """Back to the one-thread build."""
    global _lib
    _lib = None
    lib()


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    """ctypes signatures of the oracle library L."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(Params)
    L.orc_setup.argtypes = [pp]
    L.orc_setup.restype = ctypes.c_int
    L.orc_lattice.argtypes = [ip, ip, dp, ip]
    L.orc_hydrostatic_params.argtypes = [ctypes.c_double] * 4 + [dp, dp]
    L.orc_hydrostatic_params.restype = ctypes.c_int
    L.orc_dft.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
    L.orc_fft.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
    L.orc_thomas.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
    L.orc_poisson_general.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, dp, dp]
    L.orc_poisson_oddext.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, dp, dp]
    L.orc_poisson.argtypes = [pp, dp, dp]
    L.orc_efield.argtypes = [pp, dp, dp, dp]
    L.orc_perturbation.argtypes = [pp, ctypes.c_int, dp, dp, ctypes.c_double,
                                   ctypes.c_double, dp, dp]
    L.orc_init.argtypes = [pp, ctypes.c_int, dp, dp, dp, dp, dp]
    L.orc_fields.argtypes = [pp, dp, dp, dp, dp]
    L.orc_step.argtypes = [pp, dp, dp, dp, ctypes.c_long, dp]


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def setup(Nx, Ny, T, C, M, Fe, Lambda, Lambda_g=1e-6, u_ion=2e-3, wall_mode=0,
          periodic_y=0, no_poisson=0, no_force=0, ext_E=(0.0, 0.0),
          ext_F=(0.0, 0.0), x_symbol=0, ex_spectral=0, dc_printed=0) -> Params:
    p = Params()
    p.Nx, p.Ny = int(Nx), int(Ny)
    p.T, p.C, p.M, p.Fe = float(T), float(C), float(M), float(Fe)
    p.Lambda, p.Lambda_g, p.u_ion = float(Lambda), float(Lambda_g), float(u_ion)
    p.wall_mode = int(wall_mode)
    p.x_symbol = int(x_symbol)
    p.ex_spectral = int(ex_spectral)
    p.dc_printed = int(dc_printed)
    p.periodic_y, p.no_poisson, p.no_force = int(periodic_y), int(no_poisson), int(no_force)
    p.ext_E[0], p.ext_E[1] = float(ext_E[0]), float(ext_E[1])
    p.ext_F[0], p.ext_F[1] = float(ext_F[0]), float(ext_F[1])
    if lib().orc_setup(ctypes.byref(p)) != 0:
        raise ValueError("oracle: invalid parameters")
    return p


def lattice():
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    opp = (ctypes.c_int * 9)()
    lib().orc_lattice(cx, cy, w, opp)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:]))


def hydrostatic(rho0, eps, H, dphi0):
    ra, ya = ctypes.c_double(), ctypes.c_double()
    if lib().orc_hydrostatic_params(rho0, eps, H, dphi0, ctypes.byref(ra),
                                    ctypes.byref(ya)) != 0:
        raise ValueError("oracle: hydrostatic solve failed")
    return ra.value, ya.value


def dft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    ore, oim = np.empty_like(re), np.empty_like(im)
    lib().orc_dft(len(x), _dp(re), _dp(im), _dp(ore), _dp(oim), sign)
    return ore + 1j * oim


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.ascontiguousarray(x.real).copy(), np.ascontiguousarray(x.imag).copy()
    lib().orc_fft(len(x), _dp(re), _dp(im), sign)
    return re + 1j * im


def thomas(a, b, c, d) -> np.ndarray:
    a, b, c = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c))
    d = np.asarray(d, dtype=np.complex128)
    dre, dim = np.ascontiguousarray(d.real).copy(), np.ascontiguousarray(d.imag).copy()
    lib().orc_thomas(len(b), _dp(a), _dp(b), _dp(c), _dp(dre), _dp(dim))
    return dre + 1j * dim


def poisson_general(src: np.ndarray, wall_mode=0, phi_bottom=0.0, phi_top=0.0, x_symbol=0):
    """Solve [Dx^2 + Dy^2] phi = src on an Ny x Nx grid (Sec. IV.3); Dx^2 is
    spectral (Eq. 20, x_symbol 0) or the 3-point difference (x_symbol 1)."""
    src = np.ascontiguousarray(src, dtype=np.float64)
    Ny, Nx = src.shape
    phi = np.empty_like(src)
    lib().orc_poisson_general(Nx, Ny, wall_mode, x_symbol, phi_bottom, phi_top, _dp(src), _dp(phi))
    return phi


def poisson_oddext(src: np.ndarray, wall_mode=0, phi_bottom=0.0, phi_top=0.0, x_symbol=0):
    """The same solve as :func:`poisson_general` in the literal form of
    Sec. IV.3: odd extension in y (Eqs. 21-22), 2-D transform, division by
    the symbol (Eqs. 20, 24), inverse, first half (Eq. 25)."""
    src = np.ascontiguousarray(src, dtype=np.float64)
    Ny, Nx = src.shape
    phi = np.empty_like(src)
    lib().orc_poisson_oddext(Nx, Ny, wall_mode, x_symbol, phi_bottom, phi_top, _dp(src), _dp(phi))
    return phi


def poisson(p: Params, rhoc: np.ndarray) -> np.ndarray:
    rhoc = np.ascontiguousarray(rhoc, dtype=np.float64)
    phi = np.empty_like(rhoc)
    lib().orc_poisson(ctypes.byref(p), _dp(rhoc), _dp(phi))
    return phi


def efield(p: Params, phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    Ex, Ey = np.empty_like(phi), np.empty_like(phi)
    lib().orc_efield(ctypes.byref(p), _dp(phi), _dp(Ex), _dp(Ey))
    return Ex, Ey


def perturbation(p: Params, amp, phase, x, y):
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    phase = np.ascontiguousarray(phase, dtype=np.float64)
    ux, uy = ctypes.c_double(), ctypes.c_double()
    lib().orc_perturbation(ctypes.byref(p), len(amp), _dp(amp), _dp(phase),
                           float(x), float(y), ctypes.byref(ux), ctypes.byref(uy))
    return ux.value, uy.value


class State:
    """Populations f, g ([9][Ny][Nx]) and potential phi ([Ny][Nx])."""

    def __init__(self, p: Params, f: np.ndarray, g: np.ndarray, phi: np.ndarray):
        self.p, self.f, self.g, self.phi = p, f, g, phi
        self.t = 0

    def copy(self):
        s = State(self.p, self.f.copy(), self.g.copy(), self.phi.copy())
        s.t = self.t
        return s


def init_state(p: Params, amp=(1e-3,), phase=(0.0,)) -> State:
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    phase = np.ascontiguousarray(phase, dtype=np.float64)
    assert len(amp) == len(phase)
    f = np.empty((9, p.Ny, p.Nx))
    g = np.empty((9, p.Ny, p.Nx))
    phi = np.empty((p.Ny, p.Nx))
    lib().orc_init(ctypes.byref(p), len(amp), _dp(amp), _dp(phase), _dp(f), _dp(g), _dp(phi))
    return State(p, f, g, phi)


def state_from(p: Params, f: np.ndarray, g: np.ndarray) -> State:
    """Wrap given populations and solve phi for them."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    g = np.ascontiguousarray(g, dtype=np.float64).copy()
    phi = np.zeros((p.Ny, p.Nx))
    if not p.no_poisson:
        phi = poisson(p, g.sum(axis=0))
    return State(p, f, g, phi)


def step(s: State, n: int = 1, diag: bool = False):
    """Advance the state n coupled steps in place; return per-step diagnostics."""
    d = np.empty((max(n, 1), NDIAG)) if diag else None
    lib().orc_step(ctypes.byref(s.p), _dp(s.f), _dp(s.g), _dp(s.phi), int(n),
                   _dp(d) if diag else None)
    s.t += n
    return d


def fields(s: State) -> dict:
    out = np.empty((7, s.p.Ny, s.p.Nx))
    lib().orc_fields(ctypes.byref(s.p), _dp(s.f), _dp(s.g), _dp(s.phi), _dp(out))
    return {k: out[i] for i, k in enumerate(FIELDS)}
