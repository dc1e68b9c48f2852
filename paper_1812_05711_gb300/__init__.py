"""GB300 electroconvection step (arXiv:1812.05711) -- Python binding.

Thin ctypes marshalling over the C ABI in ``include/ehd.h`` (library
``libehd.so``, CUDA kernels for sm_103a).  Every step of the method runs in
those kernels; this module only converts arguments.  There is no CPU path:
if the library cannot be loaded, importing the functions raises.

PyTorch is used for device memory only: :func:`use_torch_allocator` routes the
library's device allocations through the PyTorch caching allocator, and
:class:`Run` gives each run its own ``torch.cuda.Stream``.

The module-level functions carry the C names (``ehd_create``,
``ehd_poisson``, ``ehd_step``, ``ehd_fields``, ...) and the same argument
order; numpy arrays are passed for host buffers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

FIELDS = ("rho", "ux", "uy", "rho_c", "phi", "Ex", "Ey")
FIELD_BITS = {name: 1 << i for i, name in enumerate(FIELDS)}
FIELD_ALL = 0x7F
NDIAG = 8
DIAG_NAMES = ("mass", "charge", "q_in", "q_out", "kinetic", "max_uy", "max_u", "step")
PARAM_NAMES = ("Nx", "Ny", "H", "mu_b", "eps", "nu", "rho0", "Dc", "tau_p", "tau_m",
               "taug_p", "taug_m", "rho_a", "y_a", "storage", "compute")
STORAGE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
COMPUTE = {"f64": 0, "f32": 1}
MAX_PERT_MODES = 16

STATUS = {0: "EHD_OK", -1: "EHD_EINVAL", -2: "EHD_ENOMEM", -3: "EHD_ECUDA",
          -4: "EHD_EDIVERGED", -5: "EHD_ETIMEOUT", -6: "EHD_EBUSY"}


class EhdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int), ("compute", ctypes.c_int),
        ("lambda_g", ctypes.c_double), ("u_ion", ctypes.c_double),
        ("wall_mode", ctypes.c_int), ("n_modes", ctypes.c_int),
        ("pert_amp", ctypes.c_double * MAX_PERT_MODES),
        ("pert_phase", ctypes.c_double * MAX_PERT_MODES),
        ("stream", ctypes.c_void_p),
        ("step_kernel", ctypes.c_int),
        ("x_symbol", ctypes.c_int),
        ("ex_spectral", ctypes.c_int),
        ("perturbation", ctypes.c_int),
        ("dc_printed", ctypes.c_int),
    ]


_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libehd.so (building it first if it is missing or stale)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if _build.stale():
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.ehd_default_options.argtypes = [ctypes.POINTER(Options)]
        L.ehd_default_options.restype = None
        L.ehd_create.argtypes = [ip, ip] + [ctypes.c_double] * 5 + [ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.ehd_poisson.argtypes = [vp]
        L.ehd_step.argtypes = [vp, ctypes.c_long]
        L.ehd_step_profile.argtypes = [vp, ctypes.c_long, dp]
        L.ehd_fields.argtypes = [vp, ctypes.c_uint, dp]
        L.ehd_diagnostics.argtypes = [vp, dp]
        L.ehd_load.argtypes = [vp, dp, dp]
        L.ehd_save.argtypes = [vp, dp, dp]
        L.ehd_params.argtypes = [vp, dp]
        L.ehd_footprint.argtypes = [ip, ip, ip, ctypes.POINTER(ctypes.c_size_t)]
        L.ehd_sync.argtypes = [vp]
        L.ehd_stream.argtypes = [vp]
        L.ehd_stream.restype = vp
        L.ehd_destroy.argtypes = [vp]
        L.ehd_destroy.restype = None
        L.ehd_last_error.restype = ctypes.c_char_p
        L.ehd_set_allocator.argtypes = [vp, vp, vp]
        L.ehd_tune.argtypes = [vp, ip, ip]
        L.ehd_tune.restype = ctypes.c_int
        L.ehd_tune_get.argtypes = [vp, ip]
        L.ehd_tune_get.restype = ctypes.c_int
        L.ehd_batch_create.argtypes = [ip, ctypes.c_size_t, ip, ip, vp, ctypes.POINTER(vp)]
        L.ehd_batch_add.argtypes = [vp, vp, ctypes.c_long]
        L.ehd_batch_remove.argtypes = [vp, vp]
        L.ehd_batch_tick.argtypes = [vp, ip]
        L.ehd_batch_sync.argtypes = [vp]
        L.ehd_batch_admits.argtypes = [vp, ip, ip, ip]
        L.ehd_batch_memory.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
        for name in ("ehd_batch_create", "ehd_batch_add", "ehd_batch_remove", "ehd_batch_tick", "ehd_batch_sync",
                     "ehd_batch_admits", "ehd_batch_memory"):
            getattr(L, name).restype = ctypes.c_int
        L.ehd_batch_remaining.argtypes = [vp, vp]
        L.ehd_batch_remaining.restype = ctypes.c_long
        L.ehd_batch_size.argtypes = [vp]
        L.ehd_batch_size.restype = ctypes.c_int
        L.ehd_batch_stream.argtypes = [vp]
        L.ehd_batch_stream.restype = vp
        L.ehd_batch_tune.argtypes = [vp, ip, ip]
        L.ehd_batch_tune.restype = ctypes.c_int
        L.ehd_batch_tune_get.argtypes = [vp, ip]
        L.ehd_batch_tune_get.restype = ctypes.c_int
        L.ehd_batch_destroy.argtypes = [vp]
        L.ehd_batch_destroy.restype = None
        L.ehd_poisson_noalloc.argtypes = [ip, ip, ctypes.c_double, ctypes.c_double, ip, vp, vp, vp]
        L.ehd_poisson_noalloc.restype = ctypes.c_int
        for name in ("ehd_create", "ehd_poisson", "ehd_step", "ehd_step_profile", "ehd_fields", "ehd_diagnostics",
                     "ehd_load", "ehd_save", "ehd_params", "ehd_footprint", "ehd_sync",
                     "ehd_set_allocator"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(status: int):
    if status != 0:
        raise EhdError(status, lib().ehd_last_error().decode())


def _dp(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous float64 array")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------- allocator (torch)
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_torch_blocks: dict = {}
_torch_lock = threading.Lock()
_callbacks = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator."""
    global _callbacks
    if not enable:
        _check(lib().ehd_set_allocator(None, None, None))
        _callbacks = None
        return
    import torch

    def _alloc(nbytes, ctx):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=torch.cuda.current_device())
        except RuntimeError:
            return None
        with _torch_lock:
            _torch_blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, ctx):
        with _torch_lock:
            _torch_blocks.pop(int(ptr), None)

    _callbacks = (_ALLOC_T(_alloc), _FREE_T(_free))
    _check(lib().ehd_set_allocator(ctypes.cast(_callbacks[0], ctypes.c_void_p),
                                   ctypes.cast(_callbacks[1], ctypes.c_void_p), None))


# ------------------------------------------------------- C-named functions
def ehd_default_options() -> Options:
    o = Options()
    lib().ehd_default_options(ctypes.byref(o))
    return o


def ehd_create(Nx, Ny, T, C, M, Fe, Lambda, opt: Options | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ehd_create(int(Nx), int(Ny), float(T), float(C), float(M), float(Fe), float(Lambda),
                            ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h.value


def ehd_poisson(h):
    _check(lib().ehd_poisson(h))


def ehd_step(h, n: int):
    _check(lib().ehd_step(h, int(n)))


def ehd_step_profile(h, n: int) -> dict:
    out = np.zeros(9)
    _check(lib().ehd_step_profile(h, int(n), _dp(out)))
    return {"collide_stream_ms": out[0], "charge_ms": out[1], "poisson_ms": out[2], "step_ms": out[3],
            "steps": int(out[4]), "fft_fwd_ms": out[5], "modes_ms": out[6], "fft_inv_ms": out[7],
            "mean_mode_ms": out[8]}


def ehd_fields(h, mask: int, out: np.ndarray):
    _check(lib().ehd_fields(h, int(mask), _dp(out)))


def ehd_diagnostics(h, out: np.ndarray):
    _check(lib().ehd_diagnostics(h, _dp(out)))


def ehd_load(h, f: np.ndarray, g: np.ndarray):
    _check(lib().ehd_load(h, _dp(f), _dp(g)))


def ehd_save(h, f: np.ndarray | None, g: np.ndarray | None):
    _check(lib().ehd_save(h, _dp(f) if f is not None else None, _dp(g) if g is not None else None))


def ehd_params(h, out: np.ndarray):
    _check(lib().ehd_params(h, _dp(out)))


def ehd_footprint(Nx, Ny, storage) -> int:
    b = ctypes.c_size_t()
    _check(lib().ehd_footprint(int(Nx), int(Ny), int(storage), ctypes.byref(b)))
    return b.value


def ehd_poisson_noalloc(Nx, Ny, eps, phi0, wall_mode, rhoc_ptr: int, phi_ptr: int, stream: int = 0):
    """Poisson solve on caller-owned device buffers (FP32 [Ny][Nx]) that
    allocates no device memory; see include/ehd.h."""
    _check(lib().ehd_poisson_noalloc(int(Nx), int(Ny), float(eps), float(phi0), int(wall_mode),
                                     ctypes.c_void_p(rhoc_ptr), ctypes.c_void_p(phi_ptr),
                                     ctypes.c_void_p(stream) if stream else None))


TUNE = {"slab_rows": 1, "ring_depth": 2, "step_kernel": 3, "cols_per_lane": 4, "tile_modes": 5, "pdl": 6, "fft_cta": 7,
        "y_solver": 8, "march_tma": 9, "tile_threads": 10,
        "tile_cluster": 11, "tile_tma": 12, "slab_shift": 13}


def ehd_tune(h, param, value: int):
    _check(lib().ehd_tune(h, TUNE[param] if isinstance(param, str) else int(param), int(value)))


def ehd_tune_get(h, param) -> int:
    return int(lib().ehd_tune_get(h, TUNE[param] if isinstance(param, str) else int(param)))


def ehd_sync(h):
    _check(lib().ehd_sync(h))


def ehd_stream(h) -> int:
    return lib().ehd_stream(h) or 0


def ehd_destroy(h):
    lib().ehd_destroy(h)


def ehd_last_error() -> str:
    return lib().ehd_last_error().decode()


# ------------------------------------------------------------ convenience
def make_options(storage="f32", compute=None, lambda_g=1e-6, u_ion=2e-3, wall_mode=0,
                 amp=(), phase=(), stream=None, step_kernel=-1, x_symbol=0, ex_spectral=0,
                 perturbation=0, dc_printed=0) -> Options:
    o = ehd_default_options()
    o.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    if compute is None:
        compute = "f64" if o.storage == 0 and storage == "f64" else "f32"
    o.compute = COMPUTE[compute] if isinstance(compute, str) else int(compute)
    o.lambda_g = float(lambda_g)
    o.u_ion = float(u_ion)
    o.wall_mode = int(wall_mode)
    amp, phase = list(amp), list(phase)
    if len(amp) != len(phase) or len(amp) > MAX_PERT_MODES:
        raise ValueError("amp and phase must have the same length <= 16")
    o.n_modes = len(amp)
    for k, (a, p) in enumerate(zip(amp, phase)):
        o.pert_amp[k] = float(a)
        o.pert_phase[k] = float(p)
    o.stream = stream
    o.step_kernel = int(step_kernel)
    o.x_symbol = int(x_symbol)
    o.ex_spectral = int(ex_spectral)
    o.perturbation = int(perturbation)
    o.dc_printed = int(dc_printed)
    return o


class Run:
    """One channel run on the current CUDA device.

    ``storage``: "f64" (with FP64 compute: the plain double-precision path),
    "f32", "bf16", "f16" (FP32 compute on shifted populations); ``compute``
    may force "f32" on FP64 storage.  ``amp``/``phase``: Eq. 29 x-modes.
    ``perturbation=1`` (FP32 compute): the charge populations are stored and
    collided as departures from an x-uniform base state advanced in FP64.
    ``dc_printed=1``: the charge rates of Eq. 16 as printed (D_c on tau_g+).
    """

    def __init__(self, Nx, Ny, T, C, M, Fe, Lambda, storage="f32", compute=None, lambda_g=1e-6,
                 u_ion=2e-3, wall_mode=0, amp=(), phase=(), stream=None, torch_stream=True, step_kernel=-1,
                 x_symbol=0, ex_spectral=0, perturbation=0, dc_printed=0):
        self.Nx, self.Ny = int(Nx), int(Ny)
        self._stream_obj = None
        if stream is None and torch_stream:
            import torch
            self._stream_obj = torch.cuda.Stream()
            stream = self._stream_obj.cuda_stream
        opt = make_options(storage, compute, lambda_g, u_ion, wall_mode, amp, phase, stream, step_kernel, x_symbol,
                           ex_spectral, perturbation, dc_printed)
        self.handle = ehd_create(Nx, Ny, T, C, M, Fe, Lambda, opt)

    # lifecycle
    def close(self):
        if getattr(self, "handle", None):
            ehd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # operations
    def step(self, n: int = 1):
        ehd_step(self.handle, n)
        return self

    def poisson(self):
        ehd_poisson(self.handle)

    def sync(self):
        ehd_sync(self.handle)

    def fields(self, names=FIELDS) -> dict:
        names = list(names)
        mask = 0
        for n in names:
            mask |= FIELD_BITS[n]
        order = [n for n in FIELDS if FIELD_BITS[n] & mask]
        out = np.empty((len(order), self.Ny, self.Nx))
        ehd_fields(self.handle, mask, out)
        return {n: out[i] for i, n in enumerate(order)}

    def diagnostics(self) -> dict:
        out = np.empty(NDIAG)
        ehd_diagnostics(self.handle, out)
        return dict(zip(DIAG_NAMES, out.tolist()))

    def params(self) -> dict:
        out = np.empty(16)
        ehd_params(self.handle, out)
        return dict(zip(PARAM_NAMES, out.tolist()))

    def load(self, f: np.ndarray, g: np.ndarray):
        ehd_load(self.handle, np.ascontiguousarray(f, dtype=np.float64), np.ascontiguousarray(g, dtype=np.float64))

    def save(self):
        f = np.empty((9, self.Ny, self.Nx))
        g = np.empty((9, self.Ny, self.Nx))
        ehd_save(self.handle, f, g)
        return f, g


# ------------------------------------------------------------------ batches
def ehd_batch_create(max_runs, hbm_budget, max_nx, max_ny, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ehd_batch_create(int(max_runs), int(hbm_budget), int(max_nx), int(max_ny), stream,
                                  ctypes.byref(h)))
    return h.value


def ehd_batch_admits(b, Nx, Ny, storage) -> int:
    """Status of the admission query: 0 (EHD_OK), -6 (EHD_EBUSY) or -1
    (EHD_EINVAL, never admissible); raises on other failures."""
    st = int(lib().ehd_batch_admits(b, int(Nx), int(Ny), int(storage)))
    if st not in (0, -1, -6):
        _check(st)
    return st


def ehd_batch_memory(b):
    used, budget = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().ehd_batch_memory(b, ctypes.byref(used), ctypes.byref(budget)))
    return used.value, budget.value


def ehd_batch_add(b, run_handle, steps):
    _check(lib().ehd_batch_add(b, run_handle, int(steps)))


def ehd_batch_remove(b, run_handle):
    _check(lib().ehd_batch_remove(b, run_handle))


def ehd_batch_tick(b, steps):
    _check(lib().ehd_batch_tick(b, int(steps)))


def ehd_batch_remaining(b, run_handle) -> int:
    return int(lib().ehd_batch_remaining(b, run_handle))


def ehd_batch_size(b) -> int:
    return int(lib().ehd_batch_size(b))


def ehd_batch_sync(b):
    _check(lib().ehd_batch_sync(b))


def ehd_batch_stream(b) -> int:
    return lib().ehd_batch_stream(b) or 0


BATCH_TUNE = {"slab_rows": 1, "march_ctas": 2, "row_ctas": 3, "tile_ctas": 4, "pdl": 5}


def ehd_batch_tune(b, param, value):
    _check(lib().ehd_batch_tune(b, BATCH_TUNE[param] if isinstance(param, str) else int(param), int(value)))


def ehd_batch_tune_get(b, param) -> int:
    return int(lib().ehd_batch_tune_get(b, BATCH_TUNE[param] if isinstance(param, str) else int(param)))


def ehd_batch_destroy(b):
    lib().ehd_batch_destroy(b)


class Batch:
    """Runs of uneven sizes advanced together (FP32 storage and compute)."""

    def __init__(self, max_runs, max_nx=2048, max_ny=1680, stream=None, torch_stream=True, hbm_budget=0):
        self._stream_obj = None
        if stream is None and torch_stream:
            import torch
            self._stream_obj = torch.cuda.Stream()
            stream = self._stream_obj.cuda_stream
        self.handle = ehd_batch_create(max_runs, hbm_budget, max_nx, max_ny, stream)
        self.members = {}

    def admits(self, Nx, Ny, storage="f32") -> int:
        """0: admitted now; -6 (EHD_EBUSY): wait for a slot or memory;
        -1 (EHD_EINVAL): never."""
        return ehd_batch_admits(self.handle, Nx, Ny, STORAGE[storage])

    def memory(self):
        """(bytes the members hold, HBM budget)."""
        return ehd_batch_memory(self.handle)

    def add(self, run: "Run", steps: int):
        ehd_batch_add(self.handle, run.handle, steps)
        self.members[run.handle] = run

    def remove(self, run: "Run"):
        ehd_batch_remove(self.handle, run.handle)
        self.members.pop(run.handle, None)

    def tick(self, steps: int):
        ehd_batch_tick(self.handle, steps)

    def remaining(self, run: "Run") -> int:
        return ehd_batch_remaining(self.handle, run.handle)

    def __len__(self):
        return ehd_batch_size(self.handle)

    def sync(self):
        ehd_batch_sync(self.handle)

    def tune(self, **params):
        for k, v in params.items():
            ehd_batch_tune(self.handle, k, v)

    def tuning(self) -> dict:
        return {k: ehd_batch_tune_get(self.handle, k) for k in BATCH_TUNE}

    def close(self):
        if getattr(self, "handle", None):
            ehd_batch_destroy(self.handle)
            self.handle = None
            self.members = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
