"""ctypes binding of libpimd (include/pimd.h): argument marshalling only.

Every step of the PIMD path runs in the library's CUDA kernels.  If the
library has not been built, or cannot be loaded, the calls raise: there is no
CPU fallback.  PyTorch, when present, only provides device memory (through
the library's allocator hook, see ``use_torch_allocator``) and CUDA streams.
"""
from __future__ import annotations

import collections.abc
import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpimd.so")

POT_HARMONIC = 0
POT_WATERLIKE = 1
THERMO_NONE = 0
THERMO_PILE_L = 1
BAOAB = 0
OBABO = 1
METHOD_NMPIMD = 0
METHOD_PIMD = 1
FMMODE_PHYSICAL = 0
FMMODE_NORMAL = 1
BARO_NONE = 0
BARO_BZP_ISO = 1
BARO_BZP_ANISO = 2
AXIS_X, AXIS_Y, AXIS_Z = 1, 2, 4
PREC_FP64 = 0
PREC_SPLIT = 1
MAX_BEADS = 128

STATUS = {0: "PIMD_OK", 1: "PIMD_EINVAL", 2: "PIMD_ENOMEM", 3: "PIMD_ECUDA", 4: "PIMD_ENONFINITE",
          5: "PIMD_ETIMEOUT", 6: "PIMD_EPENDING", 7: "PIMD_ENOTFOUND", 8: "PIMD_EBUDGET",
          9: "PIMD_EOVERFLOW"}


class PimdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status


class System(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("potential", ctypes.c_int32),
        ("mass", ctypes.POINTER(ctypes.c_double)),
        ("pos", ctypes.POINTER(ctypes.c_double)),
        ("vel", ctypes.POINTER(ctypes.c_double)),
        ("box", ctypes.c_double * 3),
        ("ff", ctypes.c_double * 8),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("thermostat", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("method", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("tau", ctypes.c_double), ("scale", ctypes.c_double), ("sp", ctypes.c_double),
        ("fixcom", ctypes.c_int32), ("fmmode", ctypes.c_int32),
        ("fmass", ctypes.c_double),
        ("barostat", ctypes.c_int32), ("baro_axes", ctypes.c_int32),
        ("pext", ctypes.c_double), ("taup", ctypes.c_double),
    ]


class Estimates(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("P", ctypes.c_int32), ("N", ctypes.c_int32),
        ("K_mode", ctypes.c_double * MAX_BEADS), ("S_mode", ctypes.c_double * MAX_BEADS),
        ("U_bead", ctypes.c_double * MAX_BEADS),
        ("H", ctypes.c_double), ("K_PR", ctypes.c_double), ("K_VR", ctypes.c_double),
        ("K_CV", ctypes.c_double), ("P_PR", ctypes.c_double), ("P_MD", ctypes.c_double),
        ("P_CV", ctypes.c_double), ("T_ring", ctypes.c_double),
        ("volume", ctypes.c_double), ("vir_sum", ctypes.c_double),
        ("vW", ctypes.c_double), ("K_W", ctypes.c_double), ("U_W", ctypes.c_double),
        ("J_W", ctypes.c_double), ("enthalpy", ctypes.c_double),
        ("box", ctypes.c_double * 3),
        ("vWa", ctypes.c_double * 3),
    ]

    def as_dict(self) -> dict:
        P = self.P
        out = {k: getattr(self, k) for k in ("H", "K_PR", "K_VR", "K_CV", "P_PR", "P_MD", "P_CV",
                                             "T_ring", "volume", "vir_sum", "vW", "K_W", "U_W",
                                             "J_W", "enthalpy")}
        out["box"] = np.array(list(self.box))
        out["vWa"] = np.array(list(self.vWa))
        out["step"] = int(self.step)
        out["K_mode"] = np.array(self.K_mode[:P])
        out["S_mode"] = np.array(self.S_mode[:P])
        out["U_bead"] = np.array(self.U_bead[:P])
        return out


class _EstimatesMap(collections.abc.Mapping):
    """Read-only mapping slot -> estimator dict over one pimd_estimates array;
    a slot's dict is built when it is first read (a batch holds hundreds of
    replicas; building every dict costs milliseconds of host time)."""

    def __init__(self, arr, slots):
        self._arr = arr
        self._slots = list(slots)
        self._live = set(self._slots)
        self._cache = {}

    def __getitem__(self, slot):
        if slot not in self._live:
            raise KeyError(slot)
        if slot not in self._cache:
            self._cache[slot] = self._arr[slot].as_dict()
        return self._cache[slot]

    def __iter__(self):
        return iter(self._slots)

    def __len__(self):
        return len(self._slots)


# every symbol include/pimd.h declares (checked by the CPU tests)
EXPORTS = ("pimd_set_allocator", "pimd_params_default", "pimd_status_string", "pimd_last_error",
           "pimd_create", "pimd_step", "pimd_sync", "pimd_estimators", "pimd_get_state",
           "pimd_set_state", "pimd_get_barostat", "pimd_set_barostat", "pimd_destroy",
           "pimd_set_kernel_timing", "pimd_kernel_times",
           "pimd_kernel_launches", "pimd_noise_sample", "pimd_fp64_fma_rate", "pimd_estimators_noalloc",
           "pimd_batch_replica_bytes", "pimd_batch_create", "pimd_batch_add", "pimd_batch_remove",
           "pimd_batch_run", "pimd_batch_sync", "pimd_batch_status", "pimd_batch_estimators",
           "pimd_batch_get_state", "pimd_batch_autotune", "pimd_batch_kernel_launches",
           "pimd_batch_time_kernels", "pimd_batch_set_transforms",
           "pimd_batch_destroy", "pimd_server_create", "pimd_batch_submit", "pimd_batch_poll",
           "pimd_batch_cancel", "pimd_server_job_times", "pimd_server_stats_get", "pimd_server_keep_state",
           "pimd_server_get_state", "pimd_server_destroy")
KINDS = ("step", "force", "nbr", "close", "est", "other")

_lock = threading.Lock()
_lib = None
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def lib():
    """Load libpimd.so (raises if it is missing: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpimd.so is not built (%s); run paper_2602_13553_gb300.build.build()"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.pimd_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
        L.pimd_set_allocator.restype = None
        L.pimd_params_default.argtypes = [ctypes.POINTER(Params)]
        L.pimd_params_default.restype = None
        L.pimd_status_string.argtypes = [ctypes.c_int]
        L.pimd_status_string.restype = ctypes.c_char_p
        L.pimd_last_error.argtypes = []
        L.pimd_last_error.restype = ctypes.c_char_p
        L.pimd_create.argtypes = [ctypes.POINTER(System), ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.POINTER(Params), vp,
                                  ctypes.POINTER(vp)]
        L.pimd_step.argtypes = [vp, ctypes.c_int64]
        L.pimd_sync.argtypes = [vp]
        L.pimd_estimators.argtypes = [vp, ctypes.POINTER(Estimates)]
        L.pimd_get_state.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int64)]
        L.pimd_set_state.argtypes = [vp, dp, dp, ctypes.c_int64]
        L.pimd_get_barostat.argtypes = [vp, dp, dp]
        L.pimd_set_barostat.argtypes = [vp, dp, dp]
        L.pimd_destroy.argtypes = [vp]
        L.pimd_destroy.restype = None
        L.pimd_set_kernel_timing.argtypes = [vp, ctypes.c_int]
        L.pimd_set_kernel_timing.restype = ctypes.c_int
        L.pimd_kernel_times.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64)]
        L.pimd_kernel_times.restype = ctypes.c_int
        L.pimd_kernel_launches.argtypes = [vp]
        L.pimd_kernel_launches.restype = ctypes.c_int64
        L.pimd_noise_sample.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32), dp]
        L.pimd_noise_sample.restype = ctypes.c_int
        L.pimd_fp64_fma_rate.argtypes = [ctypes.c_int32, dp]
        L.pimd_fp64_fma_rate.restype = ctypes.c_int
        for f in ("pimd_create", "pimd_step", "pimd_sync", "pimd_estimators", "pimd_get_state",
                  "pimd_set_state", "pimd_get_barostat", "pimd_set_barostat"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
        return L


def check(status: int) -> None:
    if status != 0:
        msg = lib().pimd_last_error().decode(errors="replace")
        raise PimdError(status, msg)


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fp64_fma_rate(iters: int = 20000) -> float:
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    out = ctypes.c_double()
    check(lib().pimd_fp64_fma_rate(int(iters), ctypes.byref(out)))
    return out.value


def noise_sample(seed: int, stream: int, step: int, n_atoms: int, n_modes: int):
    """Philox words [n_modes][n_atoms][4] (uint32) and FP64 deviates
    [n_modes][n_atoms][3] of one (seed, stream, step), from the device."""
    words = np.zeros((n_modes, n_atoms, 4), dtype=np.uint32)
    eta = np.zeros((n_modes, n_atoms, 3))
    check(lib().pimd_noise_sample(seed, stream, step, n_atoms, n_modes,
                                  words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _dp(eta)))
    return words, eta


def default_params(**kw) -> Params:
    p = Params()
    lib().pimd_params_default(ctypes.byref(p))
    names = {f[0] for f in Params._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown pimd_params field {k!r}")
        setattr(p, k, v)
    return p


_torch_alloc_refs = None


def use_torch_allocator() -> None:
    """Route libpimd's device allocations through PyTorch's caching allocator."""
    global _torch_alloc_refs
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or None))
        except Exception:  # reported to the library as NULL -> PIMD_ENOMEM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _torch_alloc_refs = (a, f)
    lib().pimd_set_allocator(a, f, None)


def reset_allocator() -> None:
    global _torch_alloc_refs
    lib().pimd_set_allocator(ALLOC_FN(), FREE_FN(), None)
    _torch_alloc_refs = None


class Simulation:
    """One ring-polymer system on the GPU (a pimd_handle).

    x0: [P][N][3] positions (A); v0: [P][N][3] velocities -- normal-mode
    (method nmpimd) or bead (method pimd) -- or None (thermal draw).  Keyword
    arguments map onto pimd_params fields (thermostat, integrator, method,
    precision, seed, tau, scale, sp, fixcom, fmmode, fmass, barostat, baro_axes,
    pext, taup); an unknown name raises TypeError.
    """

    def __init__(self, x0, mass, *, T, dt, potential=POT_HARMONIC, ff=(0.0,), box=(0.0, 0.0, 0.0),
                 v0=None, gamma0=0.0, stream=None, **params):
        self.x0 = np.ascontiguousarray(x0, dtype=np.float64)
        P, N, three = self.x0.shape
        assert three == 3
        self.P, self.N = P, N
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
        s = System()
        s.n_atoms = N
        s.potential = potential
        s.mass = _dp(self.mass)
        s.pos = _dp(self.x0)
        s.vel = _dp(self.v0)
        for a in range(3):
            s.box[a] = float(box[a])
        ffl = list(ff) + [0.0] * (8 - len(ff))
        for a in range(8):
            s.ff[a] = float(ffl[a])
        prm = default_params(**params)
        self._aniso = prm.barostat == BARO_BZP_ANISO
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        check(lib().pimd_create(ctypes.byref(s), P, T, dt, gamma0, ctypes.byref(prm), st,
                                ctypes.byref(h)))
        self._h = h

    def step(self, n: int) -> None:
        check(lib().pimd_step(self._h, int(n)))

    def sync(self) -> None:
        check(lib().pimd_sync(self._h))

    def estimators(self) -> dict:
        e = Estimates()
        check(lib().pimd_estimators(self._h, ctypes.byref(e)))
        return e.as_dict()

    def get_state(self, x=None, v=None):
        x = np.empty((self.P, self.N, 3)) if x is None else x
        v = np.empty((self.P, self.N, 3)) if v is None else v
        st = ctypes.c_int64()
        check(lib().pimd_get_state(self._h, _dp(x), _dp(v), ctypes.byref(st)))
        return x, v, int(st.value)

    def set_state(self, x, v, step: int) -> None:
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        check(lib().pimd_set_state(self._h, _dp(x), _dp(v), int(step)))

    def get_barostat(self):
        """(v_W in 1/ps, box edges in A) of the barostat state; v_W is a float
        (isotropic) or an array of the three edges' v_Wa (anisotropic)."""
        vw = np.zeros(3)
        box = np.zeros(3)
        check(lib().pimd_get_barostat(self._h, _dp(vw), _dp(box)))
        return (vw.copy() if self._aniso else float(vw[0])), box

    def set_barostat(self, vW, box) -> None:
        box = np.ascontiguousarray(box, dtype=np.float64)
        vw = np.zeros(3)
        vw[:] = np.asarray(vW, dtype=np.float64).reshape(-1)[:3] if self._aniso else float(vW)
        check(lib().pimd_set_barostat(self._h, _dp(vw), _dp(box)))

    def set_kernel_timing(self, enable: bool) -> None:
        check(lib().pimd_set_kernel_timing(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        ms = (ctypes.c_double * len(KINDS))()
        n = (ctypes.c_int64 * len(KINDS))()
        check(lib().pimd_kernel_times(self._h, ms, n))
        return {k: (ms[i], int(n[i])) for i, k in enumerate(KINDS)}

    def kernel_launches(self) -> int:
        return int(lib().pimd_kernel_launches(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().pimd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------
# batches and serving
# ---------------------------------------------------------------------------
class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("running", ctypes.c_int64), ("queued", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t),
                ("chunks", ctypes.c_int64), ("bead_atom_steps", ctypes.c_double),
                ("gpu_busy_s", ctypes.c_double)]


_batch_ready = False


def _batch_lib():
    global _batch_ready
    L = lib()
    if _batch_ready:
        return L
    vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    sysp, prmp = ctypes.POINTER(System), ctypes.POINTER(Params)
    sig = {
        "pimd_batch_replica_bytes": ([ctypes.c_int32, ctypes.c_int32], ctypes.c_size_t),
        "pimd_batch_create": ([ctypes.c_int32, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "pimd_batch_add": ([vp, sysp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double, prmp,
                            ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "pimd_batch_remove": ([vp, ctypes.c_int32], ctypes.c_int),
        "pimd_batch_run": ([vp, ctypes.c_int64], ctypes.c_int),
        "pimd_batch_sync": ([vp], ctypes.c_int),
        "pimd_batch_status": ([vp, i64, i64, i64], ctypes.c_int),
        "pimd_batch_estimators": ([vp, ctypes.POINTER(Estimates)], ctypes.c_int),
        "pimd_batch_get_state": ([vp, ctypes.c_int32, dp, dp, i64], ctypes.c_int),
        "pimd_batch_autotune": ([vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "pimd_batch_kernel_launches": ([vp], ctypes.c_int64),
        "pimd_batch_time_kernels": ([vp, ctypes.c_int32, dp], ctypes.c_int),
        "pimd_batch_set_transforms": ([vp, ctypes.c_int32], ctypes.c_int),
        "pimd_batch_destroy": ([vp], None),
        "pimd_server_create": ([ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64, vp, ctypes.POINTER(vp)],
                               ctypes.c_int),
        "pimd_batch_submit": ([vp, sysp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double, prmp,
                               ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "pimd_batch_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(Estimates)], ctypes.c_int),
        "pimd_batch_cancel": ([vp, ctypes.c_uint64], ctypes.c_int),
        "pimd_server_job_times": ([vp, ctypes.c_uint64, dp, dp, dp], ctypes.c_int),
        "pimd_server_stats_get": ([vp, ctypes.POINTER(ServerStats)], ctypes.c_int),
        "pimd_server_keep_state": ([vp, ctypes.c_int], ctypes.c_int),
        "pimd_server_get_state": ([vp, ctypes.c_uint64, dp, dp, i64], ctypes.c_int),
        "pimd_server_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _batch_ready = True
    return L


def make_system(x0, mass, *, potential=POT_WATERLIKE, ff=(0.0,), box=(0.0, 0.0, 0.0), v0=None):
    """A pimd_system over numpy arrays; the arrays are kept alive on the struct."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    s = System()
    s.n_atoms = x0.shape[1]
    s.potential = potential
    s.mass, s.pos, s.vel = _dp(mass), _dp(x0), _dp(v0)
    for a in range(3):
        s.box[a] = float(box[a])
    ffl = list(ff) + [0.0] * (8 - len(ff))
    for a in range(8):
        s.ff[a] = float(ffl[a])
    s._keep = (x0, mass, v0)
    return s


def replica_bytes(n_atoms: int, P: int) -> int:
    return int(_batch_lib().pimd_batch_replica_bytes(n_atoms, P))


class Batch:
    """Many independent water-like systems advanced together (pimd_batch)."""

    def __init__(self, max_replicas: int, stream=None):
        L = _batch_lib()
        h = ctypes.c_void_p()
        check(L.pimd_batch_create(max_replicas, ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self._h = h
        self.capacity = max_replicas
        self.shapes = {}

    def add(self, x0, mass, *, T, dt, nsteps, ff, box, v0=None, gamma0=0.0, **params) -> int:
        s = make_system(x0, mass, ff=ff, box=box, v0=v0)
        prm = default_params(**params)
        slot = ctypes.c_int32()
        check(_batch_lib().pimd_batch_add(self._h, ctypes.byref(s), x0.shape[0], T, dt, gamma0,
                                          ctypes.byref(prm), int(nsteps), ctypes.byref(slot)))
        self.shapes[slot.value] = (x0.shape[0], x0.shape[1])
        return slot.value

    def remove(self, slot: int) -> None:
        check(_batch_lib().pimd_batch_remove(self._h, slot))
        self.shapes.pop(slot, None)

    def run(self, nsteps: int) -> None:
        check(_batch_lib().pimd_batch_run(self._h, int(nsteps)))

    def sync(self) -> None:
        check(_batch_lib().pimd_batch_sync(self._h))

    def status(self, rebuilds: bool = False):
        st = (ctypes.c_int64 * self.capacity)()
        left = (ctypes.c_int64 * self.capacity)()
        rb = (ctypes.c_int64 * self.capacity)()
        check(_batch_lib().pimd_batch_status(self._h, st, left, rb))
        if rebuilds:
            return np.array(st[:]), np.array(left[:]), np.array(rb[:])
        return np.array(st[:]), np.array(left[:])

    def estimators(self):
        """slot -> estimator dict of every live replica (converted on first access)."""
        arr = (Estimates * self.capacity)()
        check(_batch_lib().pimd_batch_estimators(self._h, arr))
        return _EstimatesMap(arr, [s for s in range(self.capacity) if arr[s].step >= 0])

    def get_state(self, slot: int):
        P, N = self.shapes[slot]
        x = np.empty((P, N, 3))
        v = np.empty((P, N, 3))
        st = ctypes.c_int64()
        check(_batch_lib().pimd_batch_get_state(self._h, slot, _dp(x), _dp(v), ctypes.byref(st)))
        return x, v, int(st.value)

    def autotune(self, steps_per_trial: int = 2):
        tiles = (ctypes.c_int32 * (MAX_BEADS + 1))()
        check(_batch_lib().pimd_batch_autotune(self._h, steps_per_trial, tiles))
        out = {P: tiles[P] for P in range(1, MAX_BEADS + 1) if tiles[P] > 0}
        out["warp_blocks_per_sm"] = tiles[0]
        return out

    def set_transforms(self, kind: str) -> None:
        """'tensor' (warp items, 3xTF32 tensor cores) or 'ffma' (block items,
        FP32 FMA transforms)."""
        check(_batch_lib().pimd_batch_set_transforms(self._h, {"tensor": 0, "ffma": 1}[kind]))

    def kernel_launches(self) -> int:
        return int(_batch_lib().pimd_batch_kernel_launches(self._h))

    def time_kernels(self, nsteps: int) -> dict:
        ms = (ctypes.c_double * 4)()
        check(_batch_lib().pimd_batch_time_kernels(self._h, int(nsteps), ms))
        return dict(zip(("ctl", "step", "nbr", "force"), list(ms)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            _batch_lib().pimd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching PIMD job server (pimd_server)."""

    def __init__(self, hbm_budget_bytes: int, max_replicas: int = 256, chunk_steps: int = 100, stream=None,
                 keep_state: bool = False):
        L = _batch_lib()
        h = ctypes.c_void_p()
        check(L.pimd_server_create(int(hbm_budget_bytes), max_replicas, chunk_steps,
                                   ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self._h = h
        self.shapes = {}
        if keep_state:
            check(L.pimd_server_keep_state(h, 1))

    def submit(self, x0, mass, *, T, dt, nsteps, ff, box, v0=None, gamma0=0.0, **params) -> int:
        s = make_system(x0, mass, ff=ff, box=box, v0=v0)
        prm = default_params(**params)
        job = ctypes.c_uint64()
        check(_batch_lib().pimd_batch_submit(self._h, ctypes.byref(s), x0.shape[0], T, dt, gamma0,
                                             ctypes.byref(prm), int(nsteps), ctypes.byref(job)))
        self.shapes[job.value] = (x0.shape[0], x0.shape[1])
        return job.value

    def get_state(self, job: int):
        """(x, v_nm, step) of a finished job (the server must keep states)."""
        P, N = self.shapes[job]
        x = np.zeros((P, N, 3))
        v = np.zeros((P, N, 3))
        st = ctypes.c_int64()
        check(_batch_lib().pimd_server_get_state(self._h, job, _dp(x), _dp(v), ctypes.byref(st)))
        return x, v, st.value

    def poll(self, job: int):
        """None while pending; the estimator dict once done; raises on failure."""
        e = Estimates()
        st = _batch_lib().pimd_batch_poll(self._h, job, ctypes.byref(e))
        if st == 6:
            return None
        check(st)
        return e.as_dict()

    def cancel(self, job: int) -> None:
        check(_batch_lib().pimd_batch_cancel(self._h, job))

    def times(self, job: int):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(_batch_lib().pimd_server_job_times(self._h, job, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def stats(self) -> dict:
        s = ServerStats()
        check(_batch_lib().pimd_server_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            _batch_lib().pimd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
