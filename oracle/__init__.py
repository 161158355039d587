"""Plain FP64 CPU oracle of the ring-polymer PIMD step (fix pimd/langevin,
arXiv 2602.13553).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or runs it.

The arithmetic lives in ``pimd_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only builds it with gcc and marshals numpy
arrays through ctypes.  Array layout is ``[P][N][3]`` (bead or mode, atom,
component); velocities are normal-mode velocities at integer time.

Parity status: every function here is pinned by a CPU test against something
other than itself (closed forms, numpy/scipy library routines, invariants,
brute force); see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pimd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

POT_HARMONIC = 0
POT_WATERLIKE = 1
BAOAB = 0
OBABO = 1
NMPIMD = 0
PIMD = 1          # Cartesian method
FM_PHYSICAL = 0
FM_NORMAL = 1
BARO_NONE = 0
BARO_BZP = 1      # isotropic BZP barostat (App. E)
BARO_BZP_ANISO = 2  # one BZP barostat per axis in baro_axes (bits x = 1, y = 2, z = 4)


def build(force: bool = False) -> str:
    """Compile pimd_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Sim(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("P", ctypes.c_int32),
        ("potential", ctypes.c_int32), ("thermostat", ctypes.c_int32),
        ("integrator", ctypes.c_int32), ("method", ctypes.c_int32),
        ("T", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("scale", ctypes.c_double), ("sp", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("box", ctypes.c_double * 3),
        ("ff", ctypes.c_double * 8),
        ("mass", ctypes.POINTER(ctypes.c_double)),
        ("x", ctypes.POINTER(ctypes.c_double)),
        ("v", ctypes.POINTER(ctypes.c_double)),
        ("F", ctypes.POINTER(ctypes.c_double)),
        ("U", ctypes.POINTER(ctypes.c_double)),
        ("vir", ctypes.POINTER(ctypes.c_double)),
        ("step", ctypes.c_int64),
        ("fmmode", ctypes.c_int32), ("fixcom", ctypes.c_int32),
        ("fmass", ctypes.c_double),
        ("barostat", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("pext", ctypes.c_double), ("taup", ctypes.c_double), ("vW", ctypes.c_double),
        ("baro_axes", ctypes.c_int32), ("pad2", ctypes.c_int32),
        ("vWa", ctypes.c_double * 3), ("vir3", ctypes.c_double * 384),
    ]


class _Est(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("P", ctypes.c_int32), ("N", ctypes.c_int32),
        ("K_mode", ctypes.c_double * 128), ("S_mode", ctypes.c_double * 128),
        ("U_bead", ctypes.c_double * 128),
        ("H", ctypes.c_double), ("K_PR", ctypes.c_double), ("K_VR", ctypes.c_double),
        ("K_CV", ctypes.c_double), ("P_PR", ctypes.c_double), ("P_MD", ctypes.c_double),
        ("P_CV", ctypes.c_double), ("T_ring", ctypes.c_double),
        ("volume", ctypes.c_double), ("vir_sum", ctypes.c_double),
        ("vW", ctypes.c_double), ("K_W", ctypes.c_double), ("U_W", ctypes.c_double),
        ("J_W", ctypes.c_double), ("enthalpy", ctypes.c_double),
        ("vWa", ctypes.c_double * 3),
    ]


def lib():
    """Load (building on first use) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_constants.argtypes = [dp]
            L.or_de_boer.argtypes = [ctypes.c_double] * 3
            L.or_de_boer.restype = ctypes.c_double
            L.or_nm_matrix.argtypes = [ctypes.c_int, dp]
            L.or_mode_lambda.argtypes = [ctypes.c_int, dp]
            L.or_omega_n.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.or_omega_n.restype = ctypes.c_double
            L.or_mode_omega.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.or_philox4.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p, u64p]
            L.or_gauss3.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint64, dp]
            L.or_force_harmonic.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, dp, dp]
            L.or_force_water.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp, dp]
            L.or_to_nm.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.or_from_nm.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            sp = ctypes.POINTER(_Sim)
            L.or_compute_forces.argtypes = [sp]
            L.or_thermal_velocities.argtypes = [sp]
            L.or_run.argtypes = [sp, ctypes.c_int64]
            L.or_estimators.argtypes = [sp, ctypes.POINTER(_Est)]
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def constants() -> dict:
    out = np.zeros(4)
    lib().or_constants(_dp(out))
    return {"kB": out[0], "h": out[1], "hbar": out[2], "mvv2e": out[3]}


def de_boer(m_amu: float, eps_ev: float, sigma_a: float) -> float:
    return lib().or_de_boer(m_amu, eps_ev, sigma_a)


def nm_matrix(P: int) -> np.ndarray:
    M = np.zeros((P, P))
    lib().or_nm_matrix(P, _dp(M))
    return M


def mode_lambda(P: int) -> np.ndarray:
    lam = np.zeros(P)
    lib().or_mode_lambda(P, _dp(lam))
    return lam


def omega_n(P: int, T: float, sp: float = 1.0) -> float:
    return lib().or_omega_n(P, T, sp)


def mode_omega(P: int, T: float, sp: float = 1.0) -> np.ndarray:
    w = np.zeros(P)
    lib().or_mode_omega(P, T, sp, _dp(w))
    return w


def philox4(wbits: int, rounds: int, ctr, key) -> np.ndarray:
    c = (ctypes.c_uint64 * 4)(*[int(v) for v in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(v) for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().or_philox4(wbits, rounds, c, k, o)
    return np.array(list(o), dtype=np.uint64)


def gauss3(seed: int, atom: int, mode: int, stream: int, step: int) -> np.ndarray:
    out = np.zeros(3)
    lib().or_gauss3(seed, atom, mode, stream, step, _dp(out))
    return out


def to_nm(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    P, N, _ = x.shape
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.zeros_like(x)
    lib().or_to_nm(P, N, _dp(np.ascontiguousarray(M)), _dp(x), _dp(q))
    return q


def from_nm(M: np.ndarray, q: np.ndarray) -> np.ndarray:
    P, N, _ = q.shape
    q = np.ascontiguousarray(q, dtype=np.float64)
    x = np.zeros_like(q)
    lib().or_from_nm(P, N, _dp(np.ascontiguousarray(M)), _dp(q), _dp(x))
    return x


def force_harmonic(mass: np.ndarray, omega: float, x: np.ndarray):
    """x: [N][3] -> (F [N][3], U, Tr Xi)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    F = np.zeros_like(x)
    U = np.zeros(1)
    W = np.zeros(1)
    lib().or_force_harmonic(x.shape[0], _dp(mass), omega, _dp(x), _dp(F), _dp(U), _dp(W))
    return F, U[0], W[0]


def force_water(box, ff, x: np.ndarray):
    """x: [3*nmol][3] -> (F, U, Tr Xi); ff = (kb, r0, kth, th0, eps, sig, rc)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float64))
    f = np.ascontiguousarray(np.asarray(ff, dtype=np.float64)[:7])
    F = np.zeros_like(x)
    U = np.zeros(1)
    W = np.zeros(1)
    lib().or_force_water(x.shape[0] // 3, _dp(b), _dp(f), _dp(x), _dp(F), _dp(U), _dp(W))
    return F, U[0], W[0]


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return lib().or_max_threads()


class Sim:
    """One ring-polymer system advanced by the oracle.

    x0: [P][N][3] bead positions (A, unwrapped); v0: [P][N][3] velocities
    (A/ps) at integer time -- normal-mode velocities (method NMPIMD) or bead
    velocities (method PIMD, Cartesian) -- or None to draw them thermally
    (noise stream 2).  potential 0 = harmonic (ff[0] = omega in 1/ps), 1 =
    water-like (ff = kb, r0, kth, th0, eps, sig, rc).  thermostat 0 = NVE,
    1 = PILE_L.  fmmode 0 = physical, 1 = normal; fmass scales the fictitious
    masses; fixcom removes the centre-of-mass velocity every step.  barostat 1
    = isotropic BZP (App. E, normal modes) at pext (eV/A^3) with
    barostat time taup (ps); NpH without a thermostat, NpT with PILE_L;
    BAOAB or OBABO.
    barostat 2 = anisotropic BZP: one barostat per box edge in the bit mask
    baro_axes (x = 1, y = 2, z = 4), the other edges fixed.
    """

    def __init__(self, x0, mass, *, T, dt, potential=POT_HARMONIC, ff=(0.0,), box=(0.0, 0.0, 0.0),
                 v0=None, thermostat=1, integrator=BAOAB, seed=1, tau=1.0, scale=1.0, sp=1.0,
                 method=NMPIMD, fmmode=FM_PHYSICAL, fmass=1.0, fixcom=0, barostat=BARO_NONE,
                 pext=0.0, taup=1.0, vW=0.0, baro_axes=7):
        assert barostat == BARO_NONE or (method == NMPIMD and potential == POT_WATERLIKE)
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        P, N, three = x0.shape
        assert three == 3 and 1 <= P <= 128
        self.P, self.N = P, N
        self.mass = np.ascontiguousarray(mass, dtype=np.float64).copy()
        assert self.mass.shape == (N,)
        self.x = x0.copy()
        self.v = np.zeros_like(self.x) if v0 is None else np.ascontiguousarray(v0, dtype=np.float64).copy()
        self.F = np.zeros_like(self.x)
        self.U = np.zeros(P)
        self.vir = np.zeros(P)
        s = _Sim()
        s.N, s.P = N, P
        s.potential, s.thermostat, s.integrator = potential, thermostat, integrator
        s.method, s.fmmode, s.fixcom, s.fmass = method, fmmode, int(fixcom), float(fmass)
        s.barostat, s.pext, s.taup, s.vW = int(barostat), float(pext), float(taup), float(vW)
        s.baro_axes = int(baro_axes)
        s.T, s.dt, s.tau, s.scale, s.sp = T, dt, tau, scale, sp
        s.seed = seed
        for a in range(3):
            s.box[a] = float(box[a])
        ffl = list(ff) + [0.0] * (8 - len(ff))
        for a in range(8):
            s.ff[a] = float(ffl[a])
        s.mass, s.x, s.v, s.F = _dp(self.mass), _dp(self.x), _dp(self.v), _dp(self.F)
        s.U, s.vir = _dp(self.U), _dp(self.vir)
        s.step = 0
        self._s = s
        if v0 is None:
            lib().or_thermal_velocities(ctypes.byref(s))
        lib().or_compute_forces(ctypes.byref(s))

    @property
    def step(self) -> int:
        return int(self._s.step)

    @property
    def box(self) -> np.ndarray:
        return np.array(list(self._s.box))

    @property
    def vW(self) -> float:
        return float(self._s.vW)

    @property
    def vWa(self) -> np.ndarray:
        return np.array(list(self._s.vWa))

    def run(self, nsteps: int) -> None:
        lib().or_run(ctypes.byref(self._s), int(nsteps))

    def compute_forces(self) -> None:
        lib().or_compute_forces(ctypes.byref(self._s))

    def estimators(self) -> dict:
        e = _Est()
        lib().or_estimators(ctypes.byref(self._s), ctypes.byref(e))
        P = self.P
        out = {k: getattr(e, k) for k in ("H", "K_PR", "K_VR", "K_CV", "P_PR", "P_MD", "P_CV",
                                          "T_ring", "volume", "vir_sum", "vW", "K_W", "U_W", "J_W",
                                          "enthalpy")}
        out["step"] = int(e.step)
        out["vWa"] = np.array(list(e.vWa))
        out["K_mode"] = np.array(e.K_mode[:P])
        out["S_mode"] = np.array(e.S_mode[:P])
        out["U_bead"] = np.array(e.U_bead[:P])
        return out
