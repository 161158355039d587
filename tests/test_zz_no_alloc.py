"""GPU test of pimd_estimators_noalloc, the estimator entry point that
allocates nothing (for callers that own all device memory themselves).

It is called through the C ABI on state held in caller-owned device buffers
and must agree with pimd_estimators of a handle holding the same state,
within the FP64 bars of the parity tests, on consecutive calls that reuse the
library's static scratch array.  This file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import coord_err, pimd, scalar_err  # noqa: F401

pytestmark = pytest.mark.gpu

MVV2E = 1.0364269e-4
OMEGA_HO = 0.1 / (4.135667403e-3 / (2 * math.pi))


def _noalloc(pimd, x, v, F, mass, U_bead, vir, T, volume, P, N):
    import torch
    L = pimd.lib()
    f = L.pimd_estimators_noalloc
    dp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  dp, dp, dp, dp, dp, ctypes.c_double, dp, ctypes.POINTER(pimd.Estimates)]
    f.restype = ctypes.c_int
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    tx, tv, tF, tm, tU = dev(x), dev(v), dev(F), dev(mass), dev(U_bead)
    stream = torch.cuda.current_stream().cuda_stream
    e = pimd.Estimates()
    st = f(N, P, T, 1.0, volume, tx.data_ptr(), tv.data_ptr(), tF.data_ptr(), tm.data_ptr(),
           tU.data_ptr(), vir, stream, ctypes.byref(e))
    assert st == 0, L.pimd_last_error()
    return e.as_dict()


def _same(a, b, tol):
    for k in ("H", "K_PR", "K_VR", "K_CV", "T_ring"):
        assert scalar_err(a[k], b[k]) < tol, (k, a[k], b[k])
    for k in ("K_mode", "S_mode", "U_bead"):
        assert coord_err(a[k], b[k]) < tol, k
    for k in ("P_PR", "P_MD", "P_CV"):
        if math.isnan(b[k]):
            assert math.isnan(a[k])
        else:
            scale = abs(b["vir_sum"]) / (3 * b["volume"]) + abs(b[k])
            assert abs(a[k] - b[k]) < tol * scale, k


def _harmonic_case(pimd, P, N, seed, steps):
    x0, mass = inputs.harmonic(N, P, seed=seed, std=0.1)
    s = pimd.Simulation(x0, mass, T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), seed=seed)
    s.step(steps)
    x, v, _ = s.get_state()
    ref = s.estimators()
    F = -(mass * MVV2E * OMEGA_HO ** 2)[None, :, None] * x
    out = _noalloc(pimd, x, v, F, mass, ref["U_bead"], ref["vir_sum"], 300.0, 0.0, P, N)
    s.close()
    return out, ref


def test_noalloc_matches_handle_estimators(pimd, orc):
    # call 1: harmonic oscillators, 300 atoms x 8 beads
    out, ref = _harmonic_case(pimd, 8, 300, 3, 40)
    _same(out, ref, 1e-10)
    # call 2: a water-like box with a volume (pressures), different N and P;
    # the forces of the state come from the oracle's force field
    L = 12.42
    x0, mass = inputs.water_box(64, L, 16, 5, jitter=0.02)
    s = pimd.Simulation(x0, mass, T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF,
                        box=(L, L, L), seed=5)
    s.step(30)
    x, v, _ = s.get_state()
    ref = s.estimators()
    F = np.stack([orc.force_water((L, L, L), inputs.WATER_FF, x[k])[0] for k in range(16)])
    out = _noalloc(pimd, x, v, F, mass, ref["U_bead"], ref["vir_sum"], 300.0, L ** 3, 16, 192)
    s.close()
    _same(out, ref, 1e-8)
    # call 3: back to a harmonic system with more atoms than one pass of
    # blocks covers (the static grid walks several tiles per block)
    out, ref = _harmonic_case(pimd, 128, 2000, 4, 10)
    _same(out, ref, 1e-10)


def test_noalloc_rejects_sizes_beyond_limits(pimd):
    L = pimd.lib()
    f = L.pimd_estimators_noalloc
    dp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  dp, dp, dp, dp, dp, ctypes.c_double, dp, ctypes.POINTER(pimd.Estimates)]
    f.restype = ctypes.c_int
    e = pimd.Estimates()
    fake = ctypes.c_void_p(16)   # never dereferenced: the size checks come first
    assert f(10, 129, 300.0, 1.0, 0.0, fake, fake, fake, fake, fake, 0.0, None, ctypes.byref(e)) == 1
    assert b"P = 129" in L.pimd_last_error()
    assert f(2**28, 64, 300.0, 1.0, 0.0, fake, fake, fake, fake, fake, 0.0, None, ctypes.byref(e)) == 1
    assert f(0, 8, 300.0, 1.0, 0.0, fake, fake, fake, fake, fake, 0.0, None, ctypes.byref(e)) == 1
