"""GPU tests of pimd_estimators_noalloc, the estimator entry point that
allocates nothing.  It serves callers that cannot let a library allocate
device memory: an application that reserves one fixed device pool at start-up
and owns every byte of it, or a stepping loop in which a cudaMalloc would
synchronise the device and stall its other streams.

The entry point is called through the C ABI on state held in caller-owned
device buffers.  Each test calls it at least twice in a row, so the library's
static scratch array is reused with the previous call's contents still in it.
The results must agree with pimd_estimators of a handle that holds the same
state, and with the oracle's estimators of that state, within the FP64 bars
of the parity tests.  The remaining checks:
- method pimd, fmmode normal, fmass and sp are covered;
- the fields the call cannot know come back zero;
- neither the library's allocator hook nor the device's free memory moves
  across calls.
This file is collected last on purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import coord_err, pimd, scalar_err  # noqa: F401

pytestmark = pytest.mark.gpu

MVV2E = 1.0364269e-4
OMEGA_HO = 0.1 / (4.135667403e-3 / (2 * math.pi))
TAIL = ("vW", "K_W", "U_W", "J_W", "enthalpy")


def _fn(pimd):
    L = pimd.lib()
    f = L.pimd_estimators_noalloc
    dp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp, dp,
                  ctypes.c_double, ctypes.POINTER(pimd.Params), dp, ctypes.POINTER(pimd.Estimates)]
    f.restype = ctypes.c_int
    return L, f


class _DeviceState:
    """The caller's own device buffers (allocated here, before any call)."""

    def __init__(self, x, v, F, mass, U_bead):
        import torch
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        self.t = [dev(x), dev(v), dev(F), dev(mass), dev(U_bead)]
        self.P, self.N = x.shape[0], x.shape[1]

    def ptrs(self):
        return [a.data_ptr() for a in self.t]


def _call(pimd, state, vir, T, volume, params=None):
    import torch
    L, f = _fn(pimd)
    e = pimd.Estimates()
    for k in TAIL:            # a caller's struct that holds garbage
        setattr(e, k, 123.0)
    for d in range(3):
        e.box[d] = 7.0
        e.vWa[d] = 7.0
    prm = None if params is None else ctypes.byref(pimd.default_params(**params))
    stream = torch.cuda.current_stream().cuda_stream
    st = f(state.N, state.P, T, volume, *state.ptrs(), vir, prm, stream, ctypes.byref(e))
    assert st == 0, L.pimd_last_error()
    out = e.as_dict()
    for k in TAIL:
        assert out[k] == 0.0, k
    assert list(e.box) == [0.0] * 3 and list(e.vWa) == [0.0] * 3
    return out


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


def _harmonic(pimd, orc, P, N, seed, steps, **params):
    """A stepped handle's state; the oracle's estimators of the same state."""
    x0, mass = inputs.harmonic(N, P, seed=seed, std=0.1)
    kw = dict(T=300.0, dt=2.5e-4, potential=0, ff=(OMEGA_HO,), seed=seed)
    s = pimd.Simulation(x0, mass, **kw, **params)
    s.step(steps)
    x, v, _ = s.get_state()
    ref = s.estimators()
    s.close()
    c = orc.Sim(x, mass, v0=v, **kw, **params)     # forces, U and Tr Xi of this state
    return _DeviceState(x, v, c.F, mass, c.U), mass, ref, c.estimators(), float(np.sum(c.vir))


def test_noalloc_matches_handle_and_oracle(pimd, orc):
    # call 1: harmonic oscillators, 300 atoms x 8 beads, default keywords
    st, _, ref, want, vir = _harmonic(pimd, orc, 8, 300, 3, 40)
    out = _call(pimd, st, vir, 300.0, 0.0)
    _same(out, ref, 1e-10)
    _same(out, want, 1e-10)
    # call 2: a water-like box with a volume (pressures), different N and P
    L = 12.42
    x0, mass = inputs.water_box(64, L, 16, 5, jitter=0.02)
    kw = dict(T=300.0, dt=5e-4, potential=1, ff=inputs.WATER_FF, box=(L, L, L), seed=5)
    s = pimd.Simulation(x0, mass, **kw)
    s.step(30)
    x, v, _ = s.get_state()
    ref = s.estimators()
    s.close()
    c = orc.Sim(x, mass, v0=v, **kw)
    out = _call(pimd, _DeviceState(x, v, c.F, mass, c.U), float(np.sum(c.vir)), 300.0, L ** 3)
    _same(out, ref, 1e-8)
    _same(out, c.estimators(), 1e-10)
    # call 3: more atoms than one pass of blocks covers (the static grid walks
    # several tiles per block), P = 128
    st, _, ref, want, vir = _harmonic(pimd, orc, 128, 2000, 4, 10)
    out = _call(pimd, st, vir, 300.0, 0.0)
    _same(out, ref, 1e-10)
    _same(out, want, 1e-10)


@pytest.mark.parametrize("params", [
    dict(fmmode=1, fmass=2.5),                 # fictitious masses lambda_k fmass m
    dict(fmass=0.6, sp=0.8),                   # scaled masses and hbar
    dict(method=1, fmass=1.7),                 # Cartesian beads: bead forms of outputs 1, 2 and P_CV
])
def test_noalloc_method_keywords(pimd, orc, params):
    st, _, ref, want, vir = _harmonic(pimd, orc, 16, 96, 6, 25, **params)
    for _ in range(2):
        out = _call(pimd, st, vir, 300.0, 0.0, params)
        _same(out, ref, 1e-10)
        _same(out, want, 1e-10)


def test_noalloc_allocates_nothing(pimd, orc):
    """Across calls that follow the first (which looks up the scratch address
    and may load the library's device code), the allocator hook is never
    entered and the device's free memory does not move."""
    import torch
    st, _, _, want, vir = _harmonic(pimd, orc, 32, 500, 8, 5)
    _call(pimd, st, vir, 300.0, 0.0)               # set-up call
    torch.cuda.synchronize()
    calls = [0]

    def _alloc(nbytes, stream, ctx):
        calls[0] += 1
        return None

    def _free(ptr, stream, ctx):
        calls[0] += 1

    hooks = (pimd.ALLOC_FN(_alloc), pimd.FREE_FN(_free))
    restore_torch = pimd._torch_alloc_refs is not None
    pimd.lib().pimd_set_allocator(hooks[0], hooks[1], None)
    try:
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            out = _call(pimd, st, vir, 300.0, 0.0)
            _same(out, want, 1e-10)
        free1, _ = torch.cuda.mem_get_info()
    finally:
        pimd.reset_allocator()
        if restore_torch:
            pimd.use_torch_allocator()
    assert calls[0] == 0
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_limits(pimd):
    L, f = _fn(pimd)
    e = pimd.Estimates()
    fake = ctypes.c_void_p(16)   # never dereferenced: the size checks come first
    args = [fake] * 5
    assert f(10, 129, 300.0, 0.0, *args, 0.0, None, None, ctypes.byref(e)) == 1
    assert b"P = 129" in L.pimd_last_error()
    assert f(2**28, 64, 300.0, 0.0, *args, 0.0, None, None, ctypes.byref(e)) == 1
    assert f(0, 8, 300.0, 0.0, *args, 0.0, None, None, ctypes.byref(e)) == 1
    bad = pimd.default_params(method=1, fmmode=1)
    assert f(10, 8, 300.0, 0.0, *args, 0.0, ctypes.byref(bad), None, ctypes.byref(e)) == 1
