"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/*.h declares, and rejects invalid arguments before touching the GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2602_13553_gb300 import binding as b
from paper_2602_13553_gb300 import build as bld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pimd_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    bld.build()
    return b.lib()


def test_exports_every_declared_symbol(L):
    decl = declared_functions()
    assert "pimd_create" in decl and "pimd_step" in decl
    for name in sorted(decl):
        assert hasattr(L, name), name
    assert set(b.EXPORTS) <= decl


def test_params_default(L):
    p = b.default_params()
    assert (p.thermostat, p.integrator, p.method, p.precision, p.seed) == (1, 0, 0, 0, 1)
    assert (p.tau, p.scale, p.sp, p.fixcom, p.fmmode, p.fmass) == (1.0, 1.0, 1.0, 0, 0, 1.0)
    assert (p.barostat, p.pext, p.taup, p.baro_axes) == (0, 0.0, 1.0, 7)


def test_params_reject_unknown_names(L):
    with pytest.raises(TypeError):
        b.default_params(baro_axis=3)


def test_status_strings(L):
    for s in range(10):
        assert L.pimd_status_string(s)


def _create(L, sysfix, P=4, T=300.0, dt=1e-3, gamma0=0.0, prm=None):
    h = ctypes.c_void_p()
    st = L.pimd_create(ctypes.byref(sysfix), P, T, dt, gamma0,
                       ctypes.byref(prm) if prm is not None else None, None, ctypes.byref(h))
    return st, h


@pytest.fixture()
def water_sys():
    from paper_2602_13553_gb300 import inputs
    x, m = inputs.water_box(8, 14.0, 4, 1)
    s = b.System()
    s.n_atoms = 24
    s.potential = b.POT_WATERLIKE
    keep = (np.ascontiguousarray(m), np.ascontiguousarray(x))
    s.mass = b._dp(keep[0]); s.pos = b._dp(keep[1]); s.vel = None
    for a in range(3):
        s.box[a] = 14.0
    for a, v in enumerate(inputs.WATER_FF):
        s.ff[a] = v
    s._keep = keep
    return s


@pytest.mark.parametrize("case", ["P0", "P129", "T0", "dt0", "badpot", "badthermo", "badint",
                                  "fixcom2", "badmethod", "badfmmode", "fmass0", "normal_cartesian",
                                  "split_cartesian", "split_fixcom", "split_fmass", "split_normal",
                                  "badbaro", "baro_cartesian", "baro_taup0", "baro_split",
                                  "aniso_axes0", "aniso_axes8", "aniso_cartesian",
                                  "tau0", "sp0", "gamma_mismatch", "box_small",
                                  "natoms_not3", "mass0", "null_pos"])
def test_create_rejects_invalid(L, water_sys, case):
    s = water_sys
    prm = b.default_params()
    kw = {}
    if case == "P0": kw["P"] = 0
    elif case == "P129": kw["P"] = 129
    elif case == "T0": kw["T"] = 0.0
    elif case == "dt0": kw["dt"] = -1.0
    elif case == "badpot": s.potential = 7
    elif case == "badthermo": prm.thermostat = 5
    elif case == "badint": prm.integrator = 3
    elif case == "fixcom2": prm.fixcom = 2
    elif case == "badmethod": prm.method = 5
    elif case == "badfmmode": prm.fmmode = 3
    elif case == "fmass0": prm.fmass = 0.0
    elif case == "normal_cartesian": prm.method, prm.fmmode = b.METHOD_PIMD, b.FMMODE_NORMAL
    elif case == "split_cartesian": prm.precision, prm.method = b.PREC_SPLIT, b.METHOD_PIMD
    elif case == "split_fixcom": prm.precision, prm.fixcom = b.PREC_SPLIT, 1
    elif case == "split_fmass": prm.precision, prm.fmass = b.PREC_SPLIT, 2.0
    elif case == "split_normal": prm.precision, prm.fmmode = b.PREC_SPLIT, b.FMMODE_NORMAL
    elif case == "badbaro": prm.barostat = 4
    elif case == "baro_cartesian": prm.barostat, prm.method = b.BARO_BZP_ISO, b.METHOD_PIMD
    elif case == "baro_taup0": prm.barostat, prm.taup = b.BARO_BZP_ISO, 0.0
    elif case == "baro_split": prm.barostat, prm.precision = b.BARO_BZP_ISO, b.PREC_SPLIT
    elif case == "aniso_axes0": prm.barostat, prm.baro_axes = b.BARO_BZP_ANISO, 0
    elif case == "aniso_axes8": prm.barostat, prm.baro_axes = b.BARO_BZP_ANISO, 8
    elif case == "aniso_cartesian": prm.barostat, prm.method = b.BARO_BZP_ANISO, b.METHOD_PIMD
    elif case == "tau0": prm.tau = 0.0
    elif case == "sp0": prm.sp = 0.0
    elif case == "gamma_mismatch": kw["gamma0"] = 3.0
    elif case == "box_small": s.box[1] = 11.0
    elif case == "natoms_not3": s.n_atoms = 23
    elif case == "mass0":
        s._keep[0][5] = 0.0
    elif case == "null_pos": s.pos = None
    st, h = _create(L, s, prm=prm, **kw)
    assert st == 1, (case, st)
    assert h.value is None
    assert L.pimd_last_error()


def test_null_handle_calls(L):
    assert L.pimd_step(None, 1) == 1
    assert L.pimd_sync(None) == 1
    e = b.Estimates()
    assert L.pimd_estimators(None, ctypes.byref(e)) == 1
    L.pimd_destroy(None)


def test_noise_sample_rejects_bad_sizes(L):
    """Argument checks come before any CUDA call, so they run without a GPU."""
    w = (ctypes.c_uint32 * 16)()
    e = (ctypes.c_double * 12)()
    assert L.pimd_noise_sample(1, 0, 0, 0, 4, w, e) == 1          # n_atoms < 1
    assert L.pimd_noise_sample(1, 0, 0, 4, 0, w, e) == 1          # n_modes < 1
    assert L.pimd_noise_sample(1, 70000, 0, 4, 4, w, e) == 1      # stream >= 2^16
    assert L.pimd_noise_sample(1, 0, 0, 1 << 20, 32, w, e) == 1   # more than 2^24 draws
