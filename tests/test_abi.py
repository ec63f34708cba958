"""The C-ABI library loads and exports every entry point include/chem.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

import paper_2510_23993_gb300 as chem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(chem_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    chem.build()
    return chem.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("chem_init", "chem_advance", "chem_advance_f64", "chem_advance_host", "chem_destroy",
              "chem_status", "chem_strerror", "chem_rates", "chem_temperature", "chem_state_from_TpY"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_logic_without_gpu(lib):
    p = chem.chem_default_params()
    assert p.k_bulk == 1 and p.k_max == 100000 and 0 < p.rtol < 1e-3
    assert chem.chem_strerror(chem.CHEM_EMAXSTEPS).startswith("a stiff cell")
    # argument checks happen on the host before any CUDA call
    out = ctypes.c_void_p()
    assert lib.chem_init(None, None, 10, ctypes.byref(out)) == chem.CHEM_EINVAL
    st = chem.chem_stats()
    assert lib.chem_status(None, None, ctypes.byref(st)) == chem.CHEM_EINVAL


def test_bad_mechanism_rejected_before_device_use(lib, h2mech):
    import numpy as np
    bad = dict(h2mech)
    bad["W"] = np.array(h2mech["W"], copy=True)
    bad["W"][0] = -1.0
    m = chem.Mechanism(bad)
    out = ctypes.c_void_p()
    assert lib.chem_init(ctypes.byref(m.c), None, 10, ctypes.byref(out)) == chem.CHEM_EINVAL
    bad = dict(h2mech)
    th = np.array(h2mech["thermo"], copy=True)
    th[3, 8] = 4000.0   # species ranges must agree
    bad["thermo"] = th
    m = chem.Mechanism(bad)
    assert lib.chem_init(ctypes.byref(m.c), None, 10, ctypes.byref(out)) == chem.CHEM_EINVAL
    bad_params = chem.chem_default_params(k_bulk=0)
    m = chem.Mechanism(h2mech)
    assert lib.chem_init(ctypes.byref(m.c), ctypes.byref(bad_params), 10, ctypes.byref(out)) == chem.CHEM_EINVAL


def _prototypes():
    """name -> number of parameters of every chem_* function declared in include/*.h"""
    out = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(chem_\w+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    """Every entry point the binding types takes as many arguments as the header declares."""
    protos = _prototypes()
    assert len(protos) >= 35
    checked = 0
    for name, nargs in protos.items():
        fn = getattr(lib, name, None)
        if fn is None or fn.argtypes is None:
            continue
        assert len(fn.argtypes) == nargs, (name, len(fn.argtypes), nargs)
        checked += 1
    assert checked >= 30


def test_new_entry_points_check_arguments_on_the_host(lib):
    import numpy as np
    out = ctypes.c_void_p()
    assert lib.chem_mk_create(None, 10, ctypes.byref(out)) == chem.CHEM_EINVAL
    nl = ctypes.c_int32(-1)
    assert lib.chem_advance_explicit(None, None, None, None, 0, None, None, 0, 1e-8, None, 5, 10000,
                                     ctypes.byref(nl), None) == chem.CHEM_EINVAL
    assert nl.value == 0
    W = np.full(9, 0.02)
    Wp = W.ctypes.data_as(ctypes.c_void_p)
    assert lib.chem_pressure_layout(9, Wp, 7, None, 0, 0, None, None) == chem.CHEM_EINVAL      # unknown layout
    assert lib.chem_pressure_layout(9, Wp, chem.CHEM_LAYOUT_SOA, None, 0, 0, None, None) == chem.CHEM_OK   # nothing to do
    assert lib.chem_pressure_layout(10, np.full(10, 0.02).ctypes.data_as(ctypes.c_void_p), chem.CHEM_LAYOUT_AOS,
                                    None, 0, 0, None, None) == chem.CHEM_EUNSUPPORTED
    assert lib.chem_pressure_layout(9, None, chem.CHEM_LAYOUT_AOS, None, 0, 0, None, None) == chem.CHEM_EINVAL


@pytest.mark.parametrize("defect", ["A_nonpositive", "nu_4", "eff_negative", "T_range", "W_nan"])
def test_both_entry_points_refuse_the_same_bad_mechanisms(lib, h2mech, defect):
    """chem_init and chem_advance_noalloc run the same host-side checks, before any device use,
    so a mechanism that one refuses the other refuses too (CHEM_EINVAL)."""
    import numpy as np
    bad = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in h2mech.items()}
    if defect == "A_nonpositive":
        bad["A"][3] = 0.0
    elif defect == "nu_4":
        bad["nu_f"][2, 1] = 4
    elif defect == "eff_negative":
        r = int(np.nonzero(bad["third_body"])[0][0])
        bad["eff"][r, 0] = -1.0
    elif defect == "T_range":
        bad["thermo"][:, 8] = bad["thermo"][:, 7]   # T_hi == T_lo
    else:
        bad["W"][4] = np.nan
    m = chem.Mechanism(bad)
    out = ctypes.c_void_p()
    assert lib.chem_init(ctypes.byref(m.c), None, 10, ctypes.byref(out)) == chem.CHEM_EINVAL
    assert not out.value
    rc = lib.chem_advance_noalloc(ctypes.byref(m.c), None, None, None, None, 0, None, None, 0, 1e-8, None, None,
                                  None)
    assert rc == chem.CHEM_EINVAL
    # and the same parameter checks: an unknown flag bit is refused by both
    good = chem.Mechanism(h2mech)
    bad_p = chem.chem_default_params(flags=1 << 12)
    assert lib.chem_init(ctypes.byref(good.c), ctypes.byref(bad_p), 10, ctypes.byref(out)) == chem.CHEM_EINVAL
    assert lib.chem_advance_noalloc(ctypes.byref(good.c), ctypes.byref(bad_p), None, None, None, 0, None, None, 0,
                                    1e-8, None, None, None) == chem.CHEM_EINVAL


def test_fp64_peak_measurement_checks_arguments_on_the_host(lib):
    out = ctypes.c_double(-1.0)
    assert lib.chem_measure_fp64_peak(None, 5, None) == chem.CHEM_EINVAL
    assert lib.chem_measure_fp64_peak(ctypes.byref(out), 0, None) == chem.CHEM_EINVAL
    assert out.value == -1.0   # nothing written on a refused call
