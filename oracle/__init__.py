"""FP64 CPU oracle of per-cell stiff chemistry (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this package.  It is built from `oracle.c` with gcc (OpenMP over cells) and loaded with
ctypes; it shares no code with the CUDA library.  See oracle.c for what it computes and
which sections of the paper it follows.

Parity status: pinned by closed forms (first/second order, third body), invariants (sum Y,
element mass, internal energy), detailed balance against an independent entropy-maximising
equilibrium solver, the thermodynamic affinity relation q_f/q_r = exp(-dG/RT), step-halving
extrapolation of a brute-force backward-Euler integration, T(e) round trips, and the
temperature-ODE cross-check (corrected Eq. 6).
"""
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

R_GAS = 8.314462618


def build(force=False):
    """Compile oracle.c into _oracle.so (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


D, I8, U8, I32 = ctypes.c_double, ctypes.c_int8, ctypes.c_uint8, ctypes.c_int32


class _Mech:
    """Keeps contiguous copies of the mechanism arrays alive for the C calls."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech["ns"]), int(mech["nr"])
        self.W = np.ascontiguousarray(mech["W"], np.float64)
        self.thermo = np.ascontiguousarray(mech["thermo"], np.float64)
        self.nu_f = np.ascontiguousarray(mech["nu_f"], np.int8)
        self.nu_r = np.ascontiguousarray(mech["nu_r"], np.int8)
        self.A = np.ascontiguousarray(mech["A"], np.float64)
        self.b = np.ascontiguousarray(mech["b"], np.float64)
        self.Ea = np.ascontiguousarray(mech["Ea"], np.float64)
        self.rev = np.ascontiguousarray(mech["reversible"], np.uint8)
        self.tb = np.ascontiguousarray(mech["third_body"], np.uint8)
        self.eff = np.ascontiguousarray(mech["eff"], np.float64)

    def args(self):
        return (ctypes.c_int(self.ns), ctypes.c_int(self.nr), _p(self.W, D), _p(self.thermo, D),
                _p(self.nu_f, I8), _p(self.nu_r, I8), _p(self.A, D), _p(self.b, D), _p(self.Ea, D),
                _p(self.rev, U8), _p(self.tb, U8), _p(self.eff, D))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def state_from_TpY(mech, T, p, Y):
    """rho = p / (R T sum Y/W) and e = sum Y_k u_k(T) for each cell (Y is [ns, n])."""
    lib, M = _load(), _Mech(mech)
    T, p, Y = _f64(T), _f64(p), _f64(Y)
    n = T.shape[0]
    rho, e = np.empty(n), np.empty(n)
    lib.oracle_state_from_TpY(*M.args(), ctypes.c_int64(n), _p(T, D), _p(p, D), _p(Y, D),
                              ctypes.c_int64(n), _p(rho, D), _p(e, D))
    return rho, e


def temperature_from_energy(mech, Y, e, T_guess):
    lib, M = _load(), _Mech(mech)
    Y, e, T_guess = _f64(Y), _f64(e), _f64(T_guess)
    n = e.shape[0]
    T = np.empty(n)
    lib.oracle_T_from_e(*M.args(), ctypes.c_int64(n), _p(Y, D), ctypes.c_int64(n), _p(e, D),
                        _p(T_guess, D), _p(T, D))
    return T


def rates(mech, rho, T, Y, with_progress=False):
    """dY/dt [ns, n] (Eq. 5) at the given states; optionally q_f, q_r [nr, n]."""
    lib, M = _load(), _Mech(mech)
    rho, T, Y = _f64(rho), _f64(T), _f64(Y)
    n = T.shape[0]
    dYdt = np.empty((M.ns, n))
    qf = np.empty((M.nr, n)) if with_progress else None
    qr = np.empty((M.nr, n)) if with_progress else None
    lib.oracle_rates(*M.args(), ctypes.c_int64(n), _p(rho, D), _p(T, D), _p(Y, D),
                     ctypes.c_int64(n), _p(dYdt, D),
                     _p(qf, D) if with_progress else None, _p(qr, D) if with_progress else None)
    return (dYdt, qf, qr) if with_progress else dYdt


def thermo(mech, T):
    """cp/R, h/RT, s/R of every species at T [n] -> three [ns, n] arrays."""
    lib, M = _load(), _Mech(mech)
    T = _f64(T)
    n = T.shape[0]
    out = np.empty((3, M.ns, n))
    lib.oracle_thermo(*M.args(), ctypes.c_int64(n), _p(T, D), _p(out, D))
    return out[0], out[1], out[2]


def advance(mech, rho, e, T, Y, dt, rtol=1e-10, atol=1e-14, T_min=0.0, max_steps=200000):
    """Exact (to rtol) solution at t = dt of the constant-volume adiabatic reactor per cell.

    Returns (T, p, Y, steps); cells with T < T_min are returned unchanged with steps = 0 and
    p = NaN; steps = -1 marks a failed integration."""
    lib, M = _load(), _Mech(mech)
    rho, e = _f64(rho), _f64(e)
    T = np.array(T, dtype=np.float64, copy=True)
    Y = np.array(Y, dtype=np.float64, copy=True, order="C")
    n = T.shape[0]
    p = np.full(n, np.nan)
    steps = np.zeros(n, dtype=np.int32)
    lib.oracle_advance(*M.args(), ctypes.c_int64(n), _p(rho, D), _p(e, D), _p(T, D), _p(p, D),
                       _p(Y, D), ctypes.c_int64(n), ctypes.c_double(dt), ctypes.c_double(rtol),
                       ctypes.c_double(atol), ctypes.c_double(T_min), ctypes.c_int(max_steps),
                       _p(steps, I32))
    return T, p, Y, steps


def explicit(mech, rho, e, T, Y, dt, frac=0.05, y_floor=1e-10, T_min=0.0, k_max=100000):
    """The paper's explicit first-order scheme (Sec. 2.1) per cell: forward Euler substeps that
    change no Y_k by more than frac * max(|Y_k|, y_floor).  Returns (T, p, Y, steps); steps = 0
    for cells below T_min, -1 for cells that do not reach dt within k_max substeps."""
    lib, M = _load(), _Mech(mech)
    rho, e = _f64(rho), _f64(e)
    T = np.array(T, dtype=np.float64, copy=True)
    Y = np.array(Y, dtype=np.float64, copy=True, order="C")
    n = T.shape[0]
    p = np.full(n, np.nan)
    steps = np.zeros(n, dtype=np.int64)
    lib.oracle_explicit(*M.args(), ctypes.c_int64(n), _p(rho, D), _p(e, D), _p(T, D), _p(p, D), _p(Y, D),
                        ctypes.c_int64(n), ctypes.c_double(dt), ctypes.c_double(frac), ctypes.c_double(y_floor),
                        ctypes.c_double(T_min), ctypes.c_int64(k_max), _p(steps, ctypes.c_int64))
    return T, p, Y, steps


def backward_euler(mech, rho, e, T, Y, dt, nsteps):
    """Brute force: nsteps uniform backward-Euler steps of one cell (Newton to round-off)."""
    lib, M = _load(), _Mech(mech)
    y = np.array(Y, dtype=np.float64, copy=True)
    Tc = ctypes.c_double(float(T))
    ok = lib.oracle_backward_euler(*M.args(), ctypes.c_double(rho), ctypes.c_double(e), _p(y, D),
                                   ctypes.byref(Tc), ctypes.c_double(dt), ctypes.c_int64(nsteps))
    if not ok:
        raise RuntimeError("backward Euler Newton failed")
    return Tc.value, y


def temperature_ode(mech, rho, T, Y, dt, nsteps):
    """Integrate (Y, T) with the corrected Eq. 6 energy equation (RK4, nsteps steps)."""
    lib, M = _load(), _Mech(mech)
    y = np.array(Y, dtype=np.float64, copy=True)
    Tc = ctypes.c_double(float(T))
    lib.oracle_temperature_ode(*M.args(), ctypes.c_double(rho), _p(y, D), ctypes.byref(Tc),
                               ctypes.c_double(dt), ctypes.c_int64(nsteps))
    return Tc.value, y


def radau_tableau():
    lib = _load()
    A = np.empty(9)
    c = np.empty(3)
    lib.oracle_radau_tableau(_p(A, D), _p(c, D))
    return A.reshape(3, 3), c


def max_threads():
    lib = _load()
    lib.oracle_max_threads.restype = ctypes.c_int
    return int(lib.oracle_max_threads())
