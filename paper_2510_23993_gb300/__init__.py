"""GB300-native per-cell stiff chemistry: Python binding of libchem.so (include/chem.h).

The binding only marshals arguments: every step of the chemistry runs in the library's CUDA
kernels.  Functions keep the C names (chem_init, chem_advance, ...); `Context` is a small
convenience wrapper over them that accepts torch tensors.  Importing the package does not
load the library; the first call does, and fails loudly if libchem.so was not built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchem.so")

CHEM_OK = 0
CHEM_EINVAL = -1
CHEM_ENOMEM = -2
CHEM_EMAXSTEPS = -3
CHEM_ENOCONV = -4
CHEM_ECUDA = -5
CHEM_EUNSUPPORTED = -6
CHEM_FLAG_FP64_RATES = 1
CHEM_FLAG_TIMING = 2
CHEM_FLAG_ORDER_RATE = 4
CHEM_FLAG_ORDER_PREV = 8
CHEM_FLAG_TWO_PASS = 16

_P = ctypes.POINTER
_c_void_p = ctypes.c_void_p


class chem_mechanism(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int32), ("nr", ctypes.c_int32),
                ("W", _P(ctypes.c_double)), ("thermo", _P(ctypes.c_double)),
                ("nu_f", _P(ctypes.c_int8)), ("nu_r", _P(ctypes.c_int8)),
                ("A", _P(ctypes.c_double)), ("b", _P(ctypes.c_double)), ("Ea", _P(ctypes.c_double)),
                ("reversible", _P(ctypes.c_uint8)), ("third_body", _P(ctypes.c_uint8)),
                ("eff", _P(ctypes.c_double))]


class chem_params(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("T_min", ctypes.c_double),
                ("bulk_frac", ctypes.c_double), ("y_floor", ctypes.c_double),
                ("k_bulk", ctypes.c_int32), ("k_max", ctypes.c_int32), ("flags", ctypes.c_int32)]


class chem_box(ctypes.Structure):
    _fields_ = [("T", ctypes.c_void_p), ("p", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("ld", ctypes.c_int64),
                ("rho", ctypes.c_void_p), ("e", ctypes.c_void_p), ("substeps", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("dt", ctypes.c_double), ("level", ctypes.c_int32)]


class chem_tune_result(ctypes.Structure):
    _fields_ = [("k_bulk", ctypes.c_int32), ("flags", ctypes.c_int32), ("bulk_blocks_per_sm", ctypes.c_int32),
                ("stiff_blocks_per_sm", ctypes.c_int32), ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float),
                ("trials", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("stiff_block", ctypes.c_int32),
                ("quantum", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class chem_train_cfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("err_weight", ctypes.c_double), ("seed", ctypes.c_uint64)]


class chem_stats(ctypes.Structure):
    _fields_ = [("ncell", ctypes.c_int64), ("nskipped", ctypes.c_int64), ("nbulk", ctypes.c_int64),
                ("nqueued", ctypes.c_int64), ("nfailed", ctypes.c_int64), ("ninvalid", ctypes.c_int64),
                ("substeps", ctypes.c_int64), ("attempts", ctypes.c_int64), ("newton", ctypes.c_int64),
                ("status", ctypes.c_int32), ("bulk_ms", ctypes.c_float), ("stiff_ms", ctypes.c_float),
                ("factorizations", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def build(force=False, verbose=False):
    """Compile libchem.so for sm_103a (nvcc; see build_lib.py)."""
    from . import build_lib
    return build_lib.build(force=force, verbose=verbose)


def lib():
    """The loaded libchem.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2510_23993_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, d, i32 = _c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32
        L.chem_default_params.argtypes = [_P(chem_params)]
        L.chem_default_params.restype = None
        L.chem_init.argtypes = [_P(chem_mechanism), _P(chem_params), i64, _P(vp)]
        L.chem_set_params.argtypes = [vp, _P(chem_params)]
        L.chem_destroy.argtypes = [vp]
        L.chem_destroy.restype = None
        adv = [vp, vp, vp, vp, i64, vp, vp, i64, d, vp, vp]
        L.chem_advance.argtypes = adv
        L.chem_advance_f64.argtypes = adv
        L.chem_advance_host.argtypes = [vp, vp, vp, vp, vp, vp, i64, d, vp, vp]
        L.chem_advance_explicit.argtypes = [vp, vp, vp, vp, i64, vp, vp, i64, d, vp, i32, i64, _P(i32), vp]
        L.chem_mk_create.argtypes = [_P(chem_mechanism), i64, _P(vp)]
        L.chem_mk_create.restype = i32
        L.chem_mk_rates.argtypes = [vp, vp, vp, vp, i64, i64, vp, vp]
        L.chem_mk_rates.restype = i32
        L.chem_mk_destroy.argtypes = [vp]
        L.chem_mk_destroy.restype = None
        L.chem_pressure_layout.argtypes = [i32, vp, i32, vp, i64, i64, vp, vp]
        L.chem_pressure_layout.restype = i32
        L.chem_state_from_TpY.argtypes = [vp, vp, vp, vp, i64, i64, vp, vp, vp]
        L.chem_state_from_TpY_f64.argtypes = [vp, vp, vp, vp, i64, i64, vp, vp, vp]
        L.chem_temperature.argtypes = [vp, vp, i64, vp, i64, vp, vp]
        L.chem_rates.argtypes = [vp, vp, vp, vp, i64, i64, vp, vp]
        L.chem_rates_tc.argtypes = [vp, vp, vp, vp, i64, i64, vp, vp]
        L.chem_status.argtypes = [vp, vp, _P(chem_stats)]
        L.chem_advance_noalloc.argtypes = [_P(chem_mechanism), _P(chem_params), vp, vp, vp, i64, vp, vp, i64, d,
                                           vp, _P(chem_stats), vp]
        L.chem_advance_noalloc.restype = i32
        L.chem_measure_fp64_peak.argtypes = [_P(ctypes.c_double), i32, vp]
        L.chem_measure_fp64_peak.restype = i32
        L.chem_boxes_set.argtypes = [vp, _P(chem_box), i32]
        L.chem_advance_boxes.argtypes = [vp, vp]
        L.chem_boxes_capture.argtypes = [vp, vp]
        L.chem_boxes_launch.argtypes = [vp, vp]
        for name in ("chem_boxes_set", "chem_advance_boxes", "chem_boxes_capture", "chem_boxes_launch"):
            getattr(L, name).restype = i32
        L.chem_tune.argtypes = [vp, vp, vp, vp, i64, vp, vp, i64, d, vp, ctypes.c_char_p, _P(chem_tune_result), vp]
        L.chem_tune.restype = i32
        L.chem_tc_gemm.argtypes = [vp, i64, i64, vp, i64, i64, vp, i64, vp, vp, i32, i32, i32, i32, i32, vp, vp]
        L.chem_tc_gemm.restype = i32
        u64, szt = ctypes.c_uint64, ctypes.c_size_t
        L.chem_surrogate_init.argtypes = [vp, u64]
        L.chem_surrogate_nparams.argtypes = [i32]
        L.chem_surrogate_train.argtypes = [vp, vp, vp, i64, _P(chem_train_cfg), vp, vp]
        L.chem_surrogate_grads.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp, vp]
        L.chem_surrogate_forward.argtypes = [vp, vp, i32, vp, vp]
        L.chem_surrogate_infer.argtypes = [vp, vp, vp, i64, vp, vp, i64, d, vp, vp]
        L.chem_surrogate_params.argtypes = [vp, vp, vp, vp]
        L.chem_surrogate_save.argtypes = [vp, vp, szt, _P(szt)]
        L.chem_surrogate_load.argtypes = [vp, vp, szt]
        L.chem_advance_gated.argtypes = [vp, vp, vp, vp, i64, vp, vp, i64, d, d, vp, vp, _P(i64), vp]
        for name in ("chem_surrogate_init", "chem_surrogate_nparams", "chem_surrogate_train", "chem_surrogate_grads",
                     "chem_surrogate_forward", "chem_surrogate_infer", "chem_surrogate_params", "chem_surrogate_save",
                     "chem_surrogate_load", "chem_advance_gated"):
            getattr(L, name).restype = i32
        L.chem_strerror.argtypes = [i32]
        L.chem_strerror.restype = ctypes.c_char_p
        for name in ("chem_init", "chem_set_params", "chem_advance", "chem_advance_f64", "chem_advance_host",
                     "chem_advance_explicit", "chem_state_from_TpY", "chem_state_from_TpY_f64", "chem_temperature", "chem_rates",
                     "chem_rates_tc", "chem_status"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


class ChemError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {lib().chem_strerror(code).decode()} ({code})")


def _check(code, what):
    if code != CHEM_OK:
        raise ChemError(code, what)


class Mechanism:
    """Host copy of a mechanism dict (synth layout) as the C struct chem_mechanism."""

    def __init__(self, mech):
        self.ns, self.nr = int(mech["ns"]), int(mech["nr"])
        self._keep = dict(
            W=np.ascontiguousarray(mech["W"], np.float64),
            thermo=np.ascontiguousarray(mech["thermo"], np.float64),
            nu_f=np.ascontiguousarray(mech["nu_f"], np.int8),
            nu_r=np.ascontiguousarray(mech["nu_r"], np.int8),
            A=np.ascontiguousarray(mech["A"], np.float64),
            b=np.ascontiguousarray(mech["b"], np.float64),
            Ea=np.ascontiguousarray(mech["Ea"], np.float64),
            reversible=np.ascontiguousarray(mech["reversible"], np.uint8),
            third_body=np.ascontiguousarray(mech["third_body"], np.uint8),
            eff=np.ascontiguousarray(mech["eff"], np.float64))
        k = self._keep
        ptr = lambda a, t: a.ctypes.data_as(_P(t))
        self.c = chem_mechanism(self.ns, self.nr, ptr(k["W"], ctypes.c_double), ptr(k["thermo"], ctypes.c_double),
                                ptr(k["nu_f"], ctypes.c_int8), ptr(k["nu_r"], ctypes.c_int8),
                                ptr(k["A"], ctypes.c_double), ptr(k["b"], ctypes.c_double),
                                ptr(k["Ea"], ctypes.c_double), ptr(k["reversible"], ctypes.c_uint8),
                                ptr(k["third_body"], ctypes.c_uint8), ptr(k["eff"], ctypes.c_double))


def chem_default_params(**overrides):
    p = chem_params()
    lib().chem_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def chem_init(mech, params=None, max_cells=0):
    m = mech if isinstance(mech, Mechanism) else Mechanism(mech)
    h = _c_void_p()
    _check(lib().chem_init(ctypes.byref(m.c), ctypes.byref(params) if params is not None else None,
                           int(max_cells), ctypes.byref(h)), "chem_init")
    return h


def chem_destroy(ctx):
    lib().chem_destroy(ctx)


def chem_set_params(ctx, params):
    _check(lib().chem_set_params(ctx, ctypes.byref(params)), "chem_set_params")


def _dp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def chem_advance(ctx, T, p, Y, ld, rho, e, n, dt, substeps, stream=None):
    fn = lib().chem_advance_f64 if T.dtype.itemsize == 8 else lib().chem_advance
    return fn(ctx, _dp(T), _dp(p), _dp(Y), int(ld), _dp(rho), _dp(e), int(n), float(dt), _dp(substeps),
              _stream(stream))


def chem_advance_host(ctx, T, p, Y, rho, e, n, dt, substeps, stream=None):
    return lib().chem_advance_host(ctx, _dp(T), _dp(p), _dp(Y), _dp(rho), _dp(e), int(n), float(dt),
                                   _dp(substeps), _stream(stream))


def chem_advance_explicit(ctx, T, p, Y, ld, rho, e, n, dt, substeps, k_steps=5, n_star=10000, stream=None):
    """The paper's explicit scheme under Algorithm 3's bulk/sparse control; returns (code, launches)."""
    nl = ctypes.c_int32(0)
    rc = lib().chem_advance_explicit(ctx, _dp(T), _dp(p), _dp(Y), int(ld), _dp(rho), _dp(e), int(n), float(dt),
                                     _dp(substeps), int(k_steps), int(n_star), ctypes.byref(nl), _stream(stream))
    return rc, nl.value


def chem_measure_fp64_peak(reps=5, stream=None):
    """FP64 FMA throughput of the current GPU, TFLOP/s (see include/chem.h)."""
    out = ctypes.c_double(0.0)
    _check(lib().chem_measure_fp64_peak(ctypes.byref(out), int(reps), _stream(stream)), "chem_measure_fp64_peak")
    return out.value


def chem_advance_noalloc(mech, params, T, p, Y, ld, rho, e, n, dt, substeps, stats=None, stream=None):
    """chem_advance without any allocation (see include/chem.h); mech is a Mechanism."""
    return lib().chem_advance_noalloc(ctypes.byref(mech.c), ctypes.byref(params) if params is not None else None,
                                      _dp(T), _dp(p), _dp(Y), int(ld), _dp(rho), _dp(e), int(n), float(dt),
                                      _dp(substeps), ctypes.byref(stats) if stats is not None else None,
                                      _stream(stream))


def chem_tc_gemm(A, sam, sak, B, sbn, sbk, C, ldc, bias, C2, M, N, K, epi, ksplit, status, stream=None):
    return lib().chem_tc_gemm(_dp(A), int(sam), int(sak), _dp(B), int(sbn), int(sbk), _dp(C), int(ldc), _dp(bias),
                              _dp(C2), int(M), int(N), int(K), int(epi), int(ksplit), _dp(status), _stream(stream))


def chem_surrogate_init(ctx, seed=0):
    return lib().chem_surrogate_init(ctx, int(seed))


def chem_surrogate_nparams(ns):
    return lib().chem_surrogate_nparams(int(ns))


def chem_surrogate_train(ctx, X, Yt, n, cfg, loss_per_epoch=None, stream=None):
    """X [n][ns + 3] = (T, p, dt, Y), Yt [n][ns + 1] = (Y1, T1), device; loss_per_epoch: ctypes float array."""
    return lib().chem_surrogate_train(ctx, _dp(X), _dp(Yt), int(n), ctypes.byref(cfg), loss_per_epoch,
                                      _stream(stream))


def chem_surrogate_grads(ctx, X, Yt, n, err_weight, grads, loss, stream=None):
    return lib().chem_surrogate_grads(ctx, _dp(X), _dp(Yt), int(n), float(err_weight), _dp(grads), _dp(loss),
                                      _stream(stream))


def chem_surrogate_forward(ctx, X, n, out, stream=None):
    return lib().chem_surrogate_forward(ctx, _dp(X), int(n), _dp(out), _stream(stream))


def chem_surrogate_infer(ctx, T, Y, ld, rho, e, n, dt, out, stream=None):
    return lib().chem_surrogate_infer(ctx, _dp(T), _dp(Y), int(ld), _dp(rho), _dp(e), int(n), float(dt), _dp(out),
                                      _stream(stream))


def chem_surrogate_params(ctx, dst=None, src=None, stream=None):
    return lib().chem_surrogate_params(ctx, _dp(dst), _dp(src), _stream(stream))


def chem_surrogate_save(ctx):
    size = ctypes.c_size_t(0)
    _check(lib().chem_surrogate_save(ctx, None, 0, ctypes.byref(size)), "chem_surrogate_save")
    buf = ctypes.create_string_buffer(size.value)
    _check(lib().chem_surrogate_save(ctx, buf, size.value, ctypes.byref(size)), "chem_surrogate_save")
    return buf.raw


def chem_surrogate_load(ctx, blob):
    return lib().chem_surrogate_load(ctx, blob, len(blob))


def chem_advance_gated(ctx, T, p, Y, ld, rho, e, n, dt, gate_tol, accepted, substeps, n_accepted=None, stream=None):
    return lib().chem_advance_gated(ctx, _dp(T), _dp(p), _dp(Y), int(ld), _dp(rho), _dp(e), int(n), float(dt),
                                    float(gate_tol), _dp(accepted), _dp(substeps),
                                    ctypes.byref(n_accepted) if n_accepted is not None else None, _stream(stream))


def chem_boxes_set(ctx, boxes):
    """boxes: sequence of dicts with tensors T, p, Y, rho, e, substeps and floats dt, level."""
    arr = (chem_box * len(boxes))()
    for k, b in enumerate(boxes):
        arr[k] = chem_box(b["T"].data_ptr(), b["p"].data_ptr() if b.get("p") is not None else None,
                          b["Y"].data_ptr(), b["Y"].stride(0), b["rho"].data_ptr(), b["e"].data_ptr(),
                          b["substeps"].data_ptr(), b["T"].shape[0], float(b["dt"]), int(b.get("level", 0)))
    return lib().chem_boxes_set(ctx, arr, len(boxes))


def chem_advance_boxes(ctx, stream=None):
    return lib().chem_advance_boxes(ctx, _stream(stream))


def chem_boxes_capture(ctx, stream):
    return lib().chem_boxes_capture(ctx, _stream(stream))


def chem_boxes_launch(ctx, stream=None):
    return lib().chem_boxes_launch(ctx, _stream(stream))


def chem_state_from_TpY(ctx, T, p, Y, ld, n, rho, e, stream=None):
    fn = lib().chem_state_from_TpY_f64 if T.dtype.itemsize == 8 else lib().chem_state_from_TpY
    return fn(ctx, _dp(T), _dp(p), _dp(Y), int(ld), int(n), _dp(rho), _dp(e), _stream(stream))


def chem_temperature(ctx, Y, ld, e, n, T, stream=None):
    return lib().chem_temperature(ctx, _dp(Y), int(ld), _dp(e), int(n), _dp(T), _stream(stream))


def chem_rates(ctx, rho, T, Y, ld, n, dYdt, stream=None):
    return lib().chem_rates(ctx, _dp(rho), _dp(T), _dp(Y), int(ld), int(n), _dp(dYdt), _stream(stream))


def chem_rates_tc(ctx, rho, T, Y, ld, n, dYdt, stream=None):
    return lib().chem_rates_tc(ctx, _dp(rho), _dp(T), _dp(Y), int(ld), int(n), _dp(dYdt), _stream(stream))


def chem_status(ctx, stream=None):
    s = chem_stats()
    _check(lib().chem_status(ctx, _stream(stream), ctypes.byref(s)), "chem_status")
    return s


def chem_strerror(code):
    return lib().chem_strerror(int(code)).decode()


CHEM_LAYOUT_SOA, CHEM_LAYOUT_AOS, CHEM_LAYOUT_AOSOA, CHEM_LAYOUT_AOS_STAGED = 0, 1, 2, 3


def pressure_layout(W, layout, X, n, p, ld=0, stream=None):
    """p = rho R T sum_k Y_k / W_k from state records X in one of the CHEM_LAYOUT_* layouts."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    _check(lib().chem_pressure_layout(W.size, W.ctypes.data_as(ctypes.c_void_p), int(layout), _dp(X), int(ld), int(n),
                                      _dp(p), _stream(stream)), "chem_pressure_layout")


class MultiKernelRates:
    """The multi-kernel, cuBLAS-GEMM rate evaluation (chem_mk_*): the per-grid baseline strategy
    that the fused single-kernel chem_rates replaces (Sec. 3.2.1, App. C)."""

    def __init__(self, mech, max_cells):
        self.mech = mech if isinstance(mech, Mechanism) else Mechanism(mech)
        h = ctypes.c_void_p()
        _check(lib().chem_mk_create(ctypes.byref(self.mech.c), int(max_cells), ctypes.byref(h)), "chem_mk_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().chem_mk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rates(self, rho, T, Y, dYdt, n=None, stream=None):
        n = T.shape[0] if n is None else n
        for t in (rho, T, Y, dYdt):
            if not t.is_cuda:
                raise ValueError("tensors must be CUDA tensors")
        _check(lib().chem_mk_rates(self.handle, _dp(rho), _dp(T), _dp(Y), Y.stride(0), int(n), _dp(dYdt),
                                   _stream(stream)), "chem_mk_rates")


class Context:
    """One mechanism on the current CUDA device; methods take torch tensors (SoA layout)."""

    def __init__(self, mech, max_cells, params=None, **param_overrides):
        self.mech = mech if isinstance(mech, Mechanism) else Mechanism(mech)
        self.params = params if params is not None else chem_default_params(**param_overrides)
        self.handle = chem_init(self.mech, self.params, max_cells)
        self.ns = self.mech.ns

    def close(self):
        if self.handle is not None:
            chem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **overrides):
        for k, v in overrides.items():
            setattr(self.params, k, v)
        chem_set_params(self.handle, self.params)

    @staticmethod
    def _check_state(T, Y, *others):
        n = T.shape[0]
        for t in (T, Y) + others:
            if t is not None and (not t.is_cuda or not t.is_contiguous()):
                raise ValueError("tensors must be contiguous CUDA tensors")
        return n

    def advance(self, T, p, Y, rho, e, dt, substeps, stream=None):
        n = self._check_state(T, Y, p, rho, e, substeps)
        _check(chem_advance(self.handle, T, p, Y, Y.stride(0), rho, e, n, dt, substeps, stream), "chem_advance")

    def advance_explicit(self, T, p, Y, rho, e, dt, substeps, k_steps=5, n_star=10000, stream=None):
        """Explicit first-order scheme of Sec. 2.1 under Algorithm 3 (bulk launches of k_steps
        substeps while more than n_star cells are active, then one sparse launch); returns the
        number of bulk launches.  Synchronizes the stream."""
        n = self._check_state(T, Y, p, rho, e, substeps)
        rc, nl = chem_advance_explicit(self.handle, T, p, Y, Y.stride(0), rho, e, n, dt, substeps, k_steps, n_star,
                                       stream)
        _check(rc, "chem_advance_explicit")
        return nl

    def advance_host(self, T, p, Y, rho, e, dt, substeps, stream=None):
        _check(chem_advance_host(self.handle, T, p, Y, rho, e, T.shape[0], dt, substeps, stream),
               "chem_advance_host")

    def state_from_TpY(self, T, p, Y, rho, e, stream=None):
        n = self._check_state(T, Y, p, rho, e)
        _check(chem_state_from_TpY(self.handle, T, p, Y, Y.stride(0), n, rho, e, stream), "chem_state_from_TpY")

    def temperature(self, Y, e, T, stream=None):
        n = self._check_state(T, Y, e)
        _check(chem_temperature(self.handle, Y, Y.stride(0), e, n, T, stream), "chem_temperature")

    def rates(self, rho, T, Y, dYdt, stream=None):
        n = self._check_state(T, Y, rho, dYdt)
        _check(chem_rates(self.handle, rho, T, Y, Y.stride(0), n, dYdt, stream), "chem_rates")

    def rates_tc(self, rho, T, Y, dYdt, stream=None):
        """chem_rates with the stoichiometric contractions on the tensor cores (53 species)."""
        n = self._check_state(T, Y, rho, dYdt)
        _check(chem_rates_tc(self.handle, rho, T, Y, Y.stride(0), n, dYdt, stream), "chem_rates_tc")

    def status(self, stream=None):
        return chem_status(self.handle, stream).as_dict()

    def tune(self, T, p, Y, rho, e, dt, substeps, cache_path=None, stream=None):
        """Autotune the launch configuration on this field (inputs are left unchanged)."""
        res = chem_tune_result()
        cp = cache_path.encode() if cache_path else None
        _check(lib().chem_tune(self.handle, _dp(T), _dp(p), _dp(Y), Y.stride(0), _dp(rho), _dp(e), T.shape[0],
                               float(dt), _dp(substeps), cp, ctypes.byref(res), _stream(stream)), "chem_tune")
        # keep the parameter mirror in step with what the tuner applied
        order_bits = CHEM_FLAG_ORDER_RATE | CHEM_FLAG_ORDER_PREV | CHEM_FLAG_TWO_PASS
        self.params.k_bulk = res.k_bulk
        self.params.flags = (self.params.flags & ~order_bits) | res.flags
        return res.as_dict()

    def set_boxes(self, boxes):
        self._boxes = list(boxes)   # the library references these tensors
        _check(chem_boxes_set(self.handle, self._boxes), "chem_boxes_set")

    def advance_boxes(self, stream=None):
        _check(chem_advance_boxes(self.handle, stream), "chem_advance_boxes")

    def capture_boxes(self, stream):
        _check(chem_boxes_capture(self.handle, stream), "chem_boxes_capture")

    def launch_boxes(self, stream=None):
        _check(chem_boxes_launch(self.handle, stream), "chem_boxes_launch")

    # ---- surrogate
    def surrogate_init(self, seed=0):
        _check(chem_surrogate_init(self.handle, seed), "chem_surrogate_init")

    def surrogate_train(self, X, Yt, epochs=20, batch=4096, lr=1e-3, weight_decay=1e-5, err_weight=0.1, seed=0,
                        stream=None):
        """Train on device arrays X [n][ns + 3] = (T, p, dt, Y) and Yt [n][ns + 1] = (Y1, T1), the state
        after dt; returns the mean loss of each epoch."""
        for t in (X, Yt):
            if not t.is_cuda or not t.is_contiguous() or t.dtype.itemsize != 4:
                raise ValueError("X and Yt must be contiguous float32 CUDA tensors")
        cfg = chem_train_cfg(int(epochs), int(batch), float(lr), float(weight_decay), float(err_weight), int(seed))
        losses = (ctypes.c_float * max(int(epochs), 1))()
        _check(chem_surrogate_train(self.handle, X, Yt, X.shape[0], cfg, losses, stream), "chem_surrogate_train")
        return list(losses)[:int(epochs)]

    def surrogate_grads(self, X, Yt, err_weight, grads, loss, stream=None):
        _check(chem_surrogate_grads(self.handle, X, Yt, X.shape[0], err_weight, grads, loss, stream),
               "chem_surrogate_grads")

    def surrogate_forward(self, X, out, stream=None):
        _check(chem_surrogate_forward(self.handle, X, X.shape[0], out, stream), "chem_surrogate_forward")

    def surrogate_infer(self, T, Y, rho, e, dt, out, stream=None):
        n = self._check_state(T, Y, rho, e, out)
        _check(chem_surrogate_infer(self.handle, T, Y, Y.stride(0), rho, e, n, dt, out, stream), "chem_surrogate_infer")

    def surrogate_params(self, dst=None, src=None, stream=None):
        _check(chem_surrogate_params(self.handle, dst, src, stream), "chem_surrogate_params")

    def surrogate_save(self):
        return chem_surrogate_save(self.handle)

    def surrogate_load(self, blob):
        _check(chem_surrogate_load(self.handle, blob), "chem_surrogate_load")

    def advance_gated(self, T, p, Y, rho, e, dt, gate_tol, accepted, substeps, stream=None):
        """One step with the surrogate in front of the method; returns the number of accepted cells."""
        n = self._check_state(T, Y, p, rho, e, substeps, accepted)
        na = ctypes.c_int64(0)
        _check(chem_advance_gated(self.handle, T, p, Y, Y.stride(0), rho, e, n, dt, gate_tol, accepted, substeps, na,
                                  stream), "chem_advance_gated")
        return int(na.value)
