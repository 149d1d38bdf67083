"""ctypes binding of libqarray.so (include/qarray.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device
memory and streams); host matrices are numpy arrays.  The library is built
in-tree on first use if missing; when it cannot be loaded every call raises
-- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_DOT = 16
MAX_GATE = 64

QA_OK = 0
ERRORS = {
    -1: "QA_ERR_INVALID", -2: "QA_ERR_SHAPE", -3: "QA_ERR_NOT_SYMMETRIC",
    -4: "QA_ERR_NOT_PD", -5: "QA_ERR_RANGE", -6: "QA_ERR_OVERFLOW",
    -7: "QA_ERR_CUDA", -8: "QA_ERR_TIMEOUT", -9: "QA_ERR_NOMEM",
    -10: "QA_ERR_UNRESOLVED",
}
QA_FORM_MAXWELL = 0
QA_FORM_COUPLING = 1

FLAG_NEAR_TIE = 1
FLAG_BOUNDARY = 2
FLAG_QP = 4
FLAG_QP_CAP = 8
FLAG_RECHECKED = 16
FLAG_DOUBLED = 32
FLAG_UNRESOLVED = 64
FLAG_OVERFLOW = 128


class QAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class qa_raster(ctypes.Structure):
    _fields_ = [("V0", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)),
                ("w", ctypes.POINTER(ctypes.c_double)),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("W", ctypes.c_int), ("H", ctypes.c_int)]


class qa_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in (
        "pixels", "candidates", "evaluated", "qp_pixels", "flagged", "near_tie",
        "boundary", "unresolved", "overflow", "doubled", "shortlist_max",
        "resolved")] + [
        ("team", ctypes.c_int), ("inner_bits", ctypes.c_int),
        ("middle_bits", ctypes.c_int), ("timed", ctypes.c_int),
        ("ms_prep", ctypes.c_double), ("ms_search", ctypes.c_double),
        ("ms_recheck", ctypes.c_double), ("ms_soft", ctypes.c_double)]


class qa_sensor_params(ctypes.Structure):
    _fields_ = [("n_sensor", ctypes.c_int), ("shape", ctypes.c_int),
                ("width", ctypes.c_double), ("white_sigma", ctypes.c_double),
                ("pink_sigma", ctypes.c_double), ("jump_amplitude", ctypes.c_double),
                ("jump_prob", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


class qa_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


QA_SENSOR_LORENTZIAN = 0
QA_SENSOR_GAUSSIAN = 1


class qa_batch_item(ctypes.Structure):
    _fields_ = [("model", ctypes.c_void_p), ("raster", qa_raster),
                ("threshold", ctypes.c_double), ("closed", ctypes.c_int),
                ("n_charges", ctypes.c_int), ("team", ctypes.c_int),
                ("out_n", ctypes.c_void_p), ("out_U", ctypes.c_void_p),
                ("out_flags", ctypes.c_void_p)]


_lib = None
_SYMBOLS = None


def library_path() -> str:
    """The in-tree library, or the one named by QARRAY_LIB (a build made
    elsewhere)."""
    return os.environ.get("QARRAY_LIB") or _build.LIB


def load():
    """Load (building if needed) libqarray.so; raises if that fails."""
    global _lib, _SYMBOLS
    if _lib is not None:
        return _lib
    path = os.environ.get("QARRAY_LIB") or _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.c_int
    sig = {
        "qa_model_create": (I, [D, D, I, I, I, ctypes.c_double, ctypes.POINTER(P)]),
        "qa_model_update": (I, [P, D, D]),
        "qa_model_update_async": (I, [P, D, D, P]),
        "qa_model_update_dev": (I, [P, P, P, P]),
        "qa_model_destroy": (I, [P]),
        "qa_model_shape": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "qa_model_get": (I, [P, D, D, D]),
        "qa_ground_state_open": (I, [P, ctypes.POINTER(qa_raster), ctypes.c_double,
                                     P, P, P, P]),
        "qa_ground_state_closed": (I, [P, ctypes.POINTER(qa_raster), ctypes.c_double,
                                       I, P, P, P, P]),
        "qa_ground_state_points": (I, [P, P, ctypes.c_longlong, ctypes.c_double, I, I,
                                       P, P, P, P]),
        "qa_optimal_gate_voltages": (I, [P, P, I, I, I, ctypes.c_double, P, P]),
        "qa_virtual_gate_matrix": (I, [P, P, I, I, I, P]),
        "qa_charge_sensor": (I, [P, ctypes.POINTER(qa_raster), P,
                                 ctypes.POINTER(qa_sensor_params), P, P, P, P]),
        "qa_ground_state_i16": (I, [P, ctypes.POINTER(qa_raster), ctypes.c_double, I, I,
                                    P, P, P, P]),
        "qa_brute_force_open": (I, [P, ctypes.POINTER(qa_raster), I, P, P, P, P]),
        "qa_brute_force_closed": (I, [P, ctypes.POINTER(qa_raster), I, P, P, P, P]),
        "qa_soft_occupation": (I, [P, ctypes.POINTER(qa_raster), ctypes.c_double,
                                   ctypes.c_double, I, I, P, P, P]),
        "qa_soft_occupation_backward": (I, [P, ctypes.POINTER(qa_raster),
                                            ctypes.c_double, ctypes.c_double, I, I,
                                            P, P, P, P]),
        "qa_soft_occupation_ctx": (I, [P, ctypes.POINTER(qa_raster), ctypes.c_double,
                                       ctypes.c_double, I, I, P, P, P, P]),
        "qa_soft_occupation_backward_ctx": (I, [P, ctypes.POINTER(qa_raster),
                                                ctypes.c_double, ctypes.c_double, I, I,
                                                P, P, P, P, P, P]),
        "qa_fit_step": (I, [P, ctypes.POINTER(qa_raster), ctypes.c_double, ctypes.c_double,
                            I, I, P, I, P, P, P, ctypes.POINTER(qa_adam), P, P, P, P, P]),
        "qa_model_stats": (I, [P, P, ctypes.POINTER(qa_stats)]),
        "qa_model_set_timing": (I, [P, I]),
        "qa_ground_state_open_static": (I, [P, ctypes.POINTER(qa_raster),
                                            ctypes.c_double, P, P, P, P]),
        "qa_batch_create": (I, [ctypes.POINTER(qa_batch_item), I, ctypes.POINTER(P)]),
        "qa_batch_run": (I, [P, P]),
        "qa_batch_stats": (I, [P, P, ctypes.POINTER(qa_stats)]),
        "qa_batch_destroy": (I, [P]),
        "qa_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _SYMBOLS = tuple(sig)
    _lib = lib
    return lib


def exported_symbols():
    load()
    return _SYMBOLS


def qa_last_error() -> str:
    return load().qa_last_error().decode()


def _check(rc):
    if rc != QA_OK:
        raise QAError(rc, qa_last_error())


def _host(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, numel=None, name="buffer"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def make_raster(r, n_gate):
    """qa_raster from a dict {V0, u, w, x0, x1, y0, y1, W, H}; the struct
    keeps its host arrays alive.  An existing qa_raster is passed through, so
    a caller making many calls on one raster can build it once."""
    if isinstance(r, qa_raster):
        return r
    V0, pV0 = _host(r["V0"], (n_gate,))
    u, pu = _host(r["u"], (n_gate,))
    w, pw = _host(r["w"], (n_gate,))
    s = qa_raster(pV0, pu, pw, float(r["x0"]), float(r["x1"]), float(r["y0"]),
                  float(r["y1"]), int(r["W"]), int(r["H"]))
    s._keep = (V0, u, w)
    return s


# --------------------------------------------------------------------------
# the C ABI, name for name
# --------------------------------------------------------------------------

def qa_model_create(Cdd, Cgd, form=QA_FORM_MAXWELL, carrier_sign=1.0):
    Cgd = np.atleast_2d(np.asarray(Cgd, dtype=np.float64))
    n, ng = Cgd.shape
    Cd, pCd = _host(Cdd, (n, n))
    Cg, pCg = _host(Cgd, (n, ng))
    h = ctypes.c_void_p()
    _check(load().qa_model_create(pCd, pCg, n, ng, int(form), float(carrier_sign),
                                  ctypes.byref(h)))
    _SHAPES[h.value] = (n, ng)
    return h


def qa_model_update(m, Cdd, Cgd):
    n, ng = qa_model_shape(m)
    _, pCd = _host(Cdd, (n, n))
    _, pCg = _host(Cgd, (n, ng))
    _check(load().qa_model_update(m, pCd, pCg))


def qa_model_update_async(m, Cdd, Cgd, stream=None):
    n, ng = qa_model_shape(m)
    _, pCd = _host(Cdd, (n, n))
    _, pCg = _host(Cgd, (n, ng))
    _check(load().qa_model_update_async(m, pCd, pCg, _stream(stream)))


def qa_model_update_dev(m, Cdd_dev, Cgd_dev, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    _check(load().qa_model_update_dev(m, _dev(Cdd_dev, torch.float64, n * n, "Cdd"),
                                      _dev(Cgd_dev, torch.float64, n * ng, "Cgd"),
                                      _stream(stream)))


def qa_model_destroy(m):
    _SHAPES.pop(m.value if isinstance(m, ctypes.c_void_p) else m, None)
    _check(load().qa_model_destroy(m))


_SHAPES = {}  # model handle -> (n_dot, n_gate), immutable for a model's lifetime


def qa_model_shape(m):
    key = m.value if isinstance(m, ctypes.c_void_p) else m
    if key in _SHAPES:
        return _SHAPES[key]
    n = ctypes.c_int()
    ng = ctypes.c_int()
    _check(load().qa_model_shape(m, ctypes.byref(n), ctypes.byref(ng)))
    return n.value, ng.value


def qa_model_get(m):
    n, ng = qa_model_shape(m)
    Cdd = np.zeros((n, n))
    M = np.zeros((n, n))
    Cgd = np.zeros((n, ng))
    D = ctypes.POINTER(ctypes.c_double)
    _check(load().qa_model_get(m, Cdd.ctypes.data_as(D), M.ctypes.data_as(D),
                               Cgd.ctypes.data_as(D)))
    return Cdd, M, Cgd


def qa_ground_state_open(m, raster, threshold, out_n, out_U=None, out_flags=None,
                         stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_ground_state_open(
        m, ctypes.byref(r), float(threshold), _dev(out_n, torch.int8, P * n, "out_n"),
        _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


def qa_ground_state_i16(m, raster, threshold, closed, n_charges, out_n, out_U=None,
                        out_flags=None, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_ground_state_i16(
        m, ctypes.byref(r), float(threshold), int(bool(closed)), int(n_charges),
        _dev(out_n, torch.int16, P * n, "out_n"), _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


STATIC_MAX_PIXELS = 16384


def qa_ground_state_open_static(m, raster, threshold, out_n, out_U=None,
                                out_flags=None, stream=None):
    """qa_ground_state_open without any GPU allocation: the scratch is the
    library's static device array, so the raster holds at most
    STATIC_MAX_PIXELS pixels and calls on one device must not overlap."""
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_ground_state_open_static(
        m, ctypes.byref(r), float(threshold), _dev(out_n, torch.int8, P * n, "out_n"),
        _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


def qa_ground_state_closed(m, raster, threshold, n_charges, out_n, out_U=None,
                           out_flags=None, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_ground_state_closed(
        m, ctypes.byref(r), float(threshold), int(n_charges),
        _dev(out_n, torch.int8, P * n, "out_n"), _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


def qa_ground_state_points(m, V, threshold, closed, n_charges, out_n, out_U=None,
                           out_flags=None, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    P = V.shape[0]
    _check(load().qa_ground_state_points(
        m, _dev(V, torch.float64, P * ng, "V"), P, float(threshold), int(closed),
        int(n_charges), _dev(out_n, torch.int8, P * n, "out_n"),
        _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


BF_NEAR_TIE = 1
BF_AT_BOX = 2


def qa_charge_sensor(m, raster, n_dots, params, out_signal, out_n_sensor=None,
                     out_potential=None, stream=None):
    """params: dict with n_sensor, shape, width, white_sigma, pink_sigma,
    jump_amplitude, jump_prob, seed."""
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    S = int(params["n_sensor"])
    sp = qa_sensor_params(S, int(params.get("shape", 0)), float(params.get("width", 0.05)),
                          float(params.get("white_sigma", 0.0)),
                          float(params.get("pink_sigma", 0.0)),
                          float(params.get("jump_amplitude", 0.0)),
                          float(params.get("jump_prob", 0.0)), int(params.get("seed", 0)))
    _check(load().qa_charge_sensor(
        m, ctypes.byref(r), _dev(n_dots, torch.int8, P * (n - S), "n_dots"), ctypes.byref(sp),
        _dev(out_signal, torch.float32, P * S, "out_signal"),
        _dev(out_n_sensor, torch.int8, P * S, "out_n_sensor"),
        _dev(out_potential, torch.float64, P * S, "out_potential"), _stream(stream)))




def qa_optimal_gate_voltages(Cdd, Cgd, Q, form=QA_FORM_MAXWELL, carrier_sign=1.0):
    """Gate voltages minimising the free energy of charge state Q (host)."""
    Cgd = np.ascontiguousarray(Cgd, dtype=np.float64)
    n, ng = Cgd.shape
    Cdd, _ = _host(Cdd, (n, n))
    Q, _ = _host(Q, (n,))
    V = np.zeros(ng)
    _check(load().qa_optimal_gate_voltages(
        Cdd.ctypes.data, Cgd.ctypes.data, n, ng, int(form), float(carrier_sign),
        Q.ctypes.data, V.ctypes.data))
    return V


def qa_virtual_gate_matrix(Cdd, Cgd, form=QA_FORM_MAXWELL):
    """alpha = (Cdd^-1 Cgd)^+, [n_gate, n_dot] (host)."""
    Cgd = np.ascontiguousarray(Cgd, dtype=np.float64)
    n, ng = Cgd.shape
    Cdd, _ = _host(Cdd, (n, n))
    alpha = np.zeros((ng, n))
    _check(load().qa_virtual_gate_matrix(Cdd.ctypes.data, Cgd.ctypes.data, n, ng, int(form),
                                         alpha.ctypes.data))
    return alpha


def virtual_raster(Cdd, Cgd, V0, dot_x, dot_y, lo=-1.0, hi=1.0, W=100, H=100,
                   form=QA_FORM_MAXWELL):
    """Raster sweeping the virtual gates of dots dot_x (fast axis) and dot_y
    around the gate voltages V0: u, w are columns of the virtual gate matrix."""
    alpha = qa_virtual_gate_matrix(Cdd, Cgd, form)
    return {"V0": np.asarray(V0, dtype=np.float64), "u": alpha[:, dot_x].copy(),
            "w": alpha[:, dot_y].copy(), "x0": lo, "x1": hi, "y0": lo, "y1": hi,
            "W": int(W), "H": int(H)}


def qa_brute_force_open(m, raster, n_max, out_n, out_U=None, out_flags=None, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_brute_force_open(
        m, ctypes.byref(r), int(n_max), _dev(out_n, torch.int8, P * n, "out_n"),
        _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


def qa_brute_force_closed(m, raster, n_charges, out_n, out_U=None, out_flags=None,
                          stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_brute_force_closed(
        m, ctypes.byref(r), int(n_charges), _dev(out_n, torch.int8, P * n, "out_n"),
        _dev(out_U, torch.float64, P, "out_U"),
        _dev(out_flags, torch.uint8, P, "out_flags"), _stream(stream)))


def qa_soft_occupation(m, raster, kT, threshold, closed, n_charges, out_mean,
                       out_logZ=None, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_soft_occupation(
        m, ctypes.byref(r), float(kT), float(threshold), int(closed), int(n_charges),
        _dev(out_mean, torch.float32, P * n, "out_mean"),
        _dev(out_logZ, torch.float32, P, "out_logZ"), _stream(stream)))


def qa_soft_occupation_backward(m, raster, kT, threshold, closed, n_charges,
                                grad_mean, dL_dCdd, dL_dCgd, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_soft_occupation_backward(
        m, ctypes.byref(r), float(kT), float(threshold), int(closed), int(n_charges),
        _dev(grad_mean, torch.float32, P * n, "grad_mean"),
        _dev(dL_dCdd, torch.float64, n * n, "dL_dCdd"),
        _dev(dL_dCgd, torch.float64, n * ng, "dL_dCgd"), _stream(stream)))


def qa_soft_occupation_ctx(m, raster, kT, threshold, closed, n_charges, out_mean, out_logZ,
                           out_ctx, stream=None):
    """out_ctx: CUDA tensor of P * 8 bytes (e.g. int64 [P])."""
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_soft_occupation_ctx(
        m, ctypes.byref(r), float(kT), float(threshold), int(closed), int(n_charges),
        _dev(out_mean, torch.float32, P * n, "out_mean"),
        _dev(out_logZ, torch.float32, P, "out_logZ"),
        _dev(out_ctx, torch.int64, P, "out_ctx"), _stream(stream)))


def qa_soft_occupation_backward_ctx(m, raster, kT, threshold, closed, n_charges, grad_mean,
                                    mean, ctx, dL_dCdd, dL_dCgd, stream=None):
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    _check(load().qa_soft_occupation_backward_ctx(
        m, ctypes.byref(r), float(kT), float(threshold), int(closed), int(n_charges),
        _dev(grad_mean, torch.float32, P * n, "grad_mean"),
        _dev(mean, torch.float32, P * n, "mean"), _dev(ctx, torch.int64, P, "ctx"),
        _dev(dL_dCdd, torch.float64, n * n, "dL_dCdd"),
        _dev(dL_dCgd, torch.float64, n * ng, "dL_dCgd"), _stream(stream)))


def fit_state_len(n, ng):
    """Doubles of qa_fit_step's optimiser state: first and second moments of
    every parameter, then the step count t, beta1^t and beta2^t."""
    return 2 * (n * n + n * ng) + 3


def qa_fit_step(m, raster, kT, threshold, closed, n_charges, target, per_dot, Cdd, Cgd,
                opt_state, lr, beta1=0.9, beta2=0.999, eps=1e-8, loss=None, dL_dCdd=None,
                dL_dCgd=None, out_mean=None, stream=None):
    """One fused fitting step: model update, soft occupation, MSE against
    target, gradient and an Adam step on Cdd, Cgd (in place)."""
    import torch
    n, ng = qa_model_shape(m)
    r = make_raster(raster, ng)
    P = r.W * r.H
    opt = qa_adam(float(lr), float(beta1), float(beta2), float(eps))
    _check(load().qa_fit_step(
        m, ctypes.byref(r), float(kT), float(threshold), int(closed), int(n_charges),
        _dev(target, torch.float32, P * n if per_dot else P, "target"), int(bool(per_dot)),
        _dev(Cdd, torch.float64, n * n, "Cdd"), _dev(Cgd, torch.float64, n * ng, "Cgd"),
        _dev(opt_state, torch.float64, fit_state_len(n, ng), "opt_state"), ctypes.byref(opt),
        _dev(loss, torch.float32, 1, "loss"), _dev(dL_dCdd, torch.float64, n * n, "dL_dCdd"),
        _dev(dL_dCgd, torch.float64, n * ng, "dL_dCgd"),
        _dev(out_mean, torch.float32, P * n, "out_mean"), _stream(stream)))


def qa_model_set_timing(m, enable=True):
    _check(load().qa_model_set_timing(m, int(bool(enable))))


def qa_model_stats(m, stream=None):
    s = qa_stats()
    _check(load().qa_model_stats(m, _stream(stream), ctypes.byref(s)))
    return {f[0]: getattr(s, f[0]) for f in qa_stats._fields_}


# --------------------------------------------------------------------------
# convenience: a model object that allocates its outputs as torch tensors
# --------------------------------------------------------------------------

class Model:
    """Owns a qa_model handle; methods mirror the paper's DotArray calls
    (Sec. V): ground_state_open / ground_state_closed / soft occupation."""

    def __init__(self, Cdd, Cgd, form=QA_FORM_MAXWELL, carrier_sign=1.0):
        self.handle = qa_model_create(Cdd, Cgd, form, carrier_sign)
        self.n_dot, self.n_gate = qa_model_shape(self.handle)

    def close(self):
        if self.handle is not None:
            qa_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outs(self, P, energies, flags):
        import torch
        n = torch.empty((P, self.n_dot), dtype=torch.int8, device="cuda")
        U = torch.empty(P, dtype=torch.float64, device="cuda") if energies else None
        f = torch.empty(P, dtype=torch.uint8, device="cuda") if flags else None
        return n, U, f

    def ground_state_open(self, raster, threshold=1.0, energies=True, flags=True,
                          stream=None):
        P = int(raster["W"]) * int(raster["H"])
        n, U, f = self._outs(P, energies, flags)
        qa_ground_state_open(self.handle, raster, threshold, n, U, f, stream)
        return n.view(int(raster["H"]), int(raster["W"]), self.n_dot), U, f

    def ground_state_closed(self, raster, n_charges, threshold=1.0, energies=True,
                            flags=True, stream=None):
        P = int(raster["W"]) * int(raster["H"])
        n, U, f = self._outs(P, energies, flags)
        qa_ground_state_closed(self.handle, raster, threshold, n_charges, n, U, f,
                               stream)
        return n.view(int(raster["H"]), int(raster["W"]), self.n_dot), U, f

    def ground_state_i16(self, raster, threshold=1.0, closed=False, n_charges=0,
                         energies=True, flags=True, stream=None):
        import torch
        H, W = int(raster["H"]), int(raster["W"])
        _, U, f = self._outs(H * W, energies, flags)
        n = torch.empty((H, W, self.n_dot), dtype=torch.int16, device="cuda")
        qa_ground_state_i16(self.handle, raster, threshold, closed, n_charges, n, U, f, stream)
        return n, U, f

    def ground_state_points(self, V, threshold=1.0, closed=False, n_charges=0,
                            energies=True, flags=True, stream=None):
        P = int(V.shape[0])
        n, U, f = self._outs(P, energies, flags)
        qa_ground_state_points(self.handle, V, threshold, closed, n_charges, n, U, f,
                               stream)
        return n, U, f

    def brute_force_open(self, raster, n_max, energies=True, flags=True, stream=None):
        P = int(raster["W"]) * int(raster["H"])
        n, U, f = self._outs(P, energies, flags)
        qa_brute_force_open(self.handle, raster, n_max, n, U, f, stream)
        return n.view(int(raster["H"]), int(raster["W"]), self.n_dot), U, f

    def brute_force_closed(self, raster, n_charges, energies=True, flags=True, stream=None):
        P = int(raster["W"]) * int(raster["H"])
        n, U, f = self._outs(P, energies, flags)
        qa_brute_force_closed(self.handle, raster, n_charges, n, U, f, stream)
        return n.view(int(raster["H"]), int(raster["W"]), self.n_dot), U, f

    def soft_occupation(self, raster, kT, threshold=1.0, closed=False, n_charges=0,
                        stream=None):
        import torch
        P = int(raster["W"]) * int(raster["H"])
        mean = torch.empty((P, self.n_dot), dtype=torch.float32, device="cuda")
        logZ = torch.empty(P, dtype=torch.float32, device="cuda")
        qa_soft_occupation(self.handle, raster, kT, threshold, closed, n_charges, mean,
                           logZ, stream)
        return mean, logZ

    def stats(self, stream=None):
        return qa_model_stats(self.handle, stream)


# --------------------------------------------------------------------------
# batched calls
# --------------------------------------------------------------------------

def qa_batch_create(items):
    """items: list of dicts {model (handle), raster, threshold, closed,
    n_charges, team, out_n, out_U, out_flags} (torch CUDA outputs).  Returns
    (handle, keep) -- keep holds the host rasters until the call returns."""
    import torch
    arr = (qa_batch_item * len(items))()
    keep = []
    for i, it in enumerate(items):
        n, ng = qa_model_shape(it["model"])
        r = make_raster(it["raster"], ng)
        keep.append(r)
        P = r.W * r.H
        arr[i].model = it["model"].value if isinstance(it["model"], ctypes.c_void_p) else it["model"]
        arr[i].raster = r
        arr[i].threshold = float(it.get("threshold", 1.0))
        arr[i].closed = int(bool(it.get("closed", False)))
        arr[i].n_charges = int(it.get("n_charges", 0))
        arr[i].team = int(it.get("team", 0))
        arr[i].out_n = _dev(it["out_n"], torch.int8, P * n, "out_n")
        arr[i].out_U = _dev(it.get("out_U"), torch.float64, P, "out_U")
        arr[i].out_flags = _dev(it.get("out_flags"), torch.uint8, P, "out_flags")
    h = ctypes.c_void_p()
    _check(load().qa_batch_create(arr, len(items), ctypes.byref(h)))
    return h


def qa_batch_run(b, stream=None):
    _check(load().qa_batch_run(b, _stream(stream)))


def qa_batch_stats(b, stream=None):
    s = qa_stats()
    _check(load().qa_batch_stats(b, _stream(stream), ctypes.byref(s)))
    return {f[0]: getattr(s, f[0]) for f in qa_stats._fields_}


def qa_batch_destroy(b):
    _check(load().qa_batch_destroy(b))


class Batch:
    """A prepared batch of arrays with device outputs allocated per array.

    specs: list of dicts {Cdd, Cgd, raster, threshold, closed, n_charges,
    team}.  outputs[i] = (n [H, W, N] int8, U [H, W] f64, flags [H, W] u8)."""

    def __init__(self, specs):
        import torch
        self.models, self.outputs, items = [], [], []
        for sp in specs:
            m = Model(sp["Cdd"], sp["Cgd"])
            self.models.append(m)
            H, W = int(sp["raster"]["H"]), int(sp["raster"]["W"])
            n = torch.empty((H, W, m.n_dot), dtype=torch.int8, device="cuda")
            U = torch.empty((H, W), dtype=torch.float64, device="cuda")
            f = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            self.outputs.append((n, U, f))
            items.append(dict(model=m.handle, raster=sp["raster"],
                              threshold=sp.get("threshold", sp.get("t", 1.0)),
                              closed=sp.get("closed", False), n_charges=sp.get("n_charges", 0),
                              team=sp.get("team", 0), out_n=n, out_U=U, out_flags=f))
        self.handle = qa_batch_create(items)
        self.pixels = sum(int(sp["raster"]["H"]) * int(sp["raster"]["W"]) for sp in specs)

    def run(self, stream=None):
        qa_batch_run(self.handle, stream)

    def stats(self, stream=None):
        return qa_batch_stats(self.handle, stream)

    def close(self):
        if self.handle is not None:
            qa_batch_destroy(self.handle)
            self.handle = None
        for m in self.models:
            m.close()
        self.models = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
