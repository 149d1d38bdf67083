"""FP64 CPU oracle for the constant-capacitance-model ground-state method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this package.  It shares no code with the
CUDA library in ``paper_2404_04994_gb300`` and never imports it.

The arithmetic lives in ``qa_oracle.c`` (plain C, double precision, direct
energy evaluation); this module is argument marshalling through ctypes.  What
each routine follows in the paper:

* ``ground_state``  -- Sec. III (continuous minimum, Sec. III.A; default and
  thresholded candidate sets with closed filtering and threshold doubling,
  Sec. III.B, Eq. "threshold"; argmin of Eq. "argmin").
* ``soft``          -- Sec. IV.B, Eq. "softargmin", over the method's candidates.
* ``soft_grad``     -- derivative of a loss through Eq. "softargmin" with the
  candidate set frozen (the paper has no gradient; written from the definition).
* ``brute_force``   -- Table I brute-force row.
* ``continuous_min``, ``energy``, ``inverse_spd`` -- the pieces, for pinning.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
MAX_DOT = 16


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no GPU involved)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB_PATH)
             < os.path.getmtime(os.path.join(_HERE, "qa_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
            "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Raster(ctypes.Structure):
    _fields_ = [("V0", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)),
                ("w", ctypes.POINTER(ctypes.c_double)),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("W", ctypes.c_int), ("H", ctypes.c_int)]


class _Pixel(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * MAX_DOT),
                ("x", ctypes.c_double * MAX_DOT),
                ("U", ctypes.c_double),
                ("U2", ctypes.c_double),
                ("margin_floor", ctypes.c_double),
                ("margin_thresh", ctypes.c_double),
                ("t_used", ctypes.c_double),
                ("qp_cert", ctypes.c_double),
                ("qp_used", ctypes.c_int),
                ("n_cand", ctypes.c_int),
                ("status", ctypes.c_int)]


PIXEL_DTYPE = np.dtype({
    "names": [f[0] for f in _Pixel._fields_],
    "formats": [("<i4", (MAX_DOT,)), ("<f8", (MAX_DOT,)), "<f8", "<f8", "<f8",
                "<f8", "<f8", "<f8", "<i4", "<i4", "<i4"],
    "offsets": [getattr(_Pixel, f[0]).offset for f in _Pixel._fields_],
    "itemsize": ctypes.sizeof(_Pixel),
})

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        R = ctypes.POINTER(_Raster)
        lib.qo_inverse_spd.argtypes = [ctypes.c_int, D, D]
        lib.qo_energy.argtypes = [ctypes.c_int, D, I, D]
        lib.qo_energy.restype = ctypes.c_double
        lib.qo_continuous_min.argtypes = [ctypes.c_int, D, D, D, ctypes.c_int,
                                          ctypes.c_int, D, I, D]
        lib.qo_ground_state_c.argtypes = [ctypes.c_int, D, D, D, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_Pixel)]
        lib.qo_ground_state.argtypes = [ctypes.c_int, ctypes.c_int, D, D,
                                        ctypes.c_double, R, D, ctypes.c_long,
                                        ctypes.c_long, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p]
        lib.qo_soft.argtypes = [ctypes.c_int, ctypes.c_int, D, D, ctypes.c_double,
                                R, D, ctypes.c_long, ctypes.c_long,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, D, D]
        lib.qo_soft_grad.argtypes = [ctypes.c_int, ctypes.c_int, D, D,
                                     ctypes.c_double, R, D, ctypes.c_long,
                                     ctypes.c_long, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     D, ctypes.c_int, D, D, D]
        lib.qo_raster_c.argtypes = [ctypes.c_int, ctypes.c_int, D,
                                    ctypes.c_double, R, ctypes.c_long, D]
        lib.qo_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint)] * 3
        lib.qo_charge_sensor.argtypes = [ctypes.c_int, ctypes.c_int, D, D, ctypes.c_double, R,
                                         I, ctypes.c_void_p, D, I, D]
        lib.qo_brute_force.argtypes = [ctypes.c_int, D, D, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, I, D, I]
        lib.qo_brute_force.restype = ctypes.c_long
        lib.qo_brute_force2.argtypes = [ctypes.c_int, D, D, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]
        lib.qo_brute_force2.restype = ctypes.c_long
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _raster(r):
    """Build the C raster struct; keeps the arrays alive on the struct."""
    if r is None:
        return None
    V0, pV0 = _d(r["V0"])
    u, pu = _d(r["u"])
    w, pw = _d(r["w"])
    s = _Raster(pV0, pu, pw, float(r["x0"]), float(r["x1"]), float(r["y0"]),
                float(r["y1"]), int(r["W"]), int(r["H"]))
    s._keep = (V0, u, w)
    return s


def inverse_spd(A):
    A, pA = _d(A)
    n = A.shape[0]
    out = np.zeros((n, n))
    st = _load().qo_inverse_spd(n, pA, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise ValueError("matrix is not symmetric positive definite")
    return out


def energy(M, nvec, c):
    M, pM = _d(M)
    c, pc = _d(c)
    nv = np.ascontiguousarray(nvec, dtype=np.int32)
    return _load().qo_energy(M.shape[0], pM,
                             nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), pc)


def continuous_min(Cdd, c, closed=False, n_charges=0):
    """(x, qp_used, certificate) of Sec. III.A."""
    Cdd, pC = _d(Cdd)
    M, pM = _d(inverse_spd(Cdd))
    c, pc = _d(c)
    n = Cdd.shape[0]
    x = np.zeros(n)
    qp = ctypes.c_int(0)
    cert = ctypes.c_double(0.0)
    st = _load().qo_continuous_min(n, pC, pM, pc, int(closed), int(n_charges),
                                   x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(qp), ctypes.byref(cert))
    if st != 0:
        raise RuntimeError("QP: no active set satisfied the KKT conditions")
    return x, bool(qp.value), cert.value


def ground_state_c(Cdd, c, t=1.0, closed=False, n_charges=0):
    """The method for one induced-charge vector; returns a PIXEL_DTYPE record."""
    Cdd, pC = _d(Cdd)
    M, pM = _d(inverse_spd(Cdd))
    c, pc = _d(c)
    out = _Pixel()
    st = _load().qo_ground_state_c(Cdd.shape[0], pC, pM, pc, float(t),
                                   int(closed), int(n_charges), ctypes.byref(out))
    if st != 0:
        raise RuntimeError(f"oracle ground state failed ({st})")
    rec = np.frombuffer(bytes(out), dtype=PIXEL_DTYPE)[0]
    return rec


def _npix(raster, V):
    if raster is not None:
        return int(raster["W"]) * int(raster["H"])
    return int(np.asarray(V).shape[0])


def ground_state(Cdd, Cgd, raster=None, V=None, t=1.0, closed=False,
                 n_charges=0, carrier=1.0, pixels=None, n_threads=None):
    """Ground state on a raster (or a [P, n_gate] voltage list).

    ``pixels``: optional (p0, p1) range.  Returns a PIXEL_DTYPE array."""
    Cdd, pC = _d(Cdd)
    Cgd, pG = _d(Cgd)
    n, ng = Cgd.shape
    P = _npix(raster, V)
    p0, p1 = pixels if pixels is not None else (0, P)
    out = np.zeros(p1 - p0, dtype=PIXEL_DTYPE)
    rs = _raster(raster)
    Vd = None
    pV = None
    if V is not None:
        Vd, pV = _d(V)
    st = _load().qo_ground_state(
        n, ng, pC, pG, float(carrier), ctypes.byref(rs) if rs is not None else None,
        pV, p0, p1, float(t), int(closed), int(n_charges),
        int(n_threads or os.cpu_count() or 1), out.ctypes.data)
    if st != 0:
        raise RuntimeError(f"oracle ground state failed ({st})")
    return out


def soft(Cdd, Cgd, raster=None, V=None, kT=0.01, t=1.0, closed=False,
         n_charges=0, carrier=1.0, pixels=None, n_threads=None):
    """(mean [P, N], logZ [P]) of Eq. "softargmin"."""
    Cdd, pC = _d(Cdd)
    Cgd, pG = _d(Cgd)
    n, ng = Cgd.shape
    P = _npix(raster, V)
    p0, p1 = pixels if pixels is not None else (0, P)
    mean = np.zeros((p1 - p0, n))
    logZ = np.zeros(p1 - p0)
    rs = _raster(raster)
    pV = None
    if V is not None:
        Vd, pV = _d(V)
    st = _load().qo_soft(n, ng, pC, pG, float(carrier),
                         ctypes.byref(rs) if rs is not None else None, pV, p0, p1,
                         float(kT), float(t), int(closed), int(n_charges),
                         int(n_threads or os.cpu_count() or 1),
                         mean.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         logZ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise RuntimeError(f"oracle soft occupation failed ({st})")
    return mean, logZ


def soft_grad(Cdd, Cgd, grad_mean, raster=None, V=None, kT=0.01, t=1.0,
              closed=False, n_charges=0, carrier=1.0, pixels=None,
              n_threads=None):
    """(dL/dM, dL/dCdd, dL/dCgd) for L with dL/d<n> = grad_mean [P, N]."""
    Cdd, pC = _d(Cdd)
    Cgd, pG = _d(Cgd)
    n, ng = Cgd.shape
    P = _npix(raster, V)
    p0, p1 = pixels if pixels is not None else (0, P)
    g, pg = _d(np.asarray(grad_mean).reshape(p1 - p0, n))
    dM = np.zeros((n, n))
    dCdd = np.zeros((n, n))
    dCgd = np.zeros((n, ng))
    rs = _raster(raster)
    pV = None
    if V is not None:
        Vd, pV = _d(V)
    D = ctypes.POINTER(ctypes.c_double)
    st = _load().qo_soft_grad(n, ng, pC, pG, float(carrier),
                              ctypes.byref(rs) if rs is not None else None, pV,
                              p0, p1, float(kT), float(t), int(closed),
                              int(n_charges), pg,
                              int(n_threads or os.cpu_count() or 1),
                              dM.ctypes.data_as(D), dCdd.ctypes.data_as(D),
                              dCgd.ctypes.data_as(D))
    if st != 0:
        raise RuntimeError(f"oracle gradient failed ({st})")
    return dM, dCdd, dCgd


def raster_c(Cgd, raster, p, carrier=1.0):
    Cgd, pG = _d(Cgd)
    n, ng = Cgd.shape
    rs = _raster(raster)
    c = np.zeros(n)
    _load().qo_raster_c(n, ng, pG, float(carrier), ctypes.byref(rs), int(p),
                        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return c


def brute_force(M, c, closed=False, n_charges=0, n_max=3):
    """(n*, U*, hit_nmax, states) by exhaustive search (Table I)."""
    M, pM = _d(M)
    c, pc = _d(c)
    n = M.shape[0]
    out = np.zeros(n, dtype=np.int32)
    U = ctypes.c_double(0.0)
    hit = ctypes.c_int(0)
    cnt = _load().qo_brute_force(n, pM, pc, int(closed), int(n_charges),
                                 int(n_max),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 ctypes.byref(U), ctypes.byref(hit))
    return out, U.value, bool(hit.value), int(cnt)


def brute_force_raster(Cdd, Cgd, raster, closed=False, n_charges=0, n_max=3, carrier=1.0):
    """Brute force on every pixel of a raster: dict of n [P, N], U [P],
    U2 [P] (second-lowest energy) and hit [P] (open argmin at n_max)."""
    Cdd = np.ascontiguousarray(Cdd, dtype=np.float64)
    M, _ = _d(inverse_spd(Cdd))
    n = Cdd.shape[0]
    P = int(raster["W"]) * int(raster["H"])
    res = {"n": np.zeros((P, n), dtype=np.int64), "U": np.zeros(P), "U2": np.zeros(P),
           "hit": np.zeros(P, dtype=bool)}
    out = np.zeros(n, dtype=np.int32)
    U = ctypes.c_double(0.0)
    U2 = ctypes.c_double(0.0)
    hit = ctypes.c_int(0)
    for p in range(P):
        c, pc = _d(raster_c(Cgd, raster, p, carrier=carrier))
        _load().qo_brute_force2(n, M.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pc,
                                int(closed), int(n_charges), int(n_max),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                ctypes.byref(U), ctypes.byref(U2), ctypes.byref(hit))
        res["n"][p] = out
        res["U"][p] = U.value
        res["U2"][p] = U2.value
        res["hit"][p] = bool(hit.value)
    return res


def optimal_gate_voltages(Cdd, Cgd, Q, carrier=1.0):
    """Sec. IV.C, Eq. "optimal_gate_voltages" (Appendix H): V* = s (R Cgd)^+ R Q
    with R^T R = Cdd^-1, from numpy's Cholesky factor and pseudo-inverse."""
    M = inverse_spd(Cdd)
    R = np.linalg.cholesky(M).T
    return carrier * (np.linalg.pinv(R @ np.asarray(Cgd, dtype=np.float64)) @ (R @ np.asarray(Q, dtype=np.float64)))


def virtual_gate_matrix(Cdd, Cgd):
    """Sec. IV.C (Appendix I): alpha = (Cdd^-1 Cgd)^+, [n_gate, n_dot]."""
    return np.linalg.pinv(inverse_spd(Cdd) @ np.asarray(Cgd, dtype=np.float64))


class _SensorParams(ctypes.Structure):
    _fields_ = [("n_sensor", ctypes.c_int), ("shape", ctypes.c_int),
                ("width", ctypes.c_double), ("white_sigma", ctypes.c_double),
                ("pink_sigma", ctypes.c_double), ("jump_amplitude", ctypes.c_double),
                ("jump_prob", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


def philox4x32_10(ctr, key):
    """Philox4x32-10 of four 32-bit counter words and two key words."""
    c = (ctypes.c_uint * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint * 4)()
    _load().qo_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def charge_sensor(Cdd_full, Cgd_full, raster, n_dots, n_sensor=1, shape=0, width=0.05,
                  white_sigma=0.0, pink_sigma=0.0, jump_amplitude=0.0, jump_prob=0.0,
                  seed=0, carrier=1.0):
    """Sec. IV.A sensor response given the dots' ground state n_dots
    [P, n_full - n_sensor]: dict of signal, n_sensor, potential, each [P, S]."""
    Cdd_full, pC = _d(Cdd_full)
    Cgd_full, pG = _d(Cgd_full)
    nf, ng = Cgd_full.shape
    P = int(raster["W"]) * int(raster["H"])
    nd = np.ascontiguousarray(np.asarray(n_dots).reshape(P, nf - n_sensor), dtype=np.int32)
    sp = _SensorParams(int(n_sensor), int(shape), float(width), float(white_sigma),
                       float(pink_sigma), float(jump_amplitude), float(jump_prob), int(seed))
    sig = np.zeros((P, n_sensor))
    ns = np.zeros((P, n_sensor), dtype=np.int32)
    pot = np.zeros((P, n_sensor))
    rs = _raster(raster)
    st = _load().qo_charge_sensor(nf, ng, pC, pG, float(carrier), ctypes.byref(rs),
                                  nd.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  ctypes.byref(sp),
                                  sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  pot.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise ValueError("oracle charge sensor: bad input")
    return {"signal": sig, "n_sensor": ns, "potential": pot}
