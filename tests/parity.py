"""Shared helpers for the GPU-vs-oracle parity tests.

Rules (the FP32 search is held to the FP64 oracle):
* a pixel is *comparable* when the oracle's best/runner-up energy gap and its
  floor / threshold decision margins all exceed 1e-9 (and its QP, if any,
  certified); comparable pixels must match bit-exactly;
* closed arrays: a pixel whose relaxed minimum is a vertex N_hat e_j (every
  other dot active) is comparable whatever its floor margin: that integer
  point is the exact minimum and lies in every candidate set a rounding of
  x_j can give;
* energies agree within 1e-5 * max(|U|, max_i M_ii / 2);
* non-comparable pixels are counted and reported, never silently compared.
"""
import numpy as np

import oracle

GAP_EPS = 1e-9
U_RTOL = 1e-5


def vertex(rec, n):
    """Closed-array pixels whose relaxed minimum has one nonzero, integral
    coordinate (all other dots active at exactly 0)."""
    x = rec["x"][:, :n]
    pos = x > 0.0
    one = (pos.sum(1) == 1) & ((x == 0.0) | pos).all(1)
    xj = np.where(pos, x, 0.0).sum(1)
    return one & (np.abs(xj - np.rint(xj)) < GAP_EPS)


def comparable(rec, n=None, closed=False):
    floor_ok = rec["margin_floor"] > GAP_EPS
    if closed:
        floor_ok = floor_ok | vertex(rec, n)
    return ((rec["U2"] - rec["U"] > GAP_EPS) & floor_ok
            & (rec["margin_thresh"] > GAP_EPS) & (rec["qp_cert"] < 1e-9)
            & (rec["status"] == 0))


def compare(n_gpu, U_gpu, flags, rec, Cdd, label="", closed=False):
    """Assert parity; returns a small report dict."""
    n = Cdd.shape[0]
    M = np.linalg.inv(Cdd)
    ok = comparable(rec, n, closed)
    want = rec["n"][:, :n]
    got = np.asarray(n_gpu).reshape(-1, n).astype(np.int64)
    bad = ok & (got != want).any(1)
    report = {"pixels": int(len(rec)), "comparable": int(ok.sum()),
              "mismatch": int(bad.sum()),
              "flagged": int(((flags & 0x0B) != 0).sum()) if flags is not None else -1,
              "rechecked": int(((flags & 16) != 0).sum()) if flags is not None else -1}
    if bad.any():
        idx = np.where(bad)[0][:5]
        detail = [(int(i), got[i].tolist(), want[i].tolist(), float(rec["U2"][i] - rec["U"][i]),
                   int(flags[i]) if flags is not None else -1) for i in idx]
        raise AssertionError(f"{label}: {bad.sum()} comparable pixels differ: {detail}")
    if flags is not None:
        assert not (flags & 64).any(), f"{label}: unresolved pixels"
    if U_gpu is not None:
        same = (got == want).all(1)
        scale = np.maximum(np.abs(rec["U"]), 0.5 * np.max(np.diag(M)))
        err = np.abs(np.asarray(U_gpu) - rec["U"]) / scale
        worst = float(err[same].max()) if same.any() else 0.0
        assert worst <= U_RTOL, f"{label}: energy error {worst:.3e}"
        report["energy_rel_err"] = worst
    return report
