"""Shared helpers for the GPU-vs-oracle parity tests.

Rules (the FP32 search is held to the FP64 oracle):
* a pixel is *comparable* when the oracle's best/runner-up energy gap and its
  floor / threshold decision margins all exceed 1e-9 (and its QP, if any,
  certified); comparable pixels must match bit-exactly;
* energies agree within 1e-5 * max(|U|, max_i M_ii / 2);
* non-comparable pixels are counted and reported, never silently compared.
"""
import numpy as np

import oracle

GAP_EPS = 1e-9
U_RTOL = 1e-5


def comparable(rec):
    return ((rec["U2"] - rec["U"] > GAP_EPS) & (rec["margin_floor"] > GAP_EPS)
            & (rec["margin_thresh"] > GAP_EPS) & (rec["qp_cert"] < 1e-9)
            & (rec["status"] == 0))


def compare(n_gpu, U_gpu, flags, rec, Cdd, label=""):
    """Assert parity; returns a small report dict."""
    n = Cdd.shape[0]
    M = np.linalg.inv(Cdd)
    ok = comparable(rec)
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
