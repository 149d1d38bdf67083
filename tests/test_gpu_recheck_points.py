"""GPU parity of the FP64 recheck path and of the point-list entry point.

The FP64 recheck (recheck_entry, in the tail kernel k_lists) redoes a pixel in double precision when an FP32
decision of the method is not certain: the relaxed minimum within the FP32
error bound of an integer (the floor of Sec. III.B) or of a threshold band
edge 1/2 +- t/2 (Eq. "threshold"), or a QP whose FP32 certificate is weak.
These tests make sure that path runs and decides compared pixels:

* the closed 16-dot diagram (N_hat = 16, t = 1), every pixel against the
  oracle; every pixel needs the QP there (Sec. III.A.2), and the pixels at a
  nearly degenerate QP vertex go through the prep's second double-float round;
* rasters a few micro-volts wide centred on a decision boundary that the
  oracle locates by bisection, so that most pixels sit between 1e-9 (the
  parity rule's margin) and the FP32 bound from it: they are compared
  bit-exactly and can only be right if the FP64 recheck settled them;
* random voltage lists through qa_ground_state_points, the shape of the
  paper's own benchmark (16 dots, random gate voltages, Sec. VII), open and
  closed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import inputs
from parity import comparable, compare

pytestmark = pytest.mark.gpu

RECHECKED = 16


def _run(qa, Cdd, Cgd, ras, t, closed, n_charges):
    m = qa.Model(Cdd, Cgd)
    if closed:
        n, U, f = m.ground_state_closed(ras, n_charges, threshold=t)
    else:
        n, U, f = m.ground_state_open(ras, threshold=t)
    st = m.stats()
    out = (n.cpu().numpy().reshape(-1, m.n_dot).astype(np.int64), U.cpu().numpy(),
           f.cpu().numpy(), st)
    m.close()
    return out


def test_grid16_closed_full_diagram_every_pixel(qa):
    cfg = inputs.grid16(t=1.0)
    Cdd, Cgd, ras = cfg["Cdd"], cfg["Cgd"], cfg["raster"]
    n, U, f, st = _run(qa, Cdd, Cgd, ras, 1.0, True, 16)
    rec = oracle.ground_state(Cdd, Cgd, raster=ras, t=1.0, closed=True, n_charges=16)
    assert rec["qp_used"].all()
    rep = compare(n, U, f, rec, Cdd, "grid16 closed 100x100", closed=True)
    assert (n.sum(1) == 16).all()
    assert rep["comparable"] >= 9800
    assert st["unresolved"] == 0
    assert st["qp_pixels"] == 10000
    rechecked = (f & RECHECKED) != 0
    # pixels at a nearly degenerate QP vertex (a multiplier or free x_i within
    # rounding of zero) are settled by the prep's second double-float round
    # with the violated constraints toggled; any pixel still sent to the FP64
    # recheck is among the matches above (the recheck itself is driven by the
    # boundary windows below)
    assert st["boundary"] == 0 or rechecked.any()
    ok = comparable(rec, 16, True)
    print(f"closed grid16: {int(rechecked.sum())} rechecked, "
          f"{int((rechecked & ok).sum())} of them compared")


def _pixel_c(Cgd, ras, xs, ys):
    V = np.asarray(ras["V0"]) + xs * np.asarray(ras["u"]) + ys * np.asarray(ras["w"])
    return Cgd @ V


def _edge_distance(Cdd, Cgd, ras, xs, ys, dot, edge, closed, n_charges):
    """Signed distance of the relaxed minimum's coordinate `dot` from a
    decision point: edge = None -> nearest integer; else frac - edge."""
    x, _, _ = oracle.continuous_min(Cdd, _pixel_c(Cgd, ras, xs, ys), closed, n_charges)
    xi = max(x[dot], 0.0)
    if edge is None:
        return xi - math.floor(xi + 0.5)
    return (xi - math.floor(xi)) - edge


def _locate_boundary(Cdd, Cgd, ras, ys, edge, closed, n_charges):
    """A sweep coordinate xs where some dot's relaxed minimum crosses the
    decision point, found by bisection (FP64 oracle) between two raster
    columns that bracket it; returns (xs, dot)."""
    W = 200
    grid = np.linspace(ras["x0"], ras["x1"], W)
    n = Cdd.shape[0]
    for dot in range(n):
        prev = None
        for a in range(W):
            x, _, _ = oracle.continuous_min(Cdd, _pixel_c(Cgd, ras, grid[a], ys), closed,
                                            n_charges)
            xi = x[dot]
            if xi < 0.75:
                prev = None
                continue
            d = _edge_distance(Cdd, Cgd, ras, grid[a], ys, dot, edge, closed, n_charges)
            if prev is not None and prev[1] * d < 0 and abs(prev[1] - d) < 0.2:
                lo, hi, dlo = prev[0], grid[a], prev[1]
                for _ in range(80):
                    mid = 0.5 * (lo + hi)
                    dm = _edge_distance(Cdd, Cgd, ras, mid, ys, dot, edge, closed,
                                        n_charges)
                    if dm * dlo > 0:
                        lo, dlo = mid, dm
                    else:
                        hi = mid
                return 0.5 * (lo + hi), dot
            prev = (grid[a], d)
    raise AssertionError("no decision boundary on this row")


@pytest.mark.parametrize("closed,t,edge", [
    (False, 1.0, None),       # floor decision: x_i crossing an integer
    (False, 0.0, 0.5),        # rounding at t = 0: the charge map flips here
    (False, 0.25, 0.375),     # threshold band edge 1/2 - t/2
    (True, 1.0, None),
    (True, 0.0, 0.5),         # closed t = 0: one side doubles to t = 1
    (True, 0.25, 0.625),      # band edge 1/2 + t/2
])
def test_recheck_settles_pixels_next_to_a_decision_boundary(qa, closed, t, edge):
    cfg = inputs.chain4(closed=closed)
    Cdd, Cgd, ras0 = cfg["Cdd"], cfg["Cgd"], cfg["raster"]
    N = cfg["n_charges"]
    ys = 2.3
    xs, dot = _locate_boundary(Cdd, Cgd, ras0, ys, edge, closed, N)
    half = 3e-6
    ras = dict(ras0, x0=xs - half, x1=xs + half, y0=ys - 1e-6, y1=ys + 1e-6, W=96, H=5)
    n, U, f, st = _run(qa, Cdd, Cgd, ras, t, closed, N)
    rec = oracle.ground_state(Cdd, Cgd, raster=ras, t=t, closed=closed, n_charges=N)
    label = f"boundary closed={closed} t={t} edge={edge} dot={dot}"
    rep = compare(n, U, f, rec, Cdd, label, closed=closed)
    ok = comparable(rec, 4, closed)
    rechecked = (f & RECHECKED) != 0
    assert st["unresolved"] == 0
    # the window straddles the boundary: the oracle's decision changes in it
    mf = rec["margin_floor"] if edge is None else rec["margin_thresh"]
    assert mf.min() < 1e-7
    assert st["boundary"] > 0 and rechecked.sum() > 0, label
    assert (rechecked & ok).sum() >= 10, (label, rep, int(rechecked.sum()))
    if not closed and t == 0.0:
        # both answers occur in the window, and the GPU gives both
        want = {tuple(r) for r in rec["n"][:, :4]}
        assert len(want) == 2
        assert {tuple(r) for r in n[ok]} == want


@pytest.mark.parametrize("closed", [False, True])
def test_points_grid16_random_voltages(qa, closed):
    # the paper's benchmark shape: 16 dots, random gate-voltage vectors
    import torch
    cfg = inputs.grid16()
    Cdd, Cgd = cfg["Cdd"], cfg["Cgd"]
    V = inputs.random_points(16, 2000, seed=7 + int(closed))
    m = qa.Model(Cdd, Cgd)
    Vd = torch.tensor(V, device="cuda")
    if closed:
        n, U, f = m.ground_state_points(Vd, closed=True, n_charges=16)
    else:
        n, U, f = m.ground_state_points(Vd)
    st = m.stats()
    m.close()
    rec = oracle.ground_state(Cdd, Cgd, V=V, t=1.0, closed=closed, n_charges=16)
    rep = compare(n.cpu().numpy(), U.cpu().numpy(), f.cpu().numpy(), rec, Cdd,
                  f"points closed={closed}", closed=closed)
    assert rep["comparable"] >= 1900
    assert st["unresolved"] == 0
    if closed:
        assert (n.cpu().numpy().reshape(-1, 16).astype(np.int64).sum(1) == 16).all()
        assert st["qp_pixels"] == 2000
