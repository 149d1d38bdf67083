"""The parity helper's comparability rules, on hand-made oracle records (no
GPU): which pixels the GPU tests compare bit-exactly."""
import numpy as np

import oracle
from parity import GAP_EPS, comparable, vertex


def _records(xs, margin_floor, gap=1.0):
    rec = np.zeros(len(xs), dtype=oracle.PIXEL_DTYPE)
    for i, x in enumerate(xs):
        rec["x"][i, :len(x)] = x
    rec["U"] = 0.0
    rec["U2"] = gap
    rec["margin_floor"] = margin_floor
    rec["margin_thresh"] = np.inf
    return rec


def test_vertex_needs_one_integral_nonzero_coordinate():
    rec = _records([[0.0, 3.0, 0.0],            # vertex 3 e_1
                    [0.0, 3.0 + 1e-12, 0.0],    # within the tolerance
                    [0.5, 2.5, 0.0],            # two free dots
                    [0.0, 2.5, 0.0],            # one free dot, not integral
                    [0.0, 0.0, 0.0]],           # no free dot
                   margin_floor=0.0)
    np.testing.assert_array_equal(vertex(rec, 3), [True, True, False, False, False])


def test_closed_vertices_are_comparable_open_ones_are_not():
    rec = _records([[0.0, 3.0, 0.0], [0.2, 0.3, 0.7]], margin_floor=0.0)
    np.testing.assert_array_equal(comparable(rec, 3, closed=False), [False, False])
    np.testing.assert_array_equal(comparable(rec, 3, closed=True), [True, False])


def test_near_ties_and_uncertified_pixels_stay_out():
    rec = _records([[0.0, 3.0, 0.0], [0.0, 3.0, 0.0], [0.4, 1.3, 0.2]],
                   margin_floor=np.array([0.0, 0.0, 0.1]))
    rec["U2"][0] = 0.5 * GAP_EPS        # a true near tie
    rec["qp_cert"][1] = 1e-6            # QP not certified
    np.testing.assert_array_equal(comparable(rec, 3, closed=True), [False, False, True])
