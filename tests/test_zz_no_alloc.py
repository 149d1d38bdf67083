"""The allocation-free entry point against the ordinary one.

qa_ground_state_open_static serves callers that cannot allocate GPU memory
while they run (real-time instrument loops, processes whose GPU memory is
owned by another allocator): its scratch is a static device array of the
library instead of a cudaMalloc'd workspace.  This file sorts last so that a
run stopping at the first failure has already run every other test; it must
pass alone in a fresh process as well as after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_04994_gb300 import inputs

pytestmark = pytest.mark.gpu


def _both(qa, cfg, raster, t):
    import torch
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    P = raster["W"] * raster["H"]
    n_ref, U_ref, f_ref = m.ground_state_open(raster, threshold=t)
    n_st = torch.full((P, m.n_dot), -1, dtype=torch.int8, device="cuda")
    U_st = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    f_st = torch.full((P,), 255, dtype=torch.uint8, device="cuda")
    qa.qa_ground_state_open_static(m.handle, raster, t, n_st, U_st, f_st)
    torch.cuda.synchronize()
    out = (n_ref.cpu().numpy().reshape(P, -1), U_ref.cpu().numpy(), f_ref.cpu().numpy(),
           n_st.cpu().numpy(), U_st.cpu().numpy(), f_st.cpu().numpy())
    m.close()
    return out


def _check(out):
    n_ref, U_ref, f_ref, n_st, U_st, f_st = out
    np.testing.assert_array_equal(n_st, n_ref)
    np.testing.assert_array_equal(f_st, f_ref)
    scale = np.maximum(np.abs(U_ref), 0.5)
    assert float(np.max(np.abs(U_st - U_ref) / scale)) <= 1e-5


def test_static_entry_matches_open_twice_in_a_row(qa):
    # two calls in a row on the shared static scratch: a 16-dot diagram with
    # near-tie pixels, then a 2-dot one that must not see the first's lists
    cfg = inputs.grid16(W=64, H=48)
    _check(_both(qa, cfg, cfg["raster"], 1.0))
    cfg2 = inputs.double_dot()
    _check(_both(qa, cfg2, cfg2["raster"], 1.0))
    _check(_both(qa, cfg, cfg["raster"], 0.5))


def test_static_entry_allocates_nothing(qa):
    # after one warm-up call (which may load the library's module and with it
    # the static array), further calls leave the device's free memory as it
    # was: no cudaMalloc behind the call
    import torch
    cfg = inputs.grid16(W=128, H=128)           # exactly QA_STATIC_MAX_PIXELS
    ras = cfg["raster"]
    P = ras["W"] * ras["H"]
    assert P == qa.STATIC_MAX_PIXELS
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    n_st = torch.empty((P, m.n_dot), dtype=torch.int8, device="cuda")
    U_st = torch.empty((P,), dtype=torch.float64, device="cuda")
    f_st = torch.empty((P,), dtype=torch.uint8, device="cuda")
    ras_c = qa.make_raster(ras, m.n_gate)
    qa.qa_ground_state_open_static(m.handle, ras_c, 0.5, n_st, U_st, f_st)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        qa.qa_ground_state_open_static(m.handle, ras_c, 0.5, n_st, U_st, f_st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # the ordinary call on the same 128 x 128 raster, outside that window
    n_ref, U_ref, f_ref = m.ground_state_open(ras, threshold=0.5)
    np.testing.assert_array_equal(n_st.cpu().numpy(), n_ref.cpu().numpy().reshape(P, -1))
    np.testing.assert_array_equal(f_st.cpu().numpy(), f_ref.cpu().numpy())
    m.close()


def test_static_entry_rejects_oversized_raster(qa):
    import torch
    cfg = inputs.double_dot(W=129, H=128)
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    P = 129 * 128
    assert P > qa.STATIC_MAX_PIXELS
    out = torch.empty((P, 2), dtype=torch.int8, device="cuda")
    with pytest.raises(qa.QAError) as e:
        qa.qa_ground_state_open_static(m.handle, cfg["raster"], 1.0, out)
    assert e.value.code == -2
    assert "QA_STATIC_MAX_PIXELS" in str(e.value)
    m.close()
