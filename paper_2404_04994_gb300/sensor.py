"""Charge-sensor stability diagrams (Sec. IV.A): the ground state of the
non-sensing dots, then the fused sensor epilogue kernel (sensor charges,
potentials, Coulomb-peak response and noise), both through the C ABI.

The full system's Maxwell matrices hold the sensing dots last.  The dots'
ground state uses the leading blocks of Cdd and Cgd -- the sensors' charges
are left out, their capacitive loading (in the Maxwell diagonal) and every
gate, including the sensor plungers' cross-talk, are kept."""
from __future__ import annotations

import numpy as np

from . import api


def charge_sensor_diagram(Cdd_full, Cgd_full, raster, n_sensor=1, threshold=1.0,
                          closed=False, n_charges=0, shape=api.QA_SENSOR_LORENTZIAN,
                          width=0.05, white_sigma=0.0, pink_sigma=0.0, jump_amplitude=0.0,
                          jump_prob=0.0, seed=0, carrier_sign=1.0, stream=None):
    """Returns dict of device tensors: signal [H, W, S] (float32), n_dots
    [H, W, N - S], n_sensor [H, W, S] (int8), potential [H, W, S] (FP64)."""
    import torch
    Cdd_full = np.asarray(Cdd_full, dtype=np.float64)
    Cgd_full = np.asarray(Cgd_full, dtype=np.float64)
    nf = Cdd_full.shape[0]
    nd = nf - int(n_sensor)
    dots = api.Model(Cdd_full[:nd, :nd], Cgd_full[:nd, :], carrier_sign=carrier_sign)
    full = api.Model(Cdd_full, Cgd_full, carrier_sign=carrier_sign)
    try:
        if closed:
            n_dots, _, _ = dots.ground_state_closed(raster, n_charges, threshold=threshold,
                                                    stream=stream)
        else:
            n_dots, _, _ = dots.ground_state_open(raster, threshold=threshold, stream=stream)
        H, W = int(raster["H"]), int(raster["W"])
        sig = torch.empty((H, W, n_sensor), dtype=torch.float32, device="cuda")
        ns = torch.empty((H, W, n_sensor), dtype=torch.int8, device="cuda")
        pot = torch.empty((H, W, n_sensor), dtype=torch.float64, device="cuda")
        api.qa_charge_sensor(full.handle, raster, n_dots.contiguous(),
                             {"n_sensor": n_sensor, "shape": shape, "width": width,
                              "white_sigma": white_sigma, "pink_sigma": pink_sigma,
                              "jump_amplitude": jump_amplitude, "jump_prob": jump_prob,
                              "seed": seed}, sig, ns, pot, stream)
        if stream is None:
            torch.cuda.current_stream().synchronize()
        else:
            stream.synchronize()
    finally:
        dots.close()
        full.close()
    return {"signal": sig, "n_dots": n_dots, "n_sensor": ns, "potential": pot}
