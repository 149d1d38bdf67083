"""GPU charge-sensor epilogue (Sec. IV.A; C ABI -> CUDA) against the FP64
oracle: sensor charges, potentials, response and the three noises, first
with the same dot ground state fed to both sides, then end to end."""
import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import sensor
from test_sensor_oracle import dots_ground_state, raster, sensor_system

pytestmark = pytest.mark.gpu

NOISY = dict(white_sigma=0.05, pink_sigma=0.03, jump_amplitude=0.2, jump_prob=0.01, seed=11)


def _two_sensors():
    Cdd = np.array([[1.0, -0.15, -0.04, -0.01],
                    [-0.15, 1.0, -0.01, -0.06],
                    [-0.04, -0.01, 1.0, -0.02],
                    [-0.01, -0.06, -0.02, 1.0]])
    Cgd = np.array([[0.8, 0.1, 0.02, 0.01],
                    [0.12, 0.7, 0.01, 0.04],
                    [0.03, 0.02, 0.9, 0.0],
                    [0.01, 0.05, 0.0, 0.85]])
    return Cdd, Cgd


def _gpu_epilogue(qa, Cdd, Cgd, ras, nd, S, **kw):
    import torch
    m = qa.Model(Cdd, Cgd)
    H, W = ras["H"], ras["W"]
    ndt = torch.tensor(nd.reshape(H, W, -1), dtype=torch.int8, device="cuda")
    sig = torch.empty((H, W, S), dtype=torch.float32, device="cuda")
    ns = torch.empty((H, W, S), dtype=torch.int8, device="cuda")
    pot = torch.empty((H, W, S), dtype=torch.float64, device="cuda")
    qa.qa_charge_sensor(m.handle, ras, ndt, dict(n_sensor=S, **kw), sig, ns, pot)
    torch.cuda.synchronize()
    m.close()
    return (sig.cpu().numpy().reshape(-1, S), ns.cpu().numpy().reshape(-1, S).astype(np.int64),
            pot.cpu().numpy().reshape(-1, S))


@pytest.mark.parametrize("shape", [0, 1])
def test_epilogue_matches_oracle_on_shared_dot_charges(qa, shape):
    Cdd, Cgd = sensor_system()
    ras = raster(W=300, H=7)
    nd = dots_ground_state(Cdd, Cgd, ras)
    kw = dict(shape=shape, width=0.05, **NOISY)
    sig, ns, pot = _gpu_epilogue(qa, Cdd, Cgd, ras, nd, 1, **kw)
    ref = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, **kw)
    M = np.linalg.inv(Cdd)
    eps = 0.5 * M[2, 2] - np.abs(ref["potential"][:, 0])
    clear = eps > 1e-9
    np.testing.assert_array_equal(ns[clear], ref["n_sensor"][clear])
    np.testing.assert_allclose(pot[clear], ref["potential"][clear], atol=1e-10)
    np.testing.assert_allclose(sig[clear], ref["signal"][clear], atol=2e-6, rtol=1e-6)
    assert clear.mean() > 0.99


def test_two_sensors(qa):
    Cdd, Cgd = _two_sensors()
    ras = {"V0": np.array([0.0, 0.0, 2.5, 2.7]), "u": np.array([1.0, 0.0, 0.0, 0.0]),
           "w": np.array([0.0, 1.0, 0.0, 0.0]), "x0": -0.5, "x1": 4.0, "y0": -0.5, "y1": 4.0,
           "W": 45, "H": 33}
    nd = oracle.ground_state(Cdd[:2, :2], Cgd[:2, :], raster=ras, t=1.0)["n"][:, :2]
    sig, ns, pot = _gpu_epilogue(qa, Cdd, Cgd, ras, nd, 2, width=0.05, **NOISY)
    ref = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=2, width=0.05, **NOISY)
    M = np.linalg.inv(Cdd)
    eps = 0.5 * np.diag(M)[2:] - np.abs(ref["potential"])
    clear = (eps > 1e-9).all(1)
    np.testing.assert_array_equal(ns[clear], ref["n_sensor"][clear])
    np.testing.assert_allclose(sig[clear], ref["signal"][clear], atol=2e-6, rtol=1e-6)


def test_end_to_end_diagram(qa):
    Cdd, Cgd = sensor_system()
    ras = raster(W=64, H=48)
    out = sensor.charge_sensor_diagram(Cdd, Cgd, ras, n_sensor=1, width=0.05, **NOISY)
    nd_gpu = out["n_dots"].cpu().numpy().reshape(-1, 2).astype(np.int64)
    nd_ref = dots_ground_state(Cdd, Cgd, ras)
    same = (nd_gpu == nd_ref).all(1)
    assert same.mean() > 0.99
    ref = oracle.charge_sensor(Cdd, Cgd, ras, nd_ref, n_sensor=1, width=0.05, **NOISY)
    sig = out["signal"].cpu().numpy().reshape(-1)
    np.testing.assert_allclose(sig[same], ref["signal"][same, 0], atol=2e-6, rtol=1e-6)


def test_sensor_errors(qa):
    import torch
    Cdd, Cgd = sensor_system()
    ras = raster(W=8, H=4)
    m = qa.Model(Cdd, Cgd)
    nd = torch.zeros((4, 8, 2), dtype=torch.int8, device="cuda")
    sig = torch.empty((4, 8, 1), dtype=torch.float32, device="cuda")
    for bad, code in ((dict(n_sensor=3), -5), (dict(n_sensor=1, width=0.0), -5),
                      (dict(n_sensor=1, jump_prob=1.0), -5), (dict(n_sensor=1, shape=7), -1)):
        with pytest.raises(qa.QAError) as e:
            if bad["n_sensor"] == 3:
                qa.qa_charge_sensor(m.handle, ras, torch.zeros(0, dtype=torch.int8, device="cuda"),
                                    bad, torch.empty(96, dtype=torch.float32, device="cuda"))
            else:
                qa.qa_charge_sensor(m.handle, ras, nd, bad, sig)
        assert e.value.code == code
    m.close()
