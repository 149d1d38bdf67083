"""Pins of the charge-sensor oracle (Sec. IV.A) against what fixes it
independently: published Philox4x32-10 known answers, exhaustive search of the
sensor charge, the energy identity behind Eq. "potential", the Coulomb-peak
positions of a sensor-plunger sweep, and the statistics of the three noises."""
import numpy as np

import oracle


def sensor_system():
    """2 dots + 1 sensor (last), 3 gates (two plungers + the sensor plunger)."""
    Cdd = np.array([[1.0, -0.15, -0.04],
                    [-0.15, 1.0, -0.08],
                    [-0.04, -0.08, 1.0]])
    Cgd = np.array([[0.8, 0.1, 0.02],
                    [0.12, 0.7, 0.05],
                    [0.03, 0.06, 0.9]])
    return Cdd, Cgd


def raster(W=40, H=30, V2=3.0, lo=-0.5, hi=4.0, sweep_sensor=False):
    if sweep_sensor:
        return {"V0": np.array([1.2, 1.7, 0.0]), "u": np.array([0.0, 0.0, 1.0]),
                "w": np.array([0.0, 0.0, 0.0]), "x0": 0.0, "x1": 6.0, "y0": 0.0, "y1": 0.0,
                "W": W, "H": H}
    return {"V0": np.array([0.0, 0.0, V2]), "u": np.array([1.0, 0.0, 0.0]),
            "w": np.array([0.0, 1.0, 0.0]), "x0": lo, "x1": hi, "y0": lo, "y1": hi,
            "W": W, "H": H}


def dots_ground_state(Cdd, Cgd, ras):
    rec = oracle.ground_state(Cdd[:2, :2], Cgd[:2, :], raster=ras, t=1.0)
    return rec["n"][:, :2]


def test_philox_known_answers():
    # known-answer vectors published with Philox4x32-10 (Salmon et al., SC'11)
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert oracle.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2) == \
        [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    assert oracle.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344],
                                [0xa4093822, 0x299f31d0]) == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_sensor_charge_is_the_exhaustive_minimum_and_potential_identity():
    Cdd, Cgd = sensor_system()
    ras = raster()
    nd = dots_ground_state(Cdd, Cgd, ras)
    out = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1)
    M = np.linalg.inv(Cdd)
    for p in range(0, ras["W"] * ras["H"], 7):
        c = oracle.raster_c(Cgd, ras, p)
        Us = [oracle.energy(M, np.array([nd[p, 0], nd[p, 1], k]), c) for k in range(0, 30)]
        assert out["n_sensor"][p, 0] == int(np.argmin(Us))
        n = np.array([nd[p, 0], nd[p, 1], out["n_sensor"][p, 0]])
        # U(n + e_s) - U(n) = V_s + M_ss / 2
        up = oracle.energy(M, n + np.array([0, 0, 1]), c) - oracle.energy(M, n, c)
        assert abs(out["potential"][p, 0] - (up - 0.5 * M[2, 2])) < 1e-12


def test_peaks_sit_on_the_sensor_transitions():
    # sweeping only the sensor plunger: the noise-free response peaks where
    # the sensor's charge steps, and dips half way between
    Cdd, Cgd = sensor_system()
    ras = raster(W=600, H=1, sweep_sensor=True)
    nd = dots_ground_state(Cdd, Cgd, ras)
    out = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, width=0.01)
    sig = out["signal"][:, 0]
    steps = np.where(np.diff(out["n_sensor"][:, 0]) != 0)[0]
    assert len(steps) >= 3
    bounds = [0] + [(a + b) // 2 for a, b in zip(steps[:-1], steps[1:])] + [len(sig)]
    for k, s in enumerate(steps):
        lo, hi = bounds[k], bounds[k + 1]
        peak = lo + int(np.argmax(sig[lo:hi]))
        assert abs(peak - s) <= 1 and sig[peak] > 0.5   # one pixel is ~ one width here
    for a, b in zip(steps[:-1], steps[1:]):
        assert sig[(a + b) // 2] < 0.01
    gauss = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, width=0.01, shape=1)["signal"][:, 0]
    # both shapes are 1 at the peak and fall monotonically with |eps|
    assert abs(gauss.max() - sig.max()) < 0.05


def test_noise_statistics_and_determinism():
    Cdd, Cgd = sensor_system()
    ras = raster(W=256, H=64)
    nd = dots_ground_state(Cdd, Cgd, ras)
    base = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1)["signal"][:, 0]
    white = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, white_sigma=0.1, seed=5)["signal"][:, 0] - base
    assert abs(white.mean()) < 4 * 0.1 / np.sqrt(white.size)
    assert abs(white.std() - 0.1) < 0.005
    w2 = white.reshape(64, 256)
    assert abs(np.corrcoef(w2[:, :-1].ravel(), w2[:, 1:].ravel())[0, 1]) < 0.05
    pink = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, pink_sigma=0.1, seed=5)["signal"][:, 0] - base
    p2 = pink.reshape(64, 256)
    assert np.corrcoef(p2[:, :-1].ravel(), p2[:, 1:].ravel())[0, 1] > 0.5
    assert 0.05 < pink.std() < 0.15
    tel = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, jump_amplitude=0.3, jump_prob=0.02,
                               seed=5)["signal"][:, 0] - base
    t2 = np.round(tel.reshape(64, 256) / 0.3)
    assert set(np.unique(t2)) <= {0.0, 1.0}
    rate = (np.diff(t2, axis=1) != 0).mean()
    assert abs(rate - 0.02) < 0.006
    again = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, white_sigma=0.1, seed=5)["signal"][:, 0] - base
    np.testing.assert_array_equal(again, white)
    other = oracle.charge_sensor(Cdd, Cgd, ras, nd, n_sensor=1, white_sigma=0.1, seed=6)["signal"][:, 0] - base
    assert not np.allclose(other, white)
