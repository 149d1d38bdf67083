"""GPU parity of the ground-state path (C ABI -> CUDA kernels) against the
FP64 oracle, on the seeded workloads and their edge cases."""
import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import inputs
from parity import compare, vertex

pytestmark = pytest.mark.gpu


def _gpu(qa, cfg, t=None, closed=None, n_charges=None, raster=None, carrier=1.0):
    t = cfg["t"] if t is None else t
    closed = cfg["closed"] if closed is None else closed
    n_charges = cfg["n_charges"] if n_charges is None else n_charges
    ras = cfg["raster"] if raster is None else raster
    m = qa.Model(cfg["Cdd"], cfg["Cgd"], carrier_sign=carrier)
    if closed:
        n, U, f = m.ground_state_closed(ras, n_charges, threshold=t)
    else:
        n, U, f = m.ground_state_open(ras, threshold=t)
    st = m.stats()
    out = (n.cpu().numpy().reshape(-1, m.n_dot), U.cpu().numpy(), f.cpu().numpy(), st)
    m.close()
    return out


def _oracle(cfg, t=None, closed=None, n_charges=None, raster=None, carrier=1.0,
            pixels=None):
    t = cfg["t"] if t is None else t
    closed = cfg["closed"] if closed is None else closed
    n_charges = cfg["n_charges"] if n_charges is None else n_charges
    ras = cfg["raster"] if raster is None else raster
    return oracle.ground_state(cfg["Cdd"], cfg["Cgd"], raster=ras, t=t, closed=closed,
                               n_charges=n_charges, carrier=carrier, pixels=pixels)


def test_double_dot_full_raster(qa):
    cfg = inputs.double_dot()
    n, U, f, st = _gpu(qa, cfg)
    rep = compare(n, U, f, _oracle(cfg), cfg["Cdd"], "double dot")
    assert rep["comparable"] > 9900
    assert st["qp_pixels"] > 0


@pytest.mark.parametrize("closed", [False, True])
def test_chain4_full_raster(qa, closed):
    cfg = inputs.chain4(closed=closed)
    n, U, f, st = _gpu(qa, cfg)
    rec = _oracle(cfg)
    compare(n, U, f, rec, cfg["Cdd"], f"chain4 closed={closed}", closed=closed)
    if closed:
        assert (n.sum(1) == 4).all()


@pytest.mark.parametrize("t", [1.0, 0.5])
def test_grid16_small_raster(qa, t):
    # the 16-dot workload on a 24 x 21 raster over the same voltage window:
    # several search teams per block, a ragged last block
    cfg = inputs.grid16(W=24, H=21, t=t)
    n, U, f, st = _gpu(qa, cfg)
    rep = compare(n, U, f, _oracle(cfg), cfg["Cdd"], f"grid16 t={t}")
    assert rep["comparable"] >= 0.95 * 24 * 21


@pytest.mark.parametrize("t", [1.0, 0.5])
def test_grid16_full_size_sampled_rows(qa, t):
    # full 100 x 100 launch, compared on three sampled rows the oracle
    # computes one by one
    cfg = inputs.grid16(t=t)
    n, U, f, st = _gpu(qa, cfg)
    for row in (3, 50, 97):
        p0, p1 = row * 100, row * 100 + 100
        rec = _oracle(cfg, pixels=(p0, p1))
        compare(n[p0:p1], U[p0:p1], f[p0:p1], rec, cfg["Cdd"], f"grid16 row {row}")
    if t == 1.0:
        assert st["candidates"] == 100 * 100 * 2 ** 16
    assert st["unresolved"] == 0


def test_grid16_full_diagram_every_pixel(qa):
    # the benchmark's diagram, all 10^4 pixels against the oracle: checks the
    # FP32 near-tie bound of the search on every comparable pixel
    cfg = inputs.grid16(t=1.0)
    n, U, f, st = _gpu(qa, cfg)
    rep = compare(n, U, f, _oracle(cfg), cfg["Cdd"], "grid16 100x100 t=1")
    assert rep["comparable"] >= 9900
    assert st["unresolved"] == 0


@pytest.mark.parametrize("t", [1.0, 0.6, 0.25, 0.0])
def test_closed_threshold_doubling(qa, t):
    cfg = inputs.chain4(W=33, H=29, closed=True)
    n, U, f, st = _gpu(qa, cfg, t=t)
    compare(n, U, f, _oracle(cfg, t=t), cfg["Cdd"], f"closed t={t}", closed=True)
    assert (n.sum(1) == 4).all()
    if t == 0.0:
        assert st["doubled"] > 0


def test_uncoupled_dots_round_and_clip(qa):
    # Appendix E, Theorem 1 on the GPU: diagonal Cdd and Cgd
    rng = np.random.Generator(np.random.PCG64(99))
    nd = 6
    Cdd = np.diag(rng.uniform(0.6, 1.5, nd))
    Cgd = np.diag(rng.uniform(0.5, 1.0, nd))
    ras = inputs.raster(nd, 1, 4, rng.uniform(-1, 4, nd), lo=-2.0, hi=7.0, W=37, H=19)
    m = qa.Model(Cdd, Cgd)
    n, U, f = m.ground_state_open(ras, threshold=0.3)
    n = n.cpu().numpy().reshape(-1, nd)
    xs = np.linspace(-2, 7, 37)
    ys = np.linspace(-2, 7, 19)
    V = np.array([ras["V0"] + xs[p % 37] * ras["u"] + ys[p // 37] * ras["w"]
                  for p in range(37 * 19)])
    c = V @ Cgd.T
    want = np.maximum(0, np.floor(c + 0.5))
    away = (np.abs(c - np.floor(c) - 0.5) > 1e-6).all(1)
    np.testing.assert_array_equal(n[away], want[away])
    m.close()


@pytest.mark.parametrize("nd", [1, 3, 7, 9, 12])
def test_other_dot_counts(qa, nd):
    rng = inputs.rng_for(40 + nd)
    Cdd, Cgd = inputs.random_model(rng, nd, nn=(0.05, 0.25), off=(0.0, 0.1))
    gx, gy = inputs.swept_gates(nd)
    V = inputs.offsets(rng, nd, (gx, gy))
    ras = inputs.raster(nd, gx, gy, V, W=17, H=13)
    cfg = {"Cdd": Cdd, "Cgd": Cgd, "raster": ras, "t": 1.0, "closed": False,
           "n_charges": 0}
    for closed in (False, True):
        n, U, f, _ = _gpu(qa, cfg, closed=closed, n_charges=nd)
        compare(n, U, f, _oracle(cfg, closed=closed, n_charges=nd), Cdd,
                f"N={nd} closed={closed}", closed=closed)


@pytest.mark.parametrize("nd,t", [(2, 1.0), (3, 1.0), (3, 0.5), (4, 1.0)])
def test_closed_vertex_minima_settle_without_fp64(qa, nd, t):
    # closed, every dot but one empty: the relaxed minimum is N_hat e_j, an
    # integer point, so it is the ground state and needs no FP64 recheck
    rng = inputs.rng_for(70 + nd)
    Cdd, Cgd = inputs.random_model(rng, nd, nn=(0.05, 0.25), off=(0.0, 0.1))
    gx, gy = inputs.swept_gates(nd)
    V = inputs.offsets(rng, nd, (gx, gy))
    cfg = {"Cdd": Cdd, "Cgd": Cgd, "raster": inputs.raster(nd, gx, gy, V, lo=-6.0, hi=12.0, W=41, H=37),
           "t": t, "closed": True, "n_charges": nd}
    n, U, f, st = _gpu(qa, cfg)
    rec = _oracle(cfg)
    vx = vertex(rec, nd)
    assert vx.sum() >= 50
    compare(n, U, f, rec, Cdd, f"closed N={nd} vertices", closed=True)
    j = np.argmax(rec["x"][:, :nd], axis=1)
    np.testing.assert_array_equal(n[vx], nd * np.eye(nd, dtype=np.int64)[j[vx]])
    assert ((f[vx] & 2) != 0).mean() < 0.02


def test_single_pixel_and_negative_carrier(qa):
    cfg = inputs.double_dot()
    ras = dict(cfg["raster"], W=1, H=1, x0=-2.5, x1=-2.5, y0=-3.0, y1=-3.0)
    n, U, f, _ = _gpu(qa, cfg, raster=ras, carrier=-1.0)
    compare(n, U, f, _oracle(cfg, raster=ras, carrier=-1.0), cfg["Cdd"], "1 pixel")


def test_closed_zero_charges(qa):
    cfg = inputs.chain4(W=9, H=7, closed=True)
    n, U, f, _ = _gpu(qa, cfg, n_charges=0)
    assert (n == 0).all()
    compare(n, U, f, _oracle(cfg, n_charges=0), cfg["Cdd"], "N_hat = 0", closed=True)


def test_points_match_raster(qa):
    import torch
    cfg = inputs.chain4(W=40, H=30)
    ras = cfg["raster"]
    xs = np.linspace(ras["x0"], ras["x1"], 40)
    ys = np.linspace(ras["y0"], ras["y1"], 30)
    V = np.array([ras["V0"] + xs[p % 40] * ras["u"] + ys[p // 40] * ras["w"]
                  for p in range(1200)])
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    n1, U1, f1 = m.ground_state_points(torch.tensor(V, device="cuda"))
    rec = oracle.ground_state(cfg["Cdd"], cfg["Cgd"], V=V)
    compare(n1.cpu().numpy(), U1.cpu().numpy(), f1.cpu().numpy(), rec, cfg["Cdd"],
            "points")
    n0, _, _ = m.ground_state_points(torch.zeros((0, 4), dtype=torch.float64,
                                                 device="cuda"))
    assert n0.shape == (0, 4)
    m.close()


def test_errors_are_reported(qa):
    import torch
    cfg = inputs.double_dot()
    with pytest.raises(qa.QAError) as e:
        qa.Model(np.array([[1.0, 2.0], [2.0, 1.0]]), cfg["Cgd"])
    assert e.value.code == -4
    with pytest.raises(qa.QAError) as e:
        qa.Model(np.array([[1.0, -0.2], [-0.1, 1.0]]), cfg["Cgd"])
    assert e.value.code == -3
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    with pytest.raises(qa.QAError) as e:
        m.ground_state_open(cfg["raster"], threshold=1.5)
    assert e.value.code == -5
    bad = dict(cfg["raster"], x0=float("nan"))
    with pytest.raises(qa.QAError):
        m.ground_state_open(bad)
    with pytest.raises(qa.QAError) as e:
        m.ground_state_closed(cfg["raster"], -1)
    assert e.value.code == -5
    m.close()


def test_virtual_gate_raster(qa):
    # a sweep along the virtual gates of dots 1 and 2 (Sec. IV.C): u, w are
    # columns of (Cdd^-1 Cgd)^+; the map matches the oracle on that raster
    cfg = inputs.chain4()
    ras = qa.virtual_raster(cfg["Cdd"], cfg["Cgd"], np.full(4, 2.0), 1, 2, lo=-3.0, hi=3.0,
                            W=37, H=29)
    n, U, f, st = _gpu(qa, cfg, raster=ras, closed=False)
    rep = compare(n, U, f, _oracle(cfg, raster=ras, closed=False), cfg["Cdd"], "virtual raster")
    assert rep["comparable"] > 0.95 * 37 * 29


def test_async_model_update_in_stream_order(qa):
    # two models alternated through qa_model_update_async on one stream: each
    # call sees the model enqueued before it
    import torch
    c1, c2 = inputs.chain4(W=40, H=30), inputs.grid16(W=12, H=9)
    r = np.random.Generator(np.random.PCG64(3))
    Cdd2 = inputs.chain_cdd(r, 4, nn=(0.05, 0.2))
    Cgd2 = inputs.dense_cgd(r, 4)
    m = qa.Model(c1["Cdd"], c1["Cgd"])
    ref1 = qa.Model(c1["Cdd"], c1["Cgd"]).ground_state_open(c1["raster"])[0].cpu()
    ref2 = qa.Model(Cdd2, Cgd2).ground_state_open(c1["raster"])[0].cpu()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = []
        for k in range(6):
            Cdd, Cgd = (Cdd2, Cgd2) if k % 2 else (c1["Cdd"], c1["Cgd"])
            qa.qa_model_update_async(m.handle, Cdd, Cgd, s)
            outs.append(m.ground_state_open(c1["raster"], stream=s)[0])
    s.synchronize()
    for k, o in enumerate(outs):
        assert bool((o.cpu() == (ref2 if k % 2 else ref1)).all())
    with pytest.raises(qa.QAError):
        qa.qa_model_update_async(m.handle, -c1["Cdd"], c1["Cgd"], s)
    m.close()


@pytest.mark.parametrize("closed", [False, True])
def test_int16_maps_for_large_charges(qa, closed):
    # gate voltages high enough that the charges pass int8: the int16 map is
    # exact, the int8 map saturates and flags the overflow
    cfg = inputs.double_dot(W=37, H=23)
    ras = dict(cfg["raster"], x0=150.0, x1=190.0, y0=140.0, y1=170.0)
    nh = 320
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    n16, U16, f16 = m.ground_state_i16(ras, closed=closed, n_charges=nh)
    n8, U8, f8 = (m.ground_state_closed(ras, nh) if closed else m.ground_state_open(ras))
    m.close()
    n16 = n16.cpu().numpy().reshape(-1, 2).astype(np.int64)
    rec = oracle.ground_state(cfg["Cdd"], cfg["Cgd"], raster=ras, t=1.0, closed=closed,
                              n_charges=nh)
    assert n16.max() > 127
    compare(n16, U16.cpu().numpy(), f16.cpu().numpy(), rec, cfg["Cdd"], "int16 map")
    assert ((f8.cpu().numpy() & 128) != 0).any()
    assert not ((f16.cpu().numpy() & 128) != 0).any()
    np.testing.assert_array_equal(U8.cpu().numpy(), U16.cpu().numpy())
