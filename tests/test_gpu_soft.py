"""GPU parity of the finite-temperature occupation (Sec. IV.B) and its
gradient against the FP64 oracle and central finite differences."""
import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import inputs

pytestmark = pytest.mark.gpu

MEAN_TOL = 1e-5        # absolute, on <n>
GRAD_RTOL = 1e-4       # relative to the largest gradient entry


def _soft_gpu(qa, cfg, kT, t=1.0, closed=False, n_charges=0, raster=None):
    ras = cfg["raster"] if raster is None else raster
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    mean, logZ = m.soft_occupation(ras, kT, threshold=t, closed=closed, n_charges=n_charges)
    out = mean.cpu().numpy().astype(np.float64), logZ.cpu().numpy().astype(np.float64)
    m.close()
    return out


@pytest.mark.parametrize("kT", [0.01, 0.05])
def test_soft_grid8_full_raster(qa, kT):
    cfg = inputs.grid8(kT=kT)
    mean, logZ = _soft_gpu(qa, cfg, kT)
    om, ol = oracle.soft(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], kT=kT)
    err = np.abs(mean - om).max()
    assert err <= MEAN_TOL, err
    rel = np.abs(logZ - ol) / np.maximum(1.0, np.abs(ol))
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("closed", [False, True])
@pytest.mark.parametrize("t", [1.0, 0.4])
def test_soft_chain4(qa, closed, t):
    cfg = inputs.chain4(W=60, H=50, closed=closed)
    kT = 0.02
    mean, logZ = _soft_gpu(qa, cfg, kT, t=t, closed=closed, n_charges=4)
    om, ol = oracle.soft(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], kT=kT, t=t,
                         closed=closed, n_charges=4)
    assert np.abs(mean - om).max() <= MEAN_TOL
    if closed:
        np.testing.assert_allclose(mean.sum(1), 4.0, atol=1e-5)


def _chain6():
    """6-dot chain: 6 ambiguous slots at t = 1, so only two of a team's
    eight lanes hold outer patterns in the dense form."""
    r = np.random.Generator(np.random.PCG64(606))
    Cdd = inputs.chain_cdd(r, 6)
    Cgd = inputs.dense_cgd(r, 6, off=(0.0, 0.15), decay=0.6)
    ras = inputs.raster(6, 2, 3, inputs.offsets(r, 6, (2, 3), 0.5, 2.5), W=23, H=19)
    return {"Cdd": Cdd, "Cgd": Cgd, "raster": ras}


@pytest.mark.parametrize("closed", [False, True])
def test_soft_and_gradient_six_dots(qa, closed):
    cfg = _chain6()
    kT, nc = 0.02, 6
    mean, logZ = _soft_gpu(qa, cfg, kT, closed=closed, n_charges=nc)
    om, ol = oracle.soft(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], kT=kT, closed=closed,
                         n_charges=nc)
    assert np.abs(mean - om).max() <= MEAN_TOL
    rel = np.abs(logZ - ol) / np.maximum(1.0, np.abs(ol))
    assert rel.max() <= 1e-5, rel.max()
    gbar = np.random.Generator(np.random.PCG64(7)).normal(size=(23 * 19, 6))
    dC, dG = _grad_gpu(qa, cfg, kT, gbar, closed=closed, n_charges=nc)
    _, oC, oG = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, raster=cfg["raster"], kT=kT,
                                 closed=closed, n_charges=nc)
    sc = max(np.abs(oC).max(), np.abs(oG).max())
    assert np.abs(dC - oC).max() <= GRAD_RTOL * sc
    assert np.abs(dG - oG).max() <= GRAD_RTOL * sc


def test_soft_sixteen_dots_small(qa):
    cfg = inputs.grid16(W=6, H=5)
    kT = 0.05
    mean, _ = _soft_gpu(qa, cfg, kT)
    om, _ = oracle.soft(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], kT=kT)
    assert np.abs(mean - om).max() <= MEAN_TOL


def _grad_gpu(qa, cfg, kT, gbar, raster=None, t=1.0, closed=False, n_charges=0):
    import torch
    ras = cfg["raster"] if raster is None else raster
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    n, ng = m.n_dot, m.n_gate
    g = torch.tensor(gbar, dtype=torch.float32, device="cuda").contiguous()
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    dG = torch.empty((n, ng), dtype=torch.float64, device="cuda")
    qa.qa_soft_occupation_backward(m.handle, ras, kT, t, closed, n_charges, g, dC, dG)
    out = dC.cpu().numpy(), dG.cpu().numpy()
    m.close()
    return out


@pytest.mark.parametrize("kT", [0.01, 0.05])
def test_gradient_matches_oracle(qa, kT):
    cfg = inputs.grid8(W=48, H=40, kT=kT)
    P = 48 * 40
    gbar = np.random.Generator(np.random.PCG64(5)).normal(size=(P, 8))
    dC, dG = _grad_gpu(qa, cfg, kT, gbar)
    _, oC, oG = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, raster=cfg["raster"], kT=kT)
    sc = max(np.abs(oC).max(), np.abs(oG).max())
    assert np.abs(dC - oC).max() <= GRAD_RTOL * sc
    assert np.abs(dG - oG).max() <= GRAD_RTOL * sc
    np.testing.assert_allclose(dC, dC.T, atol=1e-12 * sc)


def test_gradient_closed_and_threshold(qa):
    cfg = inputs.chain4(W=30, H=20, closed=True)
    kT = 0.03
    gbar = np.random.Generator(np.random.PCG64(6)).normal(size=(600, 4))
    dC, dG = _grad_gpu(qa, cfg, kT, gbar, t=0.5, closed=True, n_charges=4)
    _, oC, oG = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, raster=cfg["raster"],
                                 kT=kT, t=0.5, closed=True, n_charges=4)
    sc = max(np.abs(oC).max(), np.abs(oG).max())
    assert np.abs(dC - oC).max() <= GRAD_RTOL * sc
    assert np.abs(dG - oG).max() <= GRAD_RTOL * sc


def test_gradient_matches_central_differences(qa):
    # FD of the FP64 oracle forward (h = 1e-4) on the loss L = sum g . <n>,
    # restricted to pixels whose continuous minimum stays well inside its
    # cell, so the frozen candidate set is the set at every perturbed point.
    cfg = inputs.grid8(W=20, H=16, kT=0.05)
    kT, h = 0.05, 1e-4
    ras = cfg["raster"]
    P = 20 * 16
    xs = np.linspace(ras["x0"], ras["x1"], 20)
    ys = np.linspace(ras["y0"], ras["y1"], 16)
    V = np.array([ras["V0"] + xs[p % 20] * ras["u"] + ys[p // 20] * ras["w"] for p in range(P)])
    keep = []
    for p in range(P):
        x, qp, _ = oracle.continuous_min(cfg["Cdd"], V[p] @ cfg["Cgd"].T)
        fr = np.maximum(x, 0) - np.floor(np.maximum(x, 0))
        keep.append(not qp and (np.minimum(fr, 1 - fr) > 0.02).all())
    keep = np.array(keep)
    gbar = np.random.Generator(np.random.PCG64(7)).normal(size=(P, 8))
    gbar[~keep] = 0.0
    dC, dG = _grad_gpu(qa, cfg, kT, gbar)

    def loss(Cdd, Cgd):
        mean, _ = oracle.soft(Cdd, Cgd, V=V[keep], kT=kT)
        return float((mean * gbar[keep]).sum())

    sc = max(np.abs(dC).max(), np.abs(dG).max())
    rng = np.random.Generator(np.random.PCG64(8))
    for _ in range(6):
        i, j = rng.integers(0, 8, 2)
        E = np.zeros((8, 8))
        E[i, j] = E[j, i] = 1.0
        fd = (loss(cfg["Cdd"] + h * E, cfg["Cgd"]) - loss(cfg["Cdd"] - h * E, cfg["Cgd"])) / (2 * h)
        an = dC[i, j] + (dC[j, i] if i != j else 0.0)
        assert abs(an - fd) <= 1e-4 * sc + 1e-5 * abs(fd), (i, j, an, fd)
        E = np.zeros((8, 8))
        E[i, j] = 1.0
        fd = (loss(cfg["Cdd"], cfg["Cgd"] + h * E) - loss(cfg["Cdd"], cfg["Cgd"] - h * E)) / (2 * h)
        assert abs(dG[i, j] - fd) <= 1e-4 * sc + 1e-5 * abs(fd), (i, j, dG[i, j], fd)


def test_autograd_function_and_fit_loop(qa):
    import torch
    from paper_2404_04994_gb300 import autograd as qag
    cfg = inputs.grid8(W=40, H=40, kT=0.05)
    kT = 0.05
    target = qag.target_diagram(cfg["Cdd_target"], cfg["Cgd_target"], cfg["raster"], kT)
    fit = qag.CapacitanceFit(cfg["Cdd"], cfg["Cgd"], cfg["raster"], target, kT, lr=2e-3)
    Ct, Gt = cfg["Cdd_target"], cfg["Cgd_target"]

    def rel_err():
        C = fit.Cdd.detach().cpu().numpy()
        G = fit.Cgd.detach().cpu().numpy()
        return (np.linalg.norm(C - Ct) / np.linalg.norm(Ct),
                np.linalg.norm(G - Gt) / np.linalg.norm(Gt))

    e0 = rel_err()
    losses = []
    for _ in range(100):
        fit.step()
        losses.append(float(fit.loss))
    e1 = rel_err()
    fit.close()
    print(f"fit: loss {losses[0]:.4g} -> {losses[-1]:.4g}; rel. error Cdd {e0[0]:.4f} -> "
          f"{e1[0]:.4f}, Cgd {e0[1]:.4f} -> {e1[1]:.4f}")
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.05 * losses[0], losses[:3] + losses[-3:]
    # one raster of two swept gates does not determine every capacitance of
    # an 8-dot grid (the other gates enter only through their summed offsets,
    # dots the sweep barely moves only through their tails), so the diagram
    # is fitted and Cgd moves toward the target model; the recovery of all
    # capacitances is asserted where the raster determines them (the double
    # dot of test_gpu_fit.py)
    assert e1[1] < e0[1], (e0, e1)
    # the Function's gradient (backward from the forward's context) equals
    # the plain backward kernel's up to the FP32 rounding of <n>
    Cdd = torch.tensor(cfg["Cdd"], device="cuda", requires_grad=True)
    Cgd = torch.tensor(cfg["Cgd"], device="cuda", requires_grad=True)
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    ras = inputs.grid8(W=12, H=10)["raster"]
    mean = qag.soft_occupation(Cdd, Cgd, m.handle, ras, kT)
    gbar = torch.randn_like(mean)
    (mean * gbar).sum().backward()
    dC, dG = _grad_gpu(qa, cfg, kT, gbar.cpu().numpy(), raster=ras)
    sc = max(np.abs(dC).max(), np.abs(dG).max())
    np.testing.assert_allclose(Cdd.grad.cpu().numpy(), dC, rtol=0, atol=1e-5 * sc)
    np.testing.assert_allclose(Cgd.grad.cpu().numpy(), dG, rtol=0, atol=1e-5 * sc)
    m.close()


@pytest.mark.parametrize("closed", [False, True])
def test_backward_with_forward_context_matches_oracle(qa, closed):
    # the backward that reuses the forward's anchor and partition sum gives
    # the oracle gradient as well (and the plain backward's, to rounding)
    import torch
    cfg = inputs.grid8(W=33, H=27, kT=0.01) if not closed else inputs.chain4(W=31, H=23, closed=True)
    kT, t = (0.01, 1.0) if not closed else (0.03, 0.5)
    nc = 0 if not closed else 4
    P = cfg["raster"]["W"] * cfg["raster"]["H"]
    n = cfg["Cdd"].shape[0]
    gbar = np.random.Generator(np.random.PCG64(8)).normal(size=(P, n))
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    ras = cfg["raster"]
    mean = torch.empty((P, n), dtype=torch.float32, device="cuda")
    pctx = torch.empty(P, dtype=torch.int64, device="cuda")
    qa.qa_soft_occupation_ctx(m.handle, ras, kT, t, closed, nc, mean, None, pctx)
    g = torch.tensor(gbar, dtype=torch.float32, device="cuda").contiguous()
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    dG = torch.empty((n, m.n_gate), dtype=torch.float64, device="cuda")
    qa.qa_soft_occupation_backward_ctx(m.handle, ras, kT, t, closed, nc, g, mean, pctx, dC, dG)
    dC2 = torch.empty_like(dC)
    dG2 = torch.empty_like(dG)
    qa.qa_soft_occupation_backward(m.handle, ras, kT, t, closed, nc, g, dC2, dG2)
    torch.cuda.synchronize()
    m.close()
    _, oC, oG = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, raster=ras, kT=kT, t=t,
                                 closed=closed, n_charges=nc)
    sc = max(np.abs(oC).max(), np.abs(oG).max())
    assert np.abs(dC.cpu().numpy() - oC).max() <= GRAD_RTOL * sc
    assert np.abs(dG.cpu().numpy() - oG).max() <= GRAD_RTOL * sc
    np.testing.assert_allclose(dC.cpu().numpy(), dC2.cpu().numpy(), atol=1e-5 * sc)
    np.testing.assert_allclose(dG.cpu().numpy(), dG2.cpu().numpy(), atol=1e-5 * sc)


def test_backward_context_after_other_calls_on_the_model(qa):
    # the backward with the forward's context reuses that forward's prep
    # records only while they are in place: a ground-state call or a soft
    # call on another raster in between replaces them, and the backward must
    # still give the oracle gradient
    import torch
    cfg = inputs.grid8(W=29, H=21, kT=0.02)
    kT = 0.02
    ras = cfg["raster"]
    other = dict(ras, W=17, H=13, x0=ras["x0"] + 0.3)
    P, n = 29 * 21, 8
    gbar = np.random.Generator(np.random.PCG64(9)).normal(size=(P, n))
    _, oC, oG = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, raster=ras, kT=kT)
    sc = max(np.abs(oC).max(), np.abs(oG).max())
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    g = torch.tensor(gbar, dtype=torch.float32, device="cuda").contiguous()
    for between in ("ground_state", "soft_other_raster", "model_update"):
        mean = torch.empty((P, n), dtype=torch.float32, device="cuda")
        pctx = torch.empty(P, dtype=torch.int64, device="cuda")
        qa.qa_soft_occupation_ctx(m.handle, ras, kT, 1.0, False, 0, mean, None, pctx)
        if between == "ground_state":
            m.ground_state_open(other)
        elif between == "soft_other_raster":
            m.soft_occupation(other, kT)
        else:
            qa.qa_model_update(m.handle, cfg["Cdd"], cfg["Cgd"])
        dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
        dG = torch.empty((n, m.n_gate), dtype=torch.float64, device="cuda")
        qa.qa_soft_occupation_backward_ctx(m.handle, ras, kT, 1.0, False, 0, g, mean, pctx, dC, dG)
        torch.cuda.synchronize()
        assert np.abs(dC.cpu().numpy() - oC).max() <= GRAD_RTOL * sc, between
        assert np.abs(dG.cpu().numpy() - oG).max() <= GRAD_RTOL * sc, between
    m.close()
