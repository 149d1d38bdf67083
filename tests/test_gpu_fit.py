"""GPU tests of the fused capacitance-fitting step (qa_fit_step).

The fused step forms the MSE gradient dL/d<n> of each pixel inside the soft
occupation kernel, reduces the gradient (Sec. IV.B, Eq. "softargmin",
differentiated with the candidate set frozen) and applies Adam in the last
stage.  It must agree with the same step taken the long way: the autograd
Function (forward kernel, torch loss, backward kernel) and torch.optim.Adam.
"""
import numpy as np
import pytest

from paper_2404_04994_gb300 import inputs

pytestmark = pytest.mark.gpu


def _perturbed(cfg, seed, scale=0.1):
    """Every non-zero entry of (Cdd, Cgd) times 1 + U[-scale, scale], Cdd kept
    symmetric: the model the target diagram is made with."""
    r = np.random.Generator(np.random.PCG64(seed))
    Ct = cfg["Cdd"].copy()
    n = Ct.shape[0]
    for i in range(n):
        for j in range(i, n):
            if Ct[i, j] != 0.0:
                Ct[i, j] *= 1.0 + r.uniform(-scale, scale)
                Ct[j, i] = Ct[i, j]
    Gt = cfg["Cgd"].copy()
    nz = Gt != 0.0
    Gt[nz] *= 1.0 + r.uniform(-scale, scale, size=int(nz.sum()))
    return Ct, Gt


def test_fused_steps_match_autograd_and_torch_adam(qa):
    # 8 steps of the fused path against 8 of autograd + torch.optim.Adam.
    # Adam moves every parameter by about lr = 2e-3 per step; the two paths
    # differ in FP32 rounding only (the autograd path forms g . <n> from the
    # forward's stored FP32 <n>, the fused one from the flip moments).
    # Observed: 1.3e-7 after 8 steps.
    from paper_2404_04994_gb300 import autograd as qag
    kT = 0.05
    cfg = inputs.grid8(W=40, H=30, kT=kT)
    target = qag.target_diagram(cfg["Cdd_target"], cfg["Cgd_target"], cfg["raster"], kT)
    a = qag.CapacitanceFit(cfg["Cdd"], cfg["Cgd"], cfg["raster"], target, kT, lr=2e-3,
                           graph=False, fused=True)
    b = qag.CapacitanceFit(cfg["Cdd"], cfg["Cgd"], cfg["raster"], target, kT, lr=2e-3,
                           graph=False, fused=False)
    for k in range(8):
        a.step()
        b.step()
        la, lb = float(a.loss), float(b.loss)
        assert abs(la - lb) <= 1e-5 * abs(lb) + 1e-9, (k, la, lb)
        np.testing.assert_allclose(a.Cdd.detach().cpu().numpy(), b.Cdd.detach().cpu().numpy(),
                                   rtol=0, atol=1e-6)
        np.testing.assert_allclose(a.Cgd.detach().cpu().numpy(), b.Cgd.detach().cpu().numpy(),
                                   rtol=0, atol=1e-6)
    cnt = 8 * 8 + 8 * 8
    st = a.state.cpu().numpy()
    assert st[2 * cnt] == 8.0
    assert st[2 * cnt + 1] == pytest.approx(0.9 ** 8, rel=1e-14)
    assert st[2 * cnt + 2] == pytest.approx(0.999 ** 8, rel=1e-14)
    a.close()
    b.close()


def test_fused_gradient_matches_autograd_per_dot_target(qa):
    # per-dot target: the gradient of one fused step against autograd's.  (A
    # trajectory comparison is not meaningful here: components of dL/dCgd
    # that vanish up to rounding -- a dot whose occupation never changes on
    # the raster -- get an Adam step of about lr * sign from their rounding.)
    import torch
    from paper_2404_04994_gb300 import api, autograd as qag
    kT = 0.05
    cfg = inputs.grid8(W=40, H=30, kT=kT)
    target = qag.target_diagram(cfg["Cdd_target"], cfg["Cgd_target"], cfg["raster"], kT,
                                per_dot=True)
    b = qag.CapacitanceFit(cfg["Cdd"], cfg["Cgd"], cfg["raster"], target, kT, graph=False,
                           fused=False)
    mean = qag.soft_occupation(b.Cdd, b.Cgd, b.model.handle, b.raster, kT)
    torch.mean((mean - b.target) ** 2).backward()
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    Cdd = torch.tensor(cfg["Cdd"], device="cuda")
    Cgd = torch.tensor(cfg["Cgd"], device="cuda")
    dC = torch.zeros_like(Cdd)
    dG = torch.zeros_like(Cgd)
    state = torch.zeros(api.fit_state_len(8, 8), dtype=torch.float64, device="cuda")
    qa.qa_fit_step(m.handle, cfg["raster"], kT, 1.0, False, 0, b.target, True, Cdd, Cgd, state,
                   2e-3, dL_dCdd=dC, dL_dCgd=dG)
    gC, gG = b.Cdd.grad.cpu().numpy(), b.Cgd.grad.cpu().numpy()
    sc = max(np.abs(gC).max(), np.abs(gG).max())
    np.testing.assert_allclose(dC.cpu().numpy(), gC, rtol=0, atol=1e-6 * sc)
    np.testing.assert_allclose(dG.cpu().numpy(), gG, rtol=0, atol=1e-6 * sc)
    m.close()
    b.close()


# closed arrays with a sum target are left out: sum_i <n_i> = N_hat on every
# pixel, so that loss has no gradient (only rounding noise)
@pytest.mark.parametrize("closed,per_dot", [(False, False), (True, True), (False, True)])
def test_fused_step_outputs_equal_the_separate_calls(qa, closed, per_dot):
    # the optional outputs of one step -- <n>, the loss and its gradient --
    # against the forward call, a numpy loss and the backward call
    import torch
    cfg = inputs.chain4(W=33, H=21, closed=closed)
    n, ng = 4, 4
    kT, t, N = 0.03, 1.0, (4 if closed else 0)
    ras = cfg["raster"]
    P = 33 * 21
    m = qa.Model(cfg["Cdd"], cfg["Cgd"])
    mean0, _ = m.soft_occupation(ras, kT, threshold=t, closed=closed, n_charges=N)
    rng = np.random.Generator(np.random.PCG64(11))
    mn = mean0.cpu().numpy()
    if per_dot:
        tgt = (mn + rng.normal(0, 0.1, mn.shape)).astype(np.float32)
    else:
        tgt = (mn.sum(1) + rng.normal(0, 0.3, P)).astype(np.float32)
    target = torch.tensor(tgt, device="cuda")
    Cdd = torch.tensor(cfg["Cdd"], device="cuda")
    Cgd = torch.tensor(cfg["Cgd"], device="cuda")
    state = torch.zeros(qa.fit_state_len(n, ng), dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    dC = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    dG = torch.zeros((n, ng), dtype=torch.float64, device="cuda")
    mean = torch.zeros((P, n), dtype=torch.float32, device="cuda")
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    qa.qa_fit_step(m.handle, ras, kT, t, closed, N, target, per_dot, Cdd, Cgd, state, lr,
                   b1, b2, eps, loss=loss, dL_dCdd=dC, dL_dCgd=dG, out_mean=mean)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(mean.cpu().numpy(), mn)
    if per_dot:
        r = mn.astype(np.float64) - tgt
        g = ((2.0 / (P * n)) * r).astype(np.float32)
    else:
        r = mn.sum(1).astype(np.float64) - tgt
        g = np.repeat((2.0 / P) * r[:, None], n, axis=1).astype(np.float32)
    assert float(loss) == pytest.approx(np.mean(r * r), rel=1e-5)
    m2 = qa.Model(cfg["Cdd"], cfg["Cgd"])
    dC2 = torch.zeros_like(dC)
    dG2 = torch.zeros_like(dG)
    qa.qa_soft_occupation_backward(m2.handle, ras, kT, t, closed, N,
                                   torch.tensor(g, device="cuda"), dC2, dG2)
    torch.cuda.synchronize()
    sc = max(np.abs(dC2.cpu().numpy()).max(), np.abs(dG2.cpu().numpy()).max())
    np.testing.assert_allclose(dC.cpu().numpy(), dC2.cpu().numpy(), rtol=0, atol=1e-5 * sc)
    np.testing.assert_allclose(dG.cpu().numpy(), dG2.cpu().numpy(), rtol=0, atol=1e-5 * sc)
    # the Adam step itself: at the first step the bias-corrected moments are g
    # and g^2, so the update is lr g / (|g| + eps) up to rounding
    for p0, p1, gr in ((cfg["Cdd"], Cdd, dC), (cfg["Cgd"], Cgd, dG)):
        gg = gr.cpu().numpy()
        want = p0 - lr * gg / (np.abs(gg) + eps)
        np.testing.assert_allclose(p1.cpu().numpy(), want, rtol=0, atol=1e-12)
    st = state.cpu().numpy()
    np.testing.assert_allclose(st[:n * n], (1 - b1) * dC.cpu().numpy().ravel(), rtol=1e-15)
    cnt = n * n + n * ng
    assert list(st[2 * cnt:]) == [1.0, b1, b2]
    with pytest.raises(qa.QAError):
        qa.qa_fit_step(m.handle, ras, kT, t, closed, N, target, per_dot, Cdd, Cgd, state, -1.0)
    with pytest.raises(qa.QAError):
        qa.qa_fit_step(m.handle, ras, kT, t, closed, N, target, per_dot, Cdd, Cgd, state, lr,
                       beta1=1.0)
    m.close()
    m2.close()


def test_fit_recovers_double_dot_capacitances(qa):
    # a double dot swept over both of its gates determines its capacitances
    # (the occupation of each dot at kT > 0 fixes the energy scale too): fused
    # Adam steps from the unperturbed model move (Cdd, Cgd) to the perturbed
    # model that made the target
    from paper_2404_04994_gb300 import autograd as qag
    kT = 0.05
    cfg = inputs.double_dot(W=60, H=60)
    Ct, Gt = _perturbed(cfg, 22)
    ras = cfg["raster"]
    target = qag.target_diagram(Ct, Gt, ras, kT, per_dot=True)
    fit = qag.CapacitanceFit(cfg["Cdd"], cfg["Cgd"], ras, target, kT, lr=5e-3)

    def rel_err():
        C = fit.Cdd.detach().cpu().numpy()
        G = fit.Cgd.detach().cpu().numpy()
        return (np.linalg.norm(C - Ct) / np.linalg.norm(Ct),
                np.linalg.norm(G - Gt) / np.linalg.norm(Gt))

    e0 = rel_err()
    losses, errs = [], {}
    for s in range(300):
        fit.step()
        losses.append(float(fit.loss))
        if s + 1 in (100, 300):
            errs[s + 1] = rel_err()
    fit.close()
    print(f"double dot fit: loss {losses[0]:.4g} -> {losses[99]:.4g} -> {losses[-1]:.4g}; "
          f"rel. error (Cdd, Cgd) {e0} -> {errs[100]} -> {errs[300]}")
    assert losses[99] < 0.01 * losses[0]
    # after 100 steps both errors are below the start, Cgd's far below
    assert errs[100][0] < e0[0] and errs[100][1] < 0.1 * e0[1], (e0, errs)
    # after 300 both are gone to the level of the fit's own convergence
    assert errs[300][0] < 0.05 * e0[0] and errs[300][1] < 0.05 * e0[1], (e0, errs)
