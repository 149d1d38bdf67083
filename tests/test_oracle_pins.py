"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares it with a closed
form, an invariant, a worked example, an independent library routine or brute
force, chosen so that a dropped term, a wrong sign/index or a transposed
operand in the oracle fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(k=0):
    return np.random.Generator(np.random.PCG64(777 + k))


# ---------------------------------------------------------------------------
# linear algebra and the energy
# ---------------------------------------------------------------------------

def test_inverse_spd_identity_and_not_pd():
    rng = _rng(1)
    for n in (1, 2, 5, 16):
        A = rng.normal(size=(n, n))
        A = A @ A.T + n * np.eye(n)
        M = oracle.inverse_spd(A)
        np.testing.assert_allclose(M @ A, np.eye(n), atol=1e-12)
    with pytest.raises(ValueError):
        oracle.inverse_spd(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_energy_worked_example():
    # M = [[2, 1], [1, 3]], n - c = (1, -2):
    # 1/2 * (2*1*1 + 2*1*(1*-2) + 3*(-2)*(-2)) = 1/2 * (2 - 4 + 12) = 5
    M = np.array([[2.0, 1.0], [1.0, 3.0]])
    assert oracle.energy(M, [1, 0], [0.0, 2.0]) == pytest.approx(5.0, abs=1e-15)
    # asymmetric placement catches a transposed index: n - c = (0, 1)
    M = np.array([[4.0, 0.5], [0.5, 1.0]])
    assert oracle.energy(M, [3, 2], [3.0, 1.0]) == pytest.approx(0.5, abs=1e-15)


def test_energy_is_free_energy_plus_constant():
    # Eq. "free_energy": F(Q) = 1/2 Q^T M Q - (M c)^T Q; U - F is independent
    # of Q and equals 1/2 c^T M c.
    rng = _rng(2)
    n = 4
    Cdd, _ = inputs.random_model(rng, n)
    M = np.linalg.inv(Cdd)
    c = rng.uniform(0, 3, n)
    for _ in range(5):
        q = rng.integers(0, 4, n)
        F = 0.5 * q @ M @ q - (M @ c) @ q
        assert oracle.energy(M, q, c) - F == pytest.approx(0.5 * c @ M @ c, abs=1e-12)


# ---------------------------------------------------------------------------
# continuous minimum (Sec. III.A, Appendices C-D)
# ---------------------------------------------------------------------------

def test_open_continuous_min_is_c_when_nonnegative():
    rng = _rng(3)
    Cdd, _ = inputs.random_model(rng, 5)
    c = rng.uniform(0.1, 4, 5)
    x, qp, cert = oracle.continuous_min(Cdd, c)
    assert not qp
    np.testing.assert_array_equal(x, c)


def test_closed_continuous_min_stationary_on_hyperplane():
    # Appendix D: the minimiser lies on 1^T x = N and M (x - c) is parallel
    # to the all-ones vector (Lagrange condition).
    rng = _rng(4)
    for n in (2, 3, 6):
        Cdd, _ = inputs.random_model(rng, n)
        M = np.linalg.inv(Cdd)
        c = rng.uniform(0.5, 2.0, n)
        N = int(round(c.sum()))
        x, qp, _ = oracle.continuous_min(Cdd, c, closed=True, n_charges=N)
        assert not qp
        assert x.sum() == pytest.approx(N, abs=1e-12)
        g = M @ (x - c)
        np.testing.assert_allclose(g, np.full(n, g.mean()), atol=1e-12)


def test_open_qp_matches_scipy_nnls():
    # min 1/2 (x - c)^T M (x - c), x >= 0  ==  min ||R x - R c||, R^T R = M
    from scipy.optimize import nnls
    rng = _rng(5)
    for trial in range(40):
        n = int(rng.integers(2, 9))
        Cdd, _ = inputs.random_model(rng, n, nn=(0.05, 0.3))
        M = np.linalg.inv(Cdd)
        c = rng.uniform(-2, 2, n)
        R = np.linalg.cholesky(M).T
        xs, _ = nnls(R, R @ c)
        x, qp, cert = oracle.continuous_min(Cdd, c)
        np.testing.assert_allclose(x, xs, atol=1e-9)
        assert cert < 1e-9


def _kkt_all_sets(M, c, closed, N):
    """Independent brute check: every active set, numpy solves."""
    n = len(c)
    hits = []
    for A in itertools.product([0, 1], repeat=n):
        F = [i for i in range(n) if not A[i]]
        x = np.zeros(n)
        lam = 0.0
        if F:
            MFF = M[np.ix_(F, F)]
            rhs = (M @ c)[F]
            if closed:
                K = np.zeros((len(F) + 1, len(F) + 1))
                K[:-1, :-1] = MFF
                K[:-1, -1] = -1.0
                K[-1, :-1] = 1.0
                sol = np.linalg.solve(K, np.concatenate([rhs, [N]]))
                x[F] = sol[:-1]
                lam = sol[-1]
            else:
                x[F] = np.linalg.solve(MFF, rhs)
        elif closed and N != 0:
            continue
        z = M @ (x - c) - lam
        act = [i for i in range(n) if A[i]]
        if (x[F] >= -1e-10).all() and (z[act] >= -1e-10).all() if act else (x[F] >= -1e-10).all():
            hits.append(x)
    return hits


def test_qp_unique_kkt_point_closed_and_open():
    rng = _rng(6)
    for trial in range(30):
        n = int(rng.integers(2, 7))
        closed = bool(trial % 2)
        Cdd, _ = inputs.random_model(rng, n, nn=(0.05, 0.3))
        M = np.linalg.inv(Cdd)
        c = rng.uniform(-2, 3, n)
        N = int(rng.integers(1, n + 2)) if closed else 0
        x, qp, cert = oracle.continuous_min(Cdd, c, closed=closed, n_charges=N)
        hits = _kkt_all_sets(M, c, closed, N)
        assert len(hits) >= 1
        for h in hits:
            np.testing.assert_allclose(h, x, atol=1e-8)
        if closed:
            assert x.sum() == pytest.approx(N, abs=1e-10)
        assert (x >= -1e-12).all()


# ---------------------------------------------------------------------------
# Appendix E, Theorem 1: uncoupled dots reduce to round-and-clip
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("t", [1.0, 0.5, 0.2, 0.0])
def test_uncoupled_dots_round_and_clip(t):
    rng = _rng(7)
    n = 5
    d = rng.uniform(0.5, 2.0, n)
    Cdd = np.diag(d)
    # dense, non-square gate matrix: a transposed or mis-indexed Cgd changes c
    ng = n + 2
    Cgd = rng.uniform(0.0, 0.3, size=(n, ng))
    Cgd[np.arange(n), np.arange(n)] += rng.uniform(0.5, 1.0, n)
    V = rng.uniform(-2.0, 8.0, size=(300, ng))
    out = oracle.ground_state(Cdd, Cgd, V=V, t=t)
    c = V @ Cgd.T
    expect = np.maximum(0, np.floor(c + 0.5)).astype(int)
    np.testing.assert_array_equal(out["n"][:, :n], expect)
    # energy of uncoupled dots: sum_i (n_i - c_i)^2 / (2 Cdd_ii)
    np.testing.assert_allclose(out["U"], (((expect - c) ** 2) / (2 * d)).sum(1),
                               rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Appendix E, Theorem 2: kappa(M) <= 1 + 4/n  =>  default method is exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 4])
def test_default_equals_brute_force_when_well_conditioned(n):
    rng = _rng(10 + n)
    checked = 0
    while checked < 150:
        Cdd, _ = inputs.random_model(rng, n, nn=(0.0, 0.25))
        M = np.linalg.inv(Cdd)
        ev = np.linalg.eigvalsh(M)
        if ev[-1] / ev[0] > 1 + 4 / n:
            continue
        c = rng.uniform(0.0, 3.5, n)
        rec = oracle.ground_state_c(Cdd, c, t=1.0)
        bn, bU, hit, _ = oracle.brute_force(M, c, n_max=int(math.ceil(c.max())) + 2)
        assert not hit
        if rec["U2"] - rec["U"] < 1e-9:
            continue
        np.testing.assert_array_equal(rec["n"][:n], bn)
        assert rec["U"] == pytest.approx(bU, abs=1e-12)
        checked += 1


def test_closed_double_dot_equals_brute_force():
    # Two dots with a fixed total: the admissible set is a line, and the
    # floor/ceil pair bracketing the continuous minimum holds the optimum.
    rng = _rng(20)
    for _ in range(200):
        Cdd, _ = inputs.random_model(rng, 2, nn=(0.05, 0.4))
        M = np.linalg.inv(Cdd)
        c = rng.uniform(-1.0, 4.0, 2)
        N = int(rng.integers(0, 5))
        rec = oracle.ground_state_c(Cdd, c, t=1.0, closed=True, n_charges=N)
        bn, bU, _, _ = oracle.brute_force(M, c, closed=True, n_charges=N)
        assert rec["n"][:2].sum() == N
        if rec["U2"] - rec["U"] > 1e-9:
            np.testing.assert_array_equal(rec["n"][:2], bn)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_closed_vertex_minimum_is_the_ground_state(n):
    # Closed, every dot but one active in the relaxed minimum: the sum
    # constraint puts x at the vertex N e_j, an integer point, which is then
    # the exact integer minimum (brute force over all compositions agrees)
    # whatever the rounding of x_j; the GPU parity rule relies on this.
    rng = _rng(30 + n)
    seen = 0
    for _ in range(300):
        Cdd, _ = inputs.random_model(rng, n, nn=(0.05, 0.3))
        M = np.linalg.inv(Cdd)
        c = rng.uniform(-4.0, 6.0, n)
        N = int(rng.integers(1, 5))
        rec = oracle.ground_state_c(Cdd, c, t=1.0, closed=True, n_charges=N)
        x = np.asarray(rec["x"][:n])
        if not ((x > 0).sum() == 1 and ((x == 0.0) | (x > 0)).all()):
            continue
        j = int(np.argmax(x))
        assert abs(x[j] - N) < 1e-9
        want = np.zeros(n, dtype=np.int64)
        want[j] = N
        np.testing.assert_array_equal(rec["n"][:n], want)
        bn, _, _, _ = oracle.brute_force(M, c, closed=True, n_charges=N)
        np.testing.assert_array_equal(bn, want)
        seen += 1
    assert seen >= 20


def test_open_negative_region_equals_brute_force_double_dot():
    # including pixels where the analytic minimum is infeasible (QP path)
    cfg = inputs.double_dot(W=40, H=40)
    out = oracle.ground_state(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"])
    M = np.linalg.inv(cfg["Cdd"])
    assert out["qp_used"].sum() > 0
    bad = 0
    for p in range(0, 1600, 7):
        c = oracle.raster_c(cfg["Cgd"], cfg["raster"], p)
        bn, bU, hit, _ = oracle.brute_force(M, c, n_max=9)
        assert not hit
        if out["U2"][p] - out["U"][p] > 1e-9:
            bad += int((out["n"][p, :2] != bn).any())
    assert bad == 0


# ---------------------------------------------------------------------------
# honeycomb geometry of the double dot
# ---------------------------------------------------------------------------

def test_double_dot_triple_point():
    # U(0,0) = U(1,0) = U(0,1) where (M c)_i = M_ii / 2, i.e.
    # c* = Cdd diag(M) / 2; around it the three states own the three sectors
    # c* + eps Cdd v, v = (-1,-1), (1,-1), (-1,1).
    Cdd = np.array([[1.3, -0.1], [-0.1, 1.3]])    # Sec. V example model
    Cgd = np.array([[1.0, 0.2], [0.2, 1.0]])
    M = np.linalg.inv(Cdd)
    cstar = Cdd @ (0.5 * np.diag(M))
    eps = 1e-3
    pts = []
    want = {(-1, -1): (0, 0), (1, -1): (1, 0), (-1, 1): (0, 1)}
    for v in want:
        c = cstar + eps * Cdd @ np.array(v, dtype=float)
        pts.append(np.linalg.solve(Cgd, c))
    out = oracle.ground_state(Cdd, Cgd, V=np.array(pts), t=1.0)
    got = [tuple(r[:2]) for r in out["n"]]
    assert got == list(want.values())


def test_double_dot_labels_change_only_across_transition_lines():
    cfg = inputs.double_dot(W=60, H=60)
    Cdd, Cgd, ras = cfg["Cdd"], cfg["Cgd"], cfg["raster"]
    out = oracle.ground_state(Cdd, Cgd, raster=ras)
    M = np.linalg.inv(Cdd)
    n = out["n"][:, :2].reshape(60, 60, 2)
    for iy in range(60):
        for ix in range(59):
            a, b = n[iy, ix], n[iy, ix + 1]
            pa, pb = iy * 60 + ix, iy * 60 + ix + 1
            ca = oracle.raster_c(Cgd, ras, pa)
            cb = oracle.raster_c(Cgd, ras, pb)
            if (a == b).all():
                continue
            # a beats b at pixel a, b beats a at pixel b
            assert oracle.energy(M, a, ca) <= oracle.energy(M, b, ca) + 1e-12
            assert oracle.energy(M, b, cb) <= oracle.energy(M, a, cb) + 1e-12


# ---------------------------------------------------------------------------
# closed arrays: exact conservation (constraint iii)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("t", [1.0, 0.3, 0.0])
def test_closed_conserves_total_charge(t):
    cfg = inputs.chain4(W=24, H=24, closed=True)
    out = oracle.ground_state(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], t=t,
                              closed=True, n_charges=4)
    assert (out["n"][:, :4].sum(1) == 4).all()
    assert (out["n"][:, :4] >= 0).all()
    if t == 0.0:
        assert (out["t_used"] >= 0.0).all()


# ---------------------------------------------------------------------------
# threshold (Sec. III.B, Appendix G, Appendix J)
# ---------------------------------------------------------------------------

def test_default_candidate_count_is_2_pow_n():
    rng = _rng(30)
    for n in (1, 3, 6):
        Cdd, _ = inputs.random_model(rng, n)
        rec = oracle.ground_state_c(Cdd, rng.uniform(1, 5, n), t=1.0)
        assert rec["n_cand"] == 2 ** n


@pytest.mark.parametrize("t", [0.25, 0.5, 0.75])
def test_expected_candidates_1_plus_t_pow_n(t):
    # Appendix G: with frac(x) uniform, E[#candidates] = (1 + t)^N.
    n = 6
    Cdd = np.eye(n)
    Cgd = np.eye(n)
    V = inputs.random_points(n, 20000, lo=5.0, hi=15.0, seed=int(t * 100))
    out = oracle.ground_state(Cdd, Cgd, V=V, t=t)
    mean = out["n_cand"].mean()
    assert mean == pytest.approx((1 + t) ** n, rel=0.02)


def test_243_fold_reduction_five_dots_five_charges():
    # Sec. I: 5 dots, 5 charges: brute force visits (5 + 1)^5 states, the
    # default method 2^5; the ratio is 243.
    rng = _rng(31)
    Cdd, _ = inputs.random_model(rng, 5)
    M = np.linalg.inv(Cdd)
    c = rng.uniform(0.5, 1.5, 5)
    _, _, _, visited = oracle.brute_force(M, c, closed=True, n_charges=5)
    rec = oracle.ground_state_c(Cdd, c, t=1.0)
    assert visited == 6 ** 5
    assert rec["n_cand"] == 2 ** 5
    assert visited // rec["n_cand"] == 243


def _fig6_maps(t, W=120):
    g = json.load(open(os.path.join(GOLDEN, "paper_examples.json")))
    Cdd = np.array(g["fig6_threshold"]["cdd"])
    Cgd = np.array(g["example_model"]["cgd"])
    ras = inputs.raster(2, 0, 1, np.zeros(2), lo=-1.0, hi=4.0, W=W, H=W)
    return oracle.ground_state(Cdd, Cgd, raster=ras, t=t)


def test_fig6_threshold_one_seventh_matches_default():
    # Appendix J: for cdd = [[1.4, -0.2], [-0.2, 1.4]] the diagram at t = 1/7
    # is identical to the default (t = 1) one.
    a = _fig6_maps(1.0)
    b = _fig6_maps(1.0 / 7.0)
    ok = (a["U2"] - a["U"] > 1e-9) & (a["margin_floor"] > 1e-9)
    assert (a["n"][ok] == b["n"][ok]).all()


def test_fig6_smaller_threshold_distorts_more():
    # Appendix J: below 1/7 the interdot segment shrinks as t decreases and
    # vanishes at t = 0: the number of differing pixels does not decrease.
    ref = _fig6_maps(1.0)
    diffs = []
    for t in (0.1, 0.05, 0.02, 0.0):
        m = _fig6_maps(t)
        diffs.append(int((m["n"] != ref["n"]).any(1).sum()))
    assert diffs[-1] > 0
    assert all(diffs[i] <= diffs[i + 1] for i in range(len(diffs) - 1))


# ---------------------------------------------------------------------------
# soft occupation (Sec. IV.B)
# ---------------------------------------------------------------------------

def test_soft_uncoupled_two_state_fermi():
    rng = _rng(40)
    n = 4
    d = rng.uniform(0.8, 1.5, n)
    Cdd = np.diag(d)
    Cgd = np.eye(n)
    V = rng.uniform(0.2, 5.0, size=(200, n))
    kT = 0.05
    mean, logZ = oracle.soft(Cdd, Cgd, V=V, kT=kT, t=1.0)
    fl = np.floor(V)
    # U(fl+1) - U(fl) = (fl + 1/2 - c) / Cdd_ii for an isolated dot
    dE = (fl + 0.5 - V) / d
    expect = fl + 1.0 / (1.0 + np.exp(dE / kT))
    np.testing.assert_allclose(mean, expect, atol=1e-12)
    # the partition function factorises over dots
    U0 = (fl - V) ** 2 / (2 * d)
    U1 = (fl + 1 - V) ** 2 / (2 * d)
    lz = np.logaddexp(-U0 / kT, -U1 / kT).sum(1)
    np.testing.assert_allclose(logZ, lz, rtol=1e-12, atol=1e-9)


def test_soft_zero_temperature_limit_and_closed_sum():
    cfg = inputs.chain4(W=16, H=16, closed=True)
    gs = oracle.ground_state(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"],
                             closed=True, n_charges=4)
    mean, _ = oracle.soft(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], kT=1e-4,
                          closed=True, n_charges=4)
    np.testing.assert_allclose(mean.sum(1), 4.0, atol=1e-12)
    clear = gs["U2"] - gs["U"] > 0.01
    np.testing.assert_allclose(mean[clear], gs["n"][clear, :4], atol=1e-12)


# ---------------------------------------------------------------------------
# gradient through the soft occupation (frozen candidate set)
# ---------------------------------------------------------------------------

def _loss(Cdd, Cgd, V, gbar, kT):
    mean, _ = oracle.soft(Cdd, Cgd, V=V, kT=kT, t=1.0)
    return float((mean * gbar).sum())


def test_soft_gradient_matches_central_differences():
    rng = _rng(50)
    n = 3
    Cdd, Cgd = inputs.random_model(rng, n, nn=(0.1, 0.2))
    # voltages whose continuous minimum is far from integers, so the frozen
    # candidate set is the set at every perturbed point
    V = rng.uniform(1.0, 4.0, size=(40, n))
    c = V @ Cgd.T
    keep = (np.abs(c - np.floor(c) - 0.5) < 0.4).all(1)
    V = V[keep]
    kT = 0.1
    gbar = rng.normal(size=(len(V), n))
    dM, dCdd, dCgd = oracle.soft_grad(Cdd, Cgd, gbar, V=V, kT=kT, t=1.0)
    np.testing.assert_allclose(dCdd, dCdd.T, atol=1e-12)
    h = 1e-5
    for i in range(n):
        for j in range(i, n):
            E = np.zeros((n, n))
            E[i, j] = E[j, i] = 1.0
            fd = (_loss(Cdd + h * E, Cgd, V, gbar, kT)
                  - _loss(Cdd - h * E, Cgd, V, gbar, kT)) / (2 * h)
            an = dCdd[i, j] + (dCdd[j, i] if i != j else 0.0)
            assert an == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for i in range(n):
        for g in range(n):
            E = np.zeros((n, n))
            E[i, g] = 1.0
            fd = (_loss(Cdd, Cgd + h * E, V, gbar, kT)
                  - _loss(Cdd, Cgd - h * E, V, gbar, kT)) / (2 * h)
            assert dCgd[i, g] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_soft_gradient_raster_equals_point_list():
    # the raster path and the voltage-list path differ only in how V is formed
    cfg = inputs.grid8(W=6, H=5)
    P = 30
    rs = cfg["raster"]
    xs = np.linspace(rs["x0"], rs["x1"], rs["W"])
    ys = np.linspace(rs["y0"], rs["y1"], rs["H"])
    V = np.array([rs["V0"] + xs[p % 6] * rs["u"] + ys[p // 6] * rs["w"]
                  for p in range(P)])
    gbar = _rng(51).normal(size=(P, 8))
    a = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, raster=rs, kT=0.05)
    b = oracle.soft_grad(cfg["Cdd"], cfg["Cgd"], gbar, V=V, kT=0.05)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# brute force (Table I) and its n_max failure mode (Appendix J, Fig. 7)
# ---------------------------------------------------------------------------

def test_brute_force_counts_and_nmax_artefact():
    M = np.eye(3)
    _, _, hit, visited = oracle.brute_force(M, np.array([5.2, 0.1, 0.3]), n_max=2)
    assert visited == 3 ** 3
    assert hit
    n, U, hit, _ = oracle.brute_force(M, np.array([1.2, 0.1, 2.7]), n_max=4)
    assert not hit
    np.testing.assert_array_equal(n, [1, 0, 3])


# ---------------------------------------------------------------------------
# the paper's example model (Sec. V)
# ---------------------------------------------------------------------------

def test_example_model_shapes_and_closed_total():
    g = json.load(open(os.path.join(GOLDEN, "paper_examples.json")))["example_model"]
    Cdd = np.array(g["cdd"])
    Cgd = np.array(g["cgd"])
    ras = inputs.raster(2, 0, 1, np.zeros(2), lo=g["lo"], hi=g["hi"],
                        W=g["pixels"], H=g["pixels"])
    op = oracle.ground_state(Cdd, Cgd, raster=ras)
    cl = oracle.ground_state(Cdd, Cgd, raster=ras, closed=True,
                             n_charges=g["n_charges"])
    assert op["n"][:, :2].reshape(100, 100, 2).shape == tuple(g["output_shape"])
    assert (cl["n"][:, :2].sum(1) == g["n_charges"]).all()
    stored = np.loadtxt(os.path.join(GOLDEN, "example_model_open_map.txt"),
                        dtype=np.int64)
    np.testing.assert_array_equal(op["n"][:, :2].reshape(100, 200), stored)


def test_threshold_test_is_inclusive():
    # Eq. "threshold" reads |frac - 1/2| <= t/2: at t = 0 a dot sitting exactly
    # on a half-integer keeps both neighbours; at t = 1 every dot does, also
    # an integer x (including an x clamped to 0 by the QP), so the default
    # method always evaluates 2^N states (Table I).
    Cdd = np.eye(2)
    rec = oracle.ground_state_c(Cdd, np.array([2.5, 1.25]), t=0.0)
    assert rec["n_cand"] == 2
    rec = oracle.ground_state_c(Cdd, np.array([2.0, 3.0]), t=1.0)
    assert rec["n_cand"] == 4
    cfg = inputs.double_dot(W=30, H=30)
    out = oracle.ground_state(cfg["Cdd"], cfg["Cgd"], raster=cfg["raster"], t=1.0)
    assert out["qp_used"].sum() > 0
    assert (out["n_cand"] == 4).all()


def test_brute_force_second_energy_single_dot():
    # one dot, M = 1/C: U(n) = (n - c)^2 / (2C); c = 0.3 -> n = 0 best, n = 1 next
    C = 2.0
    M = np.array([[1.0 / C]])
    bn, bU, hit, visited = oracle.brute_force(M, np.array([0.3]), n_max=4)
    assert bn.tolist() == [0] and visited == 5 and not hit
    r = oracle.brute_force_raster(np.array([[C]]), np.array([[1.0]]),
                                  {"V0": np.zeros(1), "u": np.ones(1), "w": np.zeros(1),
                                   "x0": 0.3, "x1": 2.8, "y0": 0.0, "y1": 0.0, "W": 2, "H": 1},
                                  n_max=4)
    np.testing.assert_array_equal(r["n"][:, 0], [0, 3])
    np.testing.assert_allclose(r["U"], [0.09 / 4, 0.04 / 4], rtol=1e-14)
    np.testing.assert_allclose(r["U2"], [0.49 / 4, 0.64 / 4], rtol=1e-14)
