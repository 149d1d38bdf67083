"""GPU brute force (Table I, brute-force row; C ABI -> CUDA) against the
FP64 oracle's exhaustive search, and against the default method where
Theorem 2 makes the default method exact."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import inputs

pytestmark = pytest.mark.gpu


def _brute_gpu(qa, Cdd, Cgd, ras, closed, bound):
    m = qa.Model(Cdd, Cgd)
    if closed:
        n, U, f = m.brute_force_closed(ras, bound)
    else:
        n, U, f = m.brute_force_open(ras, bound)
    out = (n.cpu().numpy().reshape(-1, m.n_dot).astype(np.int64), U.cpu().numpy(),
           f.cpu().numpy())
    m.close()
    return out


def _check(qa, Cdd, Cgd, ras, closed, bound, label):
    n, U, f = _brute_gpu(qa, Cdd, Cgd, ras, closed, bound)
    ref = oracle.brute_force_raster(Cdd, Cgd, ras, closed=closed, n_charges=bound if closed else 0,
                                    n_max=bound)
    gap = ref["U2"] - ref["U"]
    ok = gap > 1e-9
    bad = ok & (n != ref["n"]).any(1)
    assert not bad.any(), f"{label}: {int(bad.sum())} pixels differ, first {np.where(bad)[0][:5]}"
    assert ok.sum() >= 0.9 * len(ok)
    scale = np.maximum(1.0, np.abs(ref["U"]))
    assert np.max(np.abs(U - ref["U"]) / scale) < 1e-10, label
    # flags: near ties exactly where the oracle's gap is (numerically) zero-ish
    assert not (((f & 1) != 0) & (gap > 1e-6)).any()
    if not closed:
        np.testing.assert_array_equal((f & 2) != 0, ref["hit"])
    else:
        assert (n.sum(1) == bound).all() and (n >= 0).all()
    return n, U, f, ref


def _model(seed, n, chain=True):
    r = np.random.Generator(np.random.PCG64(seed))
    Cdd = inputs.chain_cdd(r, n) if chain else inputs.grid_cdd(r, 2, n // 2)
    Cgd = inputs.dense_cgd(r, n, diag=(0.5, 1.0), off=(0.0, 0.2))
    gx, gy = inputs.swept_gates(n)
    V = inputs.offsets(r, n, (gx, gy))
    return Cdd, Cgd, gx, gy, V


@pytest.mark.parametrize("n,nmax,W,H", [(2, 8, 23, 17), (3, 5, 13, 11), (4, 4, 9, 7)])
def test_open_matches_oracle(qa, n, nmax, W, H):
    Cdd, Cgd, gx, gy, V = _model(100 + n, n)
    ras = inputs.raster(n, gx, gy, V, lo=-1.0, hi=4.0, W=W, H=H)
    _check(qa, Cdd, Cgd, ras, False, nmax, f"open N={n}")


@pytest.mark.parametrize("n,nhat,W,H", [(2, 3, 19, 13), (3, 5, 11, 9), (4, 4, 9, 7), (1, 2, 5, 3)])
def test_closed_matches_oracle(qa, n, nhat, W, H):
    Cdd, Cgd, gx, gy, V = _model(200 + n, n)
    if n == 1:
        gx, gy = 0, 0
    ras = inputs.raster(n, gx, gy, V, W=W, H=H)
    _check(qa, Cdd, Cgd, ras, True, nhat, f"closed N={n}")


def test_box_too_small_is_flagged(qa):
    Cdd, Cgd, gx, gy, V = _model(301, 3)
    ras = inputs.raster(3, gx, gy, V, lo=2.0, hi=6.0, W=8, H=6)
    n, U, f, ref = _check(qa, Cdd, Cgd, ras, False, 2, "open N=3 small box")
    assert ref["hit"].any() and ((f & 2) != 0).any()


def test_default_method_equals_brute_force_under_theorem_2(qa):
    # Theorem 2 (App. E): with kappa(M) <= 1 + 4/n and x = c >= 0 the default
    # method (t = 1) is exact; both run on the GPU here
    r = np.random.Generator(np.random.PCG64(77))
    n = 2
    while True:
        Cdd, _ = inputs.random_model(r, n, nn=(0.0, 0.2))
        ev = np.linalg.eigvalsh(np.linalg.inv(Cdd))
        if ev[-1] / ev[0] <= 1 + 4 / n:
            break
    Cgd = np.diag(r.uniform(0.5, 1.0, n))
    ras = inputs.raster(n, 0, 1, np.zeros(n), lo=0.0, hi=5.0, W=31, H=29)
    m = qa.Model(Cdd, Cgd)
    nd, Ud, fd = m.ground_state_open(ras)
    nb, Ub, fb = m.brute_force_open(ras, 9)
    nd = nd.cpu().numpy().reshape(-1, n)
    nb = nb.cpu().numpy().reshape(-1, n)
    clear = ((fb.cpu().numpy() & 1) == 0) & ((fd.cpu().numpy() & 1) == 0)
    np.testing.assert_array_equal(nd[clear], nb[clear])
    assert clear.mean() > 0.95
    m.close()


def test_brute_force_errors(qa):
    Cdd, Cgd, gx, gy, V = _model(401, 4)
    ras = inputs.raster(4, gx, gy, V, W=4, H=4)
    m = qa.Model(Cdd, Cgd)
    with pytest.raises(qa.QAError) as e:
        m.brute_force_open(ras, -1)
    assert e.value.code == -5
    with pytest.raises(qa.QAError) as e:
        m.brute_force_closed(ras, 200)
    assert e.value.code == -5
    m.close()
    r = np.random.Generator(np.random.PCG64(9))
    big = qa.Model(inputs.grid_cdd(r, 4, 4), inputs.dense_cgd(r, 16))
    gx, gy = inputs.swept_gates(16)
    with pytest.raises(qa.QAError) as e:   # 128^16 states per pixel
        big.brute_force_open(inputs.raster(16, gx, gy, np.zeros(16), W=2, H=2), 127)
    assert e.value.code == -5
    big.close()
