"""Optimal gate voltages and virtual gates (Sec. IV.C, Appendices H and I):
the library's host FP64 routines (C ABI, no GPU) against their defining
properties -- the four Penrose conditions, exact charge targeting with square
gate matrices, the normal equations, minimum norm -- and against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import api, inputs


def _model(seed, n, ng):
    r = np.random.Generator(np.random.PCG64(seed))
    Cdd = inputs.chain_cdd(r, n)
    Cgd = inputs.dense_cgd(r, n, n_gate=ng, diag=(0.5, 1.0), off=(0.0, 0.2))
    return Cdd, Cgd


@pytest.mark.parametrize("n,ng", [(2, 2), (4, 4), (4, 6), (6, 4), (16, 16), (5, 1)])
def test_virtual_gate_matrix_is_the_pseudo_inverse(n, ng):
    Cdd, Cgd = _model(10 * n + ng, n, ng)
    A = np.linalg.inv(Cdd) @ Cgd
    X = api.qa_virtual_gate_matrix(Cdd, Cgd)
    assert X.shape == (ng, n)
    # Penrose (1955): the unique X with AXA = A, XAX = X, (AX)^T = AX, (XA)^T = XA
    tol = 1e-11 * max(1.0, np.abs(X).max())
    np.testing.assert_allclose(A @ X @ A, A, atol=tol)
    np.testing.assert_allclose(X @ A @ X, X, atol=tol)
    np.testing.assert_allclose((A @ X).T, A @ X, atol=tol)
    np.testing.assert_allclose((X @ A).T, X @ A, atol=tol)
    np.testing.assert_allclose(X, oracle.virtual_gate_matrix(Cdd, Cgd), atol=tol)
    if ng >= n:  # full row rank: moving along column i shifts only dot i's potential
        np.testing.assert_allclose(A @ X, np.eye(n), atol=tol)


def test_optimal_voltages_hit_the_charge_state_with_square_gates():
    Cdd, Cgd = _model(3, 4, 4)
    Q = np.array([1.0, 0.0, 2.0, 1.0])
    for s in (1.0, -1.0):
        V = api.qa_optimal_gate_voltages(Cdd, Cgd, Q, carrier_sign=s)
        np.testing.assert_allclose(s * Cgd @ V, Q, atol=1e-12)
        np.testing.assert_allclose(V, oracle.optimal_gate_voltages(Cdd, Cgd, Q, carrier=s), atol=1e-12)


def test_optimal_voltages_normal_equations_with_fewer_gates():
    # tall R Cgd: V* is the weighted least-squares solution, gradient zero
    Cdd, Cgd = _model(4, 5, 3)
    Q = np.array([1.0, 2.0, 0.0, 1.0, 3.0])
    V = api.qa_optimal_gate_voltages(Cdd, Cgd, Q)
    M = np.linalg.inv(Cdd)
    np.testing.assert_allclose(Cgd.T @ M @ (Q - Cgd @ V), 0.0, atol=1e-11)
    np.testing.assert_allclose(V, oracle.optimal_gate_voltages(Cdd, Cgd, Q), atol=1e-11)
    # any other voltage has a free energy at least as large
    rng = np.random.Generator(np.random.PCG64(1))
    F = lambda v: 0.5 * (Q - Cgd @ v) @ M @ (Q - Cgd @ v)
    for _ in range(20):
        assert F(V) <= F(V + 0.01 * rng.normal(size=3)) + 1e-15


def test_optimal_voltages_minimum_norm_with_more_gates():
    Cdd, Cgd = _model(5, 3, 6)
    Q = np.array([2.0, 1.0, 1.0])
    V = api.qa_optimal_gate_voltages(Cdd, Cgd, Q)
    np.testing.assert_allclose(Cgd @ V, Q, atol=1e-12)
    # orthogonal to the null space of Cgd: no smaller solution exists
    _, _, vt = np.linalg.svd(Cgd)
    null = vt[3:]
    np.testing.assert_allclose(null @ V, 0.0, atol=1e-12)


def test_coupling_form_matches_its_maxwell_conversion():
    r = np.random.Generator(np.random.PCG64(8))
    n, ng = 3, 4
    Ck = np.zeros((n, n))
    for i in range(n - 1):
        Ck[i, i + 1] = Ck[i + 1, i] = r.uniform(0.1, 0.3)
    Cg = r.uniform(0.2, 1.0, size=(n, ng))
    Cmax = -Ck.copy()
    np.fill_diagonal(Cmax, Ck.sum(1) + Cg.sum(1))
    a1 = api.qa_virtual_gate_matrix(Ck, Cg, form=api.QA_FORM_COUPLING)
    a2 = api.qa_virtual_gate_matrix(Cmax, Cg)
    np.testing.assert_allclose(a1, a2, atol=1e-13)
    Q = np.array([1.0, 1.0, 0.0])
    np.testing.assert_allclose(api.qa_optimal_gate_voltages(Ck, Cg, Q, form=api.QA_FORM_COUPLING),
                               api.qa_optimal_gate_voltages(Cmax, Cg, Q), atol=1e-13)


def test_errors():
    Cdd, Cgd = _model(6, 3, 3)
    with pytest.raises(api.QAError) as e:
        api.qa_virtual_gate_matrix(-Cdd, Cgd)
    assert e.value.code == -4
    with pytest.raises(api.QAError) as e:
        api.qa_optimal_gate_voltages(Cdd, Cgd, np.ones(3), carrier_sign=0.5)
    assert e.value.code == -1
    bad = Cdd.copy()
    bad[0, 1] += 0.1
    with pytest.raises(api.QAError) as e:
        api.qa_virtual_gate_matrix(bad, Cgd)
    assert e.value.code == -3


def test_virtual_raster_directions():
    Cdd, Cgd = _model(7, 4, 4)
    ras = api.virtual_raster(Cdd, Cgd, np.full(4, 1.0), 1, 2, W=5, H=4)
    A = np.linalg.inv(Cdd) @ Cgd
    np.testing.assert_allclose(A @ ras["u"], np.eye(4)[1], atol=1e-12)
    np.testing.assert_allclose(A @ ras["w"], np.eye(4)[2], atol=1e-12)
