"""Seeded synthetic workloads shaped like the paper's (arXiv 2404.04994).

This module only draws random numbers and lays them out: it holds none of the
method's arithmetic, imports neither the oracle nor the CUDA binding, and is
the one module both sides take their inputs from.

The paper's benchmark (Sec. VII) draws capacitances uniformly, converts them to
Maxwell form and sweeps 100 x 100 gate-voltage pixels; its datasets are not
public, so every workload here is synthetic.  Conventions:

* ``Cdd`` is the Maxwell dot-dot block (Sec. II, Eq. 2; Appendix B):
  diagonal 1, off-diagonal entries are minus the mutual capacitance.
* ``Cgd`` is the gate-to-dot block with positive entries, so that
  ``c = Cgd @ V`` is the induced charge in units of the electron charge.
* A raster is ``V(ix, iy) = V0 + xs[ix] * u + ys[iy] * w`` with
  ``xs = linspace(x0, x1, W)``, ``ys = linspace(y0, y1, H)``; pixel
  ``p = iy * W + ix`` (the GateVoltageComposer meshgrid of Sec. V).

Draw order within one array: Cdd upper triangle row-major (only the entries
the topology couples), then Cgd row-major, then the fixed-gate offsets, then
flags.  Seeds are ``20240404 + workload number``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20240404


def rng_for(workload: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + workload))


# --------------------------------------------------------------------------
# capacitance matrices
# --------------------------------------------------------------------------

def chain_cdd(rng, n, nn=(0.1, 0.3)):
    """Linear chain: nearest-neighbour mutual capacitance U[nn]."""
    C = np.eye(n)
    for i in range(n):
        for j in range(i + 1, n):
            if j == i + 1:
                m = rng.uniform(*nn)
                C[i, j] = C[j, i] = -m
    return C


def grid_cdd(rng, rows, cols, nn=(0.05, 0.25), diag=(0.0, 0.05)):
    """rows x cols grid: nearest neighbours U[nn], diagonal neighbours U[diag]."""
    n = rows * cols
    C = np.eye(n)
    for i in range(n):
        ri, ci = divmod(i, cols)
        for j in range(i + 1, n):
            rj, cj = divmod(j, cols)
            dr, dc = abs(ri - rj), abs(ci - cj)
            if dr + dc == 1:
                m = rng.uniform(*nn)
            elif dr == 1 and dc == 1:
                m = rng.uniform(*diag)
            else:
                continue
            C[i, j] = C[j, i] = -m
    return C


def dense_cgd(rng, n, n_gate=None, diag=(0.5, 1.0), off=(0.0, 0.1), decay=None):
    """Gate-to-dot block: plunger diag U[diag], crosstalk U[off] (optionally
    times decay**|i-j|)."""
    n_gate = n if n_gate is None else n_gate
    G = np.zeros((n, n_gate))
    for i in range(n):
        for g in range(n_gate):
            if i == g:
                G[i, g] = rng.uniform(*diag)
            else:
                v = rng.uniform(*off)
                if decay is not None:
                    v *= decay ** abs(i - g)
                G[i, g] = v
    return G


def raster(n_gate, gx, gy, V_fixed, lo=-1.0, hi=6.0, W=100, H=100):
    """2-D sweep of gates gx (fast axis) and gy over linspace(lo, hi)."""
    V0 = np.array(V_fixed, dtype=np.float64).copy()
    V0[gx] = 0.0
    V0[gy] = 0.0
    u = np.zeros(n_gate)
    w = np.zeros(n_gate)
    u[gx] = 1.0
    w[gy] = 1.0
    return {"V0": V0, "u": u, "w": w, "x0": lo, "x1": hi, "y0": lo, "y1": hi,
            "W": int(W), "H": int(H)}


def offsets(rng, n_gate, swept, lo=0.0, hi=3.0):
    V = np.zeros(n_gate)
    for g in range(n_gate):
        if g not in swept:
            V[g] = rng.uniform(lo, hi)
    return V


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def double_dot(W=100, H=100):
    """2-dot open double dot, T = 0, t = 1 (workload 1)."""
    r = rng_for(1)
    Cdd = chain_cdd(r, 2, nn=(0.1, 0.3))
    Cgd = dense_cgd(r, 2, diag=(0.5, 1.0), off=(0.05, 0.2))
    ras = raster(2, 0, 1, np.zeros(2), W=W, H=H)
    return {"name": "double_dot_2x100x100", "Cdd": Cdd, "Cgd": Cgd,
            "raster": ras, "t": 1.0, "closed": False, "n_charges": 0}


def chain4(W=200, H=200, closed=False):
    """4-dot linear chain over gates 2 and 3 (indices 1, 2), others at 2.0
    (workload 2); open, or closed with 4 charges."""
    r = rng_for(2)
    Cdd = chain_cdd(r, 4, nn=(0.1, 0.3))
    Cgd = dense_cgd(r, 4, diag=(0.5, 1.0), off=(0.0, 0.2), decay=0.5)
    V = np.full(4, 2.0)
    ras = raster(4, 1, 2, V, W=W, H=H)
    return {"name": f"chain4_{'closed' if closed else 'open'}_{W}x{H}",
            "Cdd": Cdd, "Cgd": Cgd, "raster": ras, "t": 1.0,
            "closed": bool(closed), "n_charges": 4 if closed else 0}


def grid16(W=100, H=100, t=1.0):
    """16-dot 4x4 grid, open, sweep of plungers 5 and 6 (workload 3)."""
    r = rng_for(3)
    Cdd = grid_cdd(r, 4, 4)
    Cgd = dense_cgd(r, 16, diag=(0.5, 1.0), off=(0.0, 0.1))
    V = offsets(r, 16, (5, 6))
    ras = raster(16, 5, 6, V, W=W, H=H)
    return {"name": f"grid16_open_t{t:g}_{W}x{H}", "Cdd": Cdd, "Cgd": Cgd,
            "raster": ras, "t": float(t), "closed": False, "n_charges": 0}


def swept_gates(n):
    """Adjacent interior pair: (5, 6) for the 16-dot grid, middle pair else."""
    if n == 16:
        return 5, 6
    return max(0, n // 2 - 1), n // 2


def batch(count=4096, sizes=(64, 128)):
    """``count`` independent arrays (workload 4): N ~ U{2..16}, 4x4-grid rule at
    N = 16, chain with nearest-neighbour U[0.05, 0.25] below; own raster of
    64^2 or 128^2; open or closed (N_hat = N) at random."""
    r = rng_for(4)
    items = []
    for a in range(count):
        n = int(r.integers(2, 17))
        if n == 16:
            Cdd = grid_cdd(r, 4, 4)
        else:
            Cdd = chain_cdd(r, n, nn=(0.05, 0.25))
        Cgd = dense_cgd(r, n, diag=(0.5, 1.0), off=(0.0, 0.1))
        gx, gy = swept_gates(n)
        V = offsets(r, n, (gx, gy))
        side = int(sizes[int(r.integers(0, 2))])
        closed = bool(r.integers(0, 2))
        items.append({"Cdd": Cdd, "Cgd": Cgd,
                      "raster": raster(n, gx, gy, V, W=side, H=side),
                      "t": 1.0, "closed": closed,
                      "n_charges": n if closed else 0})
    return items


def grid8(W=200, H=200, kT=0.01):
    """8-dot 2x4 grid for the differentiable workload (workload 5): the model,
    and a target model with every non-zero entry perturbed by U[-10%, +10%]."""
    r = rng_for(5)
    Cdd = grid_cdd(r, 2, 4)
    Cgd = dense_cgd(r, 8, diag=(0.5, 1.0), off=(0.0, 0.1))
    V = offsets(r, 8, (1, 5))
    ras = raster(8, 1, 5, V, W=W, H=H)
    Ct = Cdd.copy()
    for i in range(8):
        for j in range(i, 8):
            if Ct[i, j] != 0.0:
                Ct[i, j] *= 1.0 + r.uniform(-0.1, 0.1)
                Ct[j, i] = Ct[i, j]
    Gt = Cgd.copy()
    for i in range(8):
        for g in range(8):
            if Gt[i, g] != 0.0:
                Gt[i, g] *= 1.0 + r.uniform(-0.1, 0.1)
    return {"name": f"grid8_soft_kT{kT:g}_{W}x{H}", "Cdd": Cdd, "Cgd": Cgd,
            "raster": ras, "t": 1.0, "closed": False, "n_charges": 0,
            "kT": float(kT), "Cdd_target": Ct, "Cgd_target": Gt}


def random_points(n_gate, count, lo=-1.0, hi=6.0, seed=0):
    """Random gate-voltage list (the paper's benchmark samples random voltage
    configurations, Sec. VII)."""
    r = np.random.Generator(np.random.PCG64(SEED_BASE + 100 + seed))
    return r.uniform(lo, hi, size=(count, n_gate))


def random_model(rng, n, nn=(0.05, 0.3), off=(0.0, 0.2)):
    """Small random chain + dense Cgd, for tests."""
    Cdd = chain_cdd(rng, n, nn=nn)
    Cgd = dense_cgd(rng, n, diag=(0.5, 1.0), off=off)
    return Cdd, Cgd
