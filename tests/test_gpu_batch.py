"""The batched ground state (persistent launches over a device work queue)
against the single-array calls and the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2404_04994_gb300 import inputs
from parity import compare

pytestmark = pytest.mark.gpu


def _mixed_specs(count, sides=(12, 17), seed=0, nmax=16):
    r = np.random.Generator(np.random.PCG64(4242 + seed))
    specs = []
    for a in range(count):
        n = int(r.integers(2, nmax + 1))
        Cdd = inputs.grid_cdd(r, 4, 4) if n == 16 else inputs.chain_cdd(r, n, nn=(0.05, 0.25))
        Cgd = inputs.dense_cgd(r, n, diag=(0.5, 1.0), off=(0.0, 0.1))
        gx, gy = inputs.swept_gates(n)
        V = inputs.offsets(r, n, (gx, gy))
        side = int(sides[int(r.integers(0, len(sides)))])
        closed = bool(r.integers(0, 2))
        t = float(r.choice([1.0, 1.0, 0.5]))
        specs.append(dict(Cdd=Cdd, Cgd=Cgd, raster=inputs.raster(n, gx, gy, V, W=side, H=side - 3),
                          threshold=t, closed=closed, n_charges=n if closed else 0))
    return specs


def test_batch_matches_oracle_and_single_calls(qa):
    specs = _mixed_specs(40)
    b = qa.Batch(specs)
    b.run()
    st = b.stats()
    assert st["pixels"] == sum(s["raster"]["W"] * s["raster"]["H"] for s in specs)
    assert st["unresolved"] == 0
    for sp, (n, U, f) in zip(specs, b.outputs):
        nd = sp["Cdd"].shape[0]
        n = n.cpu().numpy().reshape(-1, nd)
        U = U.cpu().numpy().reshape(-1)
        f = f.cpu().numpy().reshape(-1)
        rec = oracle.ground_state(sp["Cdd"], sp["Cgd"], raster=sp["raster"], t=sp["threshold"],
                                  closed=sp["closed"], n_charges=sp["n_charges"])
        compare(n, U, f, rec, sp["Cdd"], f"batch N={nd} closed={sp['closed']}",
                closed=sp["closed"])
        m = qa.Model(sp["Cdd"], sp["Cgd"])
        if sp["closed"]:
            n1, U1, _ = m.ground_state_closed(sp["raster"], sp["n_charges"], threshold=sp["threshold"])
        else:
            n1, U1, _ = m.ground_state_open(sp["raster"], threshold=sp["threshold"])
        np.testing.assert_array_equal(n, n1.cpu().numpy().reshape(-1, nd))
        np.testing.assert_allclose(U, U1.cpu().numpy(), rtol=1e-9, atol=1e-12)
        m.close()
    b.close()


def test_batch_rerun_and_team_override(qa):
    specs = _mixed_specs(10, sides=(20,), seed=1)
    for sp in specs:
        sp["team"] = 4
    b = qa.Batch(specs)
    b.run()
    first = [o[0].clone() for o in b.outputs]
    b.run()
    for o, f0 in zip(b.outputs, first):
        assert bool((o[0] == f0).all())
    b.close()


def test_batch_rejects_bad_items(qa):
    sp = _mixed_specs(1)[0]
    sp["threshold"] = 2.0
    with pytest.raises(qa.QAError) as e:
        qa.Batch([sp])
    assert e.value.code == -5


def test_full_size_batch_graph_sampled_against_oracle(qa):
    # The 4096-array workload (N ~ U{2..16}, 64^2 / 128^2 rasters, open or
    # closed with N_hat = N) in the launch configuration the benchmark times:
    # one CUDA-graph replay of the batched run.  Every dot count and both
    # forms are sampled; three rows of each sampled array (first, a middle
    # one, last) are recomputed by the oracle one by one.
    import torch
    specs = inputs.batch(4096)
    b = qa.Batch(specs)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    for o in b.outputs:
        o[0].fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    st = b.stats()
    assert st["pixels"] == b.pixels
    assert st["unresolved"] == 0 and st["overflow"] == 0
    picks = {}
    for a, sp in enumerate(specs):
        key = (sp["Cdd"].shape[0], sp["closed"])
        picks.setdefault(key, []).append(a)
    chosen = sorted(v[0] for v in picks.values()) + sorted(v[-1] for v in picks.values())
    chosen = sorted(set(chosen))
    assert len({specs[a]["Cdd"].shape[0] for a in chosen}) == 15
    compared = 0
    for a in chosen:
        sp = specs[a]
        nd = sp["Cdd"].shape[0]
        W, H = sp["raster"]["W"], sp["raster"]["H"]
        n = b.outputs[a][0].cpu().numpy().reshape(-1, nd)
        U = b.outputs[a][1].cpu().numpy().reshape(-1)
        f = b.outputs[a][2].cpu().numpy().reshape(-1)
        if sp["closed"]:
            assert (n.astype(np.int64).sum(1) == nd).all()
        for row in (0, H // 2 + a % 7, H - 1):
            p0, p1 = row * W, (row + 1) * W
            rec = oracle.ground_state(sp["Cdd"], sp["Cgd"], raster=sp["raster"], t=sp["t"],
                                      closed=sp["closed"], n_charges=sp["n_charges"],
                                      pixels=(p0, p1))
            rep = compare(n[p0:p1], U[p0:p1], f[p0:p1], rec, sp["Cdd"],
                          f"batch array {a} N={nd} closed={sp['closed']} row {row}",
                          closed=sp["closed"])
            compared += rep["comparable"]
    assert compared > 0.9 * sum(3 * specs[a]["raster"]["W"] for a in chosen)
    b.close()


def test_autotuned_batch_matches_oracle_at_the_tuned_thresholds(qa):
    from paper_2404_04994_gb300 import autotune
    specs = _mixed_specs(24, sides=(16, 21), seed=3, nmax=10)
    for sp in specs:
        sp["threshold"] = 1.0
    table = autotune.tune(specs, sample_side=16, arrays_per_group=3)
    for key, e in table.items():
        assert e["team"] in autotune.TEAMS
        if e["threshold"] < 1.0:
            base = [dict(autotune.sample_spec(specs[i], 16), threshold=1.0) for i in e["arrays"]]
            ref, _ = autotune.gpu_runner(base, 1)
            got, _ = autotune.gpu_runner([dict(b, threshold=e["threshold"]) for b in base], 1)
            for r, g in zip(ref, got):
                np.testing.assert_array_equal(r, g)
    tuned = autotune.apply(specs, table)
    b = qa.Batch(tuned)
    b.run()
    assert b.stats()["unresolved"] == 0
    for sp, (n, U, f) in zip(tuned, b.outputs):
        nd = sp["Cdd"].shape[0]
        rec = oracle.ground_state(sp["Cdd"], sp["Cgd"], raster=sp["raster"], t=sp["threshold"],
                                  closed=sp["closed"], n_charges=sp["n_charges"])
        compare(n.cpu().numpy().reshape(-1, nd), U.cpu().numpy().reshape(-1),
                f.cpu().numpy().reshape(-1), rec, sp["Cdd"],
                f"tuned N={nd} t={sp['threshold']:.3f} team={sp['team']}", closed=sp["closed"])
    b.close()
