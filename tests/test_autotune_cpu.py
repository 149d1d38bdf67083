"""Host logic of the batch autotuner (no GPU): the threshold heuristic of
App. F, the admission rule (a t < 1 only if it reproduces the t = 1 map on
the sample), the team choice and the table's JSON round trip, with a fake
runner standing in for the library."""
import math

import numpy as np

from paper_2404_04994_gb300 import autotune, inputs


def test_delta_and_candidates_for_the_fig6_matrix():
    # Cdd = [[1.4, -0.2], [-0.2, 1.4]]: Delta has off-diagonal 1/7, so
    # 2 ||Delta||_2 = 2/7 and ||Delta||_F = sqrt(2)/7 = 0.202 (App. F)
    C = np.array([[1.4, -0.2], [-0.2, 1.4]])
    D = autotune.delta_matrix(C)
    np.testing.assert_allclose(D, [[0.0, 1 / 7], [1 / 7, 0.0]], rtol=1e-15)
    c = autotune.threshold_candidates([C])
    np.testing.assert_allclose(c, [math.sqrt(2) / 7, 2 / 7, 0.5], rtol=1e-12)


def test_candidates_take_the_group_maximum_and_drop_values_above_one():
    weak = np.array([[1.0, -0.05], [-0.05, 1.0]])
    strong = np.array([[1.0, -0.3], [-0.3, 1.0]])
    c = autotune.threshold_candidates([weak, strong])
    np.testing.assert_allclose(c, [math.sqrt(2) * 0.3, 0.5, 0.6], rtol=1e-12)
    dense = np.eye(7) - 0.16 * (np.ones((7, 7)) - np.eye(7))
    assert autotune.threshold_candidates([dense]) == [0.5]   # both norms >= 1


def _specs():
    r = np.random.Generator(np.random.PCG64(5))
    out = []
    for n, closed in ((2, False), (2, False), (3, True), (5, False)):
        Cdd = inputs.chain_cdd(r, n)
        Cgd = inputs.dense_cgd(r, n)
        gx, gy = inputs.swept_gates(n)
        out.append(dict(Cdd=Cdd, Cgd=Cgd, raster=inputs.raster(n, gx, gy, inputs.offsets(r, n, (gx, gy)), W=40, H=30),
                        threshold=1.0, closed=closed, n_charges=n if closed else 0))
    return out


class FakeRunner:
    """Maps equal to the t = 1 map when t >= t_ok[N], one pixel off below;
    time minimal at team best[N]."""

    def __init__(self, t_ok, best):
        self.t_ok, self.best, self.calls = t_ok, best, []

    def __call__(self, specs, reps):
        self.calls.append(specs)
        maps = []
        for sp in specs:
            n = sp["Cdd"].shape[0]
            W, H = sp["raster"]["W"], sp["raster"]["H"]
            m = np.zeros((H, W, n), dtype=np.int8)
            if sp["threshold"] < min(self.t_ok[n], 1.0):
                m[0, 0, 0] = 1
            maps.append(m)
        n = specs[0]["Cdd"].shape[0]
        team = specs[0].get("team", 0)
        ms = 1.0 + abs(math.log2(team) - math.log2(self.best[n])) if team else 9.0
        return maps, ms


def test_tune_admits_smallest_reproducing_threshold_and_fastest_team():
    specs = _specs()
    fake = FakeRunner(t_ok={2: 0.5, 3: 2.0, 5: 0.0}, best={2: 4, 3: 1, 5: 32})
    table = autotune.tune(specs, runner=fake, sample_side=8, arrays_per_group=2)
    assert set(table) == {(2, False), (3, True), (5, False)}
    e2 = table[(2, False)]
    assert e2["arrays"] == [0, 1]
    # candidates below 0.5 are rejected with their mismatch count (one per array)
    assert e2["threshold"] == 0.5 and all(v == 2 for v in e2["rejected"].values())
    assert e2["team"] == 4
    assert table[(3, True)]["threshold"] == 1.0 and table[(3, True)]["team"] == 1
    smallest = autotune.threshold_candidates([specs[3]["Cdd"]])[0]
    assert table[(5, False)]["threshold"] == smallest and table[(5, False)]["team"] == 32
    # every sample raster is sample_side square over the same window
    for call in fake.calls:
        for sp in call:
            assert sp["raster"]["W"] == sp["raster"]["H"] == 8
            assert sp["raster"]["x0"] == -1.0 and sp["raster"]["x1"] == 6.0
    tuned = autotune.apply(specs, table)
    assert [sp["team"] for sp in tuned] == [4, 4, 1, 32]
    assert tuned[0]["threshold"] == 0.5 and specs[0]["threshold"] == 1.0
    back = autotune.from_json(autotune.to_json(table))
    assert {k: (v["threshold"], v["team"]) for k, v in back.items()} == \
           {k: (v["threshold"], v["team"]) for k, v in table.items()}
