"""Multi-process host logic on CPU (gloo, world size 2): rank discovery,
sharding of independent work units, barrier and the max / sum reductions the
bench applies to its timings.  The method has no exchange step, so a sharded
run must reproduce the unsharded one exactly; that is checked with the oracle
on a small raster split by rows across the two ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2404_04994_gb300 import dist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_partitions_exactly():
    for n in (0, 1, 7, 100, 4096):
        for world in (1, 2, 3, 8):
            spans = [dist.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        import oracle
        from paper_2404_04994_gb300 import inputs
        r, loc, w = dist.init(backend="gloo")
        assert (r, loc, w) == (rank, rank, world)
        dist.barrier()
        mx = dist.max_over_ranks(float(rank + 1) * 1.5)
        sm = dist.sum_over_ranks(float(rank + 1))
        # rows of one raster sharded across ranks, each computed independently
        rng = np.random.Generator(np.random.PCG64(77))
        n = 4
        Cdd = inputs.chain_cdd(rng, n)
        Cgd = inputs.dense_cgd(rng, n)
        gx, gy = inputs.swept_gates(n)
        V = inputs.offsets(rng, n, (gx, gy))
        H, W = 9, 11
        ras = inputs.raster(n, gx, gy, V, W=W, H=H)
        r0, r1 = dist.shard(H, rank, world)
        full = oracle.ground_state(Cdd, Cgd, raster=ras, t=1.0)["n"].reshape(H, W, -1)
        mine = full[r0:r1].copy()
        import torch
        import torch.distributed as tdist
        parts = [None] * world
        tdist.all_gather_object(parts, (r0, r1, mine))
        dist.finalize()
        q.put((rank, mx, sm, parts, full))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e), None, None, None))


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_and_reassemble():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, mx, sm, parts, full = q.get(timeout=240)
        got[rank] = (mx, sm, parts, full)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        mx, sm, parts, full = got[rank]
        assert not isinstance(mx, str), mx
        assert mx == 3.0 and sm == 3.0
        spans = [(a, b) for a, b, _ in parts]
        assert spans == [dist.shard(full.shape[0], r, 2) for r in range(2)]
        np.testing.assert_array_equal(np.concatenate([m for _, _, m in parts]), full)


def test_single_process_helpers_are_identity(monkeypatch):
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert dist.env_rank() == (0, 0, 1)
    assert dist.init() == (0, 0, 1)
    assert dist.max_over_ranks(2.5) == 2.5
    assert dist.sum_over_ranks(2.5) == 2.5
    dist.barrier()
