"""The multi-GPU path's host logic on CPU: two gloo ranks shard a batch of
utterances (disjoint, complete, balanced by I*J) or split one utterance into
contiguous frequency ranges (disjoint, complete, in order, balanced), add up
their slot counts and take the maximum of their step times, as bench.py does
over NCCL."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, weights, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = bench.shard(weights, rank, ws)
    gathered = [None] * ws
    dist.all_gather_object(gathered, mine)
    slots = torch.tensor([float(sum(weights[i] for i in mine))], dtype=torch.float64)
    dist.all_reduce(slots, op=dist.ReduceOp.SUM)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)          # per-rank step time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((gathered, float(slots.item()), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    import numpy as np
    rng = np.random.default_rng(0)
    weights = [int(513 * j) for j in rng.integers(200, 2001, size=37)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, weights, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, slots, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = (set(g) for g in gathered)
    assert not (a & b) and a | b == set(range(len(weights)))
    la, lb = sum(weights[i] for i in a), sum(weights[i] for i in b)
    assert abs(la - lb) <= max(weights)                       # LPT balance bound
    assert slots == float(sum(weights)) and tmax == 2.0


def test_shard_single_rank_is_everything():
    import bench
    assert bench.shard([5, 3, 9], 0, 1) == [0, 1, 2]


def _rank_rows(rank, ws, port, I, J, out):
    import numpy as np

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    i0, i1 = bench.freq_range(I, rank, ws)
    p = {k: np.arange(I * J, dtype=np.float32).reshape(I, J) for k in ("rh0", "ru0")}
    p.update(x=np.zeros((I, J, 2), np.complex64), a=np.zeros((I, 2)), Rp=np.zeros((I, 2, 2)))
    q = bench.slice_rows(p, i0, i1)
    rows = [int(v) for v in q["rh0"][:, 0] // J]             # the frequency index of each kept row
    gathered = [None] * ws
    dist.all_gather_object(gathered, (i0, i1, rows))
    slots = torch.tensor([float((i1 - i0) * J)], dtype=torch.float64)
    dist.all_reduce(slots, op=dist.ReduceOp.SUM)
    if rank == 0:
        out.put((gathered, float(slots.item())))
    dist.destroy_process_group()


@pytest.mark.parametrize("I", [1025, 2049, 7])
def test_two_rank_frequency_ranges(I):
    """One utterance split over two ranks: contiguous ranges that are disjoint,
    cover every frequency row in order and differ in size by at most one row."""
    J = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_rows, args=(r, 2, port, I, J, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, slots = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (a0, a1, ra), (b0, b1, rb) = gathered
    assert a0 == 0 and a1 == b0 and b1 == I
    assert ra + rb == list(range(I))
    assert abs((a1 - a0) - (b1 - b0)) <= 1
    assert slots == float(I * J)


def test_frequency_ranges_cover_for_any_world_size():
    import bench
    for I in (1, 5, 513, 1025):
        for ws in (1, 2, 3, 4, 8):
            r = [bench.freq_range(I, k, ws) for k in range(ws)]
            assert r[0][0] == 0 and r[-1][1] == I
            assert all(r[k][1] == r[k + 1][0] for k in range(ws - 1))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1
