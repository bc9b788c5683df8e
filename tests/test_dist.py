"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2512_23569_gb300 import dist as hd
    from paper_2512_23569_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(hd.shard(7, rank, world))
        t = hd.max_over_ranks(1.5 + rank)
        n = hd.sum_over_ranks(len(mine))
        # each rank draws its own seeded image; the seeds never coincide
        seed = hd.image_seed(2000, rank)
        img = synth.clean_image(16, 16, 1, seed)
        q.put((rank, mine, t, n, seed, float(img.sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, n0, s0, i0), (r1, m1, t1, n1, s1, i1) = res
    assert m0 + m1 == list(range(7)) and not set(m0) & set(m1)
    assert t0 == t1 == 2.5          # max over ranks
    assert n0 == n1 == 7            # every item owned once
    assert s0 != s1 and i0 != i1    # distinct images per rank


def test_shard_bounds():
    from paper_2512_23569_gb300 import dist as hd

    for n in (0, 1, 5, 64):
        for w in (1, 2, 3, 8):
            parts = [list(hd.shard(n, r, w)) for r in range(w)]
            assert sum(parts, []) == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        hd.shard(4, 2, 2)
