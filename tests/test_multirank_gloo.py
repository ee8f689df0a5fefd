"""Multi-rank host logic on CPU (gloo, world size 2): the k-range shards of a
query cover every series exactly once, and summing the ranks' carry-save partial
sums with one all-reduce gives the whole query's sum exactly.  The partial sums
here come from the oracle; on GPUs the same exchange carries bbp_accumulate_async
outputs (bench.py --gpus N)."""

import os
import socket

import pytest
import torch.multiprocessing as mp

N_Q, P_Q, G_Q = 123_457, 96, 64


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, results):
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1008_3171_gb300 as bbp
    from oracle import bbp_oracle as o1

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W = o1.working_bits(P_Q, G_Q)
    L = W // 32
    slots = torch.zeros(L, dtype=torch.int64)
    for j in range(7):
        kb, ke = bbp.bbp_shard_range(0, j, N_Q, W, rank, world)
        part = oracle.c_partial_sum(0, j, kb, ke, N_Q, P_Q, G_Q, threads=2)
        for i in range(L):                    # carry-save: one u32 limb per int64 slot
            slots[i] += (part >> (32 * i)) & 0xFFFFFFFF
    dist.all_reduce(slots)
    if rank == 0:
        S = sum(int(v) << (32 * i) for i, v in enumerate(slots.tolist())) % (1 << W)
        results.put(S)
    dist.destroy_process_group()


def test_two_rank_exchange_is_exact():
    from oracle import bbp_oracle as o1

    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    S = results.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want, _ = o1.accumulate(o1.BELLARD, N_Q, P_Q, G_Q)
    assert S == want


@pytest.mark.parametrize("world", [1, 2, 3, 7, 64])
def test_shards_cover_every_series_once(world):
    import paper_1008_3171_gb300 as bbp
    from oracle import bbp_oracle as o1

    for n in (1, 10, 999, 10**9 + 1, 10**15):
        for W in (64, 320):
            for j, s in enumerate(o1.BELLARD.series):
                ne = o1.natural_end(o1.BELLARD, s, n - 1, W)
                prev = 0
                for r in range(world):
                    kb, ke = bbp.bbp_shard_range(0, j, n, W, r, world)
                    assert kb == prev and ke >= kb
                    prev = ke
                assert prev == ne
