"""The multi-GPU exchange with partial sums computed on the GPU (Sec. 4: independent
parts of the sum are added exactly).  Two processes share the one visible GPU; each
adds its k-range shard of every series into its own carry-save accumulators with
bbp_accumulate_async, the host copies are summed with one gloo all-reduce (the step
bench.py --gpus N does with NCCL), and rank 0 finalizes the summed limbs with
bbp_finalize_async.  Nothing on the GPU waits on the other process: the kernels run
independently and the exchange is on the host.

The result must equal the oracle's bits, or, for a position too large for the
oracle here, the paper's Table 2 row."""

import os
import socket

import pytest
import torch.multiprocessing as mp

import oracle

pytestmark = pytest.mark.gpu


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, n, P, results):
    import torch
    import torch.distributed as dist

    import paper_1008_3171_gb300 as bbp

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        plan = bbp.Plan(device=0, stream=stream.cuda_stream, guard_bits=64)
        W = plan.working_bits(P)
        slots = torch.zeros(W // 32, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(stream):
            slots.zero_()
            bbp.bbp_accumulate_async(plan.handle, 0, n, P, rank, world, slots.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        host = slots.cpu()
        dist.all_reduce(host)                       # exact: 64-bit carry-save limbs, added mod 2^64
        if rank == 0:
            summed = host.to("cuda")
            out = torch.zeros((P + 7) // 8, dtype=torch.uint8, device="cuda")
            valid = torch.zeros(1, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            bbp.bbp_finalize_async(plan.handle, 0, n, P, summed.data_ptr(), out.data_ptr(), valid.data_ptr(), 0,
                                   stream.cuda_stream)
            stream.synchronize()
            raw = bytes(out.cpu().tolist())
            results.put((int.from_bytes(raw, "big") >> (8 * len(raw) - P), int(valid.item())))
        plan.close()
    finally:
        dist.destroy_process_group()


def two_ranks(n, P):
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, n, P, results)) for r in range(2)]
    for p in procs:
        p.start()
    got = results.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return got


def test_two_rank_exchange_of_gpu_partial_sums_matches_oracle():
    n, P = 20_000_003, 256                          # moduli below 2^25: the lazy one-limb path
    assert two_ranks(n, P) == oracle.c_bits(n, P, 64)


def test_two_rank_exchange_of_gpu_partial_sums_matches_paper_row(pins):
    """n = 1e10 + 1 (Table 2, the suppressed m = 10 row): moduli up to 2^33.2, so both
    one-limb paths and the two-limb path run in each rank's shard."""
    pin = pins["suppressed_m10"]
    P = 256
    got, valid = two_ranks(pin["n"], P)
    ref = int(pin["hex"], 16) >> (4 * len(pin["hex"]) - pin["bits"])
    assert valid == P
    assert got == ref >> (pin["bits"] - P)
