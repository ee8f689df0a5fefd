#!/usr/bin/env python
"""Benchmark: BBP digit extraction of pi, n = 1e12, P = 256 (+64 guard bits), one GB300.

One step is one whole query: every series of Bellard's formula (Eq. 2), head and
tail terms, the exact reduction and the finalize (certified bits + output bytes),
through the library's public API with host output buffers.  The device time of a
step comes from CUDA events on the plan's stream; the end-to-end time is the
wall clock around the same API call (it includes the device->host read of the
result).  Between timed steps the L2 is flushed by writing a 256 MiB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

N > 1 (torchrun, one rank per GPU): each rank evaluates its shard of every
series (bbp_shard_range), the carry-save partial sums are summed exactly with one
all-reduce, and rank 0 finalizes -- total work fixed, so scaling is "strong".

--impl reference times the oracle (plain C, all host cores) on a bounded sample
of the same query: evenly spaced k-ranges of every series' head.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_POS = 10**12
P_BITS = 256
GUARD = 64
METRIC = "BBP terms/s at n=1e12 P=256; % of INT32 IMAD peak; batched p50/p99 latency"
WORKLOAD = "plain single query: Bellard formula, n=1e12, P=256 + 64 guard bits, all 7 series"
IMAD_LANES_PER_CLK_PER_SM = 64     # 32-bit multiply-add (low half) issue rate per SM, measured by bbp_imad_probe
SM_MAX_MHZ_FALLBACK = 2070.0       # GB300 maximum SM clock
# Eq. 2: the exponent of series j's term k is n - 1 + c_j - 10 k
BELLARD_STEP = 10
BELLARD_EXP_OFFSETS = (2, 0, -4, -4, -6, -1, -6)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=["single", "batched", "serving"], default="single",
                    help="single: the n=1e12 headline; batched: 4096 seeded queries, persistent vs plain; "
                         "serving: Poisson arrivals at 80%% of capacity plus one long query, engine vs plain FIFO")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--serve-count", type=int, default=200)
    ap.add_argument("--serve-long", type=int, default=10**12 + 1, help="n of the long query (P = 256)")
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--tune-table", default=None)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target wall time of one oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched persistent-vs-plain comparison that follows the single-query steps")
    return ap.parse_args()


# ---------------------------------------------------------------- oracle sample (CPU)

def oracle_sample(n: int, P: int, G: int, target_s: float, threads: int = 0):
    """Times oracle O2 on evenly spaced k-ranges of every series' head terms.

    Returns (terms, seconds, description).  The per-term cost is nearly constant
    across the head (it grows with the exponent's bit length), so evenly spaced
    ranges estimate the whole query's rate; the tail terms are negligible."""
    import oracle
    from oracle import bbp_oracle as o1

    f = o1.BELLARD
    W = o1.working_bits(P, G)
    positions = 16

    def run(span):
        total = 0
        t0 = time.perf_counter()
        for j, s in enumerate(f.series):
            he = o1.head_end(f, s, n - 1)
            for i in range(positions):
                kb = 1 + (he - span - 2) * i // (positions - 1)
                oracle.c_partial_sum(0, j, kb, kb + span, n, P, G, threads)
                total += span
        return total, time.perf_counter() - t0

    terms, secs = run(2000)                      # calibration
    rate = terms / max(secs, 1e-6)
    span = max(2000, int(rate * target_s / (len(f.series) * positions)))
    terms, secs = run(span)
    desc = (f"oracle O2 (plain C, 128-bit integers) on {len(f.series)} series x {positions} evenly spaced "
            f"head k-ranges of {span} terms ({terms} terms) of the n={n}, P={P}, G={G} query")
    return terms, secs, desc


def host_cores() -> int:
    return os.cpu_count() or 1


def per_term_imad_model(bbp, n: int, P: int, G: int) -> float:
    """Multiply instructions of the query's head terms by a per-term work model:
    16 ceil(log2 e) + 4 L + 50 for a two-limb (64-bit) modulus, 5 ceil(log2 e) + 3 L + 25
    for a one-limb modulus (below 2^31), L = W/32 limbs, e the term's exponent; summed
    exactly over the query's exponents (counted per bit length), host-only."""
    ranges, _ = bbp.bbp_explain(0, n, P, G)
    L = ((P + 31) // 32 * 32 + G) // 32
    step, cs = BELLARD_STEP, BELLARD_EXP_OFFSETS
    d = n - 1
    total = 0
    for r in ranges:
        if r["tail"]:
            continue
        c = cs[r["denominator"]]
        k_lo, k_hi = r["k_begin"], r["k_begin"] + r["count"] - 1
        one_limb = r["path"] in (0, 3)
        # e = d + c - step k; count terms per ceil(log2 e) = b, i.e. 2^(b-1) < e <= 2^b (b = 0: e <= 1)
        for b in range(0, 64):
            e_lo = 0 if b == 0 else (1 << (b - 1)) + 1
            e_hi = 1 if b == 0 else 1 << b
            # k with e_lo <= d + c - step k <= e_hi
            ka = max(k_lo, -((e_hi - d - c) // step))
            kb = min(k_hi, (d + c - e_lo) // step)
            if kb >= ka:
                per = (5 * b + 3 * L + 25) if one_limb else (16 * b + 4 * L + 50)
                total += (kb - ka + 1) * per
    return float(total)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="bbp_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):   # no nvidia-smi: the run reports no clocks
            self.proc = None
            if getattr(self, "fh", None):
                self.fh.close()
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return self.summarize(lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock under load, the maximum clock and the throttle reasons
        seen, from `nvidia-smi --query-gpu=<FIELDS> --format=csv,noheader,nounits`
        lines; None without samples."""
        rows = []
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        smax = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- streams

def work_stream(torch, dev):
    """A created CUDA stream, made torch's current stream, for every library call and
    every event of a run.  The legacy default stream will not do: its handle is 0,
    which the library reads as "the plan's own stream", so events recorded on it
    would not be ordered with the library's work."""
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    return stream


# ---------------------------------------------------------------- distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def emit(obj):
    print(json.dumps(obj), flush=True)


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:           # under torchrun only rank 0 runs and prints the reference arm
        return
    # each step: one bounded oracle sample of the same workload
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(N_POS, P_BITS, GUARD, per_step)
    terms = 0
    secs = 0.0
    desc = ""
    for _ in range(args.steps):
        t, s, desc = oracle_sample(N_POS, P_BITS, GUARD, per_step)
        terms += t
        secs += s
    value = terms / secs
    emit({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_POS, "P": P_BITS, "guard_bits": GUARD,
                   "sample": "bounded oracle sample per step"},
        "cpu_baseline": {"value": value, "unit": "terms/s", "cores": host_cores(), "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    })


# ---------------------------------------------------------------- GPU arm

def expected_bits_check(bits_value: int, valid: int) -> bool:
    """Bits 2..256 at n = 1e12 equal the first 255 bits of the paper's row for
    n = 1e12 + 1 (Table 2 source, suppressed m = 12 row)."""
    with open(os.path.join(ROOT, "tests", "golden", "paper_pins.json")) as fh:
        pins = {p["name"]: p for p in json.load(fh)["pins"]}
    row = pins["suppressed_m12"]
    ref = int(row["hex"], 16) >> (4 * len(row["hex"]) - row["bits"])
    return valid == P_BITS and (bits_value & ((1 << 255) - 1)) == ref >> (row["bits"] - 255)


def head_kernel_ncu():
    """The committed ncu record of the head kernel (DRAM bytes per launch, FMA-pipe
    use), if the kernel sources are still the ones that capture measured (else {})."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "head_kernel_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in rec["kernel_sources"]:
            with open(os.path.join(ROOT, f), "rb") as src:
                h.update(src.read())
        if h.hexdigest() == rec["kernel_sources_sha256"]:
            return rec
    except (OSError, KeyError, ValueError):
        pass
    return {}


def run_gpu(args):
    import torch

    import paper_1008_3171_gb300 as bbp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    stream = work_stream(torch, dev)
    plan = bbp.Plan(device=local, stream=stream.cuda_stream, guard_bits=GUARD, profile=True)
    W = plan.working_bits(P_BITS)
    L = W // 32
    nbytes = (P_BITS + 7) // 8
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    slots = torch.zeros(L, dtype=torch.int64, device=dev)
    d_out = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    d_valid = torch.zeros(1, dtype=torch.int32, device=dev)
    out_host = torch.zeros(nbytes + 4, dtype=torch.uint8).pin_memory()

    def step_single():
        raw, valid = bbp.bbp_bits(plan.handle, N_POS, P_BITS)
        return int.from_bytes(raw, "big"), valid

    def step_sharded():
        slots.zero_()
        bbp.bbp_accumulate_async(plan.handle, 0, N_POS, P_BITS, rank, world, slots.data_ptr(), stream.cuda_stream)
        dist.all_reduce(slots)
        if rank == 0:
            bbp.bbp_finalize_async(plan.handle, 0, N_POS, P_BITS, slots.data_ptr(), d_out.data_ptr(),
                                   d_valid.data_ptr(), 0, stream.cuda_stream)
            out_host[:nbytes].copy_(d_out, non_blocking=True)
            out_host[nbytes:].copy_(d_valid.view(torch.uint8), non_blocking=True)
        torch.cuda.synchronize()
        if rank == 0:
            raw = bytes(out_host[:nbytes].tolist())
            valid = int.from_bytes(bytes(out_host[nbytes:].tolist()), "little")
            return int.from_bytes(raw, "big"), valid
        return None, None

    step = step_single if world == 1 else step_sharded

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    dev_ms = []
    wall_s = []
    head_ms = 0.0
    imad = 0.0
    head_launches = 0
    launches = 0
    terms = 0
    verified = True
    for i in range(args.steps):
        flush.fill_(i & 0xFF)             # L2 flush, outside the timed events
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        v, valid = step()
        e1.record(stream)
        t1 = time.perf_counter()
        e1.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
        wall_s.append(t1 - t0)
        st = plan.stats()
        head_ms += st["head_ms"]
        imad += st["imad_model"]
        head_launches += st["head_launches"]
        launches += st["kernel_launches"] + (1 if world > 1 and rank == 0 else 0)
        terms += st["terms"]
        if rank == 0:
            verified = verified and expected_bits_check(v, valid)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()

    # whole-job numbers: max time over ranks, all ranks' terms
    t_dev = sum(dev_ms) / 1e3
    t_e2e = sum(wall_s)
    if world > 1:
        agg = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(agg, op=dist.ReduceOp.MAX)
        t_dev, t_e2e = agg.tolist()
        tt = torch.tensor([terms, launches], dtype=torch.int64, device=dev)
        dist.all_reduce(tt)
        terms, launches = tt.tolist()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    max_mhz = (clocks or {}).get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK
    peak = sms * IMAD_LANES_PER_CLK_PER_SM * max_mhz * 1e6 / 1e12        # T multiply instructions / s
    achieved = (imad / (head_ms / 1e3)) / 1e12 if head_ms > 0 else None
    modelled = per_term_imad_model(bbp, N_POS, P_BITS, GUARD) * args.steps / max(1, world)
    achieved_model = (modelled / (head_ms / 1e3)) / 1e12 if head_ms > 0 else None
    value = terms / t_dev
    e2e_value = terms / t_e2e
    ncu = head_kernel_ncu()

    batched = None
    if not args.no_batched and world == 1:
        import workloads

        ns, Ps = workloads.batched_queries(count=args.batch_count, seed=0)
        wn, wP = workloads.batched_queries(count=64, seed=99, lo=3.0, hi=8.0)
        bplan = bbp.Plan(device=local, stream=stream.cuda_stream, guard_bits=GUARD)   # no per-launch events
        try:
            bbp.bbp_bits_batch(bplan.handle, 0, wn, wP, with_latency=False)        # warm-up: graph, buffers
            pers, plain, identical, bterms, certified = batched_arms(bbp, bplan, stream, ns, Ps)
        finally:
            bplan.close()
        batched = {"workload": f"{len(ns)} queries, seed 0, n = floor(10^U(4,10)), P uniform in {{64,128,256}}, "
                               f"G = {GUARD}", "terms": bterms, "persistent": pers, "plain": plain,
                   "latency": "device time from the start of the arm to each query's finalize (both arms)",
                   "identical": identical, "all_certified": certified}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        c_terms, c_secs, desc = oracle_sample(N_POS, P_BITS, GUARD, args.cpu_seconds)
        cpu = {"value": c_terms / c_secs, "unit": "terms/s", "cores": host_cores(), "kind": "oracle", "sample": desc}

    emit({
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_POS, "P": P_BITS, "guard_bits": GUARD,
                   "terms_per_step": terms // args.steps, "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"k-range shards x{world}" if world > 1 else "single GPU"},
        "e2e": {"value": e2e_value, "unit": "terms/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": nbytes + 4,
                "note": "bbp_bits with host output; the query (n, P) travels as kernel arguments"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved_model, "peak": peak, "unit": "T IMAD/s",
                     "frac": (achieved_model / peak) if achieved_model else None,
                     "traffic": ncu.get("dram_bytes_per_launch"),
                     "model": "per term: 16 ceil(log2 e) + 4L + 50 IMAD per two-limb term, 5 ceil(log2 e) + 3L + 25 "
                              "per one-limb term, summed over the query's exponents",
                     "achieved_half_products": achieved,
                     "frac_half_products": (achieved / peak) if achieved else None,
                     "half_products_model": "32-bit product halves the method needs: 13 per two-limb squaring "
                                            "(14 when x1^2 needs its high word), 4 per one-limb squaring, 4 (2) per "
                                            "quotient digit, 6 for m^-1 mod 2^32",
                     "ncu_imad_pipe_frac": ncu.get("fma_pipe_frac_of_imad_rate"),
                     "kernel": "head_kernel", "head_launches": head_launches,
                     "peak_basis": f"{sms} SMs x {IMAD_LANES_PER_CLK_PER_SM} IMAD lanes/clk (mul.lo issue rate, "
                                   f"measured) x {max_mhz:.0f} MHz; achieved = modelled multiplies of the "
                                   "head terms / summed CUDA-event time of the head launches"},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "verified": verified,
        "batched": batched,
    })
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched workload

def batched_arms(bbp, plan, stream, ns, Ps):
    """One persistent graph-captured pass (bbp_bits_batch) and the plain form (one
    bbp_bits_async per query, back to back on the same stream) over the same
    queries.  Latency in both arms is device time from the arm's start to each
    query's finalize: the pass's global-timer stamps for the persistent form, a CUDA
    event after each query for the plain form.  Returns (persistent, plain, identical,
    terms, all certified); a query whose two results differ is listed in persistent["differs"]."""
    import torch

    count = len(ns)
    stride = max((int(P) + 7) // 8 for P in Ps)
    # persistent
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    vals, valid, lat = bbp.bbp_bits_batch(plan.handle, 0, ns, Ps)
    e1.record(stream)
    e1.synchronize()
    pers_s = e0.elapsed_time(e1) / 1e3
    terms = plan.stats()["terms"]
    # plain
    d_out = torch.zeros((count, stride), dtype=torch.uint8, device="cuda")
    d_valid = torch.zeros(count, dtype=torch.int32, device="cuda")
    start = torch.cuda.Event(enable_timing=True)
    evs = []
    torch.cuda.synchronize()
    start.record(stream)
    for q, (n, P) in enumerate(zip(ns, Ps)):
        bbp.bbp_bits_async(plan.handle, 0, int(n), int(P), d_out[q].data_ptr(), d_valid[q].data_ptr(), 0,
                           stream.cuda_stream)
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        evs.append(e)
    evs[-1].synchronize()
    plain_lat = [start.elapsed_time(e) for e in evs]
    plain_s = plain_lat[-1] / 1e3
    out = d_out.cpu().tolist()
    vv = d_valid.cpu().tolist()
    plain_vals = []
    for q, P in enumerate(Ps):
        nb = (int(P) + 7) // 8
        plain_vals.append(int.from_bytes(bytes(out[q][:nb]), "big") >> (8 * nb - int(P)))
    diff = [q for q in range(count) if (plain_vals[q], vv[q]) != (vals[q], valid[q])]
    identical = not diff
    persistent = {"terms_per_s": terms / pers_s, "device_s": pers_s, "p50_ms": percentile(lat, 50),
                  "p99_ms": percentile(lat, 99)}
    plain = {"terms_per_s": terms / plain_s, "device_s": plain_s, "p50_ms": percentile(plain_lat, 50),
             "p99_ms": percentile(plain_lat, 99)}
    if diff:   # which queries, with both forms' bits (hex) and certified counts
        persistent["differs"] = [{"q": q, "n": int(ns[q]), "P": int(Ps[q]), "persistent": [hex(vals[q]), valid[q]],
                                  "plain": [hex(plain_vals[q]), vv[q]]} for q in diff[:8]]
        persistent["differs_count"] = len(diff)
    return persistent, plain, identical, terms, all(v == P for v, P in zip(valid, Ps))


def percentile(values, q):
    v = sorted(values)
    if not v:
        return None
    i = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[i]


def run_batched(args):
    """4096 seeded queries (n log-uniform in [1e4, 1e10], P in {64, 128, 256}, G = 64):
    one persistent graph-captured pass (bbp_bits_batch) against the plain form (one
    query after another on the same stream); outputs must be identical.  Latency in
    both arms is device time from the arm's start to each query's finalize."""
    import torch

    import paper_1008_3171_gb300 as bbp
    import workloads

    ns, Ps = workloads.batched_queries(count=args.batch_count, seed=0)
    stream = work_stream(torch, torch.device("cuda", 0))
    plan = bbp.Plan(device=0, stream=stream.cuda_stream, guard_bits=GUARD, tune_table=args.tune_table)
    for _ in range(args.warmup):
        wn, wP = workloads.batched_queries(count=64, seed=99, lo=3.0, hi=8.0)
        bbp.bbp_bits_batch(plan.handle, 0, wn, wP, with_latency=False)
    sampler = ClockSampler(0)
    sampler.start()
    runs = [batched_arms(bbp, plan, stream, ns, Ps) for _ in range(args.steps)]
    clocks = sampler.stop()
    pers, plain, identical, terms, certified = runs[-1]
    emit({
        "metric": "batched: terms/s and p50/p99 query latency, persistent vs plain", "workload": "batched",
        "config": {"queries": len(ns), "seed": 0, "n": "floor(10^U(4,10))", "P": "uniform {64,128,256}",
                   "guard_bits": GUARD, "terms": terms, "tune_table": args.tune_table},
        "persistent": dict(pers, steps=args.steps, warmup=args.warmup), "plain": plain,
        "latency": "device time from the start of the arm to each query's finalize (both arms)",
        "identical": all(r[2] for r in runs), "all_certified": certified,
        "clocks": clocks,
    })


# ---------------------------------------------------------------- serving workload

def run_serving(args):
    """Poisson arrivals (seed 1; n log-uniform in [1e6, 1e11], P in {64, 256}) at
    `load` x measured capacity, plus one long query (P = 256) at t = 0.  The
    continuous-batching engine (bbp_submit / bbp_poll) against a plain FIFO server
    (one bbp_bits call per query in arrival order) on the same trace."""
    import threading

    import torch

    import paper_1008_3171_gb300 as bbp
    import workloads

    plan = bbp.Plan(device=0, guard_bits=GUARD, max_slots=4096, tune_table=args.tune_table)
    # capacity on a sample of the short-query distribution
    cal = workloads.serving_arrivals(96, 1.0, seed=101)
    cal_n = [n for _, n, _ in cal]
    cal_P = [P for _, _, P in cal]
    bbp.bbp_bits_batch(plan.handle, 0, cal_n, cal_P, with_latency=False)
    t0 = time.perf_counter()
    bbp.bbp_bits_batch(plan.handle, 0, cal_n, cal_P, with_latency=False)
    cal_rate = plan.stats()["terms"] / (time.perf_counter() - t0)
    mean_terms = plan.stats()["terms"] / len(cal_n)
    qps = args.serve_load * cal_rate / mean_terms
    trace = workloads.serving_arrivals(args.serve_count, qps, seed=1, long_query=(args.serve_long, 256))
    expect = {}
    torch.cuda.synchronize()

    # --- engine
    results = {}
    submitted = {}
    lock = threading.Lock()
    start = time.perf_counter() + 0.05

    def submitter():
        for i, (t_arr, n, P) in enumerate(trace):
            delay = start + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            while True:
                t = bbp.bbp_submit(plan.handle, n, P)
                if t is not None:
                    break
                time.sleep(0.001)
            with lock:
                submitted[t] = (i, P)

    th = threading.Thread(target=submitter)
    sampler = ClockSampler(0)
    sampler.start()
    th.start()
    while th.is_alive() or len(results) < len(trace):
        with lock:
            items = [(t, v) for t, v in submitted.items() if t not in results]
        for t, (i, P) in items:
            r = bbp.bbp_poll(plan.handle, t, P)
            if r is not None:
                results[t] = (i, r, time.perf_counter() - start)
        time.sleep(0.0005)
    th.join()
    engine_make = max(v[2] for v in results.values())
    info = bbp.bbp_serve_stats(plan.handle)
    lat = {}
    out = {}
    for t, (i, r, t_done) in results.items():
        lat[i] = t_done - trace[i][0]
        out[i] = r
    # --- plain FIFO server on the same trace
    plain_lat = {}
    plain_out = {}
    start = time.perf_counter()
    for i, (t_arr, n, P) in enumerate(trace):
        delay = start + t_arr - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        plain_out[i] = plan.bits(n, P)
        plain_lat[i] = time.perf_counter() - start - t_arr
    plain_make = time.perf_counter() - start
    clocks = sampler.stop()
    total_terms = info["terms"]
    short = [lat[i] for i in range(1, len(trace))]
    plain_short = [plain_lat[i] for i in range(1, len(trace))]
    emit({
        "metric": "serving: p50/p99 latency of arriving queries and terms/s, continuous batching vs plain FIFO",
        "workload": "serving",
        "config": {"arrivals": len(trace) - 1, "rate_qps": qps, "load": args.serve_load, "seed": 1,
                   "n": "floor(10^U(6,11))", "P": "uniform {64,256}", "long_query": {"n": args.serve_long, "P": 256},
                   "calibrated_terms_per_s": cal_rate, "guard_bits": GUARD},
        "engine": {"terms_per_s": total_terms / engine_make, "makespan_s": engine_make,
                   "p50_ms": 1e3 * percentile(short, 50), "p99_ms": 1e3 * percentile(short, 99),
                   "long_query_latency_s": lat[0], "iterations": info["iterations"]},
        "plain": {"terms_per_s": total_terms / plain_make, "makespan_s": plain_make,
                  "p50_ms": 1e3 * percentile(plain_short, 50), "p99_ms": 1e3 * percentile(plain_short, 99),
                  "long_query_latency_s": plain_lat[0]},
        "identical": all(out[i] == plain_out[i] for i in range(len(trace))),
        "clocks": clocks,
    })


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
