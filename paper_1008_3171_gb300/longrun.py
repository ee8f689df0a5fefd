"""Checkpointed long runs: one query's bits, computed shard by shard, with the
partial sums saved on the host after every shard, so that a run that stops (a
time budget runs out, the process or the machine is lost) resumes where it
stopped.

The paper keeps every task's partial sum in persistent storage so that the
whole computation can be killed at any time and resumed later (Sec. 4, the
MapReduce design: task outputs sigma_{j,k} are persisted and summed by a
controller).  Here a task is one shard of ``bbp_shard_range`` over every series
of the formula, and the saved state is the query's W/32 carry-save
accumulators (one uint64 per 32-bit limb, ``bbp_accumulate_async``) plus the
set of finished shards.  The accumulators add limb-wise modulo 2^64 and stay
exact while fewer than 2^31 shards are added, so shards added in any order, by
any number of runs, give the same sum as one uninterrupted run.

Command line::

    python -m paper_1008_3171_gb300.longrun --n 100000000000001 --P 256 \\
        --shards 64 --checkpoint run.json [--max-seconds 1500] [--max-shards K]

prints one JSON line per run: the shards done so far, and once every shard is
in, the bits (hex, MSB first) and how many of them the error bound certifies.
"""

from __future__ import annotations

import argparse
import json
import os
import time
from dataclasses import dataclass, field

MASK64 = (1 << 64) - 1
FORMAT = "bbp-longrun-1"


@dataclass
class Checkpoint:
    """State of one checkpointed query (host only; no GPU needed)."""

    formula: int
    n: int
    P: int
    guard_bits: int
    shards: int
    slots: list          # W/32 accumulators, unsigned 64-bit
    done: list = field(default_factory=list)   # finished shard indices, sorted
    seconds: float = 0.0                        # device time summed over runs

    @classmethod
    def fresh(cls, formula: int, n: int, P: int, guard_bits: int, shards: int, limbs: int) -> "Checkpoint":
        if shards < 1 or shards >= 1 << 31:
            raise ValueError("shards must be in [1, 2^31)")
        return cls(formula, n, P, guard_bits, shards, [0] * limbs)

    def key(self) -> tuple:
        return (self.formula, self.n, self.P, self.guard_bits, self.shards, len(self.slots))

    def remaining(self) -> list:
        have = set(self.done)
        return [s for s in range(self.shards) if s not in have]

    def add(self, shard: int, slots: list, seconds: float) -> None:
        """Records shard `shard` as finished with the accumulators `slots`
        (which already include it)."""
        if shard in self.done or not 0 <= shard < self.shards:
            raise ValueError(f"shard {shard} already done or out of range")
        if len(slots) != len(self.slots):
            raise ValueError("accumulator count changed")
        self.slots = [int(v) & MASK64 for v in slots]
        self.done = sorted(self.done + [shard])
        self.seconds += seconds

    def to_json(self) -> dict:
        return {"format": FORMAT, "formula": self.formula, "n": str(self.n), "P": self.P,
                "guard_bits": self.guard_bits, "shards": self.shards, "done": self.done,
                "slots": [str(v) for v in self.slots], "seconds": self.seconds}

    @classmethod
    def from_json(cls, d: dict) -> "Checkpoint":
        if d.get("format") != FORMAT:
            raise ValueError("not a longrun checkpoint")
        c = cls(int(d["formula"]), int(d["n"]), int(d["P"]), int(d["guard_bits"]), int(d["shards"]),
                [int(v) & MASK64 for v in d["slots"]], sorted(int(s) for s in d["done"]),
                float(d.get("seconds", 0.0)))
        if len(set(c.done)) != len(c.done) or any(not 0 <= s < c.shards for s in c.done):
            raise ValueError("corrupt shard list")
        return c

    def save(self, path: str) -> None:
        """Atomic replace: a run killed mid-write leaves the previous checkpoint."""
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(self.to_json(), fh)
            fh.flush()
            os.fsync(fh.fileno())
        os.replace(tmp, path)

    @classmethod
    def load_or_fresh(cls, path: str, fresh: "Checkpoint") -> "Checkpoint":
        """The saved checkpoint if `path` exists (it must describe the same
        query and shard count), else `fresh`."""
        if not path or not os.path.exists(path):
            return fresh
        with open(path) as fh:
            c = cls.from_json(json.load(fh))
        if c.key() != fresh.key():
            raise ValueError(f"checkpoint {path} is for another query: {c.key()} != {fresh.key()}")
        return c


def run(n: int, P: int, shards: int, checkpoint: str = "", formula: int = 0, guard_bits: int = 64,
        max_seconds: float = float("inf"), max_shards: int = -1, device: int = 0) -> dict:
    """Adds the shards that `checkpoint` does not hold yet, saving after each one,
    until all are in, `max_shards` were added or `max_seconds` would be passed
    (estimated from the slowest shard so far); then finalizes if complete."""
    import torch

    from . import Plan

    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device=device)
    plan = Plan(device=device, guard_bits=guard_bits, stream=stream.cuda_stream)
    try:
        with torch.cuda.stream(stream):  # every tensor below is made and used on `stream`
            return _run(plan, stream, n, P, shards, checkpoint, formula, guard_bits, max_seconds, max_shards,
                        device)
    finally:
        plan.close()


def _run(plan, stream, n, P, shards, checkpoint, formula, guard_bits, max_seconds, max_shards, device) -> dict:
    import torch

    from . import bbp_accumulate_async, bbp_finalize_async

    limbs = plan.working_bits(P) // 32
    ck = Checkpoint.load_or_fresh(checkpoint, Checkpoint.fresh(formula, n, P, guard_bits, shards, limbs))
    d_slots = torch.tensor([v - (1 << 64) if v >> 63 else v for v in ck.slots], dtype=torch.int64,
                           device=f"cuda:{device}")
    start = time.monotonic()
    slowest = 0.0
    added = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s in ck.remaining():
        if 0 <= max_shards <= added:
            break
        if time.monotonic() - start + slowest > max_seconds:
            break
        t0 = time.monotonic()
        ev0.record(stream)
        bbp_accumulate_async(plan.handle, formula, n, P, s, shards, d_slots.data_ptr(), stream.cuda_stream)
        ev1.record(stream)
        stream.synchronize()
        host = d_slots.cpu().tolist()
        ck.add(s, host, ev0.elapsed_time(ev1) / 1e3)
        if checkpoint:
            ck.save(checkpoint)
        slowest = max(slowest, time.monotonic() - t0)
        added += 1
    result = {"n": n, "P": P, "formula": formula, "guard_bits": guard_bits, "shards": shards,
              "done": len(ck.done), "added": added, "device_seconds": ck.seconds}
    if not ck.remaining():
        out = torch.zeros((P + 7) // 8, dtype=torch.uint8, device=f"cuda:{device}")
        valid = torch.zeros(1, dtype=torch.int32, device=f"cuda:{device}")
        bbp_finalize_async(plan.handle, formula, n, P, d_slots.data_ptr(), out.data_ptr(), valid.data_ptr(),
                           0, stream.cuda_stream)
        stream.synchronize()
        raw = bytes(out.cpu().tolist())
        bits = int.from_bytes(raw, "big") >> (8 * len(raw) - P)
        result.update({"bits_hex": f"{bits:0{(P + 3) // 4}X}", "valid_bits": int(valid.item())})
    return result


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, required=True, help="first bit position (1 = first bit after the point)")
    ap.add_argument("--P", type=int, default=256, help="bits wanted")
    ap.add_argument("--shards", type=int, default=64)
    ap.add_argument("--checkpoint", default="", help="JSON file read at start (if present) and rewritten per shard")
    ap.add_argument("--formula", type=int, default=0, help="0: Eq. 2 (Bellard), 1: Eq. 1 (BBP)")
    ap.add_argument("--guard-bits", type=int, default=64)
    ap.add_argument("--max-seconds", type=float, default=float("inf"),
                    help="stop before a shard that would end past this many seconds")
    ap.add_argument("--max-shards", type=int, default=-1, help="add at most this many shards in this run")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.n, a.P, a.shards, a.checkpoint, a.formula, a.guard_bits, a.max_seconds,
                         a.max_shards, a.device)), flush=True)


if __name__ == "__main__":
    main()
