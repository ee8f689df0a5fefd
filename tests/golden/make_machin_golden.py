"""Writes tests/golden/machin_bits.json: pi bits from Machin's formula (oracle O3)
at the positions the tests use but cannot afford to recompute every run.

Calls only oracle/ (no CUDA code).  Run: python tests/golden/make_machin_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import machin  # noqa: E402

WINDOWS = [(999_937, 256), (1_000_000, 256), (1_000_001, 256)]


def main():
    F = max(n - 1 + P for n, P in WINDOWS) + 128
    out = []
    for n, P in WINDOWS:
        v = machin.pi_bits(n, P, F=F)
        out.append({"n": n, "bits": P, "hex": format(v, "0{}X".format(P // 4))})
    with open(os.path.join(HERE, "machin_bits.json"), "w") as fh:
        json.dump({"source": "oracle/machin.py (Machin's arctangent formula), F = %d" % F,
                   "windows": out}, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
