"""Corroborates a row the paper's author suppressed from the typeset Table 2
(rows m = 9..12 sit inside an ignored block of the source) by running oracle O2
at the same position, and records the outcome in
tests/golden/o2_suppressed_m9.json.

Calls only oracle/ (no CUDA code).  About 3-6 minutes on 8 cores:
    python tests/golden/corroborate_suppressed_row.py
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    with open(os.path.join(HERE, "paper_pins.json")) as fh:
        pin = {p["name"]: p for p in json.load(fh)["pins"]}["suppressed_m9"]
    n, P, G = pin["n"], pin["bits"], 64
    t0 = time.time()
    value, valid = oracle.c_bits(n, P, G, "bellard")
    secs = time.time() - t0
    paper = int(pin["hex"], 16) >> (4 * len(pin["hex"]) - P)
    agree = 0
    for b in range(valid, 0, -1):
        if value >> (P - b) == paper >> (P - b):
            agree = b
            break
    rec = {"n": n, "bits": P, "guard_bits": G, "certified_bits": valid,
           "hex": format(value, "0{}X".format((P + 3) // 4)),
           "leading_bits_equal_to_paper": agree, "seconds": round(secs, 1),
           "threads": os.cpu_count()}
    with open(os.path.join(HERE, "o2_suppressed_m9.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    print(rec)


if __name__ == "__main__":
    main()
