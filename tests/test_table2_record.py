"""The committed record of Table 2 rows computed on the GPU (profiles/table2_rows.json)
against the paper's printed rows: every recorded bit string must equal the first P
bits of the row at its position, with all P bits certified.  The expectation is
the paper's text (tests/golden/paper_pins.json), not a GPU output."""

import json
import os

from conftest import ROOT


def test_recorded_rows_equal_the_paper(pins):
    with open(os.path.join(ROOT, "profiles", "table2_rows.json")) as fh:
        rows = json.load(fh)["rows"]
    assert rows
    by_n = {p["n"]: p for p in pins.values() if p["name"].startswith("table2_")}
    for r in rows:
        pin = by_n[r["n"]]
        P = r["P"]
        ref = int(pin["hex"], 16) >> (4 * len(pin["hex"]) - pin["bits"])
        assert P <= pin["bits"]
        assert r["valid_bits"] == P
        assert int(r["bits_hex"], 16) == ref >> (pin["bits"] - P), r["row"]
        assert r["device_seconds"] > 0 and r["terms"] > 0
