"""The C-ABI library loads and exports every function include/bbp.h declares,
and its host-only helpers agree with the oracle.  No GPU work is issued here."""

import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "bbp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(bbp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1008_3171_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bbp_plan_create", "bbp_plan_destroy", "bbp_partial_sum", "bbp_bits",
                     "bbp_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_exposes_abi_names(lib):
    import paper_1008_3171_gb300 as bbp

    for name in declared_functions():
        assert hasattr(bbp, name), name
    d = bbp.bbp_plan_opts_default()
    assert d["guard_bits"] == 64 and d["device"] == 0 and d["tune_table"] is None and d["strict"] == 0


def test_host_helpers(lib):
    import paper_1008_3171_gb300 as bbp

    assert bbp.bbp_abi_version() == 1
    assert bbp.bbp_status_str(bbp.BBP_ERANGE).startswith("position out of range")
    assert bbp.bbp_status_str(12345) == "unknown status"


def test_series_extent_matches_oracle(lib):
    import paper_1008_3171_gb300 as bbp
    from oracle import bbp_oracle as o1

    for fid, f in ((0, o1.BELLARD), (1, o1.BBP)):
        for n in (1, 2, 5, 9, 100, 12345, 10**6, 10**12 + 1, 2 * 10**15 - 3):
            for W in (64, 96, 320, 1088):
                for j, s in enumerate(f.series):
                    he, ne = bbp.bbp_series_extent(fid, j, n, W)
                    assert he == o1.head_end(f, s, n - 1)
                    assert ne == o1.natural_end(f, s, n - 1, W)


def test_series_extent_rejects_bad_arguments(lib):
    import paper_1008_3171_gb300 as bbp

    for args in ((0, 0, 0, 64), (0, 7, 10, 64), (1, 4, 10, 64), (0, 0, 10, 65), (2, 0, 10, 64)):
        with pytest.raises(bbp.BBPError) as e:
            bbp.bbp_series_extent(*args)
        assert e.value.status == bbp.BBP_EINVAL
