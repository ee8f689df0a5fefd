"""The boundary is a C ABI: include/bbp.h compiles as strict C99 and as C++17
without warnings, and a plain C program links against libbbp.so and calls the
host-only entry points (no GPU): version, status strings, default options,
series extents, shard ranges and a launch plan."""

import importlib.util
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

PROGRAM = r"""
#include <stdio.h>
#include <inttypes.h>
#include "bbp.h"

int main(void) {
  bbp_plan_opts o;
  uint64_t he = 0, ne = 0, kb = 0, ke = 0, terms = 0;
  uint32_t count = 0;
  bbp_range r[64];
  bbp_plan_opts_default(&o);
  printf("version %u %u\n", bbp_abi_version(), (unsigned)BBP_ABI_VERSION);
  printf("status %s|%s\n", bbp_status_str(BBP_EBUSY), bbp_status_str(BBP_ERANGE));
  printf("opts %u %d\n", o.guard_bits, o.device);
  int st;
  /* each call before the printf that reads its outputs (argument order is unspecified) */
  st = (int)bbp_series_extent(BBP_BELLARD, 0, 1000000, 96, &he, &ne);
  printf("extent %d %" PRIu64 " %" PRIu64 "\n", st, he, ne);
  st = (int)bbp_shard_range(BBP_BELLARD, 5, 1000000000, 192, 1, 4, &kb, &ke);
  printf("shard %d %" PRIu64 " %" PRIu64 "\n", st, kb, ke);
  st = (int)bbp_explain(BBP_BELLARD, 1000000000000ull, 256, 64, 30, r, 64, &count, &terms);
  printf("explain %d %u %" PRIu64 "\n", st, count, terms);
  printf("einval %d\n", (int)bbp_explain(BBP_BELLARD, 0, 256, 64, 30, r, 64, &count, &terms));
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    spec = importlib.util.spec_from_file_location("_bbp_build", os.path.join(ROOT, "paper_1008_3171_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_header_is_c99_and_cxx17_clean(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "bbp.h"\nint main(void) { return bbp_abi_version() == BBP_ABI_VERSION ? 0 : 1; }\n')
    inc = os.path.join(ROOT, "include")
    for cmd in (["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror"],
                ["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-x", "c++"]):
        r = subprocess.run(cmd + ["-I", inc, "-c", str(src), "-o", str(tmp_path / "h.o")], capture_output=True,
                           text=True)
        assert r.returncode == 0, r.stderr


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_c_program_links_and_calls_host_entry_points(tmp_path, lib):
    src = tmp_path / "prog.c"
    src.write_text(PROGRAM)
    libdir = os.path.dirname(lib)
    exe = tmp_path / "prog"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lbbp", f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    got = dict(l.split(" ", 1) for l in out.stdout.strip().splitlines())
    v_lib, v_hdr = got["version"].split()
    assert v_lib == v_hdr
    busy, erange = got["status"].split("|")
    assert busy and erange and busy != erange
    assert got["opts"].split()[0] == "64"
    st, he, ne = map(int, got["extent"].split())
    from oracle import bbp_oracle as o1

    s = o1.BELLARD.series[0]
    assert st == 0 and he == o1.head_end(o1.BELLARD, s, 10**6 - 1) and ne == o1.natural_end(o1.BELLARD, s, 10**6 - 1, 96)
    st, kb, ke = map(int, got["shard"].split())
    assert st == 0 and 0 < kb < ke
    st, count, terms = map(int, got["explain"].split())
    assert st == 0 and count == 49 and terms == 700_000_000_195
    assert int(got["einval"]) == -1
