"""Oracles for BBP digit extraction of pi (Sze, arXiv:1008.3171, Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or run anything in this
package.  The CUDA library and its Python binding never do, and nothing here
imports them: the two sides share no code.

* O1 ``bbp_oracle``  -- the definition in plain Python integers (slow, exact).
* O2 ``bbp_oracle.c`` -- the same definition in plain C with 128-bit integers and
  POSIX threads, loaded through ctypes; used for larger n and as the timed CPU
  baseline.
* O3 ``machin``      -- pi bits from Machin's arctangent formula, an independent
  method used to pin O1 and O2.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

from . import bbp_oracle, machin  # noqa: F401
from .bbp_oracle import BBP, BELLARD, FORMULAS, working_bits  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbp_oracle.c")
_LIB = os.path.join(_HERE, "_bbp_oracle_c.so")
_lock = threading.Lock()
_lib = None

UINT64_MAX = (1 << 64) - 1


def build_c_oracle(force: bool = False) -> str:
    """Compile O2 with the host C compiler (plain -O2, no machine-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


def c_oracle():
    """The loaded O2 library (compiled on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_c_oracle())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.bbp_oracle_partial_sum.argtypes = [
                ctypes.c_int, ctypes.c_uint, ctypes.c_uint64, ctypes.c_uint64,
                ctypes.c_uint64, ctypes.c_uint, u32p, ctypes.c_uint,
            ]
            lib.bbp_oracle_partial_sum.restype = ctypes.c_int
            lib.bbp_oracle_accumulate.argtypes = [
                ctypes.c_int, ctypes.c_uint64, ctypes.c_uint, u32p,
                ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint,
            ]
            lib.bbp_oracle_accumulate.restype = ctypes.c_int
            lib.bbp_oracle_natural_end.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_uint64, ctypes.c_uint]
            lib.bbp_oracle_natural_end.restype = ctypes.c_uint64
            lib.bbp_oracle_head_end.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_uint64]
            lib.bbp_oracle_head_end.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _formula_id(formula) -> int:
    if formula in (0, "bellard", BELLARD):
        return 0
    if formula in (1, "bbp", BBP):
        return 1
    raise ValueError(f"unknown formula {formula!r}")


def c_partial_sum(formula, j: int, k_begin: int, k_end: int | None, n: int, P: int, G: int,
                  threads: int = 0) -> int:
    """O2 version of ``bbp_oracle.partial_sum`` (same arguments, same result)."""
    W = working_bits(P, G)
    out = (ctypes.c_uint32 * (W // 32))()
    st = c_oracle().bbp_oracle_partial_sum(
        _formula_id(formula), j, k_begin, UINT64_MAX if k_end is None else k_end, n, W, out, threads)
    if st != 0:
        raise RuntimeError(f"C oracle status {st}")
    return bbp_oracle.from_limbs(out)


def c_accumulate(formula, n: int, P: int, G: int, threads: int = 0) -> tuple[int, int]:
    """O2 version of ``bbp_oracle.accumulate``: (S, N)."""
    W = working_bits(P, G)
    out = (ctypes.c_uint32 * (W // 32))()
    nt = ctypes.c_uint64(0)
    st = c_oracle().bbp_oracle_accumulate(_formula_id(formula), n, W, out, ctypes.byref(nt), threads)
    if st != 0:
        raise RuntimeError(f"C oracle status {st}")
    return bbp_oracle.from_limbs(out), nt.value


def c_bits(n: int, P: int, G: int = 64, formula="bellard", threads: int = 0) -> tuple[int, int]:
    """O2 version of ``bbp_oracle.bits``: (value of the P bits, certified count)."""
    f = FORMULAS[formula] if not isinstance(formula, bbp_oracle.Formula) else formula
    W = working_bits(P, G)
    S, N = c_accumulate(f, n, P, G, threads)
    return S >> (W - P), bbp_oracle.certified_bits(S, W, P, bbp_oracle.error_bound(f, N))


def c_natural_end(formula, j: int, n: int, P: int, G: int) -> int:
    return c_oracle().bbp_oracle_natural_end(_formula_id(formula), j, n, working_bits(P, G))
