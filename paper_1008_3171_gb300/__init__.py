"""Python binding of libbbp: BBP digit extraction of pi on one GB300 (sm_103a).

Argument marshalling only.  Every step of the computation runs in the CUDA
kernels of ``libbbp.so`` (built in-tree by ``build()``); there is no CPU
fallback, and importing this module fails loudly if the library is missing.

The functions mirror the C ABI in ``include/bbp.h`` (same names); ``Plan`` is a
small convenience wrapper around a ``bbp_plan`` handle.  Device buffers and
streams may come from PyTorch (``tensor.data_ptr()``, ``stream.cuda_stream``);
this module itself never imports torch.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbbp.so")

BBP_OK = 0
BBP_PENDING = 1
BBP_EINVAL = -1
BBP_ENOMEM = -2
BBP_ECUDA = -3
BBP_EBUSY = -4
BBP_ETIMEOUT = -5
BBP_ERANGE = -6
BBP_EINVALID_BITS = -7
BBP_ENOTFOUND = -8
BBP_ESCRATCH = -9

BBP_BELLARD = 0
BBP_BBP = 1
UINT64_MAX = (1 << 64) - 1


class BBPError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {bbp_status_str(status)} ({status})" if what else bbp_status_str(status))


class bbp_plan_opts(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("guard_bits", ctypes.c_uint32),
        ("accum_mem_budget", ctypes.c_size_t),
        ("max_slots", ctypes.c_uint32),
        ("tune_table", ctypes.c_char_p),
        ("profile", ctypes.c_uint32),
        ("strict", ctypes.c_uint32),
    ]


class bbp_serve_info(ctypes.Structure):
    _fields_ = [
        ("pending", ctypes.c_uint64),
        ("active", ctypes.c_uint64),
        ("slots", ctypes.c_uint64),
        ("iterations", ctypes.c_uint64),
        ("terms", ctypes.c_uint64),
        ("terms_per_s", ctypes.c_double),
    ]


class bbp_range(ctypes.Structure):
    _fields_ = [
        ("denominator", ctypes.c_uint32),
        ("tail", ctypes.c_uint32),
        ("path", ctypes.c_uint32),
        ("window", ctypes.c_uint32),
        ("first", ctypes.c_uint32),
        ("first_max", ctypes.c_uint32),
        ("k_begin", ctypes.c_uint64),
        ("count", ctypes.c_uint64),
        ("imad", ctypes.c_double),
    ]


class bbp_stats(ctypes.Structure):
    _fields_ = [
        ("terms", ctypes.c_uint64),
        ("head_terms", ctypes.c_uint64),
        ("head_launches", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
        ("imad_model", ctypes.c_double),
        ("head_ms", ctypes.c_double),
    ]


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile libbbp.so for sm_103a in-tree (nvcc; needs no GPU)."""
    from . import _build

    return _build.build(verbose=verbose, force=force)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libbbp.so not found at {LIB_PATH}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "bbp_abi_version": ([], u32),
        "bbp_status_str": ([ctypes.c_int], ctypes.c_char_p),
        "bbp_plan_opts_default": ([ctypes.POINTER(bbp_plan_opts)], None),
        "bbp_plan_create": ([ctypes.POINTER(vp), ctypes.POINTER(bbp_plan_opts)], ctypes.c_int),
        "bbp_plan_destroy": ([vp], ctypes.c_int),
        "bbp_working_bits": ([vp, u32], u32),
        "bbp_series_extent": ([ctypes.c_int, u32, u64, u32, u64p, u64p], ctypes.c_int),
        "bbp_partial_sum": ([vp, ctypes.c_int, u32, u64, u64, u64, u32, u32p], ctypes.c_int),
        "bbp_partial_sum_async": ([vp, ctypes.c_int, u32, u64, u64, u64, u32, vp, vp], ctypes.c_int),
        "bbp_bits": ([vp, u64, u32, ctypes.c_char_p, u32p], ctypes.c_int),
        "bbp_bits_formula": ([vp, ctypes.c_int, u64, u32, ctypes.c_char_p, u32p], ctypes.c_int),
        "bbp_bits_async": ([vp, ctypes.c_int, u64, u32, vp, vp, vp, vp], ctypes.c_int),
        "bbp_plan_stats": ([vp, ctypes.POINTER(bbp_stats)], ctypes.c_int),
        "bbp_shard_range": ([ctypes.c_int, u32, u64, u32, u32, u32, u64p, u64p], ctypes.c_int),
        "bbp_explain": ([ctypes.c_int, u64, u32, u32, u32, ctypes.POINTER(bbp_range), u32, u32p, u64p],
                        ctypes.c_int),
        "bbp_accumulate_async": ([vp, ctypes.c_int, u64, u32, u32, u32, vp, vp], ctypes.c_int),
        "bbp_finalize_async": ([vp, ctypes.c_int, u64, u32, vp, vp, vp, vp, vp], ctypes.c_int),
        "bbp_imad_probe": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bbp_partial_sum_noalloc": ([ctypes.c_int, u32, u64, u64, u64, u32, u32, vp, vp], ctypes.c_int),
        "bbp_bits_batch": ([vp, ctypes.c_int, u32, u64p, u32p, ctypes.c_char_p, u32, u32p,
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bbp_submit": ([vp, u64, u32, u64p], ctypes.c_int),
        "bbp_poll": ([vp, u64, ctypes.c_char_p, u32p], ctypes.c_int),
        "bbp_serve_stats": ([vp, ctypes.POINTER(bbp_serve_info)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _check(status: int, what: str) -> int:
    if status < 0:
        raise BBPError(status, what)
    return status


# ---------------------------------------------------------------- ABI-named functions

def bbp_abi_version() -> int:
    return _lib.bbp_abi_version()


def bbp_status_str(status: int) -> str:
    return _lib.bbp_status_str(status).decode()


def bbp_plan_opts_default() -> dict:
    """The library's default plan options (host-only; no GPU)."""
    opts = bbp_plan_opts()
    _lib.bbp_plan_opts_default(ctypes.byref(opts))
    return {f: getattr(opts, f) for f, _ in bbp_plan_opts._fields_}


def bbp_plan_create(device: int = 0, stream: Optional[int] = None, guard_bits: int = 64,
                    accum_mem_budget: int = 0, max_slots: int = 0, tune_table: Optional[str] = None,
                    profile: bool = False, strict: bool = False) -> int:
    opts = bbp_plan_opts()
    _lib.bbp_plan_opts_default(ctypes.byref(opts))
    opts.device = device
    opts.stream = stream or None
    opts.guard_bits = guard_bits
    opts.accum_mem_budget = accum_mem_budget
    opts.max_slots = max_slots
    opts.tune_table = tune_table.encode() if tune_table else None
    opts.profile = 1 if profile else 0
    opts.strict = 1 if strict else 0
    handle = ctypes.c_void_p()
    _check(_lib.bbp_plan_create(ctypes.byref(handle), ctypes.byref(opts)), "bbp_plan_create")
    return handle.value


def bbp_plan_destroy(plan: int) -> None:
    _check(_lib.bbp_plan_destroy(plan), "bbp_plan_destroy")


def bbp_working_bits(plan: int, P: int) -> int:
    return _lib.bbp_working_bits(plan, P)


def bbp_series_extent(formula: int, denominator: int, n: int, W: int) -> tuple[int, int]:
    he, ne = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.bbp_series_extent(formula, denominator, n, W, ctypes.byref(he), ctypes.byref(ne)),
           "bbp_series_extent")
    return he.value, ne.value


def bbp_partial_sum(plan: int, formula: int, denominator: int, k_begin: int, k_end: Optional[int],
                    n: int, P: int) -> list[int]:
    """W/32 little-endian limbs of sign_j * sum_k (-1)^k t_{j,k} mod 2^W."""
    W = bbp_working_bits(plan, P)
    if W == 0:
        raise BBPError(BBP_EINVAL, "bbp_partial_sum")
    out = (ctypes.c_uint32 * (W // 32))()
    _check(_lib.bbp_partial_sum(plan, formula, denominator, k_begin, UINT64_MAX if k_end is None else k_end,
                                n, P, out), "bbp_partial_sum")
    return list(out)


def bbp_partial_sum_async(plan: int, formula: int, denominator: int, k_begin: int, k_end: Optional[int],
                          n: int, P: int, d_out_limbs: int, stream: Optional[int] = None) -> None:
    _check(_lib.bbp_partial_sum_async(plan, formula, denominator, k_begin,
                                      UINT64_MAX if k_end is None else k_end, n, P, d_out_limbs, stream or None),
           "bbp_partial_sum_async")


def bbp_bits_formula(plan: int, formula: int, n: int, P: int) -> tuple[bytes, int]:
    """(ceil(P/8) MSB-first bytes of bits n..n+P-1, certified bit count)."""
    out = ctypes.create_string_buffer((P + 7) // 8)
    valid = ctypes.c_uint32()
    st = _lib.bbp_bits_formula(plan, formula, n, P, out, ctypes.byref(valid))
    if st == BBP_EINVALID_BITS:
        raise BBPError(st, f"bbp_bits_formula (certified {valid.value} of {P})")
    _check(st, "bbp_bits_formula")
    return out.raw, valid.value


def bbp_bits(plan: int, n: int, P: int) -> tuple[bytes, int]:
    return bbp_bits_formula(plan, BBP_BELLARD, n, P)


def bbp_bits_async(plan: int, formula: int, n: int, P: int, d_out: int, d_valid: int = 0, d_limbs: int = 0,
                   stream: Optional[int] = None) -> None:
    _check(_lib.bbp_bits_async(plan, formula, n, P, d_out, d_valid or None, d_limbs or None, stream or None),
           "bbp_bits_async")


def bbp_shard_range(formula: int, denominator: int, n: int, W: int, shard: int, nshards: int) -> tuple[int, int]:
    kb, ke = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.bbp_shard_range(formula, denominator, n, W, shard, nshards, ctypes.byref(kb), ctypes.byref(ke)),
           "bbp_shard_range")
    return kb.value, ke.value


def bbp_explain(formula: int, n: int, P: int, guard_bits: int = 64, wide_min_bits: int = 32) -> tuple[list, int]:
    """Host-only launch plan of a query: (ranges as dicts, terms covered).  No GPU."""
    count = ctypes.c_uint32()
    terms = ctypes.c_uint64()
    _check(_lib.bbp_explain(formula, n, P, guard_bits, wide_min_bits, None, 0, ctypes.byref(count), None),
           "bbp_explain")
    buf = (bbp_range * max(count.value, 1))()
    _check(_lib.bbp_explain(formula, n, P, guard_bits, wide_min_bits, buf, count.value, ctypes.byref(count),
                            ctypes.byref(terms)), "bbp_explain")
    names = [f for f, _ in bbp_range._fields_]
    return [{f: getattr(buf[i], f) for f in names} for i in range(count.value)], terms.value


def bbp_accumulate_async(plan: int, formula: int, n: int, P: int, shard: int, nshards: int, d_slots: int,
                         stream: Optional[int] = None) -> None:
    _check(_lib.bbp_accumulate_async(plan, formula, n, P, shard, nshards, d_slots, stream or None),
           "bbp_accumulate_async")


def bbp_finalize_async(plan: int, formula: int, n: int, P: int, d_slots: int, d_out: int, d_valid: int = 0,
                       d_limbs: int = 0, stream: Optional[int] = None) -> None:
    _check(_lib.bbp_finalize_async(plan, formula, n, P, d_slots, d_out, d_valid or None, d_limbs or None,
                                   stream or None), "bbp_finalize_async")


def bbp_bits_batch(plan: int, formula: int, ns, Ps, with_latency: bool = True):
    """Batched queries in one persistent pass.  Returns (values, valid, latency_ms):
    values[q] is the P[q] bits of query q as an integer (MSB = bit n[q])."""
    count = len(ns)
    if len(Ps) != count:
        raise ValueError("ns and Ps differ in length")
    stride = max(((int(P) + 7) // 8 for P in Ps), default=1)
    n_arr = (ctypes.c_uint64 * max(count, 1))(*[int(v) for v in ns])
    p_arr = (ctypes.c_uint32 * max(count, 1))(*[int(v) for v in Ps])
    out = ctypes.create_string_buffer(max(count, 1) * stride)
    valid = (ctypes.c_uint32 * max(count, 1))()
    lat = (ctypes.c_double * max(count, 1))()
    st = _lib.bbp_bits_batch(plan, formula, count, n_arr, p_arr, out, stride, valid, lat if with_latency else None)
    if st != BBP_EINVALID_BITS:
        _check(st, "bbp_bits_batch")
    raw = out.raw
    values = []
    for q in range(count):
        P = int(Ps[q])
        nb = (P + 7) // 8
        values.append(int.from_bytes(raw[q * stride:q * stride + nb], "big") >> (8 * nb - P))
    result = (values, list(valid)[:count], list(lat)[:count] if with_latency else None)
    if st == BBP_EINVALID_BITS:
        raise BBPError(st, "bbp_bits_batch")
    return result


def bbp_submit(plan: int, n: int, P: int) -> Optional[int]:
    """Ticket of the queued query, or None when the engine is busy (BBP_EBUSY)."""
    t = ctypes.c_uint64()
    st = _lib.bbp_submit(plan, n, P, ctypes.byref(t))
    if st == BBP_EBUSY:
        return None
    _check(st, "bbp_submit")
    return t.value


def bbp_poll(plan: int, ticket: int, P: int) -> Optional[tuple[int, int]]:
    """None while pending; else (the P bits as an integer, certified bit count)."""
    out = ctypes.create_string_buffer((P + 7) // 8)
    valid = ctypes.c_uint32()
    st = _lib.bbp_poll(plan, ticket, out, ctypes.byref(valid))
    if st == BBP_PENDING:
        return None
    _check(st, "bbp_poll")
    return int.from_bytes(out.raw, "big") >> (8 * len(out.raw) - P), valid.value


def bbp_serve_stats(plan: int) -> dict:
    info = bbp_serve_info()
    _check(_lib.bbp_serve_stats(plan, ctypes.byref(info)), "bbp_serve_stats")
    return {name: getattr(info, name) for name, _ in bbp_serve_info._fields_}


def bbp_plan_stats(plan: int) -> dict:
    st = bbp_stats()
    _check(_lib.bbp_plan_stats(plan, ctypes.byref(st)), "bbp_plan_stats")
    return {name: getattr(st, name) for name, _ in bbp_stats._fields_}


def bbp_imad_probe(plan: int, kind: int) -> float:
    v = ctypes.c_double()
    _check(_lib.bbp_imad_probe(plan, kind, ctypes.byref(v)), "bbp_imad_probe")
    return v.value


def bbp_partial_sum_noalloc(formula: int, denominator: int, k_begin: int, k_end: Optional[int], n: int, P: int,
                            guard_bits: int, d_out_limbs: int, stream: Optional[int] = None) -> None:
    """Partial sum without a plan and without any allocation, for callers that may
    not allocate device memory once running (pooled or fixed GPU memory budgets,
    loops that cannot afford cudaMalloc's synchronization).  Writes W/32 limbs to
    the caller's device buffer on the current device; asynchronous on `stream`.
    Calls on one device share a fixed 320-byte scratch array, so overlapping calls
    race; the first call on a device should come before any stream capture."""
    _check(_lib.bbp_partial_sum_noalloc(formula, denominator, k_begin, UINT64_MAX if k_end is None else k_end,
                                        n, P, guard_bits, d_out_limbs, stream or None), "bbp_partial_sum_noalloc")


# ---------------------------------------------------------------- convenience wrapper

def limbs_to_int(limbs) -> int:
    return sum(int(v) << (32 * i) for i, v in enumerate(limbs))


class Plan:
    """Owns one bbp_plan handle (closed on ``close()`` or garbage collection)."""

    def __init__(self, **opts):
        self.handle = bbp_plan_create(**opts)

    def close(self) -> None:
        if self.handle:
            bbp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def working_bits(self, P: int) -> int:
        return bbp_working_bits(self.handle, P)

    def partial_sum(self, formula: int, denominator: int, k_begin: int, k_end: Optional[int], n: int,
                    P: int) -> int:
        return limbs_to_int(bbp_partial_sum(self.handle, formula, denominator, k_begin, k_end, n, P))

    def bits(self, n: int, P: int, formula: int = BBP_BELLARD) -> tuple[int, int]:
        """(the P bits as an integer, MSB = bit n; certified bit count)."""
        raw, valid = bbp_bits_formula(self.handle, formula, n, P)
        return int.from_bytes(raw, "big") >> (8 * len(raw) - P), valid

    def stats(self) -> dict:
        return bbp_plan_stats(self.handle)

    def imad_probe(self, kind: int) -> float:
        return bbp_imad_probe(self.handle, kind)
