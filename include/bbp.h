/*
 * bbp.h -- C ABI of libbbp: BBP digit extraction of pi on one NVIDIA GB300 (sm_103a).
 *
 * The library evaluates Bellard's BBP-type series (Eq. 2 of Sze, "The Two
 * Quadrillionth Bit of pi is 0!", arXiv:1008.3171) -- or the original BBP series
 * (Eq. 1) -- to extract P bits of pi starting at binary position n, as exact
 * integer work on the GPU.  Sec. 3 (Eq. 3-5) defines the computation:
 *
 *   d = n - 1; {2^d pi} = { sum_j sign_j { sum_k (-1)^(alt k) 2^(d + c_j - step k) / (a_j k + b_j) } }
 *
 *   head terms (exponent e >= 0):  t = floor((2^e mod m) 2^W / m)
 *   tail terms (e < 0):            t = floor(2^(W+e) / m), up to the first zero
 *
 * summed as W-bit two's-complement fixed point (mod 2^W), W = roundup(P,32) + G.
 *
 * Conventions for every function below:
 *   - Bit positions count from 1 after the radix point (Sec. 2 footnote: the eight
 *     bits from position 9 are 0x3F).  n = 0 is invalid.
 *   - Limb arrays are little-endian uint32 (limb 0 least significant), W/32 limbs.
 *   - Output bit strings are MSB-first bytes: out[0] bit 7 is bit n; the unused low
 *     bits of the last byte are 0.
 *   - Every function returns a bbp_status; no C++ exception crosses the ABI.
 *   - A plan is not thread-safe: one host thread at a time per plan.
 *   - Buffers named h_* or without prefix are host memory owned by the caller;
 *     d_* are device memory on the plan's device owned by the caller.
 *   - Moduli must stay below 2^60: n up to about 1.1e18 (BBP_ERANGE beyond).
 */
#ifndef BBP_H
#define BBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BBP_ABI_VERSION 1u

typedef enum bbp_status {
  BBP_OK = 0,
  BBP_PENDING = 1,           /* bbp_poll: the query has not finished yet */
  BBP_EINVAL = -1,           /* bad argument (n = 0, P = 0, denominator out of range, ...) */
  BBP_ENOMEM = -2,           /* host or device allocation failed */
  BBP_ECUDA = -3,            /* a CUDA call failed; the plan should be destroyed */
  BBP_EBUSY = -4,            /* bbp_submit: no accumulator slot or memory free right now */
  BBP_ETIMEOUT = -5,         /* a bounded device-side wait gave up */
  BBP_ERANGE = -6,           /* n so large that a modulus would reach 2^60 */
  BBP_EINVALID_BITS = -7,    /* strict mode: fewer than P bits certified */
  BBP_ENOTFOUND = -8,        /* unknown ticket */
  BBP_ESCRATCH = -9          /* bbp_partial_sum_noalloc: W beyond its fixed scratch (1280 bits) */
} bbp_status;

/* Eq. 2 (Bellard, 7 series, step 10, alternating) or Eq. 1 (BBP, 4 series, step 4). */
typedef enum bbp_formula { BBP_BELLARD = 0, BBP_BBP = 1 } bbp_formula;

typedef struct bbp_plan_s* bbp_plan;

typedef struct bbp_plan_opts {
  int device;               /* CUDA device ordinal */
  void* stream;             /* cudaStream_t for all work; NULL: the plan creates its own (the legacy
                               default stream cannot be chosen: its handle is NULL too) */
  uint32_t guard_bits;      /* G: positive multiple of 32; 0 selects 64 */
  size_t accum_mem_budget;  /* bytes of device accumulator memory for queued queries; 0: 64 MiB */
  uint32_t max_slots;       /* concurrent queries admitted by bbp_submit; 0: 4096; at most 2^24 are used */
  const char* tune_table;   /* path of an autotune table or NULL for defaults.  JSON object; keys (others
                               ignored, out-of-range values keep the default): run (even, 2..4096, terms
                               per stream; 64), streams (1 or 2 term pairs per thread on every modulus
                               path; default 2 on moduli of 32 to 46 bits, 1 elsewhere), cta (head-kernel
                               threads per CTA, multiple of 32 up to 256; 256), limb_bump (0..2
                               accumulator classes above the smallest that holds W; 0), wide_min_bits
                               (5..32: moduli of at least this many bits use a two-limb Montgomery path;
                               32), grab (1..1024 warp tiles per queue operation in batched passes; 4).
                               None changes a result. */
  uint32_t profile;         /* 1: time head-kernel launches with CUDA events (see bbp_stats) */
  uint32_t strict;          /* 1: bbp_bits fails with BBP_EINVALID_BITS unless all P bits certify */
} bbp_plan_opts;

/* Counters of the most recent compute call on a plan. */
typedef struct bbp_stats {
  uint64_t terms;           /* terms evaluated (head + tail) */
  uint64_t head_terms;      /* head terms (modular exponentiations) */
  uint64_t head_launches;   /* head-kernel launches */
  uint64_t kernel_launches; /* all kernel launches */
  double imad_model;        /* 32-bit integer multiply instructions the head terms need (model) */
  double head_ms;           /* device time of the head launches (profile = 1), else 0 */
} bbp_stats;

/* ABI version of the loaded library; equals BBP_ABI_VERSION when headers match. */
uint32_t bbp_abi_version(void);

/* Static English text for a status code; never NULL. */
const char* bbp_status_str(bbp_status s);

/* Fills *opts with defaults (device 0, own stream, G = 64, no profiling). */
void bbp_plan_opts_default(bbp_plan_opts* opts);

/* Creates a plan on opts->device (NULL opts: defaults).  The plan owns its device
 * buffers and, if opts->stream is NULL, its stream.  Release with bbp_plan_destroy. */
bbp_status bbp_plan_create(bbp_plan* out, const bbp_plan_opts* opts);

/* Waits for the plan's stream, then frees everything the plan owns.  NULL is accepted. */
bbp_status bbp_plan_destroy(bbp_plan p);

/* W = roundup(P, 32) + G for the plan's guard bits G (host-only, no GPU work). */
uint32_t bbp_working_bits(bbp_plan p, uint32_t P);

/* Host-only extent of one series (Eq. 4): *head_end = first k with exponent < 0,
 * *natural_end = first tail k whose truncated term floor(2^(W+e)/m) is 0.
 * Needs no GPU.  EINVAL for n = 0, bad formula/denominator or W not a multiple of 32. */
bbp_status bbp_series_extent(bbp_formula f, uint32_t denominator, uint64_t n, uint32_t W,
                             uint64_t* head_end, uint64_t* natural_end);

/* Eq. 3-5, one series over one k-range:
 *   out_limbs = sign_j * sum_{k in [k_begin, min(k_end, natural_end))} (-1)^(alt k) t_{j,k}  (mod 2^W)
 * with W = bbp_working_bits(p, P).  k_end = UINT64_MAX means the natural end.
 * out_limbs: caller-owned host array of W/32 uint32.  Blocks until done.
 * EINVAL: n = 0, P = 0, denominator >= series count, k_begin > k_end. */
bbp_status bbp_partial_sum(bbp_plan p, bbp_formula f, uint32_t denominator, uint64_t k_begin,
                           uint64_t k_end, uint64_t n, uint32_t P, uint32_t* out_limbs);

/* As bbp_partial_sum, but writes W/32 limbs to device memory d_out_limbs and
 * returns once the work is queued on `stream` (NULL: the plan's stream). */
bbp_status bbp_partial_sum_async(bbp_plan p, bbp_formula f, uint32_t denominator, uint64_t k_begin,
                                 uint64_t k_end, uint64_t n, uint32_t P, uint32_t* d_out_limbs,
                                 void* stream);

/* Bits n .. n+P-1 of pi by Eq. 2.  out: caller-owned ceil(P/8) host bytes, MSB first.
 * valid_bits (may be NULL): how many leading bits the guard-bit error bound certifies
 * (|S - exact| < N + J + 1 units for N evaluated terms and J series).  Blocks. */
bbp_status bbp_bits(bbp_plan p, uint64_t n, uint32_t P, uint8_t* out, uint32_t* valid_bits);

/* bbp_bits with a choice of formula (Eq. 1 or Eq. 2). */
bbp_status bbp_bits_formula(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, uint8_t* out,
                            uint32_t* valid_bits);

/* Device-pointer form: d_out (ceil(P/8) bytes), d_valid (one uint32, may be NULL)
 * and d_limbs (W/32 uint32 of the raw sum, may be NULL) are caller-owned device
 * memory; returns once queued on `stream` (NULL: the plan's stream). */
bbp_status bbp_bits_async(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, uint8_t* d_out,
                          uint32_t* d_valid, uint32_t* d_limbs, void* stream);

/* Host-only split of series j's terms [0, natural_end) into nshards contiguous
 * shards: the head range is cut evenly, the tail goes to the last shard.
 * Writes shard `shard`'s range [*k_begin, *k_end).  Needs no GPU. */
bbp_status bbp_shard_range(bbp_formula f, uint32_t denominator, uint64_t n, uint32_t W, uint32_t shard,
                           uint32_t nshards, uint64_t* k_begin, uint64_t* k_end);

/* One launch range of a query plan (bbp_explain). */
typedef struct bbp_range {
  uint32_t denominator;  /* series index j */
  uint32_t tail;         /* 0: head terms (exponent >= 0, modular exponentiation), 1: tail terms */
  uint32_t path;         /* head: Montgomery arithmetic for the range's moduli: 0 one limb (32-bit), moduli
                            < 2^29; 3 one limb with fully reduced residues, 2^29 <= m < 2^31; 1 two limbs,
                            three-word square, m < 2^46; 2 two limbs, four-word square, m < 2^60 */
  uint32_t window;       /* head: ladder window bits (a window's multiplication is a shift) */
  uint32_t first;        /* head: bits taken by the first window (no squaring) */
  uint32_t first_max;    /* head: largest first-window value the range's moduli allow; a warp whose
                            exponents' top first + 1 bits stay within it takes that bit too */
  uint64_t k_begin;      /* first k */
  uint64_t count;        /* number of terms */
  double imad;           /* modelled 32-bit multiply halves of the range (head only; see bbp_stats) */
} bbp_range;

/* Host-only plan of the whole query at bit position n with P bits and guard_bits
 * guard bits (W = roundup(P, 32) + guard_bits): the launch ranges bbp_bits would
 * run, series by series in k order, with the moduli of at least wide_min_bits
 * bits (5..32; 32 is the default plan) on the two-limb paths.  Head terms with
 * modulus 1 (their value is 0) are not in any range.  Writes min(*count, cap)
 * ranges to `out` (caller-owned, may be NULL when cap = 0), sets *count to the
 * number of ranges and *terms (may be NULL) to the number of terms they cover.
 * Needs no GPU.  EINVAL: bad formula, n = 0, P = 0, guard_bits not a positive
 * multiple of 32, W > 1280, wide_min_bits outside 5..32; ERANGE: a modulus
 * would reach 2^60. */
bbp_status bbp_explain(bbp_formula f, uint64_t n, uint32_t P, uint32_t guard_bits, uint32_t wide_min_bits,
                       bbp_range* out, uint32_t cap, uint32_t* count, uint64_t* terms);

/* Adds shard `shard` of `nshards` of the whole query (every series, ranges from
 * bbp_shard_range) into caller-owned device carry-save accumulators
 * d_slots[0..W/32): limb i of the signed sum is added to d_slots[i] (uint64).
 * The caller zeroes d_slots once; the sum over all shards (added on one device,
 * or added limb-wise across devices, exact while fewer than 2^31 shards) is the
 * query's sum S mod 2^W in carry-save form.  Queued on `stream`; does not block.
 * This is also the checkpoint unit: slots saved after some shards resume by
 * adding the remaining shards. */
bbp_status bbp_accumulate_async(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, uint32_t shard,
                                uint32_t nshards, unsigned long long* d_slots, void* stream);

/* Turns carry-save accumulators holding a whole query's sum into output bits
 * (d_out, ceil(P/8) bytes), the certified count (d_valid, may be NULL) and the
 * raw sum (d_limbs, W/32 uint32, may be NULL); all caller-owned device memory. */
bbp_status bbp_finalize_async(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P,
                              const unsigned long long* d_slots, uint8_t* d_out, uint32_t* d_valid,
                              uint32_t* d_limbs, void* stream);

/* A batch of independent queries in one persistent pass.  The paper splits one
 * huge sum into jobs, tasks and threads (Sec. 4); here many queries of very
 * different sizes are split into jobs (one range of head terms of one series, or
 * one tail) that persistent warps consume a few warp tiles at a time from an
 * atomic queue, small queries first; each query's partial sums stay in its own
 * device accumulators and the warp that retires its last job finalizes it.  The
 * pass is captured in a CUDA graph and replayed.  Results are bit-identical to
 * bbp_bits_formula for each query.
 * n[count], P[count]: the queries (host arrays).  out: count * out_stride host
 * bytes, out_stride >= ceil(max P / 8); query q's bits at out + q * out_stride,
 * MSB first.  valid_bits[count] (may be NULL): certified bits.  latency_ms[count]
 * (may be NULL): device time from the start of the pass to each query's finalize.
 * Blocks until done.  EINVAL: a bad query, a too-small out_stride or count > 2^24.  ERANGE: a
 * modulus would reach 2^60, or a query needs 2^32 - 2^24 or more warp tiles (at the
 * default settings a tile is 4096 terms on moduli of 32 to 46 bits and 2048 terms
 * elsewhere: n above about 2.4e13), past which its 64-bit carry-save limbs could
 * overflow; run such a query with bbp_bits or bbp_accumulate_async. */
bbp_status bbp_bits_batch(bbp_plan p, bbp_formula f, uint32_t count, const uint64_t* n, const uint32_t* P,
                          uint8_t* out, uint32_t out_stride, uint32_t* valid_bits, double* latency_ms);

/* ---- serving: continuous batching of bit-position queries ----
 * An engine thread owned by the plan admits submitted queries into device
 * accumulator slots (at most min(max_slots, accum_mem_budget / 512 B) at once)
 * and runs short iterations; each iteration takes from every admitted query a
 * piece of its remaining terms (a fair share of an iteration budget sized from
 * the measured throughput), so long queries are sliced and queries that arrive
 * meanwhile join the next iteration.  Partial sums stay on the device between
 * iterations; the device finalizes a query in the iteration that runs its last
 * piece.  Results are bit-identical to bbp_bits.  bbp_submit/bbp_poll/
 * bbp_serve_stats may be called from any host thread.  (The paper's analogue is
 * its controller submitting small jobs into free cluster slots, Sec. 4.4.) */
typedef uint64_t bbp_ticket;

/* Queues the query (bits n .. n+P-1 by Eq. 2).  BBP_EBUSY: the wait queue is as
 * long as the slot pool; retry later.  EINVAL/ERANGE as bbp_bits, and ERANGE for
 * a query too large for the queue kernels' carry-save limbs (as bbp_bits_batch). */
bbp_status bbp_submit(bbp_plan p, uint64_t n, uint32_t P, bbp_ticket* t);

/* BBP_PENDING while the query runs; BBP_OK once done, then out (ceil(P/8) host
 * bytes, MSB first) and valid_bits (may be NULL) are filled and the ticket is
 * released; BBP_ENOTFOUND for an unknown or already collected ticket. */
bbp_status bbp_poll(bbp_plan p, bbp_ticket t, uint8_t* out, uint32_t* valid_bits);

typedef struct bbp_serve_info {
  uint64_t pending;      /* submitted, waiting for a slot */
  uint64_t active;       /* in slots, partly evaluated */
  uint64_t slots;        /* size of the slot pool */
  uint64_t iterations;   /* iterations run so far */
  uint64_t terms;        /* terms evaluated so far */
  double terms_per_s;    /* smoothed throughput of recent iterations */
} bbp_serve_info;

bbp_status bbp_serve_stats(bbp_plan p, bbp_serve_info* info);

/* Counters of the last compute call on this plan. */
bbp_status bbp_plan_stats(bbp_plan p, bbp_stats* out);

/* Issue-rate probe of the integer pipes, in 8 independent dependency chains per
 * thread (kind 0: mad.lo, the low half of a 32x32 product with an addend; 1: mad.hi;
 * 2: mad.wide, the full product with a 64-bit addend; 3: 32-bit add; 4: mul.hi;
 * 5: mul.wide without an addend, both halves used; 6: mul.wide followed by a
 * separate 64-bit add).  Runs one CTA of 1024 threads per SM and reports warp-lane
 * operations per SM clock (median over SMs).  EINVAL for another kind. */
bbp_status bbp_imad_probe(bbp_plan p, int kind, double* lanes_per_clk_per_sm);

/* No-allocation partial sum.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory once running -- code whose GPU
 * memory belongs to a pooling allocator it may not bypass, latency-bound loops that
 * cannot afford the device-wide synchronization of cudaMalloc/cudaFree, or plugins
 * with a fixed, preallocated budget.  Such callers cannot create a plan.
 *
 * Computes exactly what bbp_partial_sum_async computes for a plan with
 * guard_bits = G (same arguments, W = roundup(P,32) + G), on the calling thread's
 * current device, queued on `stream` (NULL: the legacy default stream); it does
 * not wait.  d_out_limbs: caller-owned device memory for W/32 uint32 limbs.
 * It calls no cudaMalloc, cudaFree or other allocating routine and needs no plan.
 *
 * Scratch: a fixed array of 40 uint64 carry-save accumulators (320 bytes) compiled
 * into the library, held by every GPU that loads it until the process exits, so
 * W is limited to 1280 bits: larger requests return BBP_ESCRATCH.  Every call on a
 * device uses the same array and zeroes it first; calls that overlap on the GPU
 * (other streams or threads) race on it and must be serialized by the caller.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture, and do not call
 * this entry point on a device after cudaDeviceReset of that device (the kept
 * address would belong to the context the reset destroyed).
 * Errors: BBP_EINVAL as bbp_partial_sum, BBP_ERANGE, BBP_ESCRATCH, BBP_ECUDA. */
bbp_status bbp_partial_sum_noalloc(bbp_formula f, uint32_t denominator, uint64_t k_begin, uint64_t k_end,
                                   uint64_t n, uint32_t P, uint32_t guard_bits, uint32_t* d_out_limbs,
                                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BBP_H */
