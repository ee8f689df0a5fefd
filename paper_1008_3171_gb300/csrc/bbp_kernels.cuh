// Kernel argument blocks and host-side launch wrappers shared by the runtime.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bbp {

// One contiguous run of head terms (exponent e >= 0) of one series:
// k in [k_begin, k_begin + count), m = a k + b, e = d + c - step k.
struct HeadArgs {
  uint64_t d;            // n - 1
  uint64_t k_begin;      // first term index
  uint64_t count;        // number of terms (> 0)
  uint32_t a, b;         // modulus m = a k + b (odd)
  int32_t c;             // exponent offset of the series
  uint32_t step;         // exponent decrease per k (10 or 4)
  uint32_t W;            // working bits, 32 L
  uint32_t L;            // limbs
  uint32_t alternating;  // 1 if the series carries (-1)^k
  uint32_t negate;       // 1 if this run's partial enters the sum negated
  uint32_t run;          // consecutive terms per stream (even)
  uint32_t window;       // ladder window bits (>= 1)
  uint32_t first;        // bits taken by the first window (0 allowed)
  uint32_t first_max;    // largest first-window value the moduli allow (>= 2^first - 1); a warp
                         // whose top first + 1 exponent bits stay within it takes one more bit
  unsigned long long* slots;  // L carry-save accumulators, limb i at slots[i]
};

// Tail terms (e < 0): t = floor(2^(W+e) / m), one thread per term.
struct TailArgs {
  uint64_t d;
  uint64_t k_begin;
  uint64_t count;
  uint32_t a, b;
  int32_t c;
  uint32_t step;
  uint32_t W;
  uint32_t L;
  uint32_t alternating;
  uint32_t negate;
  unsigned long long* slots;
};

// The tail ranges of up to kMaxTailSet series, launched together (tail terms are
// few: about W / step per series).
constexpr int kMaxTailSet = 7;
struct TailSet {
  TailArgs a[kMaxTailSet];
  uint32_t n;  // ranges in use
};

constexpr int kMaxLimbs = 40;    // W <= 1280 bits
constexpr int kHeadThreads = 256;
// Compiled accumulator capacities (limbs per thread) of the head and queue
// kernels; a query with W/32 limbs uses the smallest class that holds them.
constexpr int kLmaxClasses[] = {3, 4, 6, 10, 16, 24, 40};
constexpr int kNumLmaxClasses = static_cast<int>(sizeof(kLmaxClasses) / sizeof(kLmaxClasses[0]));
// Modulus paths: 0 one word, lazy residues (bitlen(m) <= 29); 1 two words, three-word
// square (bitlen <= 46); 2 two words, four-word square (bitlen <= 60); 3 one word,
// fully reduced residues (bitlen 30 or 31).
constexpr int kNumPaths = 4;
constexpr int kQueueVariants = kNumLmaxClasses * kNumPaths;  // limb class x modulus path

// ---------------------------------------------------------------- batches
//
// A batch of queries is a list of jobs: head jobs (one HeadArgs each: a range of
// head terms of one series of one query, whose `slots` point at that query's
// accumulators) grouped by kernel variant, plus tail jobs.  Persistent warps hand
// out `grab` tiles of the current job at a time; the warp that finishes a query's
// last job finalizes the query.
struct QueryDesc {
  uint64_t bound;       // N + J + 1: |S - exact| < bound units
  uint32_t P;           // output bits
  uint32_t L;           // limbs of the working precision
  uint32_t out_offset;  // byte offset of the query's output bits in `out`
  uint32_t pad;
};

struct BatchDev {
  const HeadArgs* jobs;            // head jobs, grouped by kernel variant
  const uint32_t* job_query;       // query index of each head job
  const uint64_t* job_tiles;       // warp tiles of each head job
  unsigned long long* job_taken;   // tiles handed out so far (atomic)
  unsigned long long* job_done;    // tiles finished so far (atomic)
  const TailArgs* tails;           // tail jobs
  const uint32_t* tail_query;
  uint32_t grab;                   // tiles per hand-out
  const QueryDesc* queries;
  unsigned long long* accum;       // kMaxLimbs carry-save accumulators per query
  unsigned int* jobs_left;         // unfinished jobs (head + tail) per query (atomic)
  uint8_t* out;                    // output bits of every query
  uint32_t* valid;                 // certified bit count per query
  unsigned long long* done_ns;     // completion time per query (device global timer, ns)
};

// Launch helpers (defined in bbp_kernels.cu).  They return cudaGetLastError().
// path: 0 = one-word moduli, bitlen <= 29; 1 = two-word moduli, bitlen <= 46;
//       2 = two-word moduli, bitlen <= 60; 3 = one-word moduli of 30 or 31 bits.
// threads: CTA size, a multiple of 32 in [32, kHeadThreads] (else cudaErrorInvalidValue).
cudaError_t launch_head(const HeadArgs& a, int path, int streams, int lmax, int blocks, cudaStream_t s,
                        int threads = kHeadThreads);
cudaError_t launch_tail(const TailArgs& a, cudaStream_t s);
cudaError_t launch_tail_set(const TailSet& set, cudaStream_t s);
cudaError_t launch_zero_slots(unsigned long long* slots, int L, cudaStream_t s);
cudaError_t launch_fold_limbs(const unsigned long long* slots, int L, uint32_t* out_limbs, cudaStream_t s);
cudaError_t launch_finalize_bits(const unsigned long long* slots, int L, uint32_t P, uint64_t bound,
                                 uint8_t* out_bytes, uint32_t* valid_bits, uint32_t* out_limbs, cudaStream_t s);
// One persistent launch over the head jobs [job_begin, job_end) of one variant;
// *cursor (relative to job_begin) must be 0.  blocks = resident CTAs.
cudaError_t launch_queue(const BatchDev& b, uint32_t job_begin, uint32_t job_end, unsigned int* cursor, int path,
                         int streams, int lmax, int blocks, cudaStream_t s);
// Tail jobs [tail_begin, tail_end); *cursor (relative to tail_begin) must be 0.
cudaError_t launch_queue_tail(const BatchDev& b, uint32_t tail_begin, uint32_t tail_end, unsigned int* cursor,
                              int blocks, cudaStream_t s);
cudaError_t launch_timestamp(unsigned long long* where, cudaStream_t s);
int queue_occupancy(int path, int streams, int lmax);
// Smallest compiled limb capacity >= L (bump > 0: that many classes larger, capped at
// the largest), or 0 when L exceeds every class.
int head_lmax_for(int L, int bump = 0);
// Resident CTAs per SM of that instantiation at `threads` per CTA.
int head_occupancy(int path, int streams, int lmax, int threads = kHeadThreads);
// Per accumulator class (bbp_lmax*.cu): the launchers the dispatchers above call.
#define BBP_DECLARE_LMAX(L)                                                                                    \
  cudaError_t launch_head_l##L(const HeadArgs& a, int path, int streams, int blocks, int threads, cudaStream_t s); \
  int head_occupancy_l##L(int path, int streams, int threads);                                                 \
  cudaError_t launch_queue_l##L(const BatchDev& b, uint32_t jb, uint32_t je, unsigned int* cursor, int path,      \
                                int streams, int blocks, cudaStream_t s);                                      \
  int queue_occupancy_l##L(int path, int streams);
BBP_DECLARE_LMAX(3)
BBP_DECLARE_LMAX(4)
BBP_DECLARE_LMAX(6)
BBP_DECLARE_LMAX(10)
BBP_DECLARE_LMAX(16)
BBP_DECLARE_LMAX(24)
BBP_DECLARE_LMAX(40)
#undef BBP_DECLARE_LMAX

cudaError_t launch_imad_probe(int kind, int blocks, int threads, int iters, unsigned long long* cycles_out,
                              uint32_t* smid_out, uint32_t* sink, cudaStream_t s);

}  // namespace bbp
