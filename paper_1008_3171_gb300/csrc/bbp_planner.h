// Host-side planning of a BBP query: which terms exist, how they split into
// kernel ranges, and what each range costs.  Pure C++, no CUDA.
#pragma once

#include <cstdint>
#include <vector>

namespace bbp {

struct SeriesDef {
  uint32_t a, b;  // modulus m = a k + b
  int32_t sign;   // +1 / -1 in front of the series
  int32_t c;      // exponent offset: the series term is 2^(d + c - step k) / m
};

struct FormulaDef {
  uint32_t step;         // exponent decrease per k
  uint32_t alternating;  // (-1)^k factor
  uint32_t count;        // number of series
  SeriesDef s[7];
};

// Eq. 2 (index 0) and Eq. 1 in the form of Eq. 3 (index 1).
const FormulaDef& formula_def(int f);

constexpr uint32_t kMaxWorkingBits = 1280;   // 40 limbs
constexpr int kWideMinBits = 32;             // moduli with bitlen >= 32 take a two-word path
constexpr int kLazyMaxBits = 29;             // one-word moduli up to this bitlen keep lazy residues (path 0)
// Lowest allowed crossover: moduli on the 64-bit path are >= 2^(kWideFloorBits-1) = 16,
// so floor(2^64 / m) * a (a <= 10), formed when R mod m is carried to the next k,
// stays below 2^64.
constexpr int kWideFloorBits = 5;
constexpr int kSmallMaxBits = 46;            // two-word path 1 (three-word square) up to this bitlen
constexpr int kMaxModulusBits = 60;          // 64-bit path bound
// The persistent queue kernels add one 32-bit partial sum per hand-out (at least
// one warp tile) to a query's 64-bit carry-save limbs; a query of fewer than this
// many head tiles (plus its few tail terms) keeps every limb's sum below 2^64.
constexpr uint64_t kMaxQueueTiles = (1ull << 32) - (1ull << 24);
// Queries of one batched pass, and serving slots: 2^24 keeps every query's 32-bit
// output byte offset (query index x 160 bytes) below 2^32.
constexpr uint32_t kMaxQueueQueries = 1u << 24;

// A contiguous run of terms of one series with one kernel configuration.
struct TermRange {
  uint32_t j;         // series index
  uint8_t tail;       // 0 head (e >= 0), 1 tail (e < 0)
  uint8_t path;       // head: 0 one word (bitlen <= 29), 1 two words (<= 46), 2 two words (<= 60),
                      //       3 one word, reduced residues (30, 31)
  uint8_t window;     // head: ladder window bits
  uint8_t first;      // head: first-window bits
  uint8_t first_max;  // head: largest first-window value the range's moduli allow
  uint64_t k_begin;   // first k
  uint64_t count;     // number of terms
  double imad;        // modelled multiply instructions for the range (head only)
};

int bitlen(uint64_t v);

// W = roundup(P, 32) + G; false when out of range.
bool working_bits(uint32_t P, uint32_t G, uint32_t* W);

// First k with exponent < 0 (Eq. 4 split) and the natural end of the tail.
uint64_t head_end(const FormulaDef& f, uint32_t j, uint64_t d);
uint64_t natural_end(const FormulaDef& f, uint32_t j, uint64_t d, uint32_t W);

// Kernel path for moduli of `lbits` bits: one-word Montgomery below
// `wide_min_bits` (path 0 up to kLazyMaxBits, path 3 for 30 and 31 bits), else a
// two-word path (1 up to kSmallMaxBits, 2 above).  wide_min_bits may be lowered from
// kWideMinBits down to kWideFloorBits (a tuning choice: small moduli on the two-word
// paths) but not raised.
int path_for_bits(int lbits, int wide_min_bits = kWideMinBits);

// Ladder parameters for moduli of at most `lbits` bits on the given path: the
// window bits, the first-window bits, and the largest first-window value w0 the
// first squaring allows (x = (R mod m) << w0 < m 2^w0 needs lbits + 2 w0 + 1 <= R's
// width); first_max >= 2^first - 1.
void window_params(int path, int lbits, uint8_t* window, uint8_t* first, uint8_t* first_max);

// Algorithmic work of one head term whose ladder exponent has nb bits, counted as
// 32-bit halves of 32x32-bit products (the low or high word of a product; a full
// 64-bit product counts 2).  Two-word moduli: per Montgomery squaring 5 (x0^2 and
// x0*2x1 in full, x1^2 low word; 6 when x1^2 needs its high word: every squaring
// of path 2 and the first squaring of path 1) plus per reduction step 4 (u = T0 m',
// high word of u m0, u m1 in full) twice; per quotient digit 4; plus 6 for
// m^-1 mod 2^32 (three lifting steps).  One-word moduli: 4 per squaring (x^2 in
// full, u, high word of u m), 2 per digit, 6 for the inverse.
double head_term_imad(int path, int nb, int first, int lmax);

// Shard `shard` of `nshards` of series j: the head [0, head_end) is cut evenly,
// the tail [head_end, natural_end) belongs to the last shard.
void shard_range(const FormulaDef& f, uint32_t j, uint64_t n, uint32_t W, uint32_t shard, uint32_t nshards,
                 uint64_t* k_begin, uint64_t* k_end);

// Appends the ranges of series j restricted to k in [k_lo, k_hi) (k_hi = UINT64_MAX:
// natural end).  Returns 0, or -6 (modulus too large) / -1 (bad argument, including
// wide_min_bits outside [kWideFloorBits, kWideMinBits]).
int plan_series(const FormulaDef& f, uint32_t j, uint64_t n, uint32_t W, uint32_t lmax, uint64_t k_lo,
                uint64_t k_hi, std::vector<TermRange>& out, int wide_min_bits = kWideMinBits);

}  // namespace bbp
