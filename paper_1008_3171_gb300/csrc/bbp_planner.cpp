// Host-side query planning for BBP digit extraction (Sze, arXiv:1008.3171, Sec. 3).
#include "bbp_planner.h"

#include <algorithm>
#include <limits>

namespace bbp {

namespace {
// Eq. 2: 2^2/(10k+1) - 1/(10k+3) - 2^-4/(10k+5) - 2^-4/(10k+7) + 2^-6/(10k+9)
//        - 2^-1/(4k+1) - 2^-6/(4k+3), times (-1)^k 2^-10k.
// Eq. 1 as in Eq. 3: 2^2/(8k+1) - 2^-1/(2k+1) - 1/(8k+5) - 2^-1/(4k+3), times 2^-4k.
const FormulaDef kFormulas[2] = {
    {10, 1, 7, {{10, 1, +1, 2}, {10, 3, -1, 0}, {10, 5, -1, -4}, {10, 7, -1, -4},
                {10, 9, +1, -6}, {4, 1, -1, -1}, {4, 3, -1, -6}}},
    {4, 0, 4, {{8, 1, +1, 2}, {2, 1, -1, -1}, {8, 5, -1, 0}, {4, 3, -1, -1}}},
};

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}

int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

// first k >= 0 with a k + b >= v
uint64_t first_k_at_least(uint64_t v, uint32_t a, uint32_t b) {
  if (v <= b) return 0;
  return (v - b + a - 1) / a;
}

constexpr uint64_t kMinRangeTerms = 1ull << 16;
}  // namespace

const FormulaDef& formula_def(int f) { return kFormulas[f == 1 ? 1 : 0]; }

int bitlen(uint64_t v) {
  int n = 0;
  while (v) { ++n; v >>= 1; }
  return n;
}

bool working_bits(uint32_t P, uint32_t G, uint32_t* W) {
  if (P == 0 || G == 0 || G % 32 != 0) return false;
  const uint64_t w = (static_cast<uint64_t>(P) + 31) / 32 * 32 + G;
  if (w > kMaxWorkingBits) return false;
  *W = static_cast<uint32_t>(w);
  return true;
}

uint64_t head_end(const FormulaDef& f, uint32_t j, uint64_t d) {
  const int64_t top = static_cast<int64_t>(d) + f.s[j].c;
  return top < 0 ? 0 : static_cast<uint64_t>(top) / f.step + 1;
}

uint64_t natural_end(const FormulaDef& f, uint32_t j, uint64_t d, uint32_t W) {
  const SeriesDef& s = f.s[j];
  for (uint64_t k = head_end(f, j, d);; ++k) {
    const int64_t p = static_cast<int64_t>(W) + static_cast<int64_t>(d) + s.c - static_cast<int64_t>(f.step * k);
    if (p < 0) return k;
    const uint64_t m = static_cast<uint64_t>(s.a) * k + s.b;
    if (p < 64 && (1ull << p) < m) return k;  // floor(2^p / m) == 0
  }
}

void window_params(int path, int lbits, uint8_t* window, uint8_t* first, uint8_t* first_max) {
  // A squaring with a window shift s keeps its result below 2m while
  //   path 0 (one word, lazy x < 2m):      lbits + s <= 30
  //   path 3 (one word, reduced x < m):    lbits + s <= 32
  //   paths 1, 2 (two words, lazy x < 2m): lbits + s <= 61
  // and s <= 2^window - 1.  The first window starts from x = (R mod m) << w0 < m 2^w0,
  // and the squaring after it (general routine on paths 1 and 2, shift at most one
  // bit) needs lbits + 2 w0 + 1 <= 32 (one word) / 64 (two words): w0 <= first_max.
  // `first` is the most bits whose every value fits (2^first - 1 <= first_max); the
  // kernel takes one bit more where the exponents' top bits happen to fit.
  const bool wide = path == 1 || path == 2;
  const int shift_cap = path == 0 ? 30 - lbits : path == 3 ? 32 - lbits : 61 - lbits;
  const int rbits = wide ? 64 : 32;
  int w = 0;
  while (w < 4 && (1 << (w + 1)) - 1 <= shift_cap) ++w;
  const int w0_max = std::max(0, (rbits - 1 - lbits) / 2);  // lbits + 2 w0 + 1 <= rbits
  int h = 0;
  while (h < 4 && (1 << (h + 1)) - 1 <= w0_max) ++h;
  *window = static_cast<uint8_t>(w);
  *first = static_cast<uint8_t>(h);
  *first_max = static_cast<uint8_t>(w0_max);
}

int path_for_bits(int lbits, int wide_min_bits) {
  if (lbits < std::min(wide_min_bits, kWideMinBits)) return lbits <= kLazyMaxBits ? 0 : 3;
  return lbits <= kSmallMaxBits ? 1 : 2;
}

double head_term_imad(int path, int nb, int first, int lmax) {
  const int h = nb > 0 ? std::min(first, nb - 1) : 0;
  const int sq = nb - h;
  if (path == 0 || path == 3) return 4.0 * sq + 2.0 * lmax + 6.0;
  if (path == 1) return 13.0 * sq + (sq > 0 ? 1.0 : 0.0) + 4.0 * lmax + 6.0;
  return 14.0 * sq + 4.0 * lmax + 6.0;
}

void shard_range(const FormulaDef& f, uint32_t j, uint64_t n, uint32_t W, uint32_t shard, uint32_t nshards,
                 uint64_t* k_begin, uint64_t* k_end) {
  const uint64_t he = head_end(f, j, n - 1);
  const uint64_t ne = natural_end(f, j, n - 1, W);
  // he * shard / nshards without overflow: he < 2^60, nshards < 2^32
  auto cut = [&](uint64_t i) -> uint64_t {
    const unsigned __int128 v = static_cast<unsigned __int128>(he) * i / nshards;
    return static_cast<uint64_t>(v);
  };
  *k_begin = cut(shard);
  *k_end = shard + 1 == nshards ? ne : cut(shard + 1);
}

namespace {
double range_imad(const FormulaDef& f, const SeriesDef& s, uint64_t d, uint32_t W, const TermRange& r, int lmax) {
  const int rb = (r.path == 1 || r.path == 2) ? 64 : 32;
  const int64_t v0 = static_cast<int64_t>(d) + s.c + static_cast<int64_t>(W) - rb;  // v at k = 0
  const int64_t k_lo = static_cast<int64_t>(r.k_begin);
  const int64_t k_hi = static_cast<int64_t>(r.k_begin + r.count) - 1;
  // terms with lo_v <= v0 - step k <= hi_v
  auto terms = [&](int64_t lo_v, int64_t hi_v) -> double {
    const int64_t ka = std::max(k_lo, ceil_div(v0 - hi_v, f.step));
    const int64_t kb = std::min(k_hi, floor_div(v0 - lo_v, f.step));
    return kb >= ka ? static_cast<double>(kb - ka + 1) : 0.0;
  };
  double total = 0;
  for (int i = 0; i < 64; ++i) {
    const int64_t lo_v = i == 0 ? 0 : (int64_t{1} << (i - 1));
    const int64_t hi_v = i == 0 ? 0 : (i == 63 ? std::numeric_limits<int64_t>::max() : (int64_t{1} << i) - 1);
    if (i >= r.first + 2 && i < 63) {
      // exponents whose top first + 1 bits are at most first_max take one more
      // first-window bit, so one squaring fewer
      const int64_t t = static_cast<int64_t>(r.first_max + 1) << (i - r.first - 1);
      total += terms(lo_v, t - 1) * head_term_imad(r.path, i, r.first + 1, lmax);
      total += terms(t, hi_v) * head_term_imad(r.path, i, r.first, lmax);
    } else {
      total += terms(lo_v, hi_v) * head_term_imad(r.path, i, r.first, lmax);
    }
  }
  return total;
}
}  // namespace

int plan_series(const FormulaDef& f, uint32_t j, uint64_t n, uint32_t W, uint32_t lmax, uint64_t k_lo,
                uint64_t k_hi, std::vector<TermRange>& out, int wide_min_bits) {
  if (n == 0 || j >= f.count || W == 0 || W % 32 != 0 || W > kMaxWorkingBits) return -1;
  if (wide_min_bits < kWideFloorBits || wide_min_bits > kWideMinBits) return -1;
  const SeriesDef& s = f.s[j];
  const uint64_t d = n - 1;
  const uint64_t he = head_end(f, j, d);
  const uint64_t ne = natural_end(f, j, d, W);
  const uint64_t hi = std::min(k_hi, ne);
  if (k_lo >= hi) return 0;
  if (static_cast<uint64_t>(s.a) * (hi - 1) + s.b >= (1ull << kMaxModulusBits)) return -6;

  // head terms, k in [head_lo, head_hi); the term with m = 1 is 0 (2^e mod 1 = 0)
  const uint64_t head_lo = std::max(k_lo, s.b == 1 ? uint64_t{1} : uint64_t{0});
  const uint64_t head_hi = std::min(hi, he);
  if (head_lo < head_hi) {
    struct Group { uint64_t k0, k1; int lmax_bits; int path; uint8_t w, h; };
    std::vector<Group> groups;
    const int l_first = bitlen(static_cast<uint64_t>(s.a) * head_lo + s.b);
    const int l_last = bitlen(static_cast<uint64_t>(s.a) * (head_hi - 1) + s.b);
    for (int l = l_first; l <= l_last; ++l) {
      uint64_t k0 = std::max(head_lo, first_k_at_least(1ull << (l - 1), s.a, s.b));
      uint64_t k1 = std::min(head_hi, first_k_at_least(1ull << l, s.a, s.b));
      if (k0 >= k1) continue;
      const int path = path_for_bits(l, wide_min_bits);
      uint8_t w, h, fm;
      window_params(path, l, &w, &h, &fm);
      if (!groups.empty() && groups.back().path == path && groups.back().w == w && groups.back().h == h &&
          groups.back().k1 == k0) {
        groups.back().k1 = k1;
        groups.back().lmax_bits = l;
      } else {
        groups.push_back(Group{k0, k1, l, path, w, h});
      }
    }
    // fold small groups into their larger-modulus neighbour (whose parameters are
    // valid for smaller moduli too) to keep the launch count down
    std::vector<Group> merged;
    for (size_t i = 0; i < groups.size(); ++i) {
      Group g = groups[i];
      while (g.k1 - g.k0 < kMinRangeTerms && i + 1 < groups.size() && groups[i + 1].path == g.path) {
        const Group& nx = groups[++i];
        g.k1 = nx.k1;
        g.lmax_bits = nx.lmax_bits;
        g.w = nx.w;
        g.h = nx.h;
      }
      if (!merged.empty() && g.k1 - g.k0 < kMinRangeTerms && merged.back().path == g.path) {
        merged.back().k1 = g.k1;
        merged.back().lmax_bits = g.lmax_bits;
        merged.back().w = g.w;
        merged.back().h = g.h;
      } else {
        merged.push_back(g);
      }
    }
    for (const Group& g : merged) {
      // the ladder parameters of the group's largest moduli hold for all of its moduli
      TermRange r{};
      window_params(g.path, g.lmax_bits, &r.window, &r.first, &r.first_max);
      r.j = j;
      r.tail = 0;
      r.path = static_cast<uint8_t>(g.path);
      r.k_begin = g.k0;
      r.count = g.k1 - g.k0;
      r.imad = range_imad(f, s, d, W, r, static_cast<int>(lmax));
      out.push_back(r);
    }
  }
  // tail terms, k in [max(k_lo, head_end), hi)
  const uint64_t tail_lo = std::max(k_lo, he);
  if (tail_lo < hi) {
    TermRange r{};
    r.j = j;
    r.tail = 1;
    r.k_begin = tail_lo;
    r.count = hi - tail_lo;
    out.push_back(r);
  }
  return 0;
}

}  // namespace bbp
