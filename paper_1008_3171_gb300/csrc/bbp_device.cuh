// Device arithmetic for BBP digit extraction on sm_103a (all exact integer work).
//
// Terms (Sze, arXiv:1008.3171, Sec. 3, Eq. 3-5): for series j with modulus
// m = a*k + b and exponent e = d + c - step*k, the W-bit fixed-point value of a
// head term (e >= 0) is t = floor((2^e mod m) 2^W / m).  With E = e + W this is
// t = floor(2^E / m) mod 2^W, and because m is odd it follows from s = 2^E mod m
// alone:   floor(2^E/m) * m = 2^E - s  ==>  t = (-s) * m^-1  (mod 2^W).
// So each term is
//   1. a Montgomery modular exponentiation s = 2^E mod m (Sec. 4.3; Montgomery,
//      "Modular multiplication without trial division", Math. Comp. 1985), and
//   2. an exact 2-adic division producing the W/32 quotient limbs least
//      significant first -- the same word-by-word reduction as Montgomery's REDC,
//      one quotient word per step (Jebelean, "An algorithm for exact division",
//      J. Symb. Comp. 1993).  The only "reciprocal" is m^-1 mod 2^32, lifted by
//      Newton-Hensel steps; there is no hardware or floating-point division.
// Base 2 makes the window multiplications of a left-to-right window ladder pure
// shifts, folded into the unreduced square before each reduction.
#pragma once

#include <cstdint>

namespace bbp {

// ---------------------------------------------------------------- small helpers

__device__ __forceinline__ uint32_t lo32(uint64_t v) { return static_cast<uint32_t>(v); }
__device__ __forceinline__ uint32_t hi32(uint64_t v) { return static_cast<uint32_t>(v >> 32); }
__device__ __forceinline__ uint64_t make64(uint32_t lo, uint32_t hi) {
  return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ int bitlen64(uint64_t v) { return 64 - __clzll(static_cast<long long>(v)); }

// -m^-1 mod 2^32 for odd m by Newton-Hensel lifting: each step x <- x (2 - m x)
// doubles the number of correct low bits.  The start x = (3 m) XOR 2 is already
// correct to 5 bits for every odd m (a known starting value; the word-level test
// checks it on every odd residue mod 2^16), so three steps give 5, 10, 20, 40 >= 32.
__device__ __forceinline__ uint32_t neg_inverse32(uint32_t m0) {
  uint32_t x = (3u * m0) ^ 2u;
  x *= 2u - m0 * x;
  x *= 2u - m0 * x;
  x *= 2u - m0 * x;
  return 0u - x;
}

// ---------------------------------------------------------------- R mod m tracking
//
// Montgomery arithmetic needs R mod m (R = 2^64 or 2^32) to start the ladder.
// Along a run of consecutive k the modulus grows by a, and
//   R = q m + r   ==>   R = q (m + a) + (r - a q),
// so r and q for the next modulus follow from a few corrections of r - a q.
// A run starts (or restarts when the correction would be long, i.e. for small m)
// with a bit-serial long division of R by m.
struct RTrack {
  uint64_t q;  // floor(R / m)
  uint64_t r;  // R mod m
};

template <int RBITS>
__device__ __forceinline__ RTrack r_mod_m_bitserial(uint64_t m) {
  // 2^(l-1) < m < 2^l for odd m > 1: start from 2^(l-1) = 0*m + 2^(l-1), then double.
  const int l = bitlen64(m);
  uint64_t r = 1ull << (l - 1);
  uint64_t q = 0;
  for (int i = l - 1; i < RBITS; ++i) {
    // r < m < 2^60, so 2r does not overflow
    r <<= 1;
    q <<= 1;
    if (r >= m) { r -= m; q |= 1; }
  }
  return RTrack{q, r};
}

template <int RBITS>
__device__ __forceinline__ void r_mod_m_advance(RTrack& t, uint64_t m_next, uint32_t a) {
  const uint64_t aq = t.q * a;
  if (aq > t.r + 4 * m_next) {                 // many corrections: restart the division
    t = r_mod_m_bitserial<RBITS>(m_next);
    return;
  }
  int64_t r = static_cast<int64_t>(t.r) - static_cast<int64_t>(aq);
  uint64_t q = t.q;
  while (r < 0) { r += static_cast<int64_t>(m_next); --q; }
  t.q = q;
  t.r = static_cast<uint64_t>(r);
}

// ---------------------------------------------------------------- 64-bit Montgomery
//
// m = (m1:m0) odd, 2^29 <= m < 2^60, R = 2^64, mp = -m^-1 mod 2^32.  Residues are
// lazy: x < 2m.  A squaring with a window shift s returns REDC(x^2 2^s) < 2m.
struct Mod64 {
  uint32_t m0, m1, mp;
};

// Inline-asm convention in this file: every block copies its inputs into
// block-local registers first and writes its outputs last, so the compiler may
// place an output in the same register as any input (equal values are merged)
// without changing the result.
//
// Multiply mix.  On GB300 the integer multiply pipe issues the low half of a
// 32x32 product (mul.lo) at 64 lanes/clk/SM, the high half (mul.hi) and the full
// product (mul.wide) at 32, and a full product with a 64-bit addend (mad.wide) at
// only 25.  So a product whose two halves are both needed is one mul.wide without
// an addend, a product of which only the high half is needed is one mul.hi, sums
// are 32-bit carry chains on the ALU, and the low word of T + u m -- zero by the
// choice of u -- is never formed: its carry is (T_0 != 0), produced as the carry
// out of T_0 + (2^32 - 1) and consumed by the next add of the chain.

// General squaring: x < 2^61 (so 2 x1 fits one word), T = x^2 2^s on four words,
// then two word-by-word REDC steps T <- (T + u m) / 2^32.  The result is below 2m
// when T < m 2^64: bitlen(m) + s <= 61 for a lazy x < 2m, and bitlen(m) + 2 w + s
// <= 64 for the unreduced first window x < m 2^w.
__device__ __forceinline__ void sqr_shift_redc64(uint32_t& x0, uint32_t& x1, uint32_t s, const Mod64& M,
                                                 bool do_shift) {
  uint32_t t0, t1, t2, t3;
  // T = x0^2 + (x0 * 2 x1) 2^32 + x1^2 2^64
  asm("{\n\t"
      ".reg .u32 a0, a1, d1, s0, s1, s2, s3, w0, w1;\n\t"
      ".reg .u64 p00, p01, p11;\n\t"
      "mov.u32        a0, %4;\n\t"
      "mov.u32        a1, %5;\n\t"
      "shl.b32        d1, a1, 1;\n\t"
      "mul.wide.u32   p00, a0, a0;\n\t"
      "mul.wide.u32   p01, a0, d1;\n\t"
      "mul.wide.u32   p11, a1, a1;\n\t"
      "mov.b64        {s0, s1}, p00;\n\t"
      "mov.b64        {w0, w1}, p01;\n\t"
      "mov.b64        {s2, s3}, p11;\n\t"
      "add.cc.u32     s1, s1, w0;\n\t"
      "addc.cc.u32    s2, s2, w1;\n\t"
      "addc.u32       s3, s3, 0;\n\t"
      "mov.u32        %0, s0;\n\t"
      "mov.u32        %1, s1;\n\t"
      "mov.u32        %2, s2;\n\t"
      "mov.u32        %3, s3;\n\t"
      "}"
      : "=r"(t0), "=r"(t1), "=r"(t2), "=r"(t3)
      : "r"(x0), "r"(x1));
  if (do_shift) {  // window multiply by 2^s, s < 32
    t3 = __funnelshift_l(t2, t3, s);
    t2 = __funnelshift_l(t1, t2, s);
    t1 = __funnelshift_l(t0, t1, s);
    t0 <<= s;
  }
  // two word-by-word Montgomery reduction steps: T <- (T + u m) / 2^32, twice.
  // Per step: u = T_0 mp; (T + u m)/2^32 = (T >> 32) + hi(u m0) + (T_0 != 0) + u m1.
  uint32_t r0, r1;
  asm("{\n\t"
      ".reg .u32 u, c, h, s0, s1, s2, s3, n0, n1, np;\n\t"
      ".reg .u64 z, a, hz;\n\t"
      "mov.u32        s0, %2;\n\t"
      "mov.u32        s1, %3;\n\t"
      "mov.u32        s2, %4;\n\t"
      "mov.u32        s3, %5;\n\t"
      "mov.u32        n0, %6;\n\t"
      "mov.u32        n1, %7;\n\t"
      "mov.u32        np, %8;\n\t"
      // step 1: word 0 vanishes; (s3 : s2 : s1) += hi(u m0) + c + u m1
      "mul.lo.u32     u, s0, np;\n\t"
      "min.u32        c, s0, 1;\n\t"
      "mul.hi.u32     h, u, n0;\n\t"
      "mul.wide.u32   z, u, n1;\n\t"
      "add.u32        h, h, c;\n\t"
      "mov.b64        a, {s1, s2};\n\t"
      "add.cc.u64     a, a, z;\n\t"
      "addc.u32       s3, s3, 0;\n\t"
      "cvt.u64.u32    hz, h;\n\t"
      "add.cc.u64     a, a, hz;\n\t"
      "addc.u32       s3, s3, 0;\n\t"
      "mov.b64        {s1, s2}, a;\n\t"
      // step 2: word 1 vanishes; the result (s3 : s2) + hi(u m0) + c + u m1 < 2m fits 64 bits,
      // so u m1 is accumulated by the multiply itself
      "mul.lo.u32     u, s1, np;\n\t"
      "min.u32        c, s1, 1;\n\t"
      "mul.hi.u32     h, u, n0;\n\t"
      "add.u32        h, h, c;\n\t"
      "mov.b64        a, {s2, s3};\n\t"
      "mad.wide.u32   a, u, n1, a;\n\t"
      "cvt.u64.u32    hz, h;\n\t"
      "add.u64        a, a, hz;\n\t"
      "mov.b64        {s2, s3}, a;\n\t"
      "mov.u32        %0, s2;\n\t"
      "mov.u32        %1, s3;\n\t"
      "}"
      : "=r"(r0), "=r"(r1)
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(M.m0), "r"(M.m1), "r"(M.mp));
  x0 = r0;
  x1 = r1;
}

// Squaring for moduli of at most 46 bits with a lazy x < 2m < 2^47:
//   T = x^2 < 2^94 fits three words (x1^2 < 2^30 needs only its low word), and
//   T' = (T + u m)/2^32 < 2^62 + 2^46 fits two words;
// the window shift is applied to T' (two words -> three) instead of T, and the
// second step reduces T' 2^s: (T' 2^s + u' m)/2^32 = (T 2^s + (u 2^s + u' 2^32) m)/2^64,
// a Montgomery reduction of x^2 2^s with another multiple of m, below 2m while
// bitlen(m) + s <= 61.  2 x1 is formed by a funnel shift, and the cross product
// and both reductions are summed in 32-bit carry chains.
__device__ __forceinline__ void sqr_redc64_p1(uint32_t& x0, uint32_t& x1, uint32_t s, const Mod64& M,
                                              bool do_shift) {
  uint32_t y0, y1, y2 = 0;
  asm("{\n\t"
      ".reg .u32 a0, a1, d1, s0, h0, b0, b1, q0, u, h, z0, z1, n0, n1, np, cy;\n\t"
      ".reg .u64 p;\n\t"
      "mov.u32        a0, %2;\n\t"
      "mov.u32        a1, %3;\n\t"
      "mov.u32        n0, %4;\n\t"
      "mov.u32        n1, %5;\n\t"
      "mov.u32        np, %6;\n\t"
      "shf.l.wrap.b32 d1, 0, a1, 1;\n\t"       // 2 x1 (x1 < 2^15)
      "mul.wide.u32   p, a0, a0;\n\t"
      "mov.b64        {s0, h0}, p;\n\t"
      "mul.wide.u32   p, a0, d1;\n\t"
      "mov.b64        {b0, b1}, p;\n\t"
      "mul.lo.u32     q0, a1, a1;\n\t"
      "mul.lo.u32     u, s0, np;\n\t"
      "mul.hi.u32     h, u, n0;\n\t"
      "mul.wide.u32   p, u, n1;\n\t"
      "mov.b64        {z0, z1}, p;\n\t"
      // T' = h0 + (b1:b0) + q0 2^32 + (z1:z0) + h + (s0 != 0)
      "add.cc.u32     cy, s0, -1;\n\t"         // carry out = (s0 != 0)
      "addc.cc.u32    h0, h0, b0;\n\t"
      "addc.u32       b1, b1, q0;\n\t"
      "add.cc.u32     h0, h0, z0;\n\t"
      "addc.u32       b1, b1, z1;\n\t"
      "add.cc.u32     %0, h0, h;\n\t"
      "addc.u32       %1, b1, 0;\n\t"
      "}"
      : "=r"(y0), "=r"(y1)
      : "r"(x0), "r"(x1), "r"(M.m0), "r"(M.m1), "r"(M.mp));
  if (do_shift) {  // T' 2^s on three words, s < 16
    y2 = __funnelshift_l(y1, 0u, s);
    y1 = __funnelshift_l(y0, y1, s);
    y0 <<= s;
  }
  uint32_t r0, r1;
  asm("{\n\t"
      ".reg .u32 u, h, b0, b1, b2, z0, z1, n0, n1, np, cy;\n\t"
      ".reg .u64 p;\n\t"
      "mov.u32        b0, %2;\n\t"
      "mov.u32        b1, %3;\n\t"
      "mov.u32        b2, %4;\n\t"
      "mov.u32        n0, %5;\n\t"
      "mov.u32        n1, %6;\n\t"
      "mov.u32        np, %7;\n\t"
      "mul.lo.u32     u, b0, np;\n\t"
      "mul.hi.u32     h, u, n0;\n\t"
      "mul.wide.u32   p, u, n1;\n\t"
      "mov.b64        {z0, z1}, p;\n\t"
      // (b2 : b1) + (z1:z0) + h + (b0 != 0) < 2m
      "add.cc.u32     cy, b0, -1;\n\t"
      "addc.cc.u32    b1, b1, z0;\n\t"
      "addc.u32       b2, b2, z1;\n\t"
      "add.cc.u32     %0, b1, h;\n\t"
      "addc.u32       %1, b2, 0;\n\t"
      "}"
      : "=r"(r0), "=r"(r1)
      : "r"(y0), "r"(y1), "r"(y2), "r"(M.m0), "r"(M.m1), "r"(M.mp));
  x0 = r0;
  x1 = r1;
}

// x < 2m  ->  x mod m
__device__ __forceinline__ void reduce_once64(uint32_t& x0, uint32_t& x1, const Mod64& M) {
  uint32_t y0, y1, borrow;
  asm("{\n\t"
      ".reg .u32 a0, a1, n0, n1, b0, b1, bw;\n\t"
      "mov.u32     a0, %3;\n\t"
      "mov.u32     a1, %4;\n\t"
      "mov.u32     n0, %5;\n\t"
      "mov.u32     n1, %6;\n\t"
      "sub.cc.u32  b0, a0, n0;\n\t"
      "subc.cc.u32 b1, a1, n1;\n\t"
      "subc.u32    bw, 0, 0;\n\t"
      "mov.u32     %0, b0;\n\t"
      "mov.u32     %1, b1;\n\t"
      "mov.u32     %2, bw;\n\t"
      "}"
      : "=r"(y0), "=r"(y1), "=r"(borrow)
      : "r"(x0), "r"(x1), "r"(M.m0), "r"(M.m1));
  if (borrow == 0) { x0 = y0; x1 = y1; }
}

// One exact-division digit: for x < m returns u = x * (-m^-1) mod 2^32 and
// replaces x by (x + u m) / 2^32 = x1 + hi(u m0) + (x0 != 0) + u m1 (still < m).
// The low word of x + u m is 0 by the choice of u, so only its carry matters.
__device__ __forceinline__ uint32_t hensel_step64(uint32_t& x0, uint32_t& x1, const Mod64& M) {
  uint32_t u, y0, y1;
  asm("{\n\t"
      ".reg .u32 q, c, h, a0, a1, n0, n1, np;\n\t"
      ".reg .u64 r, w;\n\t"
      "mov.u32        a0, %3;\n\t"
      "mov.u32        a1, %4;\n\t"
      "mov.u32        n0, %5;\n\t"
      "mov.u32        n1, %6;\n\t"
      "mov.u32        np, %7;\n\t"
      "mul.lo.u32     q, a0, np;\n\t"
      "min.u32        c, a0, 1;\n\t"
      "mul.hi.u32     h, q, n0;\n\t"
      "add.u32        h, h, c;\n\t"
      "cvt.u64.u32    r, h;\n\t"
      "cvt.u64.u32    w, a1;\n\t"
      "add.u64        r, r, w;\n\t"
      "mad.wide.u32   r, q, n1, r;\n\t"
      "mov.b64        {a0, a1}, r;\n\t"
      "mov.u32        %0, q;\n\t"
      "mov.u32        %1, a0;\n\t"
      "mov.u32        %2, a1;\n\t"
      "}"
      : "=r"(u), "=r"(y0), "=r"(y1)
      : "r"(x0), "r"(x1), "r"(M.m0), "r"(M.m1), "r"(M.mp));
  x0 = y0;
  x1 = y1;
  return u;
}

// Exact division digits: x < m (x = 2^E mod m); writes q[0..N) with
// x + (sum q_i 2^(32i)) m = 0 (mod 2^(32N)), least significant digit first.
template <int N>
__device__ __forceinline__ void hensel_digits64(uint32_t x0, uint32_t x1, const Mod64& M, uint32_t (&q)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) q[i] = hensel_step64(x0, x1, M);
}

// ---------------------------------------------------------------- 32-bit Montgomery
//
// m < 2^31 odd, R = 2^32, one word.  Lazy residues (REDUCED = false, m < 2^29):
// x < 2m, and REDC(x^2 2^s) < 2m while bitlen(m) + s <= 30.  Reduced residues
// (REDUCED = true, moduli of 30 and 31 bits): x < m after one conditional
// subtraction per squaring, so x^2 2^s < m^2 2^s fits 64 bits and REDC stays below
// 2m while bitlen(m) + s <= 32.
struct Mod32 {
  uint32_t m, mp;
};

template <bool REDUCED>
__device__ __forceinline__ uint32_t sqr_shift_redc32(uint32_t x, uint32_t s, const Mod32& M, bool do_shift) {
  uint64_t T = static_cast<uint64_t>(x) * x;  // one 32x32->64 product
  if (do_shift) T <<= s;
  const uint32_t t0 = lo32(T);
  const uint32_t t1 = hi32(T);
  const uint32_t u = t0 * M.mp;
  // t0 + lo(u m) = 0 (mod 2^32): the carry out of that word is (t0 != 0)
  const uint32_t r = t1 + __umulhi(u, M.m) + (t0 != 0u ? 1u : 0u);
  // r < 2m < 2^32: r - m wraps above r exactly when r < m
  return REDUCED ? min(r, r - M.m) : r;
}

template <int N>
__device__ __forceinline__ void hensel_digits32(uint32_t x, const Mod32& M, uint32_t (&q)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint32_t u = x * M.mp;
    x = __umulhi(u, M.m) + (x != 0u ? 1u : 0u);
    q[i] = u;
  }
}

// ---------------------------------------------------------------- multi-limb sums

// acc += t and acc -= t modulo 2^(32N), with explicit carries.
template <int N>
__device__ __forceinline__ void add_limbs(uint32_t (&acc)[N], const uint32_t (&t)[N]) {
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint64_t s = static_cast<uint64_t>(acc[i]) + t[i] + c;
    acc[i] = static_cast<uint32_t>(s);
    c = static_cast<uint32_t>(s >> 32);
  }
}

template <int N>
__device__ __forceinline__ void sub_limbs(uint32_t (&acc)[N], const uint32_t (&t)[N]) {
  uint32_t b = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint64_t s = static_cast<uint64_t>(acc[i]) - t[i] - b;
    acc[i] = static_cast<uint32_t>(s);
    b = static_cast<uint32_t>(s >> 63);
  }
}

// Exact warp sum of N-limb values mod 2^(32N), returned in every lane.  Each limb
// is split into 16-bit halves so the hardware 32-bit warp reduction cannot overflow
// (32 * (2^16 - 1) < 2^21), then carries are propagated limb by limb.
template <int N>
__device__ __forceinline__ void warp_sum_limbs(uint32_t (&v)[N], unsigned mask = 0xffffffffu) {
  uint64_t carry = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint64_t lo = __reduce_add_sync(mask, v[i] & 0xffffu);
    const uint64_t hi = __reduce_add_sync(mask, v[i] >> 16);
    const uint64_t s = lo + (hi << 16) + carry;
    v[i] = static_cast<uint32_t>(s);
    carry = s >> 32;
  }
}

}  // namespace bbp
