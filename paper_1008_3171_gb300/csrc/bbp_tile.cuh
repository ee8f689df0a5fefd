// Head-term kernels for BBP digit extraction (Sze, arXiv:1008.3171, Sec. 3 and 4.3):
// the per-warp tile loop (Montgomery window ladder for s = 2^(e+W) mod m, exact-division
// digits t = floor(2^(e+W)/m) mod 2^W, signed accumulation), the single-range head
// kernel and the persistent queue kernel.  Templates only: each accumulator class is
// instantiated in its own translation unit (bbp_inst.cuh).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bbp_device.cuh"
#include "bbp_finalize.cuh"
#include "bbp_kernels.cuh"

namespace bbp {

// ---------------------------------------------------------------- head terms
//
// Work split: a warp owns a tile of 32 * S * run consecutive terms; lane l, stream s
// owns the run starting at tile + (l S + s) run.  Along a run, m, the exponent and
// R mod m advance incrementally, and the exponents of a warp stay within
// step * 32 * S * run of each other, so the ladder length (the warp maximum of the
// exponent bit length) is almost always shared.  Each stream evaluates a pair
// (k, k+1) per step, so (-1)^k is static in the code.

// State of one stream at its current term.
struct StreamState {
  uint64_t rel;  // term index relative to k_begin (clamped to the last term)
  uint64_t m;    // modulus a k + b
  uint64_t E;    // exponent of the residue the ladder produces: e + W = d + c - step k + W
  RTrack tr;     // R = q m + r
};

// Modulus paths (the planner picks one per launch range by the moduli's bit length):
//   0: one 32-bit word, lazy residues, bitlen(m) <= 29
//   1: two words, bitlen(m) <= 46 (three-word square, shift after the first REDC step)
//   2: two words, bitlen(m) <= 60 (four-word square)
//   3: one 32-bit word, fully reduced residues, bitlen(m) of 30 or 31
template <int PATH>
struct PathTraits {
  static constexpr bool kWide = PATH == 1 || PATH == 2;
  static constexpr int kRBits = kWide ? 64 : 32;
};

template <int PATH, int NT>
__device__ __forceinline__ void square_all(uint32_t (&x0)[NT], uint32_t (&x1)[NT], const uint32_t (&m0)[NT],
                                           const uint32_t (&m1)[NT], const uint32_t (&mp)[NT],
                                           const uint32_t (&sh)[NT], bool do_shift) {
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (PATH == 1) sqr_redc64_p1(x0[t], x1[t], sh[t], Mod64{m0[t], m1[t], mp[t]}, do_shift);
    else if (PATH == 2) sqr_shift_redc64(x0[t], x1[t], sh[t], Mod64{m0[t], m1[t], mp[t]}, do_shift);
    else x0[t] = sqr_shift_redc32<PATH == 3>(x0[t], sh[t], Mod32{m0[t], mp[t]}, do_shift);
  }
}

// The first squaring of a path-1 ladder takes the unreduced first window
// x = (R mod m) << w0 < m 2^w0, beyond the three-word routine's x < 2m: it runs the
// general four-word routine, whose bound is bitlen(m) + 2 w0 + s <= 64.
template <int NT>
__device__ __forceinline__ void square_all_general(uint32_t (&x0)[NT], uint32_t (&x1)[NT], const uint32_t (&m0)[NT],
                                                   const uint32_t (&m1)[NT], const uint32_t (&mp)[NT],
                                                   const uint32_t (&sh)[NT], bool do_shift) {
#pragma unroll
  for (int t = 0; t < NT; ++t) sqr_shift_redc64(x0[t], x1[t], sh[t], Mod64{m0[t], m1[t], mp[t]}, do_shift);
}

// Quotient digits of every term, least significant first, folded straight into
// the LMAX-limb sum with a signed carry (odd terms subtracted when NEG_ODD).  A
// term of a lane past the range has x = 0, whose digits are all 0.
template <bool WIDE, bool NEG_ODD, int NT, int LMAX>
__device__ __forceinline__ void fold_digits(uint32_t (&acc)[LMAX], uint32_t (&x0)[NT], uint32_t (&x1)[NT],
                                            const uint32_t (&m0)[NT], const uint32_t (&m1)[NT],
                                            const uint32_t (&mp)[NT]) {
  int64_t carry = 0;
#pragma unroll
  for (int i = 0; i < LMAX; ++i) {
    int64_t sum = static_cast<int64_t>(acc[i]) + carry;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      uint32_t q;
      if (WIDE) {
        q = hensel_step64(x0[t], x1[t], Mod64{m0[t], m1[t], mp[t]});
      } else {
        q = x0[t] * mp[t];
        x0[t] = __umulhi(q, m0[t]) + (x0[t] != 0u ? 1u : 0u);
      }
      if (NEG_ODD && (t & 1)) sum -= q;
      else sum += q;
    }
    acc[i] = static_cast<uint32_t>(sum);
    carry = sum >> 32;
  }
}

// `len` squarings of one window group: len - 1 plain, then one with the group's
// value shifted in.  len <= 4.
template <int PATH, int NT>
__device__ __forceinline__ void square_group(int len, uint32_t (&x0)[NT], uint32_t (&x1)[NT],
                                             const uint32_t (&m0)[NT], const uint32_t (&m1)[NT],
                                             const uint32_t (&mp)[NT], const uint32_t (&sh)[NT]) {
  const uint32_t zero[NT] = {};
  switch (len) {
    case 4: square_all<PATH, NT>(x0, x1, m0, m1, mp, zero, false);  // fall through
    case 3: square_all<PATH, NT>(x0, x1, m0, m1, mp, zero, false);  // fall through
    case 2: square_all<PATH, NT>(x0, x1, m0, m1, mp, zero, false);  // fall through
    default: break;
  }
  square_all<PATH, NT>(x0, x1, m0, m1, mp, sh, true);
}

// One warp tile: terms [ti * tile, (ti + 1) * tile) of the run list of A, added
// into this lane's sum.  Every lane of the warp must call it (warp-wide reductions).
template <int LMAX, int PATH, int S>
__device__ __forceinline__ void process_tile(const HeadArgs& A, const uint64_t ti, const uint32_t lane,
                                             uint32_t (&acc)[LMAX]) {
  constexpr int NT = 2 * S;
  constexpr bool WIDE = PathTraits<PATH>::kWide;
  constexpr int RB = PathTraits<PATH>::kRBits;
  const uint64_t run = A.run;
  const uint64_t tile = 32ull * S * run;
  const uint64_t last = A.count - 1;
  const int window = static_cast<int>(A.window);
  // exponent of the residue at k: E(k) = e0 - step k
  const uint64_t e0 = A.d + static_cast<int64_t>(A.c) + A.W;
  uint64_t base[S];
  StreamState st[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    base[s] = ti * tile + (static_cast<uint64_t>(lane) * S + s) * run;
    st[s].rel = min(base[s], last);
    const uint64_t k = A.k_begin + st[s].rel;
    st[s].m = static_cast<uint64_t>(A.a) * k + A.b;
    st[s].E = e0 - static_cast<uint64_t>(A.step) * k;
    st[s].tr = r_mod_m_bitserial<RB>(st[s].m);
  }
  for (uint32_t i = 0; i < run; i += 2) {
    uint64_t v[NT];
    uint32_t x0[NT], x1[NT], m0[NT], m1[NT], mp[NT];
    bool valid[NT];
    int nbl = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int t = 2 * s + p;
        const uint64_t rel = base[s] + i + p;
        valid[t] = rel < A.count;
        if (valid[t] && rel != st[s].rel) {  // the next k of the run: advance by one
          st[s].rel = rel;
          st[s].m += A.a;
          st[s].E -= A.step;
          r_mod_m_advance<RB>(st[s].tr, st[s].m, A.a);
        }
        x0[t] = lo32(st[s].tr.r);
        x1[t] = hi32(st[s].tr.r);
        m0[t] = lo32(st[s].m);
        m1[t] = hi32(st[s].m);
        mp[t] = neg_inverse32(m0[t]);
        v[t] = st[s].E - RB;  // E >= W >= RB for head terms
        nbl = max(nbl, bitlen64(v[t]));
      }
    }
    const int nb = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<uint32_t>(nbl)));
    int h = nb > 0 ? min(static_cast<int>(A.first), nb - 1) : 0;
    if (A.first_max >= (1u << h) && h + 1 <= nb - 1) {
      // one more first-window bit (one squaring fewer) when the warp's top h + 1
      // exponent bits all stay within the first-window bound of the moduli (the
      // lane with nb bits has top bits >= 2^h, so a smaller bound never admits it)
      uint32_t top = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t) top = max(top, static_cast<uint32_t>(v[t] >> (nb - h - 1)));
      if (__reduce_max_sync(0xffffffffu, top) <= A.first_max) ++h;
    }
    const int low = nb - h;  // bits left after the first window
    uint64_t rem[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      // first window: Montgomery form of 2^w0 is (R mod m) << w0, no squaring
      const uint32_t w0 = h > 0 ? static_cast<uint32_t>(v[t] >> low) : 0u;
      if (WIDE) {
        const uint64_t x = make64(x0[t], x1[t]) << w0;
        x0[t] = lo32(x);
        x1[t] = hi32(x);
      } else {
        x0[t] <<= w0;
      }
      rem[t] = low > 0 ? (v[t] & ((1ull << low) - 1ull)) : 0ull;
    }
    // remaining bits, top down, in groups of at most `window` bits.  Any split of the
    // bits into consecutive groups gives the same power.  Path 1 always has 4-bit
    // windows (its moduli are below 2^47); there the groups are aligned from the
    // bottom, so only the first one is short and the rest run as a fixed
    // four-squaring body.  The other paths align them from the top.
    int p = low;
    const bool w4 = PATH == 1 && window == 4;
    if (PATH == 1 && p > 0) {
      // the first group, with its first squaring on the general routine
      const int len = w4 ? ((p - 1) & 3) + 1 : min(window, p);
      p -= len;
      uint32_t sh[NT];
      const uint32_t zero[NT] = {};
#pragma unroll
      for (int t = 0; t < NT; ++t) sh[t] = static_cast<uint32_t>(rem[t] >> p) & ((1u << len) - 1u);
      if (len == 1) {
        square_all_general<NT>(x0, x1, m0, m1, mp, sh, true);
      } else {
        square_all_general<NT>(x0, x1, m0, m1, mp, zero, false);
        square_group<PATH, NT>(len - 1, x0, x1, m0, m1, mp, sh);
      }
    }
    if (w4) {
      const uint32_t zero[NT] = {};
      while (p > 0) {
        p -= 4;
        uint32_t sh[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) sh[t] = static_cast<uint32_t>(rem[t] >> p) & 15u;
        square_all<PATH, NT>(x0, x1, m0, m1, mp, zero, false);
        square_all<PATH, NT>(x0, x1, m0, m1, mp, zero, false);
        square_all<PATH, NT>(x0, x1, m0, m1, mp, zero, false);
        square_all<PATH, NT>(x0, x1, m0, m1, mp, sh, true);
      }
    }
    while (p > 0) {
      const int len = min(window, p);
      p -= len;
      uint32_t sh[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) sh[t] = static_cast<uint32_t>(rem[t] >> p) & ((1u << len) - 1u);
      square_group<PATH, NT>(len, x0, x1, m0, m1, mp, sh);
    }
    // s = 2^E mod m (0 for a lane past the range), then the W-bit quotient digits
    // folded into the signed sum
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (WIDE) {
        reduce_once64(x0[t], x1[t], Mod64{m0[t], m1[t], mp[t]});
      } else if (x0[t] >= m0[t]) {
        x0[t] -= m0[t];
      }
      if (!valid[t]) {
        x0[t] = 0;
        x1[t] = 0;
      }
    }
    if (A.alternating) fold_digits<WIDE, true, NT, LMAX>(acc, x0, x1, m0, m1, mp);
    else fold_digits<WIDE, false, NT, LMAX>(acc, x0, x1, m0, m1, mp);
  }
}

template <int LMAX, int PATH, int S>
__global__ void __launch_bounds__(kHeadThreads) head_kernel(const HeadArgs A, const uint64_t ntiles) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wid = threadIdx.x >> 5;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;

  uint32_t acc[LMAX];
#pragma unroll
  for (int i = 0; i < LMAX; ++i) acc[i] = 0;
  for (uint64_t ti = warp; ti < ntiles; ti += nwarps) process_tile<LMAX, PATH, S>(A, ti, lane, acc);

  // limbs at or above L hold digits past 2^W: drop them (the sum is mod 2^W)
#pragma unroll
  for (int i = 0; i < LMAX; ++i)
    if (i >= static_cast<int>(A.L)) acc[i] = 0;

  __shared__ uint32_t red[kHeadThreads / 32][LMAX];
  warp_sum_limbs<LMAX>(acc);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < LMAX; ++i) red[wid][i] = acc[i];
  }
  __syncthreads();
  if (wid == 0) {
    const uint32_t nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < LMAX; ++i) acc[i] = lane < nw ? red[lane][i] : 0u;
    warp_sum_limbs<LMAX>(acc);
    if (lane == 0) {
      if (A.negate) {
        uint64_t carry = 1;
#pragma unroll
        for (int i = 0; i < LMAX; ++i) {
          const uint64_t s = static_cast<uint64_t>(~acc[i]) + carry;
          acc[i] = static_cast<uint32_t>(s);
          carry = s >> 32;
        }
      }
#pragma unroll
      for (int i = 0; i < LMAX; ++i)
        if (i < static_cast<int>(A.L) && acc[i]) atomicAdd(A.slots + i, static_cast<unsigned long long>(acc[i]));
    }
  }
}

// ---------------------------------------------------------------- persistent queue

// Hands out `grab` tiles of the current job to one warp (lane 0 decides, all lanes
// learn).  Every hand-out either succeeds or moves the cursor past an exhausted
// job, so the loop ends after at most (jobs left) rounds; nothing waits on other
// threads.
__device__ __forceinline__ bool next_grab(const BatchDev& B, uint32_t job_begin, uint32_t job_end,
                                          unsigned int* cursor, uint32_t lane, uint32_t* job,
                                          unsigned long long* t0) {
  uint32_t j = job_end;
  unsigned long long t = 0;
  if (lane == 0) {
    for (;;) {
      const uint32_t rel = *reinterpret_cast<volatile unsigned int*>(cursor);
      j = job_begin + rel;
      if (j >= job_end) { j = job_end; break; }
      t = atomicAdd(B.job_taken + j, static_cast<unsigned long long>(B.grab));
      if (t < B.job_tiles[j]) break;
      atomicMax(cursor, rel + 1);
    }
  }
  j = __shfl_sync(0xffffffffu, j, 0);
  t = __shfl_sync(0xffffffffu, t, 0);
  *job = j;
  *t0 = t;
  return j < job_end;
}

template <int LMAX, int PATH, int S>
__global__ void __launch_bounds__(kHeadThreads) queue_kernel(const BatchDev B, const uint32_t job_begin,
                                                             const uint32_t job_end, unsigned int* cursor) {
  const uint32_t lane = threadIdx.x & 31u;
  // the warp's current job lives in shared memory (like kernel arguments, it is
  // read-only and uniform, so it need not occupy registers)
  __shared__ HeadArgs job_sm[kHeadThreads / 32];
  HeadArgs& A = job_sm[threadIdx.x >> 5];
  uint32_t j;
  unsigned long long t0;
  while (next_grab(B, job_begin, job_end, cursor, lane, &j, &t0)) {
    static_assert(sizeof(HeadArgs) % 4 == 0, "HeadArgs is copied as 32-bit words");
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(B.jobs + j);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&A);
      for (uint32_t w = lane; w < sizeof(HeadArgs) / 4; w += 32) dst[w] = src[w];
      __syncwarp();
    }
    const unsigned long long ntiles = B.job_tiles[j];
    const unsigned long long t1 = min(t0 + B.grab, ntiles);
    uint32_t acc[LMAX];
#pragma unroll
    for (int i = 0; i < LMAX; ++i) acc[i] = 0;
    for (unsigned long long ti = t0; ti < t1; ++ti) process_tile<LMAX, PATH, S>(A, ti, lane, acc);
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
      if (i >= static_cast<int>(A.L)) acc[i] = 0;
    warp_sum_limbs<LMAX>(acc);
    if (lane == 0) {
      if (A.negate) {
        uint64_t carry = 1;
#pragma unroll
        for (int i = 0; i < LMAX; ++i) {
          const uint64_t v = static_cast<uint64_t>(~acc[i]) + carry;
          acc[i] = static_cast<uint32_t>(v);
          carry = v >> 32;
        }
      }
#pragma unroll
      for (int i = 0; i < LMAX; ++i)
        if (i < static_cast<int>(A.L) && acc[i]) atomicAdd(A.slots + i, static_cast<unsigned long long>(acc[i]));
      __threadfence();
      const unsigned long long done = atomicAdd(B.job_done + j, t1 - t0) + (t1 - t0);
      if (done == ntiles) retire_job(B, B.job_query[j]);
    }
    __syncwarp();
  }
}

}  // namespace bbp
