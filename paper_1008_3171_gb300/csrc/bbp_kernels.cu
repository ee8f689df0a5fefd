// sm_103a kernels for BBP digit extraction (Sze, arXiv:1008.3171, Sec. 3 and 4.3).
//
//   head_kernel    -- head terms A_k (e >= 0): Montgomery window ladder for
//                     s = 2^(e+W) mod m, exact-division digits t = floor(2^(e+W)/m)
//                     mod 2^W, signed accumulation, warp -> CTA -> grid reduction.
//   tail_kernel    -- tail terms B_k (e < 0): t = floor(2^W / m) >> -e.
//   fold / finalize -- carry propagation of the carry-save sum, the guard-bit
//                     validity rule, and the top P output bits.
//   imad_probe     -- issue-rate microbenchmark of the integer multiply pipe.
#include <cuda_runtime.h>

#include <algorithm>

#include "bbp_device.cuh"
#include "bbp_kernels.cuh"

namespace bbp {
namespace {

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

template <bool WIDE, bool SMALL, int NT>
__device__ __forceinline__ void square_all(uint32_t (&x0)[NT], uint32_t (&x1)[NT], const uint32_t (&m0)[NT],
                                           const uint32_t (&m1)[NT], const uint32_t (&mp)[NT],
                                           const uint32_t (&sh)[NT], bool do_shift) {
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (WIDE) sqr_shift_redc64<SMALL>(x0[t], x1[t], sh[t], Mod64{m0[t], m1[t], mp[t]}, do_shift);
    else x0[t] = sqr_shift_redc32(x0[t], sh[t], Mod32{m0[t], mp[t]}, do_shift);
  }
}

// Quotient digits of every term, least significant first, folded straight into
// the LMAX-limb sum with a signed carry (odd terms subtracted when NEG_ODD).
template <bool WIDE, bool NEG_ODD, int NT, int LMAX>
__device__ __forceinline__ void fold_digits(uint32_t (&acc)[LMAX], uint32_t (&x0)[NT], uint32_t (&x1)[NT],
                                            const uint32_t (&m0)[NT], const uint32_t (&m1)[NT],
                                            const uint32_t (&mp)[NT], const uint32_t (&vmask)[NT]) {
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
      q &= vmask[t];
      if (NEG_ODD && (t & 1)) sum -= q;
      else sum += q;
    }
    acc[i] = static_cast<uint32_t>(sum);
    carry = sum >> 32;
  }
}

// One warp tile: terms [ti * tile, (ti + 1) * tile) of the run list of A, added
// into this lane's sum.  Every lane of the warp must call it (warp-wide reductions).
template <int LMAX, int PATH, int S>
__device__ __forceinline__ void process_tile(const HeadArgs& A, const uint64_t ti, const uint32_t lane,
                                             uint32_t (&acc)[LMAX]) {
  constexpr int NT = 2 * S;
  constexpr bool WIDE = PATH > 0;         // 64-bit moduli (PATH 1: bitlen(m) <= 47, PATH 2: <= 60)
  constexpr bool SMALL = PATH == 1;
  constexpr int RB = WIDE ? 64 : 32;
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
    uint32_t x0[NT], x1[NT], m0[NT], m1[NT], mp[NT], vmask[NT];
    int nbl = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int t = 2 * s + p;
        const uint64_t rel = base[s] + i + p;
        const bool valid = rel < A.count;
        if (valid && rel != st[s].rel) {  // the next k of the run: advance by one
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
        vmask[t] = valid ? 0xffffffffu : 0u;
        v[t] = st[s].E - RB;  // E >= W >= RB for head terms
        nbl = max(nbl, bitlen64(v[t]));
      }
    }
    const int nb = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<uint32_t>(nbl)));
    const int h = nb > 0 ? min(static_cast<int>(A.first), nb - 1) : 0;
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
    // remaining bits, top down, in groups of `window` bits aligned from the top:
    // len - 1 plain squarings, then one squaring with the group's value shifted in
    const uint32_t zero[NT] = {};
    int p = low;
    while (p > 0) {
      const int len = min(window, p);
      p -= len;
      switch (len) {
        case 4: square_all<WIDE, SMALL, NT>(x0, x1, m0, m1, mp, zero, false);  // fall through
        case 3: square_all<WIDE, SMALL, NT>(x0, x1, m0, m1, mp, zero, false);  // fall through
        case 2: square_all<WIDE, SMALL, NT>(x0, x1, m0, m1, mp, zero, false);  // fall through
        default: break;
      }
      uint32_t sh[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) sh[t] = static_cast<uint32_t>(rem[t] >> p) & ((1u << len) - 1u);
      square_all<WIDE, SMALL, NT>(x0, x1, m0, m1, mp, sh, true);
    }
    // s = 2^E mod m, then the W-bit quotient digits folded into the signed sum
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (WIDE) {
        reduce_once64(x0[t], x1[t], Mod64{m0[t], m1[t], mp[t]});
      } else if (x0[t] >= m0[t]) {
        x0[t] -= m0[t];
      }
    }
    if (A.alternating) fold_digits<WIDE, true, NT, LMAX>(acc, x0, x1, m0, m1, mp, vmask);
    else fold_digits<WIDE, false, NT, LMAX>(acc, x0, x1, m0, m1, mp, vmask);
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

// ---------------------------------------------------------------- tail terms
//
// A tail term is B_k = 2^e / m with e < 0 (Eq. 5); its W-bit value is
// floor(2^(W+e)/m) = floor(floor(2^W/m) / 2^-e): the fraction of 1/m, shifted
// (Sec. 4.3: shift by b bits, then divide to W - b bits).  There are only about
// W/step of them per series, so one thread per term with plain loops.
// t (W/32 limbs, signed by (-1)^k and the series sign, mod 2^W) of tail term k.
__device__ void tail_term(const TailArgs& A, const uint64_t k, uint32_t* t) {
  const int64_t e = static_cast<int64_t>(A.d) + A.c - static_cast<int64_t>(A.step) * static_cast<int64_t>(k);
  const uint32_t L = A.L;
  const int64_t bshift = -e;  // 1 <= bshift <= W
  const uint64_t m = static_cast<uint64_t>(A.a) * k + A.b;
  uint32_t q[kMaxLimbs];
  for (uint32_t i = 0; i < L; ++i) { q[i] = 0; t[i] = 0; }
  if (e >= 0 || bshift > static_cast<int64_t>(A.W)) return;
  const uint32_t b = static_cast<uint32_t>(bshift);
  if (m == 1) {
    const uint32_t bit = A.W - b;  // floor(2^(W-b) / 1), below 2^W since b >= 1
    t[bit >> 5] = 1u << (bit & 31u);
  } else {
    uint64_t x = 1;  // 2^W mod m by doubling; m < 2^62
    for (uint32_t i = 0; i < A.W; ++i) {
      x <<= 1;
      if (x >= m) x -= m;
    }
    Mod64 M{lo32(m), hi32(m), neg_inverse32(lo32(m))};
    uint32_t x0 = lo32(x), x1 = hi32(x);
    for (uint32_t i = 0; i < L; ++i) q[i] = hensel_step64(x0, x1, M);
    // t = q >> b
    const uint32_t bl = b >> 5, bb = b & 31u;
    for (uint32_t i = 0; i < L; ++i) {
      const uint32_t src = i + bl;
      uint32_t lo = src < L ? q[src] : 0u;
      uint32_t hi = src + 1 < L ? q[src + 1] : 0u;
      t[i] = bb ? ((lo >> bb) | (hi << (32u - bb))) : lo;
    }
  }
  const bool neg = ((A.alternating && (k & 1ull)) ? 1u : 0u) ^ A.negate;
  if (neg) {
    uint64_t carry = 1;
    for (uint32_t i = 0; i < L; ++i) {
      const uint64_t s = static_cast<uint64_t>(~t[i]) + carry;
      t[i] = static_cast<uint32_t>(s);
      carry = s >> 32;
    }
  }
}

__global__ void tail_kernel(const TailArgs A) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= A.count) return;
  uint32_t t[kMaxLimbs];
  tail_term(A, A.k_begin + tid, t);
  for (uint32_t i = 0; i < A.L; ++i)
    if (t[i]) atomicAdd(A.slots + i, static_cast<unsigned long long>(t[i]));
}

// ---------------------------------------------------------------- fold / finalize

__global__ void zero_slots_kernel(unsigned long long* slots, int L) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) slots[i] = 0;
}

__device__ void fold(const unsigned long long* slots, int L, uint32_t* S) {
  unsigned long long carry = 0;
  for (int i = 0; i < L; ++i) {
    const unsigned long long s = slots[i] + carry;
    S[i] = static_cast<uint32_t>(s);
    carry = s >> 32;
  }
}

__global__ void fold_limbs_kernel(const unsigned long long* slots, int L, uint32_t* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t S[kMaxLimbs];
  fold(slots, L, S);
  for (int i = 0; i < L; ++i) out[i] = S[i];
}

// (x mod 2^low) >= B for an L-limb x and a 64-bit B
__device__ bool low_bits_at_least(const uint32_t* x, int low, uint64_t B) {
  for (int i = 2; i * 32 < low; ++i) {
    uint32_t limb = x[i];
    const int top = low - i * 32;
    if (top < 32) limb &= (1u << top) - 1u;
    if (limb) return true;
  }
  uint64_t v = (static_cast<uint64_t>(x[1]) << 32) | x[0];
  if (low < 64) v &= (1ull << low) - 1ull;
  return v >= B;
}

// Guard-bit rule: with |S - exact| < B units, the top b bits are certified iff
// B <= (S mod 2^(W-b)) <= 2^(W-b) - B.  Returns the largest certified b <= P.
__device__ uint32_t certified_bits(const uint32_t* S, int L, uint32_t P, uint64_t B) {
  const int W = 32 * L;
  uint32_t neg[kMaxLimbs];
  uint64_t carry = 1;
  for (int i = 0; i < L; ++i) {
    const uint64_t s = static_cast<uint64_t>(~S[i]) + carry;
    neg[i] = static_cast<uint32_t>(s);
    carry = s >> 32;
  }
  for (int b = static_cast<int>(P); b >= 0; --b) {
    const int low = W - b;
    if (low_bits_at_least(S, low, B) && low_bits_at_least(neg, low, B)) return static_cast<uint32_t>(b);
  }
  return 0;
}

// S = carry-propagated slots; output bytes (MSB first), certified count, raw limbs.
__device__ void finalize_into(const unsigned long long* slots, int L, uint32_t P, uint64_t bound, uint8_t* out,
                              uint32_t* valid, uint32_t* out_limbs) {
  uint32_t S[kMaxLimbs + 1];
  unsigned long long carry = 0;
  for (int i = 0; i < L; ++i) {
    const unsigned long long v = __ldcg(slots + i) + carry;  // slots were written by atomics
    S[i] = static_cast<uint32_t>(v);
    carry = v >> 32;
  }
  S[L] = 0;
  if (out_limbs)
    for (int i = 0; i < L; ++i) out_limbs[i] = S[i];
  const int W = 32 * L;
  const uint32_t nbytes = (P + 7) / 8;
  for (uint32_t i = 0; i < nbytes; ++i) {
    const int pos = W - 8 * static_cast<int>(i + 1);  // >= W - P - 7 >= 25
    const int li = pos >> 5, sh = pos & 31;
    uint32_t byte = S[li] >> sh;
    if (sh > 24) byte |= S[li + 1] << (32 - sh);
    byte &= 0xffu;
    const uint32_t have = P - 8 * i;
    if (have < 8) byte &= (0xffu << (8 - have)) & 0xffu;
    out[i] = static_cast<uint8_t>(byte);
  }
  if (valid) *valid = certified_bits(S, L, P, bound);
}

__global__ void finalize_bits_kernel(const unsigned long long* slots, int L, uint32_t P, uint64_t bound,
                                     uint8_t* out, uint32_t* valid, uint32_t* out_limbs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  finalize_into(slots, L, P, bound, out, valid, out_limbs);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
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

// Called by one thread after its part of query q's last job is in the
// accumulators (and fenced): the thread that retires the query's last job
// finalizes it.
__device__ void retire_job(const BatchDev& B, uint32_t q) {
  if (atomicSub(B.jobs_left + q, 1u) == 1u) {
    __threadfence();
    const QueryDesc Q = B.queries[q];
    finalize_into(B.accum + static_cast<uint64_t>(q) * kMaxLimbs, static_cast<int>(Q.L), Q.P, Q.bound,
                  B.out + Q.out_offset, B.valid + q, nullptr);
    B.done_ns[q] = global_ns();
  }
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

__global__ void timestamp_kernel(unsigned long long* where) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *where = global_ns();
}

// Tail jobs: one warp per job, one term per lane at a time.
__global__ void queue_tail_kernel(const BatchDev B, const uint32_t tail_begin, const uint32_t tail_end,
                                  unsigned int* cursor) {
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    uint32_t j = 0;
    if (lane == 0) j = tail_begin + atomicAdd(cursor, 1u);
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= tail_end) break;
    const TailArgs A = B.tails[j];
    uint32_t t[kMaxLimbs];
    for (uint64_t i = lane; i < A.count; i += 32) {
      tail_term(A, A.k_begin + i, t);
      for (uint32_t l = 0; l < A.L; ++l)
        if (t[l]) atomicAdd(A.slots + l, static_cast<unsigned long long>(t[l]));
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) retire_job(B, B.tail_query[j]);
    __syncwarp();
  }
}

// ---------------------------------------------------------------- IMAD probe

__device__ __forceinline__ uint32_t smid() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

template <int KIND>
__global__ void imad_probe_kernel(int iters, unsigned long long* cycles, uint32_t* smids, uint32_t* sink) {
  uint32_t a[8];
  uint64_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = threadIdx.x * 2654435761u + j;
    w[j] = a[j];
  }
  const uint32_t b = 0x9e3779b9u ^ blockIdx.x;
  const uint32_t c = 0x7f4a7c15u;
  __syncthreads();
  const unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
        if (KIND == 1) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
        if (KIND == 2) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[j]) : "r"(static_cast<uint32_t>(w[j])), "r"(b));
        if (KIND == 3) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[j]) : "r"(b));
      }
    }
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) x ^= a[j] ^ static_cast<uint32_t>(w[j]) ^ static_cast<uint32_t>(w[j] >> 32);
  if (x == 0x12345678u) sink[0] = x;
  if (threadIdx.x == 0) {
    cycles[blockIdx.x] = t1 - t0;
    smids[blockIdx.x] = smid();
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers

namespace {

template <int LMAX, int PATH, int S>
cudaError_t launch_head_t(const HeadArgs& a, int blocks, int threads, cudaStream_t s) {
  const uint64_t tile = 32ull * S * a.run;
  const uint64_t ntiles = (a.count + tile - 1) / tile;
  head_kernel<LMAX, PATH, S><<<blocks, threads, 0, s>>>(a, ntiles);
  return cudaGetLastError();
}

template <int LMAX, int PATH, int S>
int occupancy_t(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, head_kernel<LMAX, PATH, S>, threads, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int LMAX, int PATH>
int occupancy_p(int streams, int threads) {
  return streams == 2 ? occupancy_t<LMAX, PATH, 2>(threads) : occupancy_t<LMAX, PATH, 1>(threads);
}

template <int LMAX>
int occupancy_l(int path, int streams, int threads) {
  if (path == 2) return occupancy_p<LMAX, 2>(streams, threads);
  if (path == 1) return occupancy_p<LMAX, 1>(streams, threads);
  return occupancy_p<LMAX, 0>(streams, threads);
}

template <int LMAX, int PATH>
cudaError_t launch_head_p(const HeadArgs& a, int streams, int blocks, int threads, cudaStream_t s) {
  return streams == 2 ? launch_head_t<LMAX, PATH, 2>(a, blocks, threads, s)
                      : launch_head_t<LMAX, PATH, 1>(a, blocks, threads, s);
}

template <int LMAX>
cudaError_t launch_head_l(const HeadArgs& a, int path, int streams, int blocks, int threads, cudaStream_t s) {
  if (path == 2) return launch_head_p<LMAX, 2>(a, streams, blocks, threads, s);
  if (path == 1) return launch_head_p<LMAX, 1>(a, streams, blocks, threads, s);
  return launch_head_p<LMAX, 0>(a, streams, blocks, threads, s);
}

bool valid_head_threads(int threads) { return threads >= 32 && threads <= kHeadThreads && threads % 32 == 0; }
}  // namespace

int head_occupancy(int path, int streams, int lmax, int threads) {
  if (!valid_head_threads(threads)) return 1;
  switch (lmax) {
    case 3: return occupancy_l<3>(path, streams, threads);
    case 4: return occupancy_l<4>(path, streams, threads);
    case 6: return occupancy_l<6>(path, streams, threads);
    case 10: return occupancy_l<10>(path, streams, threads);
    case 16: return occupancy_l<16>(path, streams, threads);
    case 24: return occupancy_l<24>(path, streams, threads);
    case 40: return occupancy_l<40>(path, streams, threads);
    default: return 1;
  }
}

namespace {
template <int LMAX, int PATH, int S>
int queue_occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, queue_kernel<LMAX, PATH, S>, kHeadThreads, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int LMAX, int PATH>
int queue_occupancy_p(int streams) {
  return streams == 2 ? queue_occupancy_t<LMAX, PATH, 2>() : queue_occupancy_t<LMAX, PATH, 1>();
}

template <int LMAX>
int queue_occupancy_l(int path, int streams) {
  if (path == 2) return queue_occupancy_p<LMAX, 2>(streams);
  if (path == 1) return queue_occupancy_p<LMAX, 1>(streams);
  return queue_occupancy_p<LMAX, 0>(streams);
}

template <int LMAX, int PATH>
cudaError_t launch_queue_p(const BatchDev& b, uint32_t jb, uint32_t je, unsigned int* cursor, int streams,
                           int blocks, cudaStream_t s) {
  if (streams == 2) queue_kernel<LMAX, PATH, 2><<<blocks, kHeadThreads, 0, s>>>(b, jb, je, cursor);
  else queue_kernel<LMAX, PATH, 1><<<blocks, kHeadThreads, 0, s>>>(b, jb, je, cursor);
  return cudaGetLastError();
}

template <int LMAX>
cudaError_t launch_queue_l(const BatchDev& b, uint32_t jb, uint32_t je, unsigned int* cursor, int path, int streams,
                           int blocks, cudaStream_t s) {
  if (path == 2) return launch_queue_p<LMAX, 2>(b, jb, je, cursor, streams, blocks, s);
  if (path == 1) return launch_queue_p<LMAX, 1>(b, jb, je, cursor, streams, blocks, s);
  return launch_queue_p<LMAX, 0>(b, jb, je, cursor, streams, blocks, s);
}
}  // namespace

int queue_occupancy(int path, int streams, int lmax) {
  switch (lmax) {
    case 3: return queue_occupancy_l<3>(path, streams);
    case 4: return queue_occupancy_l<4>(path, streams);
    case 6: return queue_occupancy_l<6>(path, streams);
    case 10: return queue_occupancy_l<10>(path, streams);
    case 16: return queue_occupancy_l<16>(path, streams);
    case 24: return queue_occupancy_l<24>(path, streams);
    case 40: return queue_occupancy_l<40>(path, streams);
    default: return 1;
  }
}

cudaError_t launch_queue(const BatchDev& b, uint32_t job_begin, uint32_t job_end, unsigned int* cursor, int path,
                         int streams, int lmax, int blocks, cudaStream_t s) {
  switch (lmax) {
    case 3: return launch_queue_l<3>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    case 4: return launch_queue_l<4>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    case 6: return launch_queue_l<6>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    case 10: return launch_queue_l<10>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    case 16: return launch_queue_l<16>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    case 24: return launch_queue_l<24>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    case 40: return launch_queue_l<40>(b, job_begin, job_end, cursor, path, streams, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_timestamp(unsigned long long* where, cudaStream_t s) {
  timestamp_kernel<<<1, 32, 0, s>>>(where);
  return cudaGetLastError();
}

cudaError_t launch_queue_tail(const BatchDev& b, uint32_t tail_begin, uint32_t tail_end, unsigned int* cursor,
                              int blocks, cudaStream_t s) {
  if (tail_begin >= tail_end) return cudaSuccess;
  queue_tail_kernel<<<blocks, 128, 0, s>>>(b, tail_begin, tail_end, cursor);
  return cudaGetLastError();
}

int head_lmax_for(int L, int bump) {
  for (int i = 0; i < kNumLmaxClasses; ++i)
    if (kLmaxClasses[i] >= L) return kLmaxClasses[std::min(kNumLmaxClasses - 1, i + std::max(0, bump))];
  return 0;
}

cudaError_t launch_head(const HeadArgs& a, int path, int streams, int lmax, int blocks, cudaStream_t s, int threads) {
  if (!valid_head_threads(threads)) return cudaErrorInvalidValue;
  switch (lmax) {
    case 3: return launch_head_l<3>(a, path, streams, blocks, threads, s);
    case 4: return launch_head_l<4>(a, path, streams, blocks, threads, s);
    case 6: return launch_head_l<6>(a, path, streams, blocks, threads, s);
    case 10: return launch_head_l<10>(a, path, streams, blocks, threads, s);
    case 16: return launch_head_l<16>(a, path, streams, blocks, threads, s);
    case 24: return launch_head_l<24>(a, path, streams, blocks, threads, s);
    case 40: return launch_head_l<40>(a, path, streams, blocks, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tail(const TailArgs& a, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = static_cast<int>((a.count + threads - 1) / threads);
  tail_kernel<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_zero_slots(unsigned long long* slots, int L, cudaStream_t s) {
  zero_slots_kernel<<<1, 64, 0, s>>>(slots, L);
  return cudaGetLastError();
}

cudaError_t launch_fold_limbs(const unsigned long long* slots, int L, uint32_t* out_limbs, cudaStream_t s) {
  fold_limbs_kernel<<<1, 32, 0, s>>>(slots, L, out_limbs);
  return cudaGetLastError();
}

cudaError_t launch_finalize_bits(const unsigned long long* slots, int L, uint32_t P, uint64_t bound,
                                 uint8_t* out_bytes, uint32_t* valid_bits, uint32_t* out_limbs, cudaStream_t s) {
  finalize_bits_kernel<<<1, 32, 0, s>>>(slots, L, P, bound, out_bytes, valid_bits, out_limbs);
  return cudaGetLastError();
}

cudaError_t launch_imad_probe(int kind, int blocks, int threads, int iters, unsigned long long* cycles_out,
                              uint32_t* smid_out, uint32_t* sink, cudaStream_t s) {
  switch (kind) {
    case 0: imad_probe_kernel<0><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    case 1: imad_probe_kernel<1><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    case 2: imad_probe_kernel<2><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    case 3: imad_probe_kernel<3><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bbp
