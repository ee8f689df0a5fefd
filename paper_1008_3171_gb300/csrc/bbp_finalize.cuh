// Device helpers shared by the finalize kernels and the persistent queue kernels:
// carry propagation of carry-save accumulators, the guard-bit validity rule
// (Sec. 3.1's caveat about runs of equal bits, read as an error bound), the output
// bits, and the retirement of a query whose last job has finished.
#pragma once

#include <cstdint>

#include "bbp_kernels.cuh"

namespace bbp {

// (x mod 2^low) >= B for an L-limb x and a 64-bit B
__device__ inline bool low_bits_at_least(const uint32_t* x, int low, uint64_t B) {
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
__device__ inline uint32_t certified_bits(const uint32_t* S, int L, uint32_t P, uint64_t B) {
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
__device__ inline void finalize_into(const unsigned long long* slots, int L, uint32_t P, uint64_t bound, uint8_t* out,
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

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Called by one thread after its part of query q's last job is in the
// accumulators (and fenced): the thread that retires the query's last job
// finalizes it.
__device__ inline void retire_job(const BatchDev& B, uint32_t q) {
  if (atomicSub(B.jobs_left + q, 1u) == 1u) {
    __threadfence();
    const QueryDesc Q = B.queries[q];
    finalize_into(B.accum + static_cast<uint64_t>(q) * kMaxLimbs, static_cast<int>(Q.L), Q.P, Q.bound,
                  B.out + Q.out_offset, B.valid + q, nullptr);
    B.done_ns[q] = global_ns();
  }
}

}  // namespace bbp
