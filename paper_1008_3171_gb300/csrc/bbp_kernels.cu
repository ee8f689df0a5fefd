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

#include "bbp_device.cuh"
#include "bbp_kernels.cuh"

namespace bbp {
namespace {

// ---------------------------------------------------------------- head terms
//
// Work split: a warp owns a tile of 32 * S * run consecutive terms; lane l, stream s
// owns the run starting at tile + (l S + s) run.  Runs keep R mod m incremental and
// keep the exponents of a warp within 10 * 32 * S * run of each other, so the
// ladder length (warp maximum of the exponent bit length) is almost always shared.
// Each stream evaluates a pair (k, k+1) per step, so (-1)^k is static in the code.
template <int LMAX, bool WIDE, int S>
__global__ void __launch_bounds__(kHeadThreads) head_kernel(const HeadArgs A, const uint64_t ntiles) {
  constexpr int NT = 2 * S;
  constexpr int RB = WIDE ? 64 : 32;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wid = threadIdx.x >> 5;
  const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t run = A.run;
  const uint64_t tile = 32ull * S * run;
  const uint64_t last = A.count - 1;
  const uint32_t window = A.window;
  const uint32_t wmask = (1u << window) - 1u;

  uint32_t acc[LMAX];
#pragma unroll
  for (int i = 0; i < LMAX; ++i) acc[i] = 0;

  for (uint64_t ti = warp; ti < ntiles; ti += nwarps) {
    uint64_t base[S], kcur[S];
    RTrack tr[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      base[s] = ti * tile + (static_cast<uint64_t>(lane) * S + s) * run;
      kcur[s] = A.k_begin + min(base[s], last);
      tr[s] = r_mod_m_bitserial<RB>(static_cast<uint64_t>(A.a) * kcur[s] + A.b);
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
          const uint64_t k = A.k_begin + min(rel, last);
          const uint64_t m = static_cast<uint64_t>(A.a) * k + A.b;
          if (k != kcur[s]) {
            r_mod_m_advance<RB>(tr[s], m, A.a);
            kcur[s] = k;
          }
          x0[t] = lo32(tr[s].r);
          x1[t] = hi32(tr[s].r);
          m0[t] = lo32(m);
          m1[t] = hi32(m);
          mp[t] = neg_inverse32(m0[t]);
          // E = d + c - step k + W >= W >= RB for head terms; v = E - RB
          const uint64_t E = A.d + static_cast<int64_t>(A.c) - static_cast<uint64_t>(A.step) * k + A.W;
          v[t] = E - RB;
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
      // remaining bits, top down, in groups of `window` bits aligned from the top;
      // the group's value is multiplied in (a shift) with its last squaring.
      int cnt = static_cast<int>(window);
      for (int p = low - 1; p >= 0; --p) {
        --cnt;
        if (p == 0) {
          const uint32_t gm = (1u << (window - static_cast<uint32_t>(cnt))) - 1u;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const uint32_t sh = static_cast<uint32_t>(rem[t]) & gm;
            if (WIDE) sqr_shift_redc64(x0[t], x1[t], sh, Mod64{m0[t], m1[t], mp[t]}, true);
            else x0[t] = sqr_shift_redc32(x0[t], sh, Mod32{m0[t], mp[t]}, true);
          }
        } else if (cnt == 0) {
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const uint32_t sh = static_cast<uint32_t>(rem[t] >> p) & wmask;
            if (WIDE) sqr_shift_redc64(x0[t], x1[t], sh, Mod64{m0[t], m1[t], mp[t]}, true);
            else x0[t] = sqr_shift_redc32(x0[t], sh, Mod32{m0[t], mp[t]}, true);
          }
          cnt = static_cast<int>(window);
        } else {
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            if (WIDE) sqr_shift_redc64(x0[t], x1[t], 0u, Mod64{m0[t], m1[t], mp[t]}, false);
            else x0[t] = sqr_shift_redc32(x0[t], 0u, Mod32{m0[t], mp[t]}, false);
          }
        }
      }
      // s = 2^E mod m, then the W-bit quotient digits, then the signed sum
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        uint32_t q[LMAX];
        if (WIDE) {
          Mod64 M{m0[t], m1[t], mp[t]};
          reduce_once64(x0[t], x1[t], M);
          hensel_digits64<LMAX>(x0[t], x1[t], M, q);
        } else {
          Mod32 M{m0[t], mp[t]};
          const uint32_t x = x0[t] >= m0[t] ? x0[t] - m0[t] : x0[t];
          hensel_digits32<LMAX>(x, M, q);
        }
        if (valid[t]) {
          if ((t & 1) && A.alternating) sub_limbs<LMAX>(acc, q);
          else add_limbs<LMAX>(acc, q);
        }
      }
    }
  }

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
__global__ void tail_kernel(const TailArgs A) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= A.count) return;
  const uint64_t k = A.k_begin + tid;
  const int64_t e = static_cast<int64_t>(A.d) + A.c - static_cast<int64_t>(A.step) * static_cast<int64_t>(k);
  const uint32_t L = A.L;
  const int64_t bshift = -e;  // 1 <= bshift <= W
  const uint64_t m = static_cast<uint64_t>(A.a) * k + A.b;
  uint32_t q[kMaxLimbs];
  uint32_t t[kMaxLimbs];
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
  uint64_t carry = 1;
  for (uint32_t i = 0; i < L; ++i) {
    uint32_t v = t[i];
    if (neg) {
      const uint64_t s = static_cast<uint64_t>(~v) + carry;
      v = static_cast<uint32_t>(s);
      carry = s >> 32;
    }
    if (v) atomicAdd(A.slots + i, static_cast<unsigned long long>(v));
  }
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

__global__ void finalize_bits_kernel(const unsigned long long* slots, int L, uint32_t P, uint64_t bound,
                                     uint8_t* out, uint32_t* valid, uint32_t* out_limbs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t S[kMaxLimbs + 1];
  fold(slots, L, S);
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
constexpr int kLmaxList[] = {3, 4, 6, 10, 16, 40};

template <int LMAX, bool WIDE, int S>
cudaError_t launch_head_t(const HeadArgs& a, int blocks, cudaStream_t s) {
  const uint64_t tile = 32ull * S * a.run;
  const uint64_t ntiles = (a.count + tile - 1) / tile;
  head_kernel<LMAX, WIDE, S><<<blocks, kHeadThreads, 0, s>>>(a, ntiles);
  return cudaGetLastError();
}

template <int LMAX, bool WIDE, int S>
int occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, head_kernel<LMAX, WIDE, S>, kHeadThreads, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int LMAX>
int occupancy_l(int wide, int streams) {
  if (wide) return streams == 2 ? occupancy_t<LMAX, true, 2>() : occupancy_t<LMAX, true, 1>();
  return streams == 2 ? occupancy_t<LMAX, false, 2>() : occupancy_t<LMAX, false, 1>();
}

template <int LMAX>
cudaError_t launch_head_l(const HeadArgs& a, int wide, int streams, int blocks, cudaStream_t s) {
  if (wide) return streams == 2 ? launch_head_t<LMAX, true, 2>(a, blocks, s) : launch_head_t<LMAX, true, 1>(a, blocks, s);
  return streams == 2 ? launch_head_t<LMAX, false, 2>(a, blocks, s) : launch_head_t<LMAX, false, 1>(a, blocks, s);
}
}  // namespace

int head_occupancy(int wide, int streams, int lmax) {
  switch (lmax) {
    case 3: return occupancy_l<3>(wide, streams);
    case 4: return occupancy_l<4>(wide, streams);
    case 6: return occupancy_l<6>(wide, streams);
    case 10: return occupancy_l<10>(wide, streams);
    case 16: return occupancy_l<16>(wide, streams);
    case 40: return occupancy_l<40>(wide, streams);
    default: return 1;
  }
}

int head_lmax_for(int L) {
  for (int v : kLmaxList)
    if (v >= L) return v;
  return 0;
}

cudaError_t launch_head(const HeadArgs& a, int wide, int streams, int lmax, int blocks, cudaStream_t s) {
  switch (lmax) {
    case 3: return launch_head_l<3>(a, wide, streams, blocks, s);
    case 4: return launch_head_l<4>(a, wide, streams, blocks, s);
    case 6: return launch_head_l<6>(a, wide, streams, blocks, s);
    case 10: return launch_head_l<10>(a, wide, streams, blocks, s);
    case 16: return launch_head_l<16>(a, wide, streams, blocks, s);
    case 40: return launch_head_l<40>(a, wide, streams, blocks, s);
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
