// sm_103a kernels for BBP digit extraction (Sze, arXiv:1008.3171, Sec. 3 and 4.3),
// except the head-term kernels (bbp_tile.cuh, instantiated per accumulator class in
// bbp_lmax*.cu), and the host-side dispatch to all of them.
//
//   tail_kernel    -- tail terms B_k (e < 0): t = floor(2^W / m) >> -e.
//   fold / finalize -- carry propagation of the carry-save sum, the guard-bit
//                     validity rule, and the top P output bits.
//   queue_tail_kernel -- tail jobs of a batched pass.
//   imad_probe     -- issue-rate microbenchmark of the integer multiply pipe.
#include <cuda_runtime.h>

#include <algorithm>

#include "bbp_device.cuh"
#include "bbp_finalize.cuh"
#include "bbp_kernels.cuh"

namespace bbp {
namespace {

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

// The tail ranges of several series in one launch: thread i takes the i-th term of
// the ranges laid end to end.
__global__ void tail_set_kernel(const TailSet S) {
  uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint32_t r = 0;
  while (r < S.n && i >= S.a[r].count) i -= S.a[r++].count;
  if (r >= S.n) return;
  const TailArgs& A = S.a[r];
  uint32_t t[kMaxLimbs];
  tail_term(A, A.k_begin + i, t);
  for (uint32_t l = 0; l < A.L; ++l)
    if (t[l]) atomicAdd(A.slots + l, static_cast<unsigned long long>(t[l]));
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

__global__ void finalize_bits_kernel(const unsigned long long* slots, int L, uint32_t P, uint64_t bound,
                                     uint8_t* out, uint32_t* valid, uint32_t* out_limbs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  finalize_into(slots, L, P, bound, out, valid, out_limbs);
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
        if (KIND == 4) asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a[j]) : "r"(b));
        if (KIND == 5) {  // full product without an addend; both halves feed the next operand
          asm volatile("{\n\t.reg .u32 l, h, s;\n\t"
                       "mov.b64        {l, h}, %0;\n\t"
                       "add.u32        s, l, h;\n\t"
                       "mul.wide.u32   %0, s, %1;\n\t}"
                       : "+l"(w[j]) : "r"(b));
        }
        if (KIND == 6) {  // full product, its 64-bit addend applied by a separate add
          asm volatile("{\n\t.reg .u32 l, h;\n\t.reg .u64 p;\n\t"
                       "mov.b64        {l, h}, %0;\n\t"
                       "mul.wide.u32   p, l, %1;\n\t"
                       "add.u64        %0, %0, p;\n\t}"
                       : "+l"(w[j]) : "r"(b));
        }
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

// ---------------------------------------------------------------- dispatch

namespace {
bool valid_head_threads(int threads) { return threads >= 32 && threads <= kHeadThreads && threads % 32 == 0; }
}  // namespace

#define BBP_LMAX_CASES(X) X(3) X(4) X(6) X(10) X(16) X(24) X(40)

int head_occupancy(int path, int streams, int lmax, int threads) {
  if (!valid_head_threads(threads)) return 1;
  switch (lmax) {
#define BBP_CASE(L) \
  case L: return head_occupancy_l##L(path, streams, threads);
    BBP_LMAX_CASES(BBP_CASE)
#undef BBP_CASE
    default: return 1;
  }
}

int queue_occupancy(int path, int streams, int lmax) {
  switch (lmax) {
#define BBP_CASE(L) \
  case L: return queue_occupancy_l##L(path, streams);
    BBP_LMAX_CASES(BBP_CASE)
#undef BBP_CASE
    default: return 1;
  }
}

cudaError_t launch_queue(const BatchDev& b, uint32_t job_begin, uint32_t job_end, unsigned int* cursor, int path,
                         int streams, int lmax, int blocks, cudaStream_t s) {
  switch (lmax) {
#define BBP_CASE(L) \
  case L: return launch_queue_l##L(b, job_begin, job_end, cursor, path, streams, blocks, s);
    BBP_LMAX_CASES(BBP_CASE)
#undef BBP_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_head(const HeadArgs& a, int path, int streams, int lmax, int blocks, cudaStream_t s, int threads) {
  if (!valid_head_threads(threads)) return cudaErrorInvalidValue;
  switch (lmax) {
#define BBP_CASE(L) \
  case L: return launch_head_l##L(a, path, streams, blocks, threads, s);
    BBP_LMAX_CASES(BBP_CASE)
#undef BBP_CASE
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

cudaError_t launch_tail(const TailArgs& a, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = static_cast<int>((a.count + threads - 1) / threads);
  tail_kernel<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tail_set(const TailSet& set, cudaStream_t s) {
  uint64_t total = 0;
  for (uint32_t r = 0; r < set.n; ++r) total += set.a[r].count;
  if (total == 0) return cudaSuccess;
  const int threads = 128;
  tail_set_kernel<<<static_cast<unsigned>((total + threads - 1) / threads), threads, 0, s>>>(set);
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
    case 4: imad_probe_kernel<4><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    case 5: imad_probe_kernel<5><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    case 6: imad_probe_kernel<6><<<blocks, threads, 0, s>>>(iters, cycles_out, smid_out, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bbp
