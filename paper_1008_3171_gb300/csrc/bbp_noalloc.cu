// bbp_partial_sum_noalloc: a partial sum that allocates nothing.
//
// Who needs it: code that must not call cudaMalloc/cudaFree once it is running --
// for example a host application whose device memory is owned by a pooling
// allocator it may not bypass (a raw cudaMalloc can fail once the pool has
// reserved the GPU, and cudaFree synchronizes the whole device), a latency-bound
// loop that cannot afford those implicit synchronizations, or a plugin that runs
// with a fixed, preallocated memory budget.  Such a caller cannot create a plan
// (a plan allocates its accumulators), so this entry point takes its scratch from
// a fixed array compiled into the library instead, and its outputs from the caller.
//
// The scratch: kNoAllocMaxLimbs carry-save accumulators (8 bytes each, 320 bytes)
// in a file-scope __device__ array.  Every GPU that loads the library holds them
// until the process exits.  All calls on a device share the one array and the
// array keeps the last call's contents: each call zeroes it first, and calls that
// overlap on the GPU (different streams, or other threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "bbp.h"
#include "bbp_kernels.cuh"
#include "bbp_planner.h"

namespace {

constexpr int kNoAllocMaxLimbs = 40;  // W <= 1280 bits
constexpr int kMaxDevices = 64;
constexpr int kRun = 64;              // terms per stream run (the plan default)

static __device__ __align__(256) unsigned long long g_noalloc_slots[kNoAllocMaxLimbs];

// Host-side record of the array's device address and the SM count, per device.
std::mutex g_setup_mutex;
unsigned long long* g_slots_addr[kMaxDevices];
int g_sm_count[kMaxDevices];

// First call on a device: look up the device address of the array with that
// device current.  The symbol's host-side name is only a stand-in and must never
// be handed to a kernel.
bbp_status scratch_for_current_device(unsigned long long** slots, int* sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BBP_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return BBP_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_slots_addr[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_slots) != cudaSuccess || !addr) return BBP_ECUDA;
    int count = 0;
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count <= 0)
      return BBP_ECUDA;
    g_sm_count[dev] = count;
    g_slots_addr[dev] = static_cast<unsigned long long*>(addr);
  }
  *slots = g_slots_addr[dev];
  *sms = g_sm_count[dev];
  return BBP_OK;
}

uint64_t first_k_with_bits(uint32_t bits, uint32_t a, uint32_t b) {  // first k with a k + b >= 2^(bits-1)
  const uint64_t v = 1ull << (bits - 1);
  return v <= b ? 0 : (v - b + a - 1) / a;
}

}  // namespace

extern "C" bbp_status bbp_partial_sum_noalloc(bbp_formula f, uint32_t denominator, uint64_t k_begin,
                                              uint64_t k_end, uint64_t n, uint32_t P, uint32_t guard_bits,
                                              uint32_t* d_out_limbs, void* stream) {
  using namespace bbp;
  if ((f != BBP_BELLARD && f != BBP_BBP) || n == 0 || P == 0 || k_begin > k_end || !d_out_limbs) return BBP_EINVAL;
  const FormulaDef& F = formula_def(f);
  if (denominator >= F.count || guard_bits == 0 || guard_bits % 32 != 0) return BBP_EINVAL;
  const uint64_t W64 = (static_cast<uint64_t>(P) + 31) / 32 * 32 + guard_bits;
  if (W64 > 32ull * kNoAllocMaxLimbs) return BBP_ESCRATCH;
  const uint32_t W = static_cast<uint32_t>(W64);
  const uint32_t L = W / 32;
  const int lmax = head_lmax_for(static_cast<int>(L));
  if (lmax == 0) return BBP_ESCRATCH;

  unsigned long long* slots = nullptr;
  int sms = 0;
  const bbp_status setup = scratch_for_current_device(&slots, &sms);
  if (setup != BBP_OK) return setup;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  const SeriesDef& s = F.s[denominator];
  const uint64_t d = n - 1;
  const uint64_t he = head_end(F, denominator, d);
  const uint64_t ne = natural_end(F, denominator, d, W);
  const uint64_t hi = std::min(k_end, ne);
  if (k_begin < hi && static_cast<uint64_t>(s.a) * (hi - 1) + s.b >= (1ull << kMaxModulusBits)) return BBP_ERANGE;

  if (launch_zero_slots(slots, static_cast<int>(L), st) != cudaSuccess) return BBP_ECUDA;

  // head terms: one launch per modulus path the range touches (bit lengths up to 29,
  // 30-31, 32-46, 47-60), each with the window parameters of its largest modulus and
  // the term pairs per thread of a plan with default settings
  const uint64_t h0 = std::max(k_begin, s.b == 1 ? uint64_t{1} : uint64_t{0});
  const uint64_t h1 = std::min(hi, he);
  if (h0 < h1) {
    const uint32_t first_bits[3] = {kLazyMaxBits + 1, kWideMinBits, kSmallMaxBits + 1};  // paths 3, 1, 2
    uint64_t cuts[5] = {h0, h0, h0, h0, h1};
    for (int i = 0; i < 3; ++i) cuts[i + 1] = std::min(std::max(first_k_with_bits(first_bits[i], s.a, s.b), h0), h1);
    for (int part = 0; part < 4; ++part) {
      const uint64_t kb = cuts[part], ke = cuts[part + 1];
      if (kb >= ke) continue;
      const int lbits = bitlen(static_cast<uint64_t>(s.a) * (ke - 1) + s.b);
      const int path = path_for_bits(lbits);
      const int streams = path == 1 ? 2 : 1;
      uint8_t window, first, first_max;
      window_params(path, lbits, &window, &first, &first_max);
      HeadArgs a{};
      a.d = d;
      a.k_begin = kb;
      a.count = ke - kb;
      a.a = s.a;
      a.b = s.b;
      a.c = s.c;
      a.step = F.step;
      a.W = W;
      a.L = L;
      a.alternating = F.alternating;
      a.negate = ((s.sign < 0) != (F.alternating && (kb & 1ull))) ? 1u : 0u;
      a.run = kRun;
      a.window = window;
      a.first = first;
      a.first_max = first_max;
      a.slots = slots;
      const uint64_t tile = 32ull * static_cast<uint64_t>(streams) * kRun;
      const uint64_t ntiles = (a.count + tile - 1) / tile;
      const uint64_t want = (ntiles + kHeadThreads / 32 - 1) / (kHeadThreads / 32);
      const uint64_t cap = static_cast<uint64_t>(head_occupancy(path, streams, lmax)) * static_cast<uint64_t>(sms);
      const int blocks = static_cast<int>(std::max<uint64_t>(1, std::min(want, cap)));
      if (launch_head(a, path, streams, lmax, blocks, st) != cudaSuccess) return BBP_ECUDA;
    }
  }
  // tail terms
  const uint64_t t0 = std::max(k_begin, he);
  if (t0 < hi) {
    TailArgs a{};
    a.d = d;
    a.k_begin = t0;
    a.count = hi - t0;
    a.a = s.a;
    a.b = s.b;
    a.c = s.c;
    a.step = F.step;
    a.W = W;
    a.L = L;
    a.alternating = F.alternating;
    a.negate = s.sign < 0 ? 1u : 0u;
    a.slots = slots;
    if (launch_tail(a, st) != cudaSuccess) return BBP_ECUDA;
  }
  if (launch_fold_limbs(slots, static_cast<int>(L), d_out_limbs, st) != cudaSuccess) return BBP_ECUDA;
  return BBP_OK;
}
