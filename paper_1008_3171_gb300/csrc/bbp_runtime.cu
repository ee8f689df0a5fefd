// C ABI of libbbp (include/bbp.h): plans, single-query paths and statistics.
//
// A query (Sze, arXiv:1008.3171, Sec. 3) is planned on the host into term ranges
// (bbp_planner.cpp), each range is one kernel launch (bbp_kernels.cu) that folds
// its signed partial sum into L carry-save 64-bit accumulators on the device, and
// a finalize kernel turns the accumulators into the W-bit sum, the certified bit
// count and the top P bits.  Nothing of the arithmetic runs on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "bbp.h"
#include "bbp_kernels.cuh"
#include "bbp_planner.h"
#include "bbp_runtime.h"

using namespace bbp;

namespace bbp {

bbp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? BBP_OK : BBP_ECUDA; }

}  // namespace bbp

#define BBP_CUDA(expr)                                  \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return BBP_ECUDA;            \
  } while (0)

namespace {

constexpr uint32_t kDefaultGuard = 64;
constexpr int kDefaultRun = 64;

bool valid_formula(int f) { return f == BBP_BELLARD || f == BBP_BBP; }

int pick_lmax(uint32_t W, int bump) { return head_lmax_for(static_cast<int>(W / 32), bump); }

}  // namespace

extern "C" {

uint32_t bbp_abi_version(void) { return BBP_ABI_VERSION; }

const char* bbp_status_str(bbp_status s) {
  switch (s) {
    case BBP_OK: return "ok";
    case BBP_PENDING: return "pending";
    case BBP_EINVAL: return "invalid argument";
    case BBP_ENOMEM: return "out of memory";
    case BBP_ECUDA: return "CUDA error";
    case BBP_EBUSY: return "busy: no slot or accumulator memory free";
    case BBP_ETIMEOUT: return "bounded device wait expired";
    case BBP_ERANGE: return "position out of range (modulus would reach 2^60)";
    case BBP_EINVALID_BITS: return "fewer bits certified than requested";
    case BBP_ENOTFOUND: return "unknown ticket";
    case BBP_ESCRATCH: return "working precision exceeds the fixed scratch of the no-allocation entry point";
  }
  return "unknown status";
}

void bbp_plan_opts_default(bbp_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->guard_bits = kDefaultGuard;
}

bbp_status bbp_plan_create(bbp_plan* out, const bbp_plan_opts* opts) {
  if (!out) return BBP_EINVAL;
  *out = nullptr;
  bbp_plan_opts o;
  bbp_plan_opts_default(&o);
  if (opts) o = *opts;
  if (o.guard_bits == 0) o.guard_bits = kDefaultGuard;
  if (o.guard_bits % 32 != 0 || o.guard_bits >= kMaxWorkingBits) return BBP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return BBP_ECUDA;
  if (o.device < 0 || o.device >= ndev) return BBP_EINVAL;
  BBP_CUDA(cudaSetDevice(o.device));
  bbp_plan p = new (std::nothrow) bbp_plan_s();
  if (!p) return BBP_ENOMEM;
  p->device = o.device;
  p->guard = o.guard_bits;
  p->profile = o.profile != 0;
  p->strict = o.strict != 0;
  p->accum_budget = o.accum_mem_budget ? o.accum_mem_budget : (64u << 20);
  p->max_slots = o.max_slots ? o.max_slots : 4096u;
  p->run = kDefaultRun;
  p->streams = 0;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, o.device) != cudaSuccess) {
    delete p;
    return BBP_ECUDA;
  }
  p->sm_count = prop.multiProcessorCount;
  if (o.stream) {
    p->stream = static_cast<cudaStream_t>(o.stream);
    p->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete p;
      return BBP_ECUDA;
    }
    p->own_stream = true;
  }
  bool ok = cudaMalloc(&p->d_slots, sizeof(unsigned long long) * kMaxLimbs) == cudaSuccess &&
            cudaMalloc(&p->d_limbs, sizeof(uint32_t) * kMaxLimbs) == cudaSuccess &&
            cudaMalloc(&p->d_bytes, kMaxWorkingBits / 8) == cudaSuccess &&
            cudaMalloc(&p->d_valid, sizeof(uint32_t)) == cudaSuccess &&
            cudaMallocHost(&p->h_stage, 4096) == cudaSuccess &&
            cudaEventCreate(&p->ev0) == cudaSuccess && cudaEventCreate(&p->ev1) == cudaSuccess;
  if (!ok) {
    bbp_plan_destroy(p);
    return BBP_ENOMEM;
  }
  if (o.tune_table) load_tune_table(p, o.tune_table);
  *out = p;
  return BBP_OK;
}

bbp_status bbp_plan_destroy(bbp_plan p) {
  if (!p) return BBP_OK;
  cudaSetDevice(p->device);
  release_serve_state(p);
  if (p->stream) cudaStreamSynchronize(p->stream);
  release_batch_state(p);
  cudaFree(p->d_slots);
  cudaFree(p->d_limbs);
  cudaFree(p->d_bytes);
  cudaFree(p->d_valid);
  cudaFreeHost(p->h_stage);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
  return BBP_OK;
}

uint32_t bbp_working_bits(bbp_plan p, uint32_t P) {
  uint32_t W = 0;
  if (!p || !working_bits(P, p->guard, &W)) return 0;
  return W;
}

bbp_status bbp_series_extent(bbp_formula f, uint32_t denominator, uint64_t n, uint32_t W, uint64_t* he,
                             uint64_t* ne) {
  if (!valid_formula(f) || n == 0 || W == 0 || W % 32 != 0) return BBP_EINVAL;
  const FormulaDef& F = formula_def(f);
  if (denominator >= F.count) return BBP_EINVAL;
  if (he) *he = head_end(F, denominator, n - 1);
  if (ne) *ne = natural_end(F, denominator, n - 1, W);
  return BBP_OK;
}

bbp_status bbp_plan_stats(bbp_plan p, bbp_stats* out) {
  if (!p || !out) return BBP_EINVAL;
  *out = p->stats;
  return BBP_OK;
}

}  // extern "C"

namespace bbp {

// Launches every range of `ranges` (all of one query, same W) into `slots`.
bbp_status launch_ranges(bbp_plan p, int f, uint64_t n, uint32_t W, const std::vector<TermRange>& ranges,
                         unsigned long long* slots, cudaStream_t st) {
  const FormulaDef& F = formula_def(f);
  const uint32_t L = W / 32;
  const int lmax = pick_lmax(W, p->limb_bump);
  if (lmax == 0) return BBP_EINVAL;
  float total_ms = 0;
  TailSet tails{};
  for (const TermRange& r : ranges) {
    const SeriesDef& s = F.s[r.j];
    const bool odd_start = F.alternating && (r.k_begin & 1ull);
    if (r.tail) {  // collected, and launched together once the set is full or the ranges end
      TailArgs& a = tails.a[tails.n++];
      a = TailArgs{};
      a.d = n - 1;
      a.k_begin = r.k_begin;
      a.count = r.count;
      a.a = s.a;
      a.b = s.b;
      a.c = s.c;
      a.step = F.step;
      a.W = W;
      a.L = L;
      a.alternating = F.alternating;
      a.negate = s.sign < 0 ? 1u : 0u;
      a.slots = slots;
      p->stats.terms += r.count;
      if (tails.n == kMaxTailSet) {
        BBP_CUDA(launch_tail_set(tails, st));
        p->stats.kernel_launches++;
        tails.n = 0;
      }
      continue;
    }
    HeadArgs a{};
    a.d = n - 1;
    a.k_begin = r.k_begin;
    a.count = r.count;
    a.a = s.a;
    a.b = s.b;
    a.c = s.c;
    a.step = F.step;
    a.W = W;
    a.L = L;
    a.alternating = F.alternating;
    a.negate = ((s.sign < 0) != odd_start) ? 1u : 0u;
    a.window = r.window;
    a.first = r.first;
    a.first_max = r.first_max;
    a.slots = slots;
    const int streams = head_streams(p, r.path);
    const int warps_per_block = p->cta / 32;
    const int occ = head_occupancy(r.path, streams, lmax, p->cta);
    const uint64_t resident_warps = static_cast<uint64_t>(occ) * p->sm_count * warps_per_block;
    // a short range takes fewer consecutive terms per stream, so that its tiles
    // spread over the GPU's resident warps instead of a few warps running long runs
    uint32_t run = static_cast<uint32_t>(p->run);
    auto tiles_for = [&](uint32_t rn) { return (r.count + 32ull * streams * rn - 1) / (32ull * streams * rn); };
    while (run % 4 == 0 && tiles_for(run) < resident_warps) run /= 2;
    a.run = run;
    const uint64_t ntiles = tiles_for(run);
    const uint64_t want = (ntiles + warps_per_block - 1) / warps_per_block;
    const int blocks = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(occ) * p->sm_count)));
    if (p->profile) BBP_CUDA(cudaEventRecord(p->ev0, st));
    BBP_CUDA(launch_head(a, r.path, streams, lmax, blocks, st, p->cta));
    if (p->profile) {
      BBP_CUDA(cudaEventRecord(p->ev1, st));
      BBP_CUDA(cudaEventSynchronize(p->ev1));
      float ms = 0;
      BBP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
      total_ms += ms;
    }
    p->stats.kernel_launches++;
    p->stats.head_launches++;
    p->stats.terms += r.count;
    p->stats.head_terms += r.count;
    p->stats.imad_model += r.imad;
  }
  if (tails.n > 0) {
    BBP_CUDA(launch_tail_set(tails, st));
    p->stats.kernel_launches++;
  }
  p->stats.head_ms += total_ms;
  return BBP_OK;
}

bbp_status plan_query(bbp_plan p, int f, uint64_t n, uint32_t W, int j_only, uint64_t k_lo, uint64_t k_hi,
                      std::vector<TermRange>& ranges, uint64_t* n_terms) {
  const FormulaDef& F = formula_def(f);
  const int lmax = pick_lmax(W, p->limb_bump);
  uint64_t N = 0;
  for (uint32_t j = 0; j < F.count; ++j) {
    if (j_only >= 0 && static_cast<int>(j) != j_only) continue;
    const int st = plan_series(F, j, n, W, static_cast<uint32_t>(lmax), k_lo, k_hi, ranges, p->wide_min_bits);
    if (st == -6) return BBP_ERANGE;
    if (st != 0) return BBP_EINVAL;
    N += natural_end(F, j, n - 1, W);
  }
  if (n_terms) *n_terms = N;
  return BBP_OK;
}

}  // namespace bbp

extern "C" {

bbp_status bbp_partial_sum_async(bbp_plan p, bbp_formula f, uint32_t denominator, uint64_t k_begin,
                                 uint64_t k_end, uint64_t n, uint32_t P, uint32_t* d_out_limbs, void* stream) {
  if (!p || !valid_formula(f) || n == 0 || P == 0 || k_begin > k_end || !d_out_limbs) return BBP_EINVAL;
  if (denominator >= formula_def(f).count) return BBP_EINVAL;
  uint32_t W;
  if (!working_bits(P, p->guard, &W)) return BBP_EINVAL;
  std::vector<TermRange> ranges;
  const bbp_status st = plan_query(p, f, n, W, static_cast<int>(denominator), k_begin, k_end, ranges, nullptr);
  if (st != BBP_OK) return st;
  BBP_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
  p->stats = bbp_stats{};
  BBP_CUDA(launch_zero_slots(p->d_slots, static_cast<int>(W / 32), s));
  const bbp_status ls = launch_ranges(p, f, n, W, ranges, p->d_slots, s);
  if (ls != BBP_OK) return ls;
  BBP_CUDA(launch_fold_limbs(p->d_slots, static_cast<int>(W / 32), d_out_limbs, s));
  p->stats.kernel_launches += 2;
  return BBP_OK;
}

bbp_status bbp_partial_sum(bbp_plan p, bbp_formula f, uint32_t denominator, uint64_t k_begin, uint64_t k_end,
                           uint64_t n, uint32_t P, uint32_t* out_limbs) {
  if (!p || !out_limbs) return BBP_EINVAL;
  bbp_status st = bbp_partial_sum_async(p, f, denominator, k_begin, k_end, n, P, p->d_limbs, p->stream);
  if (st != BBP_OK) return st;
  const uint32_t L = bbp_working_bits(p, P) / 32;
  BBP_CUDA(cudaMemcpyAsync(p->h_stage, p->d_limbs, sizeof(uint32_t) * L, cudaMemcpyDeviceToHost, p->stream));
  BBP_CUDA(cudaStreamSynchronize(p->stream));
  std::memcpy(out_limbs, p->h_stage, sizeof(uint32_t) * L);
  return BBP_OK;
}

bbp_status bbp_bits_async(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, uint8_t* d_out, uint32_t* d_valid,
                          uint32_t* d_limbs, void* stream) {
  if (!p || !valid_formula(f) || n == 0 || P == 0 || !d_out) return BBP_EINVAL;
  uint32_t W;
  if (!working_bits(P, p->guard, &W)) return BBP_EINVAL;
  std::vector<TermRange> ranges;
  uint64_t N = 0;
  const bbp_status st = plan_query(p, f, n, W, -1, 0, UINT64_MAX, ranges, &N);
  if (st != BBP_OK) return st;
  BBP_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
  p->stats = bbp_stats{};
  BBP_CUDA(launch_zero_slots(p->d_slots, static_cast<int>(W / 32), s));
  const bbp_status ls = launch_ranges(p, f, n, W, ranges, p->d_slots, s);
  if (ls != BBP_OK) return ls;
  const uint64_t bound = N + formula_def(f).count + 1;  // |S - exact| < N + J + 1 units
  BBP_CUDA(launch_finalize_bits(p->d_slots, static_cast<int>(W / 32), P, bound, d_out, d_valid, d_limbs, s));
  p->stats.kernel_launches += 2;
  return BBP_OK;
}

bbp_status bbp_shard_range(bbp_formula f, uint32_t denominator, uint64_t n, uint32_t W, uint32_t shard,
                           uint32_t nshards, uint64_t* k_begin, uint64_t* k_end) {
  if (!valid_formula(f) || n == 0 || W == 0 || W % 32 != 0 || nshards == 0 || shard >= nshards) return BBP_EINVAL;
  const FormulaDef& F = formula_def(f);
  if (denominator >= F.count) return BBP_EINVAL;
  uint64_t kb = 0, ke = 0;
  shard_range(F, denominator, n, W, shard, nshards, &kb, &ke);
  if (k_begin) *k_begin = kb;
  if (k_end) *k_end = ke;
  return BBP_OK;
}

bbp_status bbp_explain(bbp_formula f, uint64_t n, uint32_t P, uint32_t guard_bits, uint32_t wide_min_bits,
                       bbp_range* out, uint32_t cap, uint32_t* count, uint64_t* terms) {
  uint32_t W;
  if (!valid_formula(f) || n == 0 || !count || (cap > 0 && !out) || !working_bits(P, guard_bits, &W))
    return BBP_EINVAL;
  if (wide_min_bits < static_cast<uint32_t>(kWideFloorBits) || wide_min_bits > static_cast<uint32_t>(kWideMinBits))
    return BBP_EINVAL;
  const FormulaDef& F = formula_def(f);
  const int lmax = head_lmax_for(static_cast<int>(W / 32));
  if (lmax == 0) return BBP_EINVAL;
  std::vector<TermRange> ranges;
  for (uint32_t j = 0; j < F.count; ++j) {
    const int st = plan_series(F, j, n, W, static_cast<uint32_t>(lmax), 0, UINT64_MAX, ranges,
                               static_cast<int>(wide_min_bits));
    if (st == -6) return BBP_ERANGE;
    if (st != 0) return BBP_EINVAL;
  }
  uint64_t total = 0;
  for (size_t i = 0; i < ranges.size(); ++i) {
    const TermRange& r = ranges[i];
    total += r.count;
    if (i < cap) {
      bbp_range& o = out[i];
      o.denominator = r.j;
      o.tail = r.tail;
      o.path = r.path;
      o.window = r.window;
      o.first = r.first;
      o.first_max = r.first_max;
      o.k_begin = r.k_begin;
      o.count = r.count;
      o.imad = r.imad;
    }
  }
  *count = static_cast<uint32_t>(ranges.size());
  if (terms) *terms = total;
  return BBP_OK;
}

bbp_status bbp_accumulate_async(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, uint32_t shard, uint32_t nshards,
                                unsigned long long* d_slots, void* stream) {
  if (!p || !valid_formula(f) || n == 0 || P == 0 || !d_slots || nshards == 0 || shard >= nshards)
    return BBP_EINVAL;
  uint32_t W;
  if (!working_bits(P, p->guard, &W)) return BBP_EINVAL;
  const FormulaDef& F = formula_def(f);
  std::vector<TermRange> ranges;
  for (uint32_t j = 0; j < F.count; ++j) {
    uint64_t kb, ke;
    shard_range(F, j, n, W, shard, nshards, &kb, &ke);
    const bbp_status st = plan_query(p, f, n, W, static_cast<int>(j), kb, ke, ranges, nullptr);
    if (st != BBP_OK) return st;
  }
  BBP_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
  p->stats = bbp_stats{};
  return launch_ranges(p, f, n, W, ranges, d_slots, s);
}

bbp_status bbp_finalize_async(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, const unsigned long long* d_slots,
                              uint8_t* d_out, uint32_t* d_valid, uint32_t* d_limbs, void* stream) {
  if (!p || !valid_formula(f) || n == 0 || P == 0 || !d_slots || !d_out) return BBP_EINVAL;
  uint32_t W;
  if (!working_bits(P, p->guard, &W)) return BBP_EINVAL;
  uint64_t N = 0;
  const FormulaDef& F = formula_def(f);
  for (uint32_t j = 0; j < F.count; ++j) N += natural_end(F, j, n - 1, W);
  BBP_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
  BBP_CUDA(launch_finalize_bits(d_slots, static_cast<int>(W / 32), P, N + F.count + 1, d_out, d_valid, d_limbs, s));
  return BBP_OK;
}

bbp_status bbp_bits_formula(bbp_plan p, bbp_formula f, uint64_t n, uint32_t P, uint8_t* out, uint32_t* valid_bits) {
  if (!p || !out) return BBP_EINVAL;
  bbp_status st = bbp_bits_async(p, f, n, P, p->d_bytes, p->d_valid, nullptr, p->stream);
  if (st != BBP_OK) return st;
  const uint32_t nbytes = (P + 7) / 8;
  uint8_t* h = static_cast<uint8_t*>(p->h_stage);
  BBP_CUDA(cudaMemcpyAsync(h, p->d_bytes, nbytes, cudaMemcpyDeviceToHost, p->stream));
  BBP_CUDA(cudaMemcpyAsync(h + 2048, p->d_valid, sizeof(uint32_t), cudaMemcpyDeviceToHost, p->stream));
  BBP_CUDA(cudaStreamSynchronize(p->stream));
  std::memcpy(out, h, nbytes);
  uint32_t valid;
  std::memcpy(&valid, h + 2048, sizeof(valid));
  if (valid_bits) *valid_bits = valid;
  if (p->strict && valid < P) return BBP_EINVALID_BITS;
  return BBP_OK;
}

bbp_status bbp_bits(bbp_plan p, uint64_t n, uint32_t P, uint8_t* out, uint32_t* valid_bits) {
  return bbp_bits_formula(p, BBP_BELLARD, n, P, out, valid_bits);
}

bbp_status bbp_imad_probe(bbp_plan p, int kind, double* lanes_per_clk_per_sm) {
  if (!p || !lanes_per_clk_per_sm || kind < 0 || kind > 6) return BBP_EINVAL;
  BBP_CUDA(cudaSetDevice(p->device));
  const int blocks = p->sm_count;
  const int threads = 1024;
  const int iters = 4096;
  unsigned long long* d_cycles = nullptr;
  uint32_t* d_smid = nullptr;
  uint32_t* d_sink = nullptr;
  BBP_CUDA(cudaMalloc(&d_cycles, sizeof(unsigned long long) * blocks));
  BBP_CUDA(cudaMalloc(&d_smid, sizeof(uint32_t) * blocks));
  BBP_CUDA(cudaMalloc(&d_sink, sizeof(uint32_t)));
  cudaError_t e = launch_imad_probe(kind, blocks, threads, iters, d_cycles, d_smid, d_sink, p->stream);
  std::vector<unsigned long long> cycles(blocks);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cycles.data(), d_cycles, sizeof(unsigned long long) * blocks,
                                            cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  cudaFree(d_cycles);
  cudaFree(d_smid);
  cudaFree(d_sink);
  if (e != cudaSuccess) return BBP_ECUDA;
  std::sort(cycles.begin(), cycles.end());
  const double med = static_cast<double>(cycles[cycles.size() / 2]);
  const double ops = static_cast<double>(threads) * iters * 64.0;
  *lanes_per_clk_per_sm = med > 0 ? ops / med : 0.0;
  return BBP_OK;
}

}  // extern "C"
