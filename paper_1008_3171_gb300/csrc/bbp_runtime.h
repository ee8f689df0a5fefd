// Internal state of a bbp_plan, shared by the runtime translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bbp.h"
#include "bbp_planner.h"

struct bbp_plan_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t guard = 64;
  bool profile = false;
  bool strict = false;
  size_t accum_budget = 0;
  uint32_t max_slots = 0;
  int sm_count = 0;
  // head-kernel tuning (terms per stream run; term pairs per thread, 0 = by path)
  int run = 64;
  int streams = 0;
  int grab = 4;  // batched pass: warp tiles handed out per queue operation
  int cta = 256;  // single-query head launches: threads per CTA (multiple of 32, <= 256)
  int limb_bump = 0;  // single-query head launches: accumulator limb class this many sizes above the smallest
  int wide_min_bits = bbp::kWideMinBits;  // moduli of at least this many bits take the 64-bit Montgomery path
  // single-query buffers
  unsigned long long* d_slots = nullptr;  // kMaxLimbs carry-save accumulators
  uint32_t* d_limbs = nullptr;
  uint8_t* d_bytes = nullptr;
  uint32_t* d_valid = nullptr;
  void* h_stage = nullptr;  // 4 KiB pinned staging
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bbp_stats stats{};
  // batched state (bbp_batch.cu) and serving engine (bbp_serve.cu)
  struct BatchState* batch = nullptr;
  struct ServeEngine* serve = nullptr;
};

namespace bbp {

// Term pairs per thread of the head and queue kernels on a modulus path: the tune
// table's value, else two on path 1 (the three-word squaring has the registers for
// a second independent pair at three CTAs per SM) and one elsewhere.
inline int head_streams(const bbp_plan_s* p, int path) { return p->streams > 0 ? p->streams : (path == 1 ? 2 : 1); }
// Terms of one warp tile on that path.
inline uint64_t tile_terms(const bbp_plan_s* p, int path) {
  return 32ull * static_cast<uint64_t>(head_streams(p, path)) * static_cast<uint64_t>(p->run);
}

bbp_status cuda_status(cudaError_t e);
bbp_status plan_query(bbp_plan p, int f, uint64_t n, uint32_t W, int j_only, uint64_t k_lo, uint64_t k_hi,
                      std::vector<TermRange>& ranges, uint64_t* n_terms);
bbp_status launch_ranges(bbp_plan p, int f, uint64_t n, uint32_t W, const std::vector<TermRange>& ranges,
                         unsigned long long* slots, cudaStream_t st);
void load_tune_table(bbp_plan p, const char* path);
void release_batch_state(bbp_plan p);
void release_serve_state(bbp_plan p);

}  // namespace bbp
