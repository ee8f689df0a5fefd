// Batched queries: one persistent, graph-captured pass over a chunk queue.
//
// Every query of a batch is planned into jobs (bbp_planner.cpp): head jobs -- one
// range of head terms of one series, with the ladder parameters of its moduli --
// and tail jobs.  Queries are sorted by size and cut into waves whose work grows
// geometrically (the smallest queries first) up to 1/12 of the batch, so the
// largest queries finish over the last several waves rather than together at the
// end of one; a wave is one tail launch plus one
// persistent launch per kernel variant (limb capacity x modulus path) in which
// warps take `grab` tiles of the current job at a time (queue_kernel), so queries
// of very different sizes share the GPU at tile granularity and small ones finish
// early.  Each query's signed partial sums accumulate in its own carry-save
// slots; the warp that retires its last job finalizes it on the device and stamps
// the completion time.  The whole pass -- uploads, resets, launches, downloads --
// is captured once into a CUDA graph and replayed (the executable graph is updated
// in place when the next batch has the same shape).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "bbp.h"
#include "bbp_kernels.cuh"
#include "bbp_planner.h"
#include "bbp_runtime.h"

using namespace bbp;

namespace {

constexpr int kVariants = kQueueVariants;
constexpr uint32_t kOutStride = kMaxWorkingBits / 8;  // bytes of output per query slot

int lmax_index(int lmax) {
  for (int i = 0; i < kNumLmaxClasses; ++i)
    if (kLmaxClasses[i] == lmax) return i;
  return -1;
}

template <typename T>
bool grow_device(T** p, size_t* cap, size_t want) {
  if (*cap >= want && *p) return true;
  cudaFree(*p);
  *p = nullptr;
  const size_t n = std::max<size_t>(want, 1) * 2;
  if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
    *cap = 0;
    return false;
  }
  *cap = n;
  return true;
}

template <typename T>
bool grow_host(T** p, size_t* cap, size_t want) {
  if (*cap >= want && *p) return true;
  cudaFreeHost(*p);
  *p = nullptr;
  const size_t n = std::max<size_t>(want, 1) * 2;
  if (cudaMallocHost(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
    *cap = 0;
    return false;
  }
  *cap = n;
  return true;
}

}  // namespace

struct BatchState {
  // device buffers and their capacities (elements)
  HeadArgs* d_jobs = nullptr;               size_t c_jobs = 0;
  uint32_t* d_job_query = nullptr;          size_t c_job_query = 0;
  uint64_t* d_job_tiles = nullptr;          size_t c_job_tiles = 0;
  unsigned long long* d_job_ctr = nullptr;  size_t c_job_ctr = 0;  // taken[0..J) then done[0..J)
  TailArgs* d_tails = nullptr;              size_t c_tails = 0;
  uint32_t* d_tail_query = nullptr;         size_t c_tail_query = 0;
  QueryDesc* d_queries = nullptr;           size_t c_queries = 0;
  unsigned long long* d_accum = nullptr;    size_t c_accum = 0;
  unsigned int* d_jobs_left = nullptr;      size_t c_jobs_left = 0;
  uint8_t* d_out = nullptr;                 size_t c_out = 0;
  uint32_t* d_valid = nullptr;              size_t c_valid = 0;
  unsigned long long* d_done = nullptr;     size_t c_done = 0;   // [0] = start time, [1 + q] = done
  unsigned int* d_cursors = nullptr;        size_t c_cursors = 0;  // per wave: kVariants + 1 (tail)
  // pinned host staging
  HeadArgs* h_jobs = nullptr;               size_t hc_jobs = 0;
  uint32_t* h_job_query = nullptr;          size_t hc_job_query = 0;
  uint64_t* h_job_tiles = nullptr;          size_t hc_job_tiles = 0;
  TailArgs* h_tails = nullptr;              size_t hc_tails = 0;
  uint32_t* h_tail_query = nullptr;         size_t hc_tail_query = 0;
  QueryDesc* h_queries = nullptr;           size_t hc_queries = 0;
  unsigned int* h_jobs_left = nullptr;      size_t hc_jobs_left = 0;
  uint8_t* h_out = nullptr;                 size_t hc_out = 0;
  uint32_t* h_valid = nullptr;              size_t hc_valid = 0;
  unsigned long long* h_done = nullptr;     size_t hc_done = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;  // capture needs a stream other than the legacy default stream
  cudaEvent_t ready = nullptr;
};

namespace bbp {

void release_batch_state(bbp_plan p) {
  BatchState* b = p->batch;
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->ready) cudaEventDestroy(b->ready);
  cudaFree(b->d_jobs);
  cudaFree(b->d_job_query);
  cudaFree(b->d_job_tiles);
  cudaFree(b->d_job_ctr);
  cudaFree(b->d_tails);
  cudaFree(b->d_tail_query);
  cudaFree(b->d_queries);
  cudaFree(b->d_accum);
  cudaFree(b->d_jobs_left);
  cudaFree(b->d_out);
  cudaFree(b->d_valid);
  cudaFree(b->d_done);
  cudaFree(b->d_cursors);
  cudaFreeHost(b->h_jobs);
  cudaFreeHost(b->h_job_query);
  cudaFreeHost(b->h_job_tiles);
  cudaFreeHost(b->h_tails);
  cudaFreeHost(b->h_tail_query);
  cudaFreeHost(b->h_queries);
  cudaFreeHost(b->h_jobs_left);
  cudaFreeHost(b->h_out);
  cudaFreeHost(b->h_valid);
  cudaFreeHost(b->h_done);
  delete b;
  p->batch = nullptr;
}

constexpr int kMaxWaves = 24;

// Plans `count` queries into the batch's pinned staging buffers.
struct BatchPlan {
  uint32_t njobs = 0, ntails = 0, nwaves = 0;
  uint32_t group_begin[kMaxWaves * kVariants + 1] = {};  // head jobs of (wave, variant)
  uint32_t tail_begin[kMaxWaves + 1] = {};               // tail jobs of a wave
  uint64_t terms = 0, head_terms = 0;
  double imad = 0;
};

static bbp_status plan_batch(bbp_plan p, int f, uint32_t count, const uint64_t* n, const uint32_t* P,
                             BatchState* b, BatchPlan* bp) {
  const FormulaDef& F = formula_def(f);
  std::vector<std::vector<HeadArgs>> vj(kVariants);
  std::vector<std::vector<uint32_t>> vq(kVariants);
  std::vector<std::vector<uint64_t>> vt(kVariants);
  std::vector<TailArgs> tails;
  std::vector<uint32_t> tail_q;
  std::vector<QueryDesc> queries(count);
  std::vector<unsigned int> jobs_left(count, 0);
  std::vector<uint64_t> qterms(count, 0);
  std::vector<TermRange> ranges;
  for (uint32_t q = 0; q < count; ++q) {
    uint32_t W;
    if (n[q] == 0 || !working_bits(P[q], p->guard, &W)) return BBP_EINVAL;
    const uint32_t L = W / 32;
    const int lmax = head_lmax_for(static_cast<int>(L));
    if (lmax == 0) return BBP_EINVAL;
    unsigned long long* slots = b->d_accum + static_cast<uint64_t>(q) * kMaxLimbs;
    ranges.clear();
    uint64_t N = 0;
    for (uint32_t j = 0; j < F.count; ++j) {
      const int st = plan_series(F, j, n[q], W, static_cast<uint32_t>(lmax), 0, UINT64_MAX, ranges, p->wide_min_bits);
      if (st == -6) return BBP_ERANGE;
      if (st != 0) return BBP_EINVAL;
      N += natural_end(F, j, n[q] - 1, W);
    }
    uint64_t qtiles = 0;
    for (const TermRange& r : ranges)
      if (!r.tail) qtiles += (r.count + tile_terms(p, r.path) - 1) / tile_terms(p, r.path);
    if (qtiles > kMaxQueueTiles) return BBP_ERANGE;  // carry-save limbs could pass 2^64
    for (const TermRange& r : ranges) {
      const SeriesDef& s = F.s[r.j];
      qterms[q] += r.count;
      bp->terms += r.count;
      if (r.tail) {
        TailArgs a{};
        a.d = n[q] - 1;
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
        tails.push_back(a);
        tail_q.push_back(q);
      } else {
        HeadArgs a{};
        a.d = n[q] - 1;
        a.k_begin = r.k_begin;
        a.count = r.count;
        a.a = s.a;
        a.b = s.b;
        a.c = s.c;
        a.step = F.step;
        a.W = W;
        a.L = L;
        a.alternating = F.alternating;
        a.negate = ((s.sign < 0) != (F.alternating && (r.k_begin & 1ull))) ? 1u : 0u;
        a.run = static_cast<uint32_t>(p->run);
        a.window = r.window;
        a.first = r.first;
        a.first_max = r.first_max;
        a.slots = slots;
        const int v = lmax_index(lmax) * kNumPaths + r.path;
        vj[v].push_back(a);
        vq[v].push_back(q);
        vt[v].push_back((r.count + tile_terms(p, r.path) - 1) / tile_terms(p, r.path));
        bp->head_terms += r.count;
        bp->imad += r.imad;
      }
      jobs_left[q]++;
    }
    if (jobs_left[q] == 0) {  // no term at all: a zero-length tail job still retires it
      TailArgs a{};
      a.W = W;
      a.L = L;
      a.slots = slots;
      tails.push_back(a);
      tail_q.push_back(q);
      jobs_left[q] = 1;
    }
    QueryDesc& Q = queries[q];
    Q.bound = N + F.count + 1;
    Q.P = P[q];
    Q.L = L;
    Q.out_offset = q * kOutStride;
  }
  // waves: queries by size, each wave twice the work of the ones before it, at most 1/12 of the total
  std::vector<uint32_t> qorder(count);
  std::iota(qorder.begin(), qorder.end(), 0u);
  std::stable_sort(qorder.begin(), qorder.end(), [&](uint32_t x, uint32_t y) { return qterms[x] < qterms[y]; });
  std::vector<uint32_t> wave_of(count, 0);
  {
    uint64_t total = 0;
    for (uint64_t t : qterms) total += t;
    const uint64_t first = std::max<uint64_t>(total / 4096, 1);  // the first wave: 1/4096 of the work
    const uint64_t step_cap = std::max<uint64_t>(total / 12, 1);  // no wave beyond 1/12 of the work
    uint64_t done = 0, target = first;
    uint32_t w = 0;
    for (uint32_t i = 0; i < count; ++i) {
      const uint32_t q = qorder[i];
      if (done >= target && w + 1 < static_cast<uint32_t>(kMaxWaves)) {
        ++w;
        target = std::min(std::max(target, done) * 2, done + step_cap);
      }
      wave_of[q] = w;
      done += qterms[q];
    }
    bp->nwaves = w + 1;
  }
  uint32_t nj = 0;
  for (int v = 0; v < kVariants; ++v) nj += static_cast<uint32_t>(vj[v].size());
  if (!grow_host(&b->h_jobs, &b->hc_jobs, nj) || !grow_host(&b->h_job_query, &b->hc_job_query, nj) ||
      !grow_host(&b->h_job_tiles, &b->hc_job_tiles, nj) || !grow_host(&b->h_tails, &b->hc_tails, tails.size()) ||
      !grow_host(&b->h_tail_query, &b->hc_tail_query, tails.size()) ||
      !grow_host(&b->h_queries, &b->hc_queries, count) || !grow_host(&b->h_jobs_left, &b->hc_jobs_left, count))
    return BBP_ENOMEM;
  uint32_t at = 0;
  for (uint32_t w = 0; w < bp->nwaves; ++w) {
    for (int v = 0; v < kVariants; ++v) {
      bp->group_begin[w * kVariants + v] = at;
      std::vector<uint32_t> order;
      for (uint32_t i = 0; i < vj[v].size(); ++i)
        if (wave_of[vq[v][i]] == w) order.push_back(i);
      std::stable_sort(order.begin(), order.end(),
                       [&](uint32_t x, uint32_t y) { return qterms[vq[v][x]] < qterms[vq[v][y]]; });
      for (uint32_t i : order) {
        b->h_jobs[at] = vj[v][i];
        b->h_job_query[at] = vq[v][i];
        b->h_job_tiles[at] = vt[v][i];
        ++at;
      }
    }
  }
  bp->group_begin[bp->nwaves * kVariants] = at;
  uint32_t tat = 0;
  for (uint32_t w = 0; w < bp->nwaves; ++w) {
    bp->tail_begin[w] = tat;
    for (size_t i = 0; i < tails.size(); ++i)
      if (wave_of[tail_q[i]] == w) {
        b->h_tails[tat] = tails[i];
        b->h_tail_query[tat] = tail_q[i];
        ++tat;
      }
  }
  bp->tail_begin[bp->nwaves] = tat;
  bp->njobs = nj;
  bp->ntails = static_cast<uint32_t>(tails.size());
  std::copy(queries.begin(), queries.end(), b->h_queries);
  std::copy(jobs_left.begin(), jobs_left.end(), b->h_jobs_left);
  return BBP_OK;
}

}  // namespace bbp

#define BBP_TRY(expr)                              \
  do {                                             \
    if ((expr) != cudaSuccess) return BBP_ECUDA;   \
  } while (0)

extern "C" bbp_status bbp_bits_batch(bbp_plan p, bbp_formula f, uint32_t count, const uint64_t* n, const uint32_t* P,
                                     uint8_t* out, uint32_t out_stride, uint32_t* valid_bits, double* latency_ms) {
  if (!p || (f != BBP_BELLARD && f != BBP_BBP) || (count && (!n || !P || !out))) return BBP_EINVAL;
  if (count == 0) return BBP_OK;
  if (count > kMaxQueueQueries) return BBP_EINVAL;
  uint32_t maxbytes = 0;
  for (uint32_t q = 0; q < count; ++q) maxbytes = std::max(maxbytes, (P[q] + 7) / 8);
  if (out_stride < maxbytes) return BBP_EINVAL;
  BBP_TRY(cudaSetDevice(p->device));
  if (!p->batch) {
    p->batch = new (std::nothrow) BatchState();
    if (!p->batch) return BBP_ENOMEM;
  }
  BatchState* b = p->batch;
  // device buffers first (job descriptors hold accumulator addresses)
  if (!grow_device(&b->d_accum, &b->c_accum, static_cast<size_t>(count) * kMaxLimbs) ||
      !grow_device(&b->d_queries, &b->c_queries, count) || !grow_device(&b->d_jobs_left, &b->c_jobs_left, count) ||
      !grow_device(&b->d_out, &b->c_out, static_cast<size_t>(count) * kOutStride) ||
      !grow_device(&b->d_valid, &b->c_valid, count) || !grow_device(&b->d_done, &b->c_done, count + 1ull) ||
      !grow_host(&b->h_out, &b->hc_out, static_cast<size_t>(count) * kOutStride) ||
      !grow_host(&b->h_valid, &b->hc_valid, count) || !grow_host(&b->h_done, &b->hc_done, count + 1ull))
    return BBP_ENOMEM;
  if (!grow_device(&b->d_cursors, &b->c_cursors, static_cast<size_t>(kMaxWaves) * (kVariants + 1)))
    return BBP_ENOMEM;
  BatchPlan bp;
  bbp_status st = plan_batch(p, f, count, n, P, b, &bp);
  if (st != BBP_OK) return st;
  if (!grow_device(&b->d_jobs, &b->c_jobs, bp.njobs) || !grow_device(&b->d_job_query, &b->c_job_query, bp.njobs) ||
      !grow_device(&b->d_job_tiles, &b->c_job_tiles, bp.njobs) ||
      !grow_device(&b->d_job_ctr, &b->c_job_ctr, 2ull * bp.njobs) ||
      !grow_device(&b->d_tails, &b->c_tails, bp.ntails) || !grow_device(&b->d_tail_query, &b->c_tail_query, bp.ntails))
    return BBP_ENOMEM;

  BatchDev dev{};
  dev.jobs = b->d_jobs;
  dev.job_query = b->d_job_query;
  dev.job_tiles = b->d_job_tiles;
  dev.job_taken = b->d_job_ctr;
  dev.job_done = b->d_job_ctr + bp.njobs;
  dev.tails = b->d_tails;
  dev.tail_query = b->d_tail_query;
  dev.grab = static_cast<uint32_t>(p->grab);
  dev.queries = b->d_queries;
  dev.accum = b->d_accum;
  dev.jobs_left = b->d_jobs_left;
  dev.out = b->d_out;
  dev.valid = b->d_valid;
  dev.done_ns = b->d_done + 1;

  if (!b->stream && cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return BBP_ECUDA;
  if (!b->ready && cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess) return BBP_ECUDA;
  // order after earlier work on the plan's stream, then run on the batch stream
  BBP_TRY(cudaEventRecord(b->ready, p->stream));
  BBP_TRY(cudaStreamWaitEvent(b->stream, b->ready, 0));
  cudaStream_t s = b->stream;
  // capture the pass
  cudaGraph_t graph = nullptr;
  BBP_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(cudaMemcpyAsync(b->d_jobs, b->h_jobs, sizeof(HeadArgs) * bp.njobs, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(b->d_job_query, b->h_job_query, sizeof(uint32_t) * bp.njobs, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(b->d_job_tiles, b->h_job_tiles, sizeof(uint64_t) * bp.njobs, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(b->d_tails, b->h_tails, sizeof(TailArgs) * bp.ntails, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(b->d_tail_query, b->h_tail_query, sizeof(uint32_t) * bp.ntails, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(b->d_queries, b->h_queries, sizeof(QueryDesc) * count, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(b->d_jobs_left, b->h_jobs_left, sizeof(unsigned int) * count, cudaMemcpyHostToDevice, s));
  chk(cudaMemsetAsync(b->d_job_ctr, 0, sizeof(unsigned long long) * 2 * bp.njobs, s));
  chk(cudaMemsetAsync(b->d_cursors, 0, sizeof(unsigned int) * kMaxWaves * (kVariants + 1), s));
  chk(cudaMemsetAsync(b->d_accum, 0, sizeof(unsigned long long) * kMaxLimbs * count, s));
  chk(launch_timestamp(b->d_done, s));
  uint64_t launches = 1, head_launches = 0;
  for (uint32_t w = 0; w < bp.nwaves; ++w) {
    unsigned int* cur = b->d_cursors + static_cast<size_t>(w) * (kVariants + 1);
    if (bp.tail_begin[w] < bp.tail_begin[w + 1]) {
      chk(launch_queue_tail(dev, bp.tail_begin[w], bp.tail_begin[w + 1], cur + kVariants, p->sm_count * 4, s));
      ++launches;
    }
    for (int v = 0; v < kVariants; ++v) {
      const uint32_t jb = bp.group_begin[w * kVariants + v], je = bp.group_begin[w * kVariants + v + 1];
      if (jb == je) continue;
      const int lmax = kLmaxClasses[v / kNumPaths], path = v % kNumPaths;
      const int blocks = queue_occupancy(path, head_streams(p, path), lmax) * p->sm_count;
      chk(launch_queue(dev, jb, je, cur + v, path, head_streams(p, path), lmax, blocks, s));
      ++launches;
      ++head_launches;
    }
  }
  chk(cudaMemcpyAsync(b->h_out, b->d_out, static_cast<size_t>(count) * kOutStride, cudaMemcpyDeviceToHost, s));
  chk(cudaMemcpyAsync(b->h_valid, b->d_valid, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost, s));
  chk(cudaMemcpyAsync(b->h_done, b->d_done, sizeof(unsigned long long) * (count + 1ull), cudaMemcpyDeviceToHost, s));
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return BBP_ECUDA;
  }
  bool updated = false;
  if (b->exec) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(b->exec, graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  if (!b->exec && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    b->exec = nullptr;
    return BBP_ECUDA;
  }
  cudaGraphDestroy(graph);
  if (p->profile) BBP_TRY(cudaEventRecord(p->ev0, s));
  BBP_TRY(cudaGraphLaunch(b->exec, s));
  if (p->profile) BBP_TRY(cudaEventRecord(p->ev1, s));
  BBP_TRY(cudaStreamSynchronize(s));
  p->stats = bbp_stats{};
  p->stats.terms = bp.terms;
  p->stats.head_terms = bp.head_terms;
  p->stats.head_launches = head_launches;
  p->stats.kernel_launches = launches;
  p->stats.imad_model = bp.imad;
  if (p->profile) {
    float ms = 0;
    BBP_TRY(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    p->stats.head_ms = ms;
  }
  for (uint32_t q = 0; q < count; ++q) {
    std::memcpy(out + static_cast<size_t>(q) * out_stride, b->h_out + static_cast<size_t>(q) * kOutStride,
                (P[q] + 7) / 8);
    if (valid_bits) valid_bits[q] = b->h_valid[q];
    if (latency_ms) latency_ms[q] = static_cast<double>(b->h_done[1 + q] - b->h_done[0]) * 1e-6;
  }
  if (p->strict)
    for (uint32_t q = 0; q < count; ++q)
      if (b->h_valid[q] < P[q]) return BBP_EINVALID_BITS;
  return BBP_OK;
}
