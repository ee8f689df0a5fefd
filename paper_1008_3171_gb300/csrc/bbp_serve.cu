// Serving: continuous batching of bit-position queries (bbp_submit / bbp_poll).
//
// An engine thread owns a pool of device accumulator slots (admission is by free
// slots, i.e. by accumulator memory) and runs iterations.  Each iteration takes
// from every active query a piece of its remaining work -- at most a fair share of
// an iteration budget sized to a target duration from the measured throughput --
// so a long query is sliced over many iterations while short queries that arrive
// meanwhile join the next iteration and finish in one or two.  The pieces of an
// iteration are head-term ranges and tails of different queries, consumed by the
// same persistent queue kernels as a batch; each query's partial sums stay in its
// slot between iterations.  A query's job counter carries one extra hold while it
// has work left, so the device finalizes it (bits, certified count) exactly in the
// iteration that runs its last piece; the host then publishes the result to
// bbp_poll and frees the slot.  Iterations run one at a time: a query that
// arrives while one runs joins the next.  (Planning iteration i+1 while i runs was
// measured on the serving workload: the same terms/s, and every arrival waits one
// iteration longer, so the median latency rose from 46 to 72 ms.)
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bbp.h"
#include "bbp_kernels.cuh"
#include "bbp_planner.h"
#include "bbp_runtime.h"

using namespace bbp;

namespace {

constexpr int kVariants = kQueueVariants;
constexpr uint32_t kOutStride = kMaxWorkingBits / 8;
constexpr double kIterTargetSeconds = 0.025;  // target duration of one iteration
constexpr double kInitialRate = 2.0e10;       // terms/s before the first measurement

int lmax_index(int lmax) {
  for (int i = 0; i < kNumLmaxClasses; ++i)
    if (kLmaxClasses[i] == lmax) return i;
  return -1;
}

template <typename T>
bool grow_dev(T** p, size_t* cap, size_t want) {
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
bool grow_pinned(T** p, size_t* cap, size_t want) {
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

// A query's work: head ranges (HeadArgs without `slots`, with their tile count and
// kernel variant) and tail ranges, taken in order.
struct Work {
  bool tail;
  int variant;
  uint64_t tiles;  // head: warp tiles of the range
  uint64_t tile;   // head: terms per warp tile on the range's path
  HeadArgs head;
  TailArgs tailargs;
};

enum State { kPending = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Query {
  uint64_t ticket = 0;
  uint64_t n = 0;
  uint32_t P = 0, W = 0, L = 0;
  int slot = -1;
  int state = kPending;
  bbp_status error = BBP_OK;
  std::vector<Work> work;
  size_t next = 0;         // next work item
  uint64_t tile_off = 0;   // tiles of work[next] already handed out
  uint64_t bound = 0;      // N + J + 1
  uint64_t total_terms = 0;
  bool final_in_flight = false;
  std::vector<uint8_t> out;
  uint32_t valid = 0;
};

}  // namespace

// Pinned host staging of one iteration: what it uploads, what it downloads, and
// the queries it finishes.
struct HostStage {
  HeadArgs* jobs = nullptr;          size_t c_jobs = 0;
  uint32_t* job_query = nullptr;     size_t c_job_query = 0;
  uint64_t* job_tiles = nullptr;     size_t c_job_tiles = 0;
  TailArgs* tails = nullptr;         size_t c_tails = 0;
  uint32_t* tail_query = nullptr;    size_t c_tail_query = 0;
  QueryDesc* queries = nullptr;      // one per slot
  unsigned int* jobs_left = nullptr; // one per slot
  uint8_t* out = nullptr;            // kOutStride bytes per slot
  uint32_t* valid = nullptr;         // one per slot
  cudaEvent_t start = nullptr, done = nullptr;
  std::vector<Query*> finishing;     // queries whose last piece runs in this iteration
  uint64_t terms = 0;
  bool in_flight = false;
};

struct ServeEngine {
  bbp_plan plan = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::thread thread;
  bool stop = false;
  bool started = false;
  uint64_t next_ticket = 1;
  std::deque<Query*> pending;
  std::vector<Query*> active;        // admitted, with work left to hand out
  std::unordered_map<uint64_t, Query*> tickets;
  std::vector<int> free_slots;
  uint32_t max_slots = 0;
  double rate = kInitialRate;  // measured terms/s
  // device state (shared by consecutive iterations: stream order separates them)
  cudaStream_t stream = nullptr;
  unsigned long long* d_accum = nullptr;
  QueryDesc* d_queries = nullptr;
  unsigned int* d_jobs_left = nullptr;
  uint8_t* d_out = nullptr;
  uint32_t* d_valid = nullptr;
  unsigned long long* d_done = nullptr;
  unsigned int* d_cursors = nullptr;
  HeadArgs* d_jobs = nullptr;            size_t c_jobs = 0;
  uint32_t* d_job_query = nullptr;       size_t c_job_query = 0;
  uint64_t* d_job_tiles = nullptr;       size_t c_job_tiles = 0;
  unsigned long long* d_job_ctr = nullptr; size_t c_job_ctr = 0;
  TailArgs* d_tails = nullptr;           size_t c_tails = 0;
  uint32_t* d_tail_query = nullptr;      size_t c_tail_query = 0;
  HostStage stage;
  // statistics
  uint64_t iterations = 0;
  uint64_t terms_done = 0;
};

namespace {

// Host planning of one query into work items (the same ranges as bbp_bits).
bbp_status plan_query_work(bbp_plan p, uint64_t n, uint32_t P, Query* q) {
  uint32_t W;
  if (n == 0 || !working_bits(P, p->guard, &W)) return BBP_EINVAL;
  const uint32_t L = W / 32;
  const int lmax = head_lmax_for(static_cast<int>(L));
  if (lmax == 0) return BBP_EINVAL;
  const FormulaDef& F = formula_def(BBP_BELLARD);
  std::vector<TermRange> ranges;
  uint64_t N = 0;
  for (uint32_t j = 0; j < F.count; ++j) {
    const int st = plan_series(F, j, n, W, static_cast<uint32_t>(lmax), 0, UINT64_MAX, ranges, p->wide_min_bits);
    if (st == -6) return BBP_ERANGE;
    if (st != 0) return BBP_EINVAL;
    N += natural_end(F, j, n - 1, W);
  }
  q->n = n;
  q->P = P;
  q->W = W;
  q->L = L;
  q->bound = N + F.count + 1;
  for (const TermRange& r : ranges) {
    const SeriesDef& s = F.s[r.j];
    Work w{};
    w.tail = r.tail != 0;
    q->total_terms += r.count;
    if (w.tail) {
      TailArgs& a = w.tailargs;
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
    } else {
      HeadArgs& a = w.head;
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
      a.negate = s.sign < 0 ? 1u : 0u;  // the parity of the piece's first k is applied per piece
      a.run = static_cast<uint32_t>(p->run);
      a.window = r.window;
      a.first = r.first;
      a.first_max = r.first_max;
      w.tile = tile_terms(p, r.path);
      w.tiles = (r.count + w.tile - 1) / w.tile;
      w.variant = lmax_index(lmax) * kNumPaths + r.path;
    }
    q->work.push_back(w);
  }
  uint64_t tiles = 0;
  for (const Work& w : q->work)
    if (!w.tail) tiles += w.tiles;
  if (tiles > kMaxQueueTiles) return BBP_ERANGE;  // carry-save limbs could pass 2^64
  if (q->work.empty()) {  // nothing to sum: a zero-length tail still retires the query
    Work w{};
    w.tail = true;
    w.tailargs.W = W;
    w.tailargs.L = L;
    q->work.push_back(w);
  }
  return BBP_OK;
}

struct Piece {
  bool tail;
  int variant;
  uint64_t tiles;
  HeadArgs head;
  TailArgs tailargs;
  uint32_t slot;
};

// Takes about `budget_terms` terms (at least one item) of q's remaining work, in
// whole warp tiles of each range.
void take_pieces(ServeEngine* E, Query* q, uint64_t budget_terms, std::vector<Piece>& out, uint64_t* terms) {
  const FormulaDef& F = formula_def(BBP_BELLARD);
  unsigned long long* slots = E->d_accum + static_cast<uint64_t>(q->slot) * kMaxLimbs;
  bool first = true;
  while (q->next < q->work.size() && (first || budget_terms > 0)) {
    first = false;
    Work& w = q->work[q->next];
    Piece pc{};
    pc.slot = static_cast<uint32_t>(q->slot);
    pc.tail = w.tail;
    if (w.tail) {
      pc.tailargs = w.tailargs;
      pc.tailargs.slots = slots;
      *terms += w.tailargs.count;
      budget_terms = budget_terms > w.tailargs.count ? budget_terms - w.tailargs.count : 0;
      ++q->next;
      q->tile_off = 0;
    } else {
      const uint64_t tile = w.tile;
      const uint64_t avail = w.tiles - q->tile_off;
      const uint64_t take = std::max<uint64_t>(1, std::min(avail, budget_terms / tile));
      HeadArgs a = w.head;
      a.k_begin = w.head.k_begin + q->tile_off * tile;
      const uint64_t end = std::min(w.head.k_begin + w.head.count, a.k_begin + take * tile);
      a.count = end - a.k_begin;
      const bool neg_series = w.head.negate != 0;
      a.negate = (neg_series != (F.alternating && (a.k_begin & 1ull))) ? 1u : 0u;
      a.slots = slots;
      pc.head = a;
      pc.variant = w.variant;
      pc.tiles = (a.count + tile - 1) / tile;
      *terms += a.count;
      budget_terms = budget_terms > take * tile ? budget_terms - take * tile : 0;
      q->tile_off += take;
      if (q->tile_off >= w.tiles) {
        ++q->next;
        q->tile_off = 0;
      }
    }
    out.push_back(pc);
  }
}

bool alloc_engine(ServeEngine* E) {
  const size_t S = E->max_slots;
  bool ok = cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&E->d_accum, sizeof(unsigned long long) * kMaxLimbs * S) == cudaSuccess &&
            cudaMalloc(&E->d_queries, sizeof(QueryDesc) * S) == cudaSuccess &&
            cudaMalloc(&E->d_jobs_left, sizeof(unsigned int) * S) == cudaSuccess &&
            cudaMalloc(&E->d_out, static_cast<size_t>(kOutStride) * S) == cudaSuccess &&
            cudaMalloc(&E->d_valid, sizeof(uint32_t) * S) == cudaSuccess &&
            cudaMalloc(&E->d_done, sizeof(unsigned long long) * S) == cudaSuccess &&
            cudaMalloc(&E->d_cursors, sizeof(unsigned int) * (kVariants + 1)) == cudaSuccess;
  {
    HostStage& h = E->stage;
    ok = ok && cudaMallocHost(&h.queries, sizeof(QueryDesc) * S) == cudaSuccess &&
         cudaMallocHost(&h.jobs_left, sizeof(unsigned int) * S) == cudaSuccess &&
         cudaMallocHost(&h.out, static_cast<size_t>(kOutStride) * S) == cudaSuccess &&
         cudaMallocHost(&h.valid, sizeof(uint32_t) * S) == cudaSuccess &&
         cudaEventCreate(&h.start) == cudaSuccess && cudaEventCreate(&h.done) == cudaSuccess;
    if (ok) {
      std::memset(h.queries, 0, sizeof(QueryDesc) * S);
      std::memset(h.jobs_left, 0, sizeof(unsigned int) * S);
    }
  }
  return ok;
}

void free_engine(ServeEngine* E) {
  if (E->stream) cudaStreamSynchronize(E->stream);
  cudaFree(E->d_accum);
  cudaFree(E->d_queries);
  cudaFree(E->d_jobs_left);
  cudaFree(E->d_out);
  cudaFree(E->d_valid);
  cudaFree(E->d_done);
  cudaFree(E->d_cursors);
  cudaFree(E->d_jobs);
  cudaFree(E->d_job_query);
  cudaFree(E->d_job_tiles);
  cudaFree(E->d_job_ctr);
  cudaFree(E->d_tails);
  cudaFree(E->d_tail_query);
  {
    HostStage& h = E->stage;
    cudaFreeHost(h.jobs);
    cudaFreeHost(h.job_query);
    cudaFreeHost(h.job_tiles);
    cudaFreeHost(h.tails);
    cudaFreeHost(h.tail_query);
    cudaFreeHost(h.queries);
    cudaFreeHost(h.jobs_left);
    cudaFreeHost(h.out);
    cudaFreeHost(h.valid);
    if (h.start) cudaEventDestroy(h.start);
    if (h.done) cudaEventDestroy(h.done);
  }
  if (E->stream) cudaStreamDestroy(E->stream);
}

// Plans one iteration over the active queries into staging H and enqueues it
// (uploads, launches, result download, events).  Queries whose
// last piece is in it move to H.finishing.  Returns false on a CUDA error.
bool enqueue_iteration(ServeEngine* E, HostStage& H, std::vector<Query*>& batch, std::vector<int>& fresh_slots) {
  bbp_plan p = E->plan;
  const uint64_t budget_terms = std::max<uint64_t>(1, static_cast<uint64_t>(E->rate * kIterTargetSeconds));
  const uint64_t share = std::max<uint64_t>(1, budget_terms / std::max<size_t>(1, batch.size()));
  std::vector<Piece> pieces;
  uint64_t terms = 0;
  std::vector<uint32_t> npieces(batch.size(), 0);
  H.finishing.clear();
  for (size_t i = 0; i < batch.size(); ++i) {
    Query* q = batch[i];
    const size_t before = pieces.size();
    take_pieces(E, q, share, pieces, &terms);
    npieces[i] = static_cast<uint32_t>(pieces.size() - before);
    q->final_in_flight = q->next >= q->work.size();
    if (q->final_in_flight) H.finishing.push_back(q);
  }
  H.terms = terms;
  // group head pieces by variant, tails apart
  std::vector<uint32_t> vb(kVariants + 1, 0);
  std::vector<const Piece*> heads, tails;
  for (int v = 0; v < kVariants; ++v) {
    vb[v] = static_cast<uint32_t>(heads.size());
    for (const Piece& pc : pieces)
      if (!pc.tail && pc.variant == v) heads.push_back(&pc);
  }
  vb[kVariants] = static_cast<uint32_t>(heads.size());
  for (const Piece& pc : pieces)
    if (pc.tail) tails.push_back(&pc);
  const size_t nh = heads.size(), nt = tails.size();
  if (!grow_pinned(&H.jobs, &H.c_jobs, nh) || !grow_pinned(&H.job_query, &H.c_job_query, nh) ||
      !grow_pinned(&H.job_tiles, &H.c_job_tiles, nh) || !grow_pinned(&H.tails, &H.c_tails, nt) ||
      !grow_pinned(&H.tail_query, &H.c_tail_query, nt) || !grow_dev(&E->d_jobs, &E->c_jobs, nh) ||
      !grow_dev(&E->d_job_query, &E->c_job_query, nh) || !grow_dev(&E->d_job_tiles, &E->c_job_tiles, nh) ||
      !grow_dev(&E->d_job_ctr, &E->c_job_ctr, 2 * nh) || !grow_dev(&E->d_tails, &E->c_tails, nt) ||
      !grow_dev(&E->d_tail_query, &E->c_tail_query, nt))
    return false;
  for (size_t i = 0; i < nh; ++i) {
    H.jobs[i] = heads[i]->head;
    H.job_query[i] = heads[i]->slot;
    H.job_tiles[i] = heads[i]->tiles;
  }
  for (size_t i = 0; i < nt; ++i) {
    H.tails[i] = tails[i]->tailargs;
    H.tail_query[i] = tails[i]->slot;
  }
  for (size_t i = 0; i < batch.size(); ++i) {
    Query* q = batch[i];
    QueryDesc& Q = H.queries[q->slot];
    Q.bound = q->bound;
    Q.P = q->P;
    Q.L = q->L;
    Q.out_offset = static_cast<uint32_t>(q->slot) * kOutStride;
    H.jobs_left[q->slot] = npieces[i] + (q->final_in_flight ? 0u : 1u);  // hold while work remains
  }
  cudaStream_t s = E->stream;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(cudaEventRecord(H.start, s));
  for (int slot : fresh_slots)
    chk(cudaMemsetAsync(E->d_accum + static_cast<uint64_t>(slot) * kMaxLimbs, 0,
                        sizeof(unsigned long long) * kMaxLimbs, s));
  // the whole slot tables in two copies (slots not in this iteration have no jobs)
  chk(cudaMemcpyAsync(E->d_queries, H.queries, sizeof(QueryDesc) * E->max_slots, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(E->d_jobs_left, H.jobs_left, sizeof(unsigned int) * E->max_slots, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(E->d_jobs, H.jobs, sizeof(HeadArgs) * nh, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(E->d_job_query, H.job_query, sizeof(uint32_t) * nh, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(E->d_job_tiles, H.job_tiles, sizeof(uint64_t) * nh, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(E->d_tails, H.tails, sizeof(TailArgs) * nt, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(E->d_tail_query, H.tail_query, sizeof(uint32_t) * nt, cudaMemcpyHostToDevice, s));
  chk(cudaMemsetAsync(E->d_job_ctr, 0, sizeof(unsigned long long) * 2 * std::max<size_t>(nh, 1), s));
  chk(cudaMemsetAsync(E->d_cursors, 0, sizeof(unsigned int) * (kVariants + 1), s));
  BatchDev dev{};
  dev.jobs = E->d_jobs;
  dev.job_query = E->d_job_query;
  dev.job_tiles = E->d_job_tiles;
  dev.job_taken = E->d_job_ctr;
  dev.job_done = E->d_job_ctr + nh;
  dev.tails = E->d_tails;
  dev.tail_query = E->d_tail_query;
  dev.grab = 1;  // short iterations: hand out single tiles so every launch ends evenly
  dev.queries = E->d_queries;
  dev.accum = E->d_accum;
  dev.jobs_left = E->d_jobs_left;
  dev.out = E->d_out;
  dev.valid = E->d_valid;
  dev.done_ns = E->d_done;
  chk(launch_queue_tail(dev, 0, static_cast<uint32_t>(nt), E->d_cursors + kVariants, p->sm_count * 4, s));
  for (int v = 0; v < kVariants; ++v) {
    if (vb[v] == vb[v + 1]) continue;
    const int lmax = kLmaxClasses[v / kNumPaths], path = v % kNumPaths;
    const int blocks = queue_occupancy(path, head_streams(p, path), lmax) * p->sm_count;
    chk(launch_queue(dev, vb[v], vb[v + 1], E->d_cursors + v, path, head_streams(p, path), lmax, blocks, s));
  }
  if (!H.finishing.empty()) {  // results of the queries that finish in this iteration
    chk(cudaMemcpyAsync(H.out, E->d_out, static_cast<size_t>(kOutStride) * E->max_slots, cudaMemcpyDeviceToHost, s));
    chk(cudaMemcpyAsync(H.valid, E->d_valid, sizeof(uint32_t) * E->max_slots, cudaMemcpyDeviceToHost, s));
  }
  chk(cudaEventRecord(H.done, s));
  H.in_flight = e == cudaSuccess;
  return e == cudaSuccess;
}

// Waits for an enqueued iteration and publishes the queries it finished (under
// E->mu, which bbp_poll and bbp_serve_stats take too).
bool finish_iteration(ServeEngine* E, HostStage& H) {
  if (!H.in_flight) return true;
  H.in_flight = false;
  if (cudaEventSynchronize(H.done) != cudaSuccess) return false;
  float ms = 0;
  const bool timed = cudaEventElapsedTime(&ms, H.start, H.done) == cudaSuccess && ms > 0.1f && H.terms > 0;
  std::lock_guard<std::mutex> lock(E->mu);
  if (timed) E->rate = 0.7 * E->rate + 0.3 * (static_cast<double>(H.terms) / (1e-3 * ms));
  E->iterations++;
  E->terms_done += H.terms;
  for (Query* q : H.finishing) {
    q->out.assign(H.out + static_cast<size_t>(q->slot) * kOutStride,
                  H.out + static_cast<size_t>(q->slot) * kOutStride + (q->P + 7) / 8);
    q->valid = H.valid[q->slot];
    q->state = kDone;
    E->free_slots.push_back(q->slot);
    q->slot = -1;
    q->work.clear();
    q->work.shrink_to_fit();
  }
  H.finishing.clear();
  return true;
}

// An iteration could not be enqueued or did not complete: every admitted query
// fails (bbp_poll returns BBP_ECUDA) and gives its slot back, so that later
// submissions are admitted again (a fresh slot is zeroed on admission).
void fail_all(ServeEngine* E) {
  std::lock_guard<std::mutex> lock(E->mu);
  auto fail = [&](Query* q) {
    q->state = kFailed;
    q->error = BBP_ECUDA;
    if (q->slot >= 0) E->free_slots.push_back(q->slot);
    q->slot = -1;
    q->work.clear();
  };
  for (Query* q : E->stage.finishing) fail(q);
  E->stage.finishing.clear();
  E->stage.in_flight = false;
  for (Query* q : E->active) fail(q);
  E->active.clear();
}

void engine_main(ServeEngine* E) {
  cudaSetDevice(E->plan->device);
  for (;;) {
    std::vector<Query*> batch;
    std::vector<int> fresh;
    {
      std::unique_lock<std::mutex> lock(E->mu);
      E->cv.wait(lock, [&] { return E->stop || !E->pending.empty() || !E->active.empty(); });
      if (E->stop) return;
      while (!E->pending.empty() && !E->free_slots.empty()) {  // admission by free accumulator slots
        Query* q = E->pending.front();
        E->pending.pop_front();
        q->slot = E->free_slots.back();
        E->free_slots.pop_back();
        q->state = kActive;
        E->active.push_back(q);
        fresh.push_back(q->slot);
      }
      batch = E->active;
    }
    bool ok = enqueue_iteration(E, E->stage, batch, fresh);
    {
      std::lock_guard<std::mutex> lock(E->mu);  // queries handed out completely leave the active list
      std::vector<Query*> still;
      for (Query* q : E->active)
        if (!q->final_in_flight) still.push_back(q);
      E->active.swap(still);
    }
    ok = ok && finish_iteration(E, E->stage);
    if (!ok) fail_all(E);
  }
}

ServeEngine* engine_of(bbp_plan p, bbp_status* st) {
  *st = BBP_OK;
  if (p->serve) return p->serve;
  ServeEngine* E = new (std::nothrow) ServeEngine();
  if (!E) {
    *st = BBP_ENOMEM;
    return nullptr;
  }
  E->plan = p;
  const size_t per_slot = sizeof(unsigned long long) * kMaxLimbs + kOutStride + 64;
  E->max_slots = static_cast<uint32_t>(
      std::max<size_t>(1, std::min<size_t>({p->max_slots, p->accum_budget / per_slot, kMaxQueueQueries})));
  cudaSetDevice(p->device);
  if (!alloc_engine(E)) {
    free_engine(E);
    delete E;
    *st = BBP_ENOMEM;
    return nullptr;
  }
  for (int s = static_cast<int>(E->max_slots) - 1; s >= 0; --s) E->free_slots.push_back(s);
  E->thread = std::thread(engine_main, E);
  E->started = true;
  p->serve = E;
  return E;
}

}  // namespace

namespace bbp {

void release_serve_state(bbp_plan p) {
  ServeEngine* E = p->serve;
  if (!E) return;
  {
    std::lock_guard<std::mutex> lock(E->mu);
    E->stop = true;
  }
  E->cv.notify_all();
  if (E->thread.joinable()) E->thread.join();
  if (E->stream) cudaStreamSynchronize(E->stream);
  for (auto& kv : E->tickets) delete kv.second;
  free_engine(E);
  delete E;
  p->serve = nullptr;
}

}  // namespace bbp

extern "C" {

bbp_status bbp_submit(bbp_plan p, uint64_t n, uint32_t P, bbp_ticket* t) {
  if (!p || !t) return BBP_EINVAL;
  Query* q = new (std::nothrow) Query();
  if (!q) return BBP_ENOMEM;
  const bbp_status ps = plan_query_work(p, n, P, q);
  if (ps != BBP_OK) {
    delete q;
    return ps;
  }
  bbp_status st;
  ServeEngine* E = engine_of(p, &st);
  if (!E) {
    delete q;
    return st;
  }
  {
    std::lock_guard<std::mutex> lock(E->mu);
    // admission: a query waits for a slot only while the queue is shorter than the pool
    if (E->pending.size() >= E->max_slots) {
      delete q;
      return BBP_EBUSY;
    }
    q->ticket = E->next_ticket++;
    E->tickets[q->ticket] = q;
    E->pending.push_back(q);
    *t = q->ticket;
  }
  E->cv.notify_all();
  return BBP_OK;
}

bbp_status bbp_poll(bbp_plan p, bbp_ticket t, uint8_t* out, uint32_t* valid_bits) {
  if (!p) return BBP_EINVAL;
  ServeEngine* E = p->serve;
  if (!E) return BBP_ENOTFOUND;
  std::lock_guard<std::mutex> lock(E->mu);
  auto it = E->tickets.find(t);
  if (it == E->tickets.end()) return BBP_ENOTFOUND;
  Query* q = it->second;
  if (q->state == kPending || q->state == kActive) return BBP_PENDING;
  const bbp_status st = q->state == kFailed ? q->error : BBP_OK;
  if (st == BBP_OK) {
    if (out) std::memcpy(out, q->out.data(), q->out.size());
    if (valid_bits) *valid_bits = q->valid;
  }
  E->tickets.erase(it);
  delete q;
  return st;
}

bbp_status bbp_serve_stats(bbp_plan p, bbp_serve_info* info) {
  if (!p || !info) return BBP_EINVAL;
  std::memset(info, 0, sizeof(*info));
  ServeEngine* E = p->serve;
  if (!E) return BBP_OK;
  std::lock_guard<std::mutex> lock(E->mu);
  info->pending = E->pending.size();
  info->active = E->active.size();
  info->slots = E->max_slots;
  info->iterations = E->iterations;
  info->terms = E->terms_done;
  info->terms_per_s = E->rate;
  return BBP_OK;
}

}  // extern "C"
