// Launchers of the head and queue kernels for one accumulator class.  A
// translation unit defines BBP_LMAX (limbs per thread) and includes this file,
// so the seven classes compile in parallel; bbp_kernels.cu dispatches to them.
#pragma once

#ifndef BBP_LMAX
#error "define BBP_LMAX (accumulator limbs) before including bbp_inst.cuh"
#endif

#include "bbp_tile.cuh"

#define BBP_CAT2(a, b) a##b
#define BBP_CAT(a, b) BBP_CAT2(a, b)

namespace bbp {
namespace {

template <int PATH, int S>
cudaError_t launch_head_t(const HeadArgs& a, int blocks, int threads, cudaStream_t s) {
  const uint64_t tile = 32ull * S * a.run;
  const uint64_t ntiles = (a.count + tile - 1) / tile;
  head_kernel<BBP_LMAX, PATH, S><<<blocks, threads, 0, s>>>(a, ntiles);
  return cudaGetLastError();
}

template <int PATH, int S>
int head_occupancy_t(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, head_kernel<BBP_LMAX, PATH, S>, threads, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int PATH, int S>
cudaError_t launch_queue_t(const BatchDev& b, uint32_t jb, uint32_t je, unsigned int* cursor, int blocks,
                           cudaStream_t s) {
  queue_kernel<BBP_LMAX, PATH, S><<<blocks, kHeadThreads, 0, s>>>(b, jb, je, cursor);
  return cudaGetLastError();
}

template <int PATH, int S>
int queue_occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, queue_kernel<BBP_LMAX, PATH, S>, kHeadThreads, 0) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace

// path 0..3 (kNumPaths), streams 1 or 2 (anything else runs 1)
cudaError_t BBP_CAT(launch_head_l, BBP_LMAX)(const HeadArgs& a, int path, int streams, int blocks, int threads,
                                             cudaStream_t s) {
  const bool two = streams == 2;
  switch (path) {
    case 0: return two ? launch_head_t<0, 2>(a, blocks, threads, s) : launch_head_t<0, 1>(a, blocks, threads, s);
    case 1: return two ? launch_head_t<1, 2>(a, blocks, threads, s) : launch_head_t<1, 1>(a, blocks, threads, s);
    case 2: return two ? launch_head_t<2, 2>(a, blocks, threads, s) : launch_head_t<2, 1>(a, blocks, threads, s);
    case 3: return two ? launch_head_t<3, 2>(a, blocks, threads, s) : launch_head_t<3, 1>(a, blocks, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

int BBP_CAT(head_occupancy_l, BBP_LMAX)(int path, int streams, int threads) {
  const bool two = streams == 2;
  switch (path) {
    case 0: return two ? head_occupancy_t<0, 2>(threads) : head_occupancy_t<0, 1>(threads);
    case 1: return two ? head_occupancy_t<1, 2>(threads) : head_occupancy_t<1, 1>(threads);
    case 2: return two ? head_occupancy_t<2, 2>(threads) : head_occupancy_t<2, 1>(threads);
    case 3: return two ? head_occupancy_t<3, 2>(threads) : head_occupancy_t<3, 1>(threads);
    default: return 1;
  }
}

cudaError_t BBP_CAT(launch_queue_l, BBP_LMAX)(const BatchDev& b, uint32_t jb, uint32_t je, unsigned int* cursor,
                                              int path, int streams, int blocks, cudaStream_t s) {
  const bool two = streams == 2;
  switch (path) {
    case 0: return two ? launch_queue_t<0, 2>(b, jb, je, cursor, blocks, s) : launch_queue_t<0, 1>(b, jb, je, cursor, blocks, s);
    case 1: return two ? launch_queue_t<1, 2>(b, jb, je, cursor, blocks, s) : launch_queue_t<1, 1>(b, jb, je, cursor, blocks, s);
    case 2: return two ? launch_queue_t<2, 2>(b, jb, je, cursor, blocks, s) : launch_queue_t<2, 1>(b, jb, je, cursor, blocks, s);
    case 3: return two ? launch_queue_t<3, 2>(b, jb, je, cursor, blocks, s) : launch_queue_t<3, 1>(b, jb, je, cursor, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

int BBP_CAT(queue_occupancy_l, BBP_LMAX)(int path, int streams) {
  const bool two = streams == 2;
  switch (path) {
    case 0: return two ? queue_occupancy_t<0, 2>() : queue_occupancy_t<0, 1>();
    case 1: return two ? queue_occupancy_t<1, 2>() : queue_occupancy_t<1, 1>();
    case 2: return two ? queue_occupancy_t<2, 2>() : queue_occupancy_t<2, 1>();
    case 3: return two ? queue_occupancy_t<3, 2>() : queue_occupancy_t<3, 1>();
    default: return 1;
  }
}

}  // namespace bbp
