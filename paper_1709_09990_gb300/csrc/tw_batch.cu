// Batched wavefront expansion: one persistent launch expands the current level
// of every active graph of a batch (per-graph frontier segments), so that many
// small graphs share launches instead of paying one launch and one host round
// trip per level each.  The per-state work is the same as in the single-graph
// kernel (tw_expand_core.cuh); states are 64-bit (n <= 64).
//
// Work items are chunks of 32 states.  Graph s owns the chunks
// [chunk_begin[s], chunk_begin[s+1]); a warp finds its graph by binary search
// and reloads the graph's adjacency rows into its own slice of shared memory
// when the graph changes.  Each graph has its own table segment, output
// segment and counters.  Outputs record the parent's index in its level, so a
// finished graph's ordering is recovered by one thread chasing parent indices
// (the added vertex is the bit in which a state and its parent differ).
#include <cuda_runtime.h>

#include "tw_expand_core.cuh"
#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

using core::kFull;
constexpr int kBatchWarps = 4;

__global__ void __launch_bounds__(kBatchWarps * 32, 6)
    expand_batch_kernel(const BatchSeg* __restrict__ segs, const unsigned long long* __restrict__ chunk_begin,
                        int nseg, unsigned long long total_chunks, const unsigned long long* __restrict__ keys,
                        const unsigned long long* __restrict__ adj_all, unsigned long long* table,
                        unsigned long long* out_keys, uint32_t* out_parent, BatchCounters* ctr, int max_probes) {
  using K = unsigned long long;
  __shared__ K sAdj[kBatchWarps][64];
  __shared__ K sState[kBatchWarps][32];
  __shared__ uint16_t sQueue[kBatchWarps][32 * 64];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const unsigned long long stride = (unsigned long long)gridDim.x * kBatchWarps;
  int cur = -1;
  BatchSeg sg{};
  K valid = 0;
  core::LevelOut<K, true> out{};
  for (unsigned long long c = (unsigned long long)blockIdx.x * kBatchWarps + warp; c < total_chunks; c += stride) {
    if (cur < 0 || c < chunk_begin[cur] || c >= chunk_begin[cur + 1]) {
      int lo = 0, hi = nseg - 1;  // last s with chunk_begin[s] <= c
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk_begin[mid] <= c)
          lo = mid;
        else
          hi = mid - 1;
      }
      cur = lo;
      sg = segs[cur];
      __syncwarp();
      const K* a = adj_all + (size_t)sg.graph * 64;
      sAdj[warp][lane] = lane < sg.n ? a[lane] : 0ull;
      sAdj[warp][lane + 32] = lane + 32 < sg.n ? a[lane + 32] : 0ull;
      __syncwarp();
      valid = kfirst_n<K>(sg.n);
      out.keys = out_keys + sg.o_off;
      out.pred = nullptr;
      out.parent = out_parent + sg.o_off;
      out.cap = sg.o_cap;
      out.count = &ctr[cur].out_count;
      out.overflow = &ctr[cur].overflow;
    }
    const unsigned long long local = c - chunk_begin[cur];
    const unsigned long long idx = local * 32ull + lane;
    const bool active = idx < sg.in_count;
    const K S = active ? keys[sg.in_off + idx] : valid;
    const K feas = active ? core::feasible_extensions<K>(S, sAdj[warp], valid, valid, sg.k) : 0ull;
    const int total = core::build_queue<K>(S, feas, lane, sState[warp], sQueue[warp]);
    if (lane == 0 && total) atomicAdd(&ctr[cur].generated, (unsigned long long)total);
    out.parent_base = (uint32_t)(local * 32ull);
    core::insert_queue<K, true>(sQueue[warp], sState[warp], total, lane, table + sg.t_off, sg.t_slots, max_probes,
                                out);
    __syncwarp();
  }
}

// Copies segment s of (keys, parents) from src to dst; src_off == ~0 writes
// the single empty-set state instead (level 0 of a new run).
__global__ void copy_segments_kernel(const CopySeg* __restrict__ segs, int nseg,
                                     const unsigned long long* __restrict__ src_keys,
                                     const uint32_t* __restrict__ src_par, unsigned long long* dst_keys,
                                     uint32_t* dst_par) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const CopySeg cs = segs[s];
    if (cs.src_off == ~0ull) {
      if (threadIdx.x == 0) {
        dst_keys[cs.dst_off] = 0ull;
        dst_par[cs.dst_off] = 0u;
      }
      continue;
    }
    for (unsigned long long i = threadIdx.x; i < cs.count; i += blockDim.x) {
      dst_keys[cs.dst_off + i] = src_keys[cs.src_off + i];
      dst_par[cs.dst_off + i] = src_par[cs.src_off + i];
    }
  }
}

// One block per segment (grid-stride): the sum and xor of the level
// fingerprints of the segment's keys.
__global__ void fingerprint_segments_kernel(const CopySeg* __restrict__ segs, int nseg,
                                            const unsigned long long* __restrict__ keys, unsigned long long* out) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const CopySeg cs = segs[s];
    unsigned long long sum = 0, x = 0;
    for (unsigned long long i = threadIdx.x; i < cs.count; i += blockDim.x) {
      const unsigned long long f = kfingerprint(keys[cs.src_off + i]);
      sum += f;
      x ^= f;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      sum += __shfl_xor_sync(kFull, sum, d);
      x ^= __shfl_xor_sync(kFull, x, d);
    }
    if ((threadIdx.x & 31) == 0 && (sum | x)) {
      atomicAdd(&out[2 * s], sum);
      atomicXor(&out[2 * s + 1], x);
    }
  }
}

// One thread per finished graph: walk the parent indices from the first state
// of the last level down to level 0, then append the vertices outside the
// final set in increasing order.
__global__ void walk_batch_kernel(const WalkSeg* __restrict__ walks, int nwalk,
                                  const unsigned long long* __restrict__ level_off,
                                  const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ par,
                                  int32_t* orders) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwalk) return;
  const WalkSeg ws = walks[w];
  const unsigned long long* lo = level_off + ws.level_base;
  int32_t* order = orders + ws.order_off;
  unsigned long long idx = 0;
  unsigned long long S = keys[lo[ws.last]];
  const unsigned long long fin = S;
  for (int j = ws.last; j >= 1; --j) {
    const uint32_t p = par[lo[j] + idx];
    const unsigned long long prev = keys[lo[j - 1] + p];
    order[j - 1] = __ffsll(S ^ prev) - 1;
    S = prev;
    idx = p;
  }
  int pos = ws.last;
  for (int v = 0; v < ws.n; ++v)
    if (!((fin >> v) & 1ull)) order[pos++] = v;
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

cudaError_t launch_expand_batch(const BatchSeg* segs, const unsigned long long* chunk_begin, int nseg,
                                unsigned long long total_chunks, const unsigned long long* keys,
                                const unsigned long long* adj_all, unsigned long long* table,
                                unsigned long long* out_keys, uint32_t* out_parent, BatchCounters* ctr, int max_probes,
                                cudaStream_t s) {
  if (total_chunks == 0 || nseg == 0) return cudaSuccess;
  static thread_local int grid_cache = 0;
  if (grid_cache == 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_batch_kernel, kBatchWarps * 32, 0);
    grid_cache = sms() * (per_sm > 0 ? per_sm : 1);
  }
  const unsigned long long blocks_needed = (total_chunks + kBatchWarps - 1) / kBatchWarps;
  const int grid = (int)(blocks_needed < (unsigned long long)grid_cache ? blocks_needed : grid_cache);
  expand_batch_kernel<<<grid, kBatchWarps * 32, 0, s>>>(segs, chunk_begin, nseg, total_chunks, keys, adj_all, table,
                                                        out_keys, out_parent, ctr, max_probes);
  return cudaGetLastError();
}

cudaError_t launch_copy_segments(const CopySeg* segs, int nseg, const unsigned long long* src_keys,
                                 const uint32_t* src_par, unsigned long long* dst_keys, uint32_t* dst_par,
                                 cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  const int grid = nseg < sms() * 8 ? nseg : sms() * 8;
  copy_segments_kernel<<<grid, 256, 0, s>>>(segs, nseg, src_keys, src_par, dst_keys, dst_par);
  return cudaGetLastError();
}

cudaError_t launch_fingerprint_segments(const CopySeg* segs, int nseg, const unsigned long long* keys,
                                        unsigned long long* out, cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  const int grid = nseg < sms() * 8 ? nseg : sms() * 8;
  fingerprint_segments_kernel<<<grid, 256, 0, s>>>(segs, nseg, keys, out);
  return cudaGetLastError();
}

cudaError_t launch_walk_batch(const WalkSeg* walks, int nwalk, const unsigned long long* level_off,
                              const unsigned long long* keys, const uint32_t* par, int32_t* orders, cudaStream_t s) {
  if (nwalk == 0) return cudaSuccess;
  walk_batch_kernel<<<(nwalk + 127) / 128, 128, 0, s>>>(walks, nwalk, level_off, keys, par, orders);
  return cudaGetLastError();
}

}  // namespace tw
