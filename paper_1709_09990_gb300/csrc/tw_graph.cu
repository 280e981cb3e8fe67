// Kernels of the graph-driven level loop.  A decide(k) run (Listing 1,
// Section 3.1 of arXiv 1709.09990) is captured once per (graph size, k,
// buffers) as init, plan, then (clear, expand, plan) per level; every kernel
// reads the level it works on from a GraphState in device memory, so one
// graph launch runs all levels with a single host synchronisation at the end.
// Kernels of levels after the run has ended return at once.
#include <cuda_runtime.h>

#include "tw_expand_core.cuh"
#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

using core::ExpandParams;
using core::ResidentWarps;

template <class K>
__global__ void graph_init_kernel(GraphState* st, K* keys) {
  st->cur = 0;
  st->level_off[0] = 0ull;
  st->level_cnt[0] = 1ull;
  st->done = st->bail = st->yes = 0;
  st->generated = 0ull;
  st->peak_bytes = 0ull;
  st->table_slots = st->out_off = st->out_cap = 0ull;
  keys[0] = kzero<K>();  // L_0 = {empty set}
}

// Records the level built by the previous expand (unless first), then plans
// the next level: the same growth estimate and 25% table slack as the host
// loop; the output may use the rest of the arena.
__global__ void graph_plan_kernel(GraphState* st, LevelCounters* ctr, unsigned long long arena_cap,
                                  unsigned long long table_cap, unsigned long long direct_table_bytes, int n, int k,
                                  int load_pct, int w, int first) {
  if (st->done || st->bail) return;
  if (!first) {
    const unsigned long long cnt = ctr->out_count;
    if (ctr->overflow != 0u || cnt > st->out_cap || cnt * 100ull > st->table_slots * 90ull) {
      st->bail = 1;
      return;
    }
    const int c = st->cur + 1;
    st->cur = c;
    st->level_off[c] = st->out_off;
    st->level_cnt[c] = cnt;
    st->generated += ctr->generated;
    const unsigned long long live = st->out_off + cnt;  // every level is kept
    const unsigned long long bytes = live * (unsigned long long)(w + 1) + st->table_slots * (unsigned long long)w;
    if (bytes > st->peak_bytes) st->peak_bytes = bytes;
    if (cnt == 0ull) {
      st->done = 1;
      st->yes = 0;
      return;
    }
    if (c == n - k - 1) {
      st->done = 1;
      st->yes = 1;
      return;
    }
  }
  const int i = st->cur;
  // (integer plan: a chain of FP64 divisions in one thread costs about ten
  // microseconds per level on this part)
  unsigned long long table_est = 0, slots = 0;
  core::plan_level(st->level_cnt[i], i > 0 ? st->level_cnt[i - 1] : 0ull, n, i, load_pct, &table_est, &slots);
  const unsigned long long out_off = st->level_off[i] + st->level_cnt[i];
  // levels for the partitioned insert, and levels that do not fit, go back
  // to the host loop
  if (slots > table_cap || slots * (unsigned long long)w > direct_table_bytes || out_off >= arena_cap ||
      arena_cap - out_off < table_est) {
    st->bail = 1;
    return;
  }
  st->table_slots = slots;
  st->out_off = out_off;
  st->out_cap = arena_cap - out_off;
  ctr->out_count = 0ull;
  ctr->generated = 0ull;
  ctr->overflow = 0u;
}

__global__ void graph_clear_kernel(const GraphState* __restrict__ st, uint4* __restrict__ t, int w) {
  if (st->done || st->bail) return;
  const size_t n16 = (st->table_slots * (unsigned long long)w + 15ull) / 16ull;
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) t[i] = ones;
}

template <class K, int kWarps, bool kMMW>
__global__ void __launch_bounds__(kWarps * 32, ResidentWarps<K>::value / kWarps)
    graph_expand_kernel(const GraphState* __restrict__ st, const ExpandParams<K> base) {
  constexpr int kBits = KeyTraits<K>::kBits;
  __shared__ K sAdj[kBits];
  __shared__ K sState[kWarps * 32];
  __shared__ uint16_t sQueue[kWarps * 32 * kBits];
  if (st->done || st->bail) return;
  ExpandParams<K> p = base;
  const int cur = st->cur;
  p.in_keys = base.in_keys + st->level_off[cur];
  p.n_in = st->level_cnt[cur];
  p.out_keys = base.out_keys + st->out_off;
  p.out_pred = base.out_pred + st->out_off;
  p.out_cap = st->out_cap;
  p.table_slots = st->table_slots;
  core::expand_level<K, kWarps, TW_INSERT_UNROLL, kMMW>(p, sAdj, sState, sQueue);
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <class K, int kWarps>
cudaError_t expand_t(const GraphState* st, const ExpandLaunch& a, cudaStream_t s) {
  ExpandParams<K> p;
  p.in_keys = static_cast<const K*>(a.in_keys);
  p.n_in = 0;
  p.adj = static_cast<const K*>(a.adj);
  p.n = a.n;
  p.k = a.k;
  p.table = static_cast<K*>(a.table);
  p.table_slots = 0;
  p.max_probes = a.max_probes;
  p.out_keys = static_cast<K*>(a.out_keys);
  p.out_pred = a.out_pred;
  p.out_cap = 0;
  p.ctr = a.ctr;
  p.allowed = core::kfrom_words<K>(a.allowed[0], a.allowed[1]);
  p.mmw = a.mmw;
  p.ranges = 1;
  p.range = 0;
  int per_sm = 0;
  if (a.mmw) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, graph_expand_kernel<K, kWarps, true>, kWarps * 32, 0);
    graph_expand_kernel<K, kWarps, true><<<sm_count() * (per_sm > 0 ? per_sm : 1), kWarps * 32, 0, s>>>(st, p);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, graph_expand_kernel<K, kWarps, false>, kWarps * 32, 0);
    graph_expand_kernel<K, kWarps, false><<<sm_count() * (per_sm > 0 ? per_sm : 1), kWarps * 32, 0, s>>>(st, p);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_graph_init(KeyClass kc, GraphState* st, void* keys, cudaStream_t s) {
  switch (kc) {
    case kKey32: graph_init_kernel<uint32_t><<<1, 1, 0, s>>>(st, static_cast<uint32_t*>(keys)); break;
    case kKey64: graph_init_kernel<unsigned long long><<<1, 1, 0, s>>>(st, static_cast<unsigned long long*>(keys)); break;
    default: graph_init_kernel<K128><<<1, 1, 0, s>>>(st, static_cast<K128*>(keys)); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_graph_plan(GraphState* st, LevelCounters* ctr, unsigned long long arena_cap,
                              unsigned long long table_cap, unsigned long long direct_table_bytes, int n, int k,
                              int load_pct, int key_bytes, int first, cudaStream_t s) {
  graph_plan_kernel<<<1, 1, 0, s>>>(st, ctr, arena_cap, table_cap, direct_table_bytes, n, k, load_pct, key_bytes,
                                    first);
  return cudaGetLastError();
}

cudaError_t launch_graph_clear(KeyClass kc, const GraphState* st, void* table, cudaStream_t s) {
  graph_clear_kernel<<<sm_count() * 4, 256, 0, s>>>(st, static_cast<uint4*>(table), (int)key_bytes(kc));
  return cudaGetLastError();
}

cudaError_t launch_graph_expand(const GraphState* st, const ExpandLaunch& a, cudaStream_t s) {
  switch (a.kc) {
    case kKey32: return expand_t<uint32_t, 4>(st, a, s);
    case kKey64: return expand_t<unsigned long long, 4>(st, a, s);
    default: return expand_t<K128, 4>(st, a, s);
  }
}

}  // namespace tw
