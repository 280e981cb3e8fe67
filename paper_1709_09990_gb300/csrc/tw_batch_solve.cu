// Persistent batched solve: one launch for a whole batch of graphs (n <= 64).
//
// Every block is a worker with its own workspace (a level arena and two
// tables in device memory).  A block takes the next graph from a queue (one
// atomic add), runs that graph's decide runs itself - Listing 1 level by level
// (Section 3.1), the block's warps taking the chunks of 32 states in turn, with
// only block barriers between levels - until the treewidth is certified (yes
// at tw, and no at tw-1 or tw equal to the lower bound), walks back through
// its levels for the ordering, and takes the next graph.  The per-graph k
// sweep starts at the lower bound, or at a proposed bound (learned-k), and
// moves up on no and down on yes.  A graph whose levels outgrow the block's
// workspace is marked and left to the single-graph path; nothing else leaves
// the device until the batch is done.
//
// In decide mode every graph runs one decide at its own k and reports its
// answer, level sizes and level fingerprints (tw_decide_batch).
#include <climits>

#include <cuda_runtime.h>

#include "tw_expand_core.cuh"
#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

using core::ExpandParams;
using K = unsigned long long;
constexpr unsigned kFull = 0xffffffffu;


// The block's view of its workspace.
struct Work {
  K* arena;
  uint8_t* pred;
  K* table[2];
  unsigned long long dirty[2];  // slots of each table to empty before use
  LevelCounters* ctr;
  unsigned long long* off;      // level offsets of the run in the arena
  unsigned long long* cnt;      // level sizes
};

// Sum and xor of the level fingerprints of keys[0, count) by the block.
__device__ void block_fingerprint(const K* keys, unsigned long long count, unsigned long long* sRed,
                                  unsigned long long* sum_out, unsigned long long* xor_out) {
  unsigned long long s = 0, x = 0;
  for (unsigned long long i = threadIdx.x; i < count; i += blockDim.x) {
    const unsigned long long f = kfingerprint(kload_cg(&keys[i]));
    s += f;
    x ^= f;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    s += __shfl_xor_sync(kFull, s, d);
    x ^= __shfl_xor_sync(kFull, x, d);
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sRed[2 * warp] = s;
    sRed[2 * warp + 1] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ts = 0, tx = 0;
    for (int w = 0; w < nw; ++w) {
      ts += sRed[2 * w];
      tx ^= sRed[2 * w + 1];
    }
    *sum_out = ts;
    *xor_out = tx;
  }
  __syncthreads();
}

// decide(k) of one graph by one block into its workspace.  Returns false when
// the levels outgrow the workspace; else *yes and *last (the final level).
// With fp_sum / fp_xor (decide mode) the level fingerprints are written.
template <int kWarps>
__device__ __noinline__ bool block_decide(const BatchSolveArgs& a, const K* adj, int n, int k, Work& w, K* sAdj, K* sState,
                             uint16_t* sQueue, unsigned long long* sRed, bool* yes, int* last,
                             unsigned long long* stats, unsigned long long* fp_sum, unsigned long long* fp_xor) {
  for (int t = 0; t < 2; ++t) {
    for (unsigned long long j = threadIdx.x; j < w.dirty[t]; j += blockDim.x) w.table[t][j] = kones<K>();
    w.dirty[t] = 0;
  }
  if (threadIdx.x == 0) {
    w.arena[0] = kzero<K>();
    w.off[0] = 0ull;
    w.cnt[0] = 1ull;
  }
  if (fp_sum && threadIdx.x == 0) {
    fp_sum[0] = 0ull;  // fp of the empty set
    fp_xor[0] = 0ull;
  }
  __syncthreads();
  *last = 0;
  if (k >= n - 1) {
    *yes = true;
    return true;
  }
  unsigned long long off = 0, cnt = 1, prev_cnt = 0;
  for (int i = 0; i <= n - k - 2; ++i) {
    // the plan of the level in integer arithmetic (FP64 is slow on this part)
    unsigned long long table_est = 0, slots = 0;
    core::plan_level(cnt, prev_cnt, n, i, a.load_pct, &table_est, &slots);
    const unsigned long long out_off = off + cnt;
    if (out_off >= a.A || a.A - out_off < table_est) return false;
    if (slots > a.T) slots = a.T;
    const int t = i & 1;
    unsigned long long got = 0, gen = 0;
    for (;;) {
      // a table that fills is emptied and the level expanded again with a
      // larger one (up to the workspace's table size)
      if (threadIdx.x == 0) *w.ctr = LevelCounters{};
      __syncthreads();
      ExpandParams<K> p;
      p.in_keys = w.arena + off;
      p.n_in = cnt;
      p.adj = adj;
      p.n = n;
      p.k = k;
      p.table = w.table[t];
      p.table_slots = slots;
      p.max_probes = a.max_probes;
      p.out_keys = w.arena + out_off;
      p.out_pred = w.pred + out_off;
      p.out_cap = a.A - out_off;
      p.ctr = w.ctr;
      p.allowed = kones<K>();
      p.mmw = 0;
      p.ranges = 1;
      p.range = 0;
      core::expand_level<K, kWarps, TW_INSERT_UNROLL, false, false, true, true>(p, sAdj, sState, sQueue);
      for (unsigned long long j = threadIdx.x; j < w.dirty[1 - t]; j += blockDim.x) w.table[1 - t][j] = kones<K>();
      w.dirty[1 - t] = 0;
      w.dirty[t] = max(w.dirty[t], slots);
      __syncthreads();
      got = __ldcg(&w.ctr->out_count);
      const unsigned int ovf = __ldcg(&w.ctr->overflow);
      gen = __ldcg(&w.ctr->generated);
      __syncthreads();
      if ((ovf & 1u) || got > p.out_cap) return false;  // the arena is full
      if (!(ovf & 2u) && got * 100ull <= slots * 90ull) break;
      if (slots >= a.T) return false;
      slots = min(a.T, max(2 * slots, (got * 100ull) / (unsigned long long)a.load_pct + 1024ull));
      for (unsigned long long j = threadIdx.x; j < w.dirty[t]; j += blockDim.x) w.table[t][j] = kones<K>();
      w.dirty[t] = 0;
      __syncthreads();
    }
    stats[0] += cnt;
    stats[1] += cnt * (unsigned long long)(n - i);
    stats[2] += gen;
    if (threadIdx.x == 0) {
      w.off[i + 1] = out_off;
      w.cnt[i + 1] = got;
    }
    if (fp_sum) block_fingerprint(w.arena + out_off, got, sRed, &fp_sum[i + 1], &fp_xor[i + 1]);
    prev_cnt = cnt;
    off = out_off;
    cnt = got;
    *last = i + 1;
    if (got == 0ull) {
      *yes = false;
      __syncthreads();
      return true;
    }
  }
  *yes = true;
  __syncthreads();
  return true;
}

template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32, 24 / kWarps) batch_solve_kernel(const BatchSolveArgs a) {
  __shared__ K sAdj[64];
  __shared__ K sState[kWarps * 32];
  __shared__ uint16_t sQueue[kWarps * 32 * 64];
  __shared__ unsigned long long sRed[2 * kWarps];
  __shared__ K sWalk;
  __shared__ int sFound;
  __shared__ int sGraph;
  const size_t slot = blockIdx.x;
  Work w;
  w.arena = a.arena + slot * a.A;
  w.pred = a.pred + slot * a.A;
  w.table[0] = a.tables + slot * 2 * a.T;
  w.table[1] = w.table[0] + a.T;
  w.dirty[0] = w.dirty[1] = a.T;  // the workspace starts with anything in it
  w.ctr = a.ctr + slot;
  w.off = a.level_off + slot * 130;
  w.cnt = a.level_cnt + slot * 130;
  unsigned long long stats[3] = {0ull, 0ull, 0ull};
  unsigned long long runs = 0;
  for (;;) {
    if (threadIdx.x == 0) sGraph = (int)atomicAdd(a.next_graph, 1u);
    __syncthreads();
    const int g = sGraph;
    __syncthreads();
    if (g >= a.num_graphs) break;
    const int n = a.n[g];
    const K* adj = a.adj + (size_t)g * 64;
    bool yes = false;
    int last = 0;
    if (a.decide_mode) {
      unsigned long long* fs = a.fp_sum ? a.fp_sum + (size_t)g * 129 : nullptr;
      unsigned long long* fx = a.fp_xor ? a.fp_xor + (size_t)g * 129 : nullptr;
      const bool ok = block_decide<kWarps>(a, adj, n, a.k_start[g], w, sAdj, sState, sQueue, sRed, &yes, &last,
                                           stats, fs, fx);
      ++runs;
      if (threadIdx.x == 0) {
        a.status[g] = ok ? 0 : 2;
        a.yes[g] = yes ? 1 : 0;
        a.last[g] = last;
      }
      if (ok)
        for (int j = threadIdx.x; j <= last; j += blockDim.x) a.level_size[(size_t)g * 129 + j] = __ldcg(&w.cnt[j]);
      __syncthreads();
      continue;
    }
    // the k sweep with certification
    const int lb = a.lb[g];
    int k = a.k_start[g];
    int yes_min = INT_MAX, no_max = lb - 1, yes_in_arena = -1;
    bool ok = true;
    for (;;) {
      ok = block_decide<kWarps>(a, adj, n, k, w, sAdj, sState, sQueue, sRed, &yes, &last, stats, nullptr, nullptr);
      ++runs;
      if (!ok) break;
      if (yes) {
        yes_min = min(yes_min, k);
        yes_in_arena = k;
      } else {
        no_max = max(no_max, k);
        yes_in_arena = -1;
      }
      if (yes_min == no_max + 1) break;
      k = yes_min == INT_MAX ? no_max + 1 : yes_min - 1;
    }
    if (ok && yes_in_arena != yes_min) {
      // the last run was a no: run the yes at tw again for its levels
      ok = block_decide<kWarps>(a, adj, n, yes_min, w, sAdj, sState, sQueue, sRed, &yes, &last, stats, nullptr,
                                nullptr);
      ++runs;
    }
    if (!ok) {
      if (threadIdx.x == 0) {
        a.status[g] = 2;
        a.tw[g] = -1;
      }
      __syncthreads();
      continue;
    }
    if (a.orders) core::walk_block<K>(w.arena, w.pred, w.off, w.cnt, last, n, a.orders + a.order_off[g], &sWalk, &sFound);
    if (threadIdx.x == 0) {
      a.status[g] = 0;
      a.tw[g] = yes_min;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.totals[0], stats[0]);
    atomicAdd(&a.totals[1], stats[1]);
    atomicAdd(&a.totals[2], stats[2]);
    atomicAdd(&a.totals[3], runs);
  }
}

}  // namespace

int batch_solve_blocks(int warps) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (warps == 8)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_solve_kernel<8>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_solve_kernel<4>, 128, 0);
  return sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_batch_solve(const BatchSolveArgs& a, int blocks, int warps, cudaStream_t s) {
  if (a.num_graphs == 0) return cudaSuccess;
  if (warps == 8)
    batch_solve_kernel<8><<<blocks, 256, 0, s>>>(a);
  else
    batch_solve_kernel<4><<<blocks, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tw
