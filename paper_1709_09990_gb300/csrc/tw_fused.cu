// Fused solve of one small graph: the whole k sweep (Section 3.1's iterative
// deepening of Listing 1), the backward walk and the tree decomposition in a
// single cooperative launch.
//
// For graphs whose levels hold a few thousand states, the host-driven or
// graph-driven level loops spend their time in launches and host round trips,
// not in the expansion.  Here every block of a cooperative grid runs the same
// loop: expand level i (grid-stride over chunks of 32 states, the kernel body
// of tw_expand_core.cuh) while emptying the table the previous level used,
// then one grid barrier.  Every block reads the level's counters after the
// barrier and takes the same decisions (the next table size, stop, answer),
// so the loop needs no other synchronisation.  Two tables alternate; all
// levels of a decide run stay in one arena for the walk.
//
// The run gives up (status "bail") when a level would not fit the arena or
// the table, or when a table fills; the host then continues the sweep with
// its own loop from that k.  Every barrier wait is bounded: a barrier that
// does not complete within a second (the global timer) sets an error flag,
// and all blocks return.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "tw_expand_core.cuh"
#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

using core::ExpandParams;
using core::ResidentWarps;
constexpr int kFusedWarps = 4;
constexpr unsigned long long kBarrierNs = 1000000000ull;  // a barrier wait gives up after a second

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded grid barrier over all blocks of a cooperative launch (which are
// co-resident).  The block's threads meet at a block barrier; its thread 0
// arrives with an acquire-release add (which also publishes the block's
// writes); the last block to arrive resets the count and advances the
// generation with a release; the others poll the generation with acquire
// loads, or give up after kBarrierNs and set st->error.  Returns false once
// any block has given up.
__device__ bool grid_barrier(FusedState* st) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire(&st->gen);
    const unsigned int prev = atom_add_acq_rel(&st->arrive, 1u);
    if (prev == gridDim.x - 1) {
      st_relaxed(&st->arrive, 0u);
      red_add_release(&st->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned int polls = 0;
      while (ld_acquire(&st->gen) == g) {
        if ((++polls & 255u) == 0u) {
          if (ld_acquire(&st->error) != 0u) break;
          if (global_ns() - t0 > kBarrierNs) {
            atomicExch(&st->error, 1u);
            break;
          }
        }
      }
    }
  }
  __syncthreads();
  return *(volatile unsigned int*)&st->error == 0u;
}

__device__ double binom_f(int n, int r) {
  if (r < 0 || r > n) return 0.0;
  double b = 1.0;
  for (int i = 1; i <= r; ++i) b = b * (double)(n - r + i) / (double)i;
  return b;
}

template <class K>
struct FusedArgs {
  const K* adj;                       // n rows in the state layout
  const unsigned long long* adj64;    // n rows of words64 words (tree decomposition)
  int n, words64, k0, k_last, max_probes, load_pct;
  K* keys;                            // level arena
  uint8_t* pred;
  unsigned long long arena_cap;
  K* table[2];
  unsigned long long table_cap;       // slots of each table
  FusedState* st;
  int32_t* order;
  int32_t* parent;
  unsigned long long* bags;
};

template <class K>
__global__ void __launch_bounds__(kFusedWarps * 32, ResidentWarps<K>::value / kFusedWarps)
    fused_solve_kernel(const FusedArgs<K> a) {
  constexpr int kBits = KeyTraits<K>::kBits;
  __shared__ K sAdj[kBits];
  __shared__ K sState[kFusedWarps * 32];
  __shared__ uint16_t sQueue[kFusedWarps * 32 * kBits];
  __shared__ K128 sTdAdj[128];
  __shared__ int sPos[128];
  __shared__ K sWalk;
  __shared__ int sFound;
  FusedState* st = a.st;
  const int n = a.n;
  const unsigned long long gtid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long gthreads = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long dirty[2] = {a.table_cap, a.table_cap};  // slots to empty before use
  int answer_k = -1, last = 0, bail_k = -1;
  bool bail = false;
  for (int k = a.k0; k <= a.k_last && answer_k < 0 && !bail; ++k) {
    // a new decide run: empty both tables, zero the per-level counters, L_0
    for (int t = 0; t < 2; ++t)
      for (unsigned long long j = gtid; j < dirty[t]; j += gthreads) a.table[t][j] = kones<K>();
    dirty[0] = dirty[1] = 0;
    if (blockIdx.x == 0) {
      for (int j = threadIdx.x; j <= n; j += blockDim.x) {
        st->ctr[j] = LevelCounters{};
        st->level_cnt[j] = 0ull;
      }
      if (threadIdx.x == 0) {
        a.keys[0] = kzero<K>();
        st->level_off[0] = 0ull;
        st->level_cnt[0] = 1ull;
      }
    }
    if (!grid_barrier(st)) return;
    if (k >= n - 1) {
      answer_k = k;
      last = 0;
      break;
    }
    unsigned long long off = 0, cnt = 1, prev_cnt = 0;
    for (int i = 0; i <= n - k - 2; ++i) {
      // the plan of level i -> i+1, the same in every block
      const double bound = fmin((double)cnt * (double)(n - i), binom_f(n, i + 1)) + 1.0;
      double est = (double)n;
      if (i > 0) {
        double r = prev_cnt > 0 ? (double)cnt / (double)prev_cnt : 1.0;
        r = fmin(fmax(r, 0.25), (double)(n - i));
        est = (double)cnt * r;
      }
      const double table_est = fmin(est * 1.25 + 1024.0, bound);
      unsigned long long slots = (unsigned long long)ceil(table_est * 100.0 / (double)a.load_pct);
      if (slots < 64ull) slots = 64ull;
      const unsigned long long out_off = off + cnt;
      if (slots > a.table_cap || out_off >= a.arena_cap || (double)(a.arena_cap - out_off) < table_est) {
        bail = true;
        bail_k = k;
        break;
      }
      const int t = i & 1;
      ExpandParams<K> p;
      p.in_keys = a.keys + off;
      p.n_in = cnt;
      p.adj = a.adj;
      p.n = n;
      p.k = k;
      p.table = a.table[t];
      p.table_slots = slots;
      p.max_probes = a.max_probes;
      p.out_keys = a.keys + out_off;
      p.out_pred = a.pred + out_off;
      p.out_cap = a.arena_cap - out_off;
      p.ctr = &st->ctr[i + 1];
      p.allowed = kones<K>();
      p.mmw = 0;
      p.ranges = 1;
      p.range = 0;
      core::expand_level<K, kFusedWarps, TW_INSERT_UNROLL, false, false, false, true>(p, sAdj, sState, sQueue);
      // meanwhile empty the table the previous level used
      for (unsigned long long j = gtid; j < dirty[1 - t]; j += gthreads) a.table[1 - t][j] = kones<K>();
      dirty[1 - t] = 0;
      dirty[t] = slots;
      if (!grid_barrier(st)) return;
      const LevelCounters& c = st->ctr[i + 1];
      const unsigned long long got = __ldcg(&c.out_count);
      const unsigned int ovf = __ldcg(&c.overflow);
      if (ovf != 0u || got > p.out_cap || got * 100ull > slots * 90ull) {
        bail = true;
        bail_k = k;
        break;
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->level_off[i + 1] = out_off;
        st->level_cnt[i + 1] = got;
        st->states_expanded += cnt;
        st->candidates += cnt * (unsigned long long)(n - i);
        st->generated += __ldcg(&c.generated);
      }
      prev_cnt = cnt;
      off = out_off;
      cnt = got;
      last = i + 1;
      if (got == 0ull) break;                        // no: the next k
      if (i + 1 == n - k - 1) answer_k = k;          // yes
    }
  }
  if (blockIdx.x != 0) return;
  if (bail || answer_k < 0) {
    // gave up at bail_k (every k before it answered no), or every k up to
    // k_last answered no
    if (threadIdx.x == 0) {
      st->status = bail ? 2 : 1;
      st->tw = -1;
      st->last = bail ? bail_k : last;
    }
    return;
  }
  // the backward walk through the kept levels, then the tree decomposition
  core::walk_block<K>(a.keys, a.pred, st->level_off, st->level_cnt, last, n, a.order, &sWalk, &sFound);
  __threadfence_block();
  core::td_block(a.adj64, n, a.words64, a.order, a.parent, a.bags, sTdAdj, sPos);
  if (threadIdx.x == 0) {
    st->status = 1;
    st->tw = answer_k;
    st->last = last;
  }
}

template <class K>
cudaError_t launch_t(const FusedLaunch& f, cudaStream_t s) {
  FusedArgs<K> a;
  a.adj = static_cast<const K*>(f.adj);
  a.adj64 = f.adj64;
  a.n = f.n;
  a.words64 = f.words64;
  a.k0 = f.k0;
  a.k_last = f.k_last;
  a.max_probes = f.max_probes;
  a.load_pct = f.load_pct;
  a.keys = static_cast<K*>(f.keys);
  a.pred = f.pred;
  a.arena_cap = f.arena_cap;
  a.table[0] = static_cast<K*>(f.table0);
  a.table[1] = static_cast<K*>(f.table1);
  a.table_cap = f.table_cap;
  a.st = f.st;
  a.order = f.order;
  a.parent = f.parent;
  a.bags = f.bags;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_solve_kernel<K>, kFusedWarps * 32, 0);
  if (per_sm < 1) return cudaErrorNotSupported;
  // one block per SM: enough warps for levels of a few thousand states, and
  // few arrivals per barrier
  const int grid = sms;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(fused_solve_kernel<K>), dim3(grid),
                                     dim3(kFusedWarps * 32), args, 0, s);
}

}  // namespace

cudaError_t launch_fused_solve(const FusedLaunch& f, cudaStream_t s) {
  switch (f.kc) {
    case kKey32: return launch_t<uint32_t>(f, s);
    case kKey64: return launch_t<unsigned long long>(f, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tw
