// Fused solve of one small graph: the k sweep (Section 3.1's iterative
// deepening of Listing 1), the backward walk and the tree decomposition in a
// single cooperative launch.
//
// For graphs whose levels hold a few thousand states, the host-driven or
// graph-driven level loops spend their time in launches and host round trips,
// not in the expansion, and a level costs about the latency of one chunk of
// 32 states plus a barrier.  Here the grid is split into groups of blocks and
// consecutive decide runs of the sweep (k, k+1, ...) run at the same time,
// one per group, so the sweep takes about as many level steps as its longest
// run instead of their sum.  Within a group every block runs the same loop:
// expand level i (the group's blocks take the chunks of 32 states in turn,
// the kernel body of tw_expand_core.cuh) while emptying the table the
// previous level used, then one barrier of the group.  Every block reads the
// level's counters after the barrier and takes the same decisions (the next
// table size, stop, answer), so the loop needs no other synchronisation.  Two
// tables alternate per group; all levels of a run stay in the group's arena
// for the walk.  The answer is that of the sequential sweep: the smallest k
// that answers yes, with every smaller k answering no.
//
// A run gives up (status "bail") when a level would not fit the arena or the
// table, or when a table fills; the host then continues the sweep with its
// own loop from that k.  Every barrier wait is bounded: a barrier that does
// not complete within a second (the global timer) sets an error flag, and all
// blocks return.
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

// Bounded barrier over `count` co-resident blocks of a cooperative launch,
// on the counter `arrive` and the generation word `gen`.  The block's threads
// meet at a block barrier; its thread 0 arrives with an acquire-release add
// (which also publishes the block's writes); the last block to arrive resets
// the count and advances the generation with a release; the others poll the
// generation with acquire loads, or give up after kBarrierNs and set *error.
// Returns false once any block has given up.
__device__ bool barrier_wait(unsigned int* arrive, unsigned int* gen, unsigned int count, unsigned int* error) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire(gen);
    const unsigned int prev = atom_add_acq_rel(arrive, 1u);
    if (prev == count - 1) {
      st_relaxed(arrive, 0u);
      red_add_release(gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned int polls = 0;
      while (ld_acquire(gen) == g) {
        if ((++polls & 255u) == 0u) {
          if (ld_acquire(error) != 0u) break;
          if (global_ns() - t0 > kBarrierNs) {
            atomicExch(error, 1u);
            break;
          }
        }
      }
    }
  }
  __syncthreads();
  return *(volatile unsigned int*)error == 0u;
}

template <class K>
struct FusedArgs {
  const K* adj;                       // n rows in the state layout
  const unsigned long long* adj64;    // n rows of words64 words (tree decomposition)
  int n, words64, k0, k_last, max_probes, load_pct, groups, tables_clean;
  const int32_t* lb_dev;              // or null: lower bounds on the device that raise k0
  K* keys[kFusedMaxGroups];           // per group: level arena
  uint8_t* pred[kFusedMaxGroups];
  unsigned long long arena_cap;
  K* table[kFusedMaxGroups][2];
  unsigned long long table_cap;       // slots of each table
  FusedState* st[kFusedMaxGroups];
  int32_t* order;
  int32_t* parent;
  unsigned long long* bags;
};

// One decide run at bound k by the blocks of one group (gb = this block's
// index in the group, nb = the group's blocks).  Returns 0 (no), 1 (yes),
// 2 (gave up: a level would not fit the arena or a table) or -2 (a barrier
// gave up); *last = index of the final level built.
template <class K>
__device__ int group_decide(const FusedArgs<K>& a, int grp, unsigned int gb, unsigned int nb, int k,
                            unsigned long long dirty[2], int* last, K* sAdj, K* sState, uint16_t* sQueue) {
  FusedState* st = a.st[grp];
  unsigned int* error = &a.st[0]->error;
  K* keys = a.keys[grp];
  const int n = a.n;
  const unsigned long long gtid = (unsigned long long)gb * blockDim.x + threadIdx.x;
  const unsigned long long gthreads = (unsigned long long)nb * blockDim.x;
  // a new decide run: empty both tables, zero the per-level counters, L_0
  for (int t = 0; t < 2; ++t)
    for (unsigned long long j = gtid; j < dirty[t]; j += gthreads) a.table[grp][t][j] = kones<K>();
  dirty[0] = dirty[1] = 0;
  if (gb == 0) {
    for (int j = threadIdx.x; j <= n; j += blockDim.x) {
      st->ctr[j] = LevelCounters{};
      st->level_cnt[j] = 0ull;
    }
    if (threadIdx.x == 0) {
      keys[0] = kzero<K>();
      st->level_off[0] = 0ull;
      st->level_cnt[0] = 1ull;
      st->run_states = st->run_candidates = st->run_generated = 0ull;
    }
  }
  if (!barrier_wait(&st->arrive, &st->gen, nb, error)) return -2;
  *last = 0;
  if (k >= n - 1) return 1;
  unsigned long long off = 0, cnt = 1, prev_cnt = 0;
  for (int i = 0; i <= n - k - 2; ++i) {
    // the plan of level i -> i+1, the same in every block of the group
    // (integer arithmetic: this part's FP64 rate is a small fraction of its
    // integer rate)
    unsigned long long table_est = 0, slots = 0;
    core::plan_level(cnt, prev_cnt, n, i, a.load_pct, &table_est, &slots);
    const unsigned long long out_off = off + cnt;
    if (slots > a.table_cap || out_off >= a.arena_cap || a.arena_cap - out_off < table_est) return 2;
    const int t = i & 1;
    ExpandParams<K> p;
    p.in_keys = keys + off;
    p.n_in = cnt;
    p.adj = a.adj;
    p.n = n;
    p.k = k;
    p.table = a.table[grp][t];
    p.max_probes = a.max_probes;
    p.out_keys = keys + out_off;
    p.out_pred = a.pred[grp] + out_off;
    p.out_cap = a.arena_cap - out_off;
    p.ctr = &st->ctr[i + 1];
    p.allowed = kones<K>();
    p.mmw = 0;
    p.ranges = 1;
    p.range = 0;
    unsigned long long got = 0;
    for (int attempt = 0;; ++attempt) {
      p.table_slots = slots;
      core::expand_level<K, kFusedWarps, TW_INSERT_UNROLL, false, false, false, true, true>(p, sAdj, sState,
                                                                                           sQueue, gb, nb);
      // meanwhile empty the table the previous level used
      for (unsigned long long j = gtid; j < dirty[1 - t]; j += gthreads) a.table[grp][1 - t][j] = kones<K>();
      dirty[1 - t] = 0;
      dirty[t] = slots;
      if (!barrier_wait(&st->arrive, &st->gen, nb, error)) return -2;
      got = __ldcg(&st->ctr[i + 1].out_count);
      const unsigned int ovf = __ldcg(&st->ctr[i + 1].overflow);
      if (ovf == 0u) break;  // every pair placed, every new set appended: the level is exact
      // the arena is full, or the largest table is: the host goes on
      if ((ovf & 1u) || got > p.out_cap || slots >= a.table_cap || attempt > 0) return 2;
      // a pair reached the probe limit: run the level again with the largest
      // table, once every block has read the counters
      if (!barrier_wait(&st->arrive, &st->gen, nb, error)) return -2;
      for (unsigned long long j = gtid; j < slots; j += gthreads) a.table[grp][t][j] = kones<K>();
      if (gb == 0 && threadIdx.x == 0) st->ctr[i + 1] = LevelCounters{};
      slots = a.table_cap;
      if (!barrier_wait(&st->arrive, &st->gen, nb, error)) return -2;
    }
    if (gb == 0 && threadIdx.x == 0) {
      st->level_off[i + 1] = out_off;
      st->level_cnt[i + 1] = got;
      st->run_states += cnt;
      st->run_candidates += cnt * (unsigned long long)(n - i);
      st->run_generated += __ldcg(&st->ctr[i + 1].generated);
    }
    prev_cnt = cnt;
    off = out_off;
    cnt = got;
    *last = i + 1;
    if (got == 0ull) return 0;
    if (i + 1 == n - k - 1) return 1;
  }
  return 0;  // (not reached: the loop ends at level n-k-1)
}

// The blocks form `groups` groups of nb = gridDim.x / groups blocks (the
// remainder idles).  Window w runs decide(k0 + w*groups + g) in group g; at
// the window's end every block meets at a barrier of the whole grid, reads
// the runs' results in k order and takes the same decision: the first run
// that did not answer no ends the sweep (a yes is the answer; a run that gave
// up hands the sweep to the host at its k), runs at larger k of that window
// are speculative and not counted; if every run answered no, the next window
// starts.  The first block of the group that answered walks back and builds
// the tree decomposition.
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
  FusedState* st0 = a.st[0];
  const unsigned int nb = gridDim.x / (unsigned int)a.groups;
  const int grp = (int)(blockIdx.x / nb);  // == groups for the idle remainder
  const unsigned int gb = blockIdx.x % nb;
  // slots to empty before use (all, unless the previous launch left every
  // table empty)
  unsigned long long dirty[2] = {a.tables_clean ? 0ull : a.table_cap, a.tables_clean ? 0ull : a.table_cap};
  int status = 0, answer_k = -1, answer_grp = -1, answer_last = 0;
  int k0 = a.k0;
  if (a.lb_dev) k0 = max(k0, max(__ldcg(&a.lb_dev[0]), __ldcg(&a.lb_dev[1])));
  if (blockIdx.x == 0 && threadIdx.x == 0) st0->k_start = k0;
  for (int k_base = k0; status == 0; k_base += a.groups) {
    if (grp < a.groups) {
      const int k = k_base + grp;
      int result = -1, last = 0;
      if (k <= a.k_last) {
        result = group_decide<K>(a, grp, gb, nb, k, dirty, &last, sAdj, sState, sQueue);
        if (result == -2) return;
      }
      if (gb == 0 && threadIdx.x == 0) {
        a.st[grp]->result = result;
        a.st[grp]->run_last = last;
      }
    }
    if (!barrier_wait(&st0->w_arrive, &st0->w_gen, gridDim.x, &st0->error)) return;
    // the same decision in every block
    int counted = 0;
    for (int g = 0; g < a.groups && status == 0; ++g) {
      const int k = k_base + g;
      if (k > a.k_last) {
        status = 1;  // no up to k_last
        break;
      }
      const int r = __ldcg(&a.st[g]->result);
      answer_grp = g;  // (the last run read so far: its levels describe a sweep that found no yes)
      answer_last = __ldcg(&a.st[g]->run_last);
      if (r == 2) {
        // the host runs this k again from the start: its partial run is not
        // counted
        status = 2;
        answer_k = k;
        break;
      }
      ++counted;
      if (r == 1) {
        status = 1;
        answer_k = k;
      }
    }
    if (status == 0 && k_base + a.groups > a.k_last) status = 1;  // every k answered no
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      for (int g = 0; g < counted; ++g) {
        st0->states_expanded += __ldcg(&a.st[g]->run_states);
        st0->candidates += __ldcg(&a.st[g]->run_candidates);
        st0->generated += __ldcg(&a.st[g]->run_generated);
      }
    }
    // the results are read by every block before the next window overwrites them
    if (status == 0 && !barrier_wait(&st0->w_arrive, &st0->w_gen, gridDim.x, &st0->error)) return;
  }
  // leave the group's tables empty for the next launch
  if (grp < a.groups) {
    const unsigned long long gtid = (unsigned long long)gb * blockDim.x + threadIdx.x;
    const unsigned long long gthreads = (unsigned long long)nb * blockDim.x;
    for (int t = 0; t < 2; ++t)
      for (unsigned long long j = gtid; j < dirty[t]; j += gthreads) a.table[grp][t][j] = kones<K>();
  }
  if (status == 2) {
    // gave up at answer_k (every k before it answered no)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st0->status = 2;
      st0->tw = -1;
      st0->last = answer_k;
      st0->group = -1;
    }
    return;
  }
  if (answer_k < 0) {
    // every k up to k_last answered no: the levels of the last run
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st0->status = 1;
      st0->tw = -1;
      st0->last = answer_last;
      st0->group = answer_grp < 0 ? 0 : answer_grp;
    }
    return;
  }
  if (blockIdx.x != (unsigned int)answer_grp * nb) return;
  // the backward walk through the answering group's levels, then the tree
  // decomposition
  FusedState* sg = a.st[answer_grp];
  core::walk_block<K>(a.keys[answer_grp], a.pred[answer_grp], sg->level_off, sg->level_cnt, answer_last, a.n,
                      a.order, &sWalk, &sFound);
  __threadfence_block();
  core::td_block(a.adj64, a.n, a.words64, a.order, a.parent, a.bags, sTdAdj, sPos);
  if (threadIdx.x == 0) {
    st0->status = 1;
    st0->tw = answer_k;
    st0->last = answer_last;
    st0->group = answer_grp;
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
  a.groups = f.groups < 1 ? 1 : (f.groups > kFusedMaxGroups ? kFusedMaxGroups : f.groups);
  a.tables_clean = f.tables_clean;
  a.lb_dev = f.lb_dev;
  for (int g = 0; g < kFusedMaxGroups; ++g) {
    const int h = g < a.groups ? g : 0;
    a.keys[g] = static_cast<K*>(f.keys[h]);
    a.pred[g] = f.pred[h];
    a.table[g][0] = static_cast<K*>(f.table0[h]);
    a.table[g][1] = static_cast<K*>(f.table1[h]);
    a.st[g] = f.st[h];
  }
  a.arena_cap = f.arena_cap;
  a.table_cap = f.table_cap;
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
  // two blocks per SM: each of the three groups has about a hundred blocks
  // (400 warps, so a level of a few thousand states is one chunk per warp)
  // and a barrier of a group takes about a hundred arrivals
  const int grid = sms * (per_sm >= 2 ? 2 : 1);
  if (grid < a.groups) return cudaErrorNotSupported;
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
