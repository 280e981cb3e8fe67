// Wavefront expansion, duplicate removal, and ordering reconstruction.
//
// One level of Listing 1 (van der Zanden & Bodlaender, arXiv 1709.09990,
// Section 3.1): every set S of L_i is extended by every vertex v outside S
// whose degree after eliminating S, |Q(S, v)|, is at most k.  The extensions
// S u {v} are deduplicated (Section 3.2) in an exact open-addressing hash
// table and appended to L_{i+1} together with the predecessor vertex v.
//
// GB300 mapping.  A warp takes 32 consecutive states (coalesced key loads).
//  1. Thread-per-state: the components of G[S] are found by a bitset flood
//     fill over the adjacency rows held in shared memory, one row read per
//     vertex of S at most.  Each component C contributes its outer boundary
//     B_C = N(C) \ S.
//     Then Q(S, v) = (N(v) u U{B_C : v in B_C}) \ (S u {v}), the bitset form
//     of the depth-first search inside Listing 1: a vertex outside S
//     is reached from v through S exactly when it borders a component of G[S]
//     that v borders.  Components with |B_C| >= k+2 make every v in B_C
//     infeasible at once; up to 8 other boundaries stay in registers, and a
//     state with more falls back to a flood fill per candidate v.  Only the
//     canonical candidates are tested: v below min(S), or v on the boundary
//     of the component of min(S); that generates every set of L_{i+1} (see
//     feasible_extensions) from about a third as many parents.  The flood
//     fill is lazy: the component of min(S) first, then only the components
//     next to a candidate that passes |N(v) \ S| <= k.
//  2. Warp-cooperative insert: the feasible (S, v) pairs of the 32 states are
//     packed into a per-warp shared-memory queue, and the whole warp inserts
//     32 of them at a time with one 4/8/16-byte compare-and-swap each, so
//     lanes do not idle on states with few extensions.
//  3. The winners of a round append (S u {v}, v) to L_{i+1} with one atomic
//     add per warp.
#include <cuda_runtime.h>

#include "tw_expand_core.cuh"
#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

using core::ExpandParams;
using core::ResidentWarps;
using core::kFull;

template <class K, int kWarps, int U, bool kMMW = false, bool kRanged = false>
__global__ void __launch_bounds__(kWarps * 32, ResidentWarps<K>::value / kWarps)
    expand_insert_kernel(const ExpandParams<K> p) {
  constexpr int kBits = KeyTraits<K>::kBits;
  __shared__ K sAdj[kBits];
  __shared__ K sState[kWarps * 32];
  __shared__ uint16_t sQueue[kWarps * 32 * kBits];
  core::expand_level<K, kWarps, U, kMMW, kRanged>(p, sAdj, sState, sQueue);
}

// One hash range of a level whose table is built slice by slice; the output
// list may continue in a second buffer (out_tail from position out_split on).
template <class K, int U>
__global__ void __launch_bounds__(4 * 32, ResidentWarps<K>::value / 4)
    expand_ranged_kernel(const ExpandParams<K> p, K* out_tail, unsigned long long out_split) {
  constexpr int kBits = KeyTraits<K>::kBits;
  __shared__ K sAdj[kBits];
  __shared__ K sState[4 * 32];
  __shared__ uint16_t sQueue[4 * 32 * kBits];
  core::expand_level<K, 4, U, false, true>(p, sAdj, sState, sQueue, 0u, 0u, out_tail, out_split);
}

// A ranged launch: 4 warps per block, one block per SM slot.
template <class K, int U>
cudaError_t launch_ranged(const ExpandParams<K>& p, K* out_tail, unsigned long long out_split,
                          unsigned long long blocks_needed, cudaStream_t s) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_ranged_kernel<K, U>, 128, 0);
  unsigned long long grid = (unsigned long long)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > blocks_needed) grid = blocks_needed;
  expand_ranged_kernel<K, U><<<(int)grid, 128, 0, s>>>(p, out_tail, out_split);
  return cudaGetLastError();
}

template <class K, int kWarps, int U>
cudaError_t launch_expand_u(const ExpandParams<K>& p, unsigned long long blocks_needed, int grid, KeyClass kc,
                            cudaStream_t s) {
  if (grid <= 0) {
    // resident blocks per SM x SMs, cached per (device, width, warps, U)
    static thread_local int cached_dev = -1, cached_grid[3][3][2] = {{{0}}};
    int dev = 0;
    cudaGetDevice(&dev);
    const int wi = kWarps == 2 ? 0 : (kWarps == 4 ? 1 : 2);
    const int ui = U == TW_INSERT_UNROLL ? 0 : 1;
    if (cached_dev != dev) {
      for (auto& a : cached_grid)
        for (auto& r : a)
          for (int& x : r) x = 0;
      cached_dev = dev;
    }
    int& g = cached_grid[(int)kc][wi][ui];
    if (g == 0) {
      int sms = 0, per_sm = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_insert_kernel<K, kWarps, U>, kWarps * 32, 0);
      g = sms * (per_sm > 0 ? per_sm : 1);
    }
    grid = g;
  }
  if ((unsigned long long)grid > blocks_needed) grid = (int)blocks_needed;
  expand_insert_kernel<K, kWarps, U><<<grid, kWarps * 32, 0, s>>>(p);
  return cudaGetLastError();
}

template <class K, int kWarps>
cudaError_t launch_expand_t(const ExpandLaunch& a, cudaStream_t s) {
  ExpandParams<K> p;
  p.in_keys = static_cast<const K*>(a.in_keys);
  p.n_in = a.n_in;
  p.adj = static_cast<const K*>(a.adj);
  p.n = a.n;
  p.k = a.k;
  p.table = static_cast<K*>(a.table);
  p.table_slots = a.table_slots;
  p.max_probes = a.max_probes;
  p.out_keys = static_cast<K*>(a.out_keys);
  p.out_pred = a.out_pred;
  p.out_cap = a.out_cap;
  p.ctr = a.ctr;
  p.allowed = core::kfrom_words<K>(a.allowed[0], a.allowed[1]);
  p.mmw = a.mmw;
  p.ranges = a.ranges > 0 ? a.ranges : 1;
  p.range = a.range;
  if (a.n_in == 0) return cudaSuccess;
  const unsigned long long chunks = (a.n_in + 31ull) / 32ull;
  const unsigned long long blocks_needed = (chunks + kWarps - 1) / kWarps;
  if (a.ranges > 0) {
    const unsigned long long need4 = (chunks + 3) / 4;
    K* tail = static_cast<K*>(a.out_tail);
    if (a.table_slots * sizeof(K) > core::kDeepTableBytes)
      return launch_ranged<K, 2 * TW_INSERT_UNROLL>(p, tail, a.out_split, need4, s);
    return launch_ranged<K, TW_INSERT_UNROLL>(p, tail, a.out_split, need4, s);
  }
  if (a.mmw) {
    // minor-min-width pruning (opt-in): its own instantiation, 4 warps
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_insert_kernel<K, 4, TW_INSERT_UNROLL, true>, 128, 0);
    unsigned long long grid = (unsigned long long)sms * (per_sm > 0 ? per_sm : 1);
    const unsigned long long need = (chunks + 3) / 4;
    if (grid > need) grid = need;
    expand_insert_kernel<K, 4, TW_INSERT_UNROLL, true><<<(int)grid, 128, 0, s>>>(p);
    return cudaGetLastError();
  }
  // Tables far larger than L2 miss on most probes: keep twice as many
  // compare-and-swaps in flight per lane there.
  if (a.table_slots * sizeof(K) > core::kDeepTableBytes)
    return launch_expand_u<K, kWarps, 2 * TW_INSERT_UNROLL>(p, blocks_needed, a.grid, a.kc, s);
  return launch_expand_u<K, kWarps, TW_INSERT_UNROLL>(p, blocks_needed, a.grid, a.kc, s);
}

template <class K>
cudaError_t launch_expand_k(const ExpandLaunch& a, cudaStream_t s) {
  switch (a.block_threads) {
    case 64: return launch_expand_t<K, 2>(a, s);
    case 256: return launch_expand_t<K, 8>(a, s);
    default: return launch_expand_t<K, 4>(a, s);
  }
}

// The 128-bit queue of 8 warps would exceed the 48 KB static shared limit.
template <>
cudaError_t launch_expand_k<K128>(const ExpandLaunch& a, cudaStream_t s) {
  return a.block_threads == 64 ? launch_expand_t<K128, 2>(a, s) : launch_expand_t<K128, 4>(a, s);
}

// ---------------------------------------------------------------- clearing
__global__ void clear_kernel(uint4* __restrict__ t, size_t n16, LevelCounters* ctr) {
  if (ctr && blockIdx.x == 0 && threadIdx.x < sizeof(LevelCounters) / sizeof(unsigned long long))
    reinterpret_cast<unsigned long long*>(ctr)[threadIdx.x] = 0ull;
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) t[i] = ones;
}

// ------------------------------------------------------------- widening
__global__ void widen32_kernel(const uint32_t* __restrict__ src, unsigned long long* __restrict__ dst,
                               unsigned long long count) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    dst[i] = src[i];
}

// ------------------------------------------------------------ fingerprints
template <class K>
__global__ void fingerprint_kernel(const K* __restrict__ keys, unsigned long long count, LevelCounters* ctr) {
  unsigned long long s = 0, x = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const unsigned long long f = kfingerprint(keys[i]);
    s += f;
    x ^= f;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    s += __shfl_xor_sync(kFull, s, d);
    x ^= __shfl_xor_sync(kFull, x, d);
  }
  if ((threadIdx.x & 31) == 0 && (s | x)) {
    atomicAdd(&ctr->fp_sum, s);
    atomicXor(&ctr->fp_xor, x);
  }
}

// ------------------------------------------------------------ backward walk
template <class K>
__global__ void walk_init_kernel(const K* keys, K* walk, int last) {
  walk[last] = keys[0];
}

template <class K>
__global__ void walk_step_kernel(const K* __restrict__ keys, const uint8_t* __restrict__ pred,
                                 unsigned long long count, K* walk, int j, int32_t* order) {
  const K target = walk[j];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    if (keys[i] == target) {
      const int v = pred[i];
      order[j - 1] = v;
      walk[j - 1] = target & ~kbit<K>(v);
    }
  }
}

template <class K>
__global__ void walk_finish_kernel(const K* walk, int last, int n, int32_t* order) {
  const K fin = walk[last];
  int pos = last;
  for (int v = 0; v < n; ++v)
    if (!ktest(fin, v)) order[pos++] = v;
}

// --------------------------------------------------- tree decomposition
__global__ void td_kernel(const unsigned long long* __restrict__ adj64, int n, int words64,
                          const int32_t* __restrict__ order, int32_t* parent, unsigned long long* bags) {
  __shared__ K128 sAdj[128];
  __shared__ int sPos[128];
  core::td_block(adj64, n, words64, order, parent, bags, sAdj, sPos);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int stream_grid(unsigned long long work, int per_block) {
  unsigned long long g = (work + per_block - 1) / per_block;
  const unsigned long long cap = (unsigned long long)sm_count() * 8ull;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_expand(const ExpandLaunch& a, cudaStream_t s) {
  switch (a.kc) {
    case kKey32: return launch_expand_k<uint32_t>(a, s);
    case kKey64: return launch_expand_k<unsigned long long>(a, s);
    default: return launch_expand_k<K128>(a, s);
  }
}

cudaError_t launch_clear(void* table, size_t table_bytes, LevelCounters* ctr, cudaStream_t s) {
  const size_t n16 = table_bytes / 16;
  clear_kernel<<<stream_grid(n16 > 0 ? n16 : 1, 256 * 4), 256, 0, s>>>(static_cast<uint4*>(table), n16, ctr);
  return cudaGetLastError();
}

cudaError_t launch_widen32(const uint32_t* src, unsigned long long* dst, unsigned long long count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  widen32_kernel<<<stream_grid(count, 256 * 4), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_fingerprint(KeyClass kc, const void* keys, unsigned long long count, LevelCounters* ctr,
                               cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int g = stream_grid(count, 256 * 4);
  switch (kc) {
    case kKey32: fingerprint_kernel<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(keys), count, ctr); break;
    case kKey64:
      fingerprint_kernel<unsigned long long><<<g, 256, 0, s>>>(static_cast<const unsigned long long*>(keys), count, ctr);
      break;
    default: fingerprint_kernel<K128><<<g, 256, 0, s>>>(static_cast<const K128*>(keys), count, ctr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_walk_init(KeyClass kc, const void* keys, void* walk, int last, cudaStream_t s) {
  switch (kc) {
    case kKey32: walk_init_kernel<uint32_t><<<1, 1, 0, s>>>(static_cast<const uint32_t*>(keys), static_cast<uint32_t*>(walk), last); break;
    case kKey64:
      walk_init_kernel<unsigned long long><<<1, 1, 0, s>>>(static_cast<const unsigned long long*>(keys),
                                                           static_cast<unsigned long long*>(walk), last);
      break;
    default: walk_init_kernel<K128><<<1, 1, 0, s>>>(static_cast<const K128*>(keys), static_cast<K128*>(walk), last); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_walk_step(KeyClass kc, const void* keys, const uint8_t* pred, unsigned long long count, void* walk,
                             int j, int32_t* order, cudaStream_t s) {
  const int g = stream_grid(count > 0 ? count : 1, 256 * 4);
  switch (kc) {
    case kKey32:
      walk_step_kernel<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(keys), pred, count,
                                                   static_cast<uint32_t*>(walk), j, order);
      break;
    case kKey64:
      walk_step_kernel<unsigned long long><<<g, 256, 0, s>>>(static_cast<const unsigned long long*>(keys), pred, count,
                                                             static_cast<unsigned long long*>(walk), j, order);
      break;
    default:
      walk_step_kernel<K128><<<g, 256, 0, s>>>(static_cast<const K128*>(keys), pred, count, static_cast<K128*>(walk), j,
                                               order);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_walk_finish(KeyClass kc, const void* walk, int last, int n, int32_t* order, cudaStream_t s) {
  switch (kc) {
    case kKey32: walk_finish_kernel<uint32_t><<<1, 1, 0, s>>>(static_cast<const uint32_t*>(walk), last, n, order); break;
    case kKey64:
      walk_finish_kernel<unsigned long long><<<1, 1, 0, s>>>(static_cast<const unsigned long long*>(walk), last, n, order);
      break;
    default: walk_finish_kernel<K128><<<1, 1, 0, s>>>(static_cast<const K128*>(walk), last, n, order); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_td(const unsigned long long* adj64, int n, int words64, const int32_t* order, int32_t* parent,
                      unsigned long long* bags, cudaStream_t s) {
  td_kernel<<<1, 128, 0, s>>>(adj64, n, words64, order, parent, bags);
  return cudaGetLastError();
}

}  // namespace tw
