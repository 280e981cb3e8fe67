// Partitioned insert for levels whose hash table is far larger than L2.
//
// A compare-and-swap into a table that lives in DRAM costs a random 32-byte
// sector read and, for a winner, a write-back; on GB300 such random accesses
// saturate at roughly a quarter of the streaming bandwidth, while the same
// compare-and-swaps into an L2-resident table run several times faster.  For
// large levels the insert is therefore split in two launches:
//  A. emit: the per-state search of tw_expand_core.cuh; each block then
//     counting-sorts the feasible pairs of its 4 x 32 states by hash range
//     (P ranges, shared-memory histogram), reserves space in each range's
//     region with one global atomic per range, and writes the pairs there;
//  B. insert: the regions are inserted range after range (blocks in launch
//     order follow the ranges), so the slice of the table a range maps to
//     stays in L2 while it is being filled.  Winners append to L_{i+1}.
// Results are the same sets as the direct kernel; only the order of L_{i+1}
// differs.
#include <cuda_runtime.h>

#include "tw_expand_core.cuh"
#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

using core::ExpandParams;
using core::kFull;
constexpr int kWarps = 4;
constexpr int kItemsPerThread = 4;
#ifndef TW_PART_STREAMING
#define TW_PART_STREAMING 1  // candidate traffic marked evict-first, so the table slice keeps L2
#endif

template <class T>
__device__ __forceinline__ void store_stream(T* p, T v) {
#if TW_PART_STREAMING
  __stcs(p, v);
#else
  *p = v;
#endif
}
template <class T>
__device__ __forceinline__ T load_stream(const T* p) {
#if TW_PART_STREAMING
  return __ldcs(p);
#else
  return *p;
#endif
}
__device__ __forceinline__ void store_stream(K128* p, K128 v) {
#if TW_PART_STREAMING
  __stcs(reinterpret_cast<ulonglong2*>(p), make_ulonglong2(v.lo, v.hi));
#else
  *p = v;
#endif
}
__device__ __forceinline__ K128 load_stream(const K128* p) {
#if TW_PART_STREAMING
  const ulonglong2 t = __ldcs(reinterpret_cast<const ulonglong2*>(p));
  return K128{t.x, t.y};
#else
  return *p;
#endif
}
__device__ __forceinline__ void store_stream(uint8_t* p, uint8_t v) {
#if TW_PART_STREAMING
  __stcs(reinterpret_cast<signed char*>(p), (signed char)v);
#else
  *p = v;
#endif
}
__device__ __forceinline__ uint8_t load_stream(const uint8_t* p) {
#if TW_PART_STREAMING
  return (uint8_t)__ldcs(reinterpret_cast<const signed char*>(p));
#else
  return *p;
#endif
}

// Range of a hash: its high word scaled to [0, P); monotone in the hash like
// the home slot, so range p covers a contiguous slice of the table.
__device__ __forceinline__ int range_of(unsigned long long h, int P) { return (int)__umul64hi(h, (unsigned long long)P); }

template <class K>
__global__ void __launch_bounds__(kWarps * 32, 6)
    emit_kernel(const ExpandParams<K> p, int P, K* __restrict__ cand_key, uint8_t* __restrict__ cand_v,
                unsigned long long region_cap, unsigned long long* __restrict__ region_cnt,
                unsigned int* __restrict__ overflow) {
  constexpr int kBits = KeyTraits<K>::kBits;
  __shared__ K sAdj[kBits];
  __shared__ K sState[kWarps * 32];
  __shared__ uint16_t sQueue[kWarps * 32 * kBits];
  __shared__ int sTotal[kWarps];
  __shared__ int sHist[kMaxRanges];
  __shared__ int sCursor[kMaxRanges];
  __shared__ unsigned long long sBase[kMaxRanges];
  for (int i = threadIdx.x; i < p.n; i += blockDim.x) sAdj[i] = p.adj[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const K valid = kfirst_n<K>(p.n);
  unsigned long long generated_total = 0;
  const unsigned long long n_blocks = (p.n_in + kWarps * 32 - 1) / (kWarps * 32);
  for (unsigned long long b = blockIdx.x; b < n_blocks; b += gridDim.x) {
    const unsigned long long idx = b * (kWarps * 32) + warp * 32 + lane;
    const bool active = idx < p.n_in;
    const K S = active ? p.in_keys[idx] : valid;
    K feas = active ? core::feasible_extensions<K>(S, sAdj, valid, p.allowed, p.k) : kzero<K>();
    if (p.mmw) feas = core::mmw_filter<K>(S, feas, sAdj, p.n, p.k, lane);
    const int total = core::build_queue<K>(S, feas, lane, sState + warp * 32, sQueue + warp * 32 * kBits);
    if (lane == 0) sTotal[warp] = total;
    for (int r = threadIdx.x; r < P; r += blockDim.x) sHist[r] = 0;
    __syncthreads();
    int start[kWarps + 1];
    start[0] = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) start[w + 1] = start[w] + sTotal[w];
    const int T = start[kWarps];
    generated_total += (unsigned long long)(threadIdx.x == 0 ? T : 0);
    // histogram of the block's pairs over the ranges
    for (int e = threadIdx.x; e < T; e += blockDim.x) {
      int w = 0;
      while (e >= start[w + 1]) ++w;
      const uint16_t q = sQueue[w * 32 * kBits + (e - start[w])];
      const K key = sState[w * 32 + (q >> 8)] | kbit<K>(q & 0xff);
      atomicAdd(&sHist[range_of(khash(key), P)], 1);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < P; r += blockDim.x) {
      sCursor[r] = 0;
      sBase[r] = sHist[r] ? atomicAdd(&region_cnt[r], (unsigned long long)sHist[r]) : 0ull;
    }
    __syncthreads();
    // scatter: the block's pairs of one range land next to each other
    for (int e = threadIdx.x; e < T; e += blockDim.x) {
      int w = 0;
      while (e >= start[w + 1]) ++w;
      const uint16_t q = sQueue[w * 32 * kBits + (e - start[w])];
      const K key = sState[w * 32 + (q >> 8)] | kbit<K>(q & 0xff);
      const int r = range_of(khash(key), P);
      const unsigned long long pos = sBase[r] + (unsigned long long)atomicAdd(&sCursor[r], 1);
      if (pos < region_cap) {
        store_stream(&cand_key[(unsigned long long)r * region_cap + pos], key);
        store_stream(&cand_v[(unsigned long long)r * region_cap + pos], (uint8_t)(q & 0xff));
      } else {
        atomicOr(overflow, 1u);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && generated_total) atomicAdd(&p.ctr->generated, generated_total);
}

// Inserts item j of the concatenation of the regions (range-major) for each
// thread's kItemsPerThread consecutive items; first probes are issued before
// any result is inspected.
template <class K>
__global__ void __launch_bounds__(256)
    insert_ranges_kernel(const K* __restrict__ cand_key, const uint8_t* __restrict__ cand_v,
                         unsigned long long region_cap, const unsigned long long* __restrict__ prefix, int P,
                         unsigned long long first_item, unsigned long long end_item, K* __restrict__ table,
                         unsigned long long slots, int max_probes, K* __restrict__ out_keys,
                         uint8_t* __restrict__ out_pred, unsigned long long out_cap, LevelCounters* ctr) {
  __shared__ unsigned long long sPrefix[kMaxRanges + 1];
  for (int i = threadIdx.x; i <= P; i += blockDim.x) sPrefix[i] = prefix[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  const unsigned long long total = end_item;
  const K empty = kones<K>();
  const unsigned long long warp_first =
      first_item + ((unsigned long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32ull * kItemsPerThread;
  // (warps past the end stay for the block's output reservation below)
  K key[kItemsPerThread];
  int vv[kItemsPerThread];
  unsigned long long h[kItemsPerThread];
  int st[kItemsPerThread];
  // range of the thread's first item: binary search in the shared prefix sums
  // (the last r with sPrefix[r] <= item); later items only move forward
  int r = 0;
  {
    const unsigned long long j0 = warp_first + lane;
    int lo = 0, hi = P - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sPrefix[mid] <= j0)
        lo = mid;
      else
        hi = mid - 1;
    }
    r = lo;
  }
#pragma unroll
  for (int u = 0; u < kItemsPerThread; ++u) {
    const unsigned long long j = warp_first + (unsigned long long)u * 32ull + lane;
    st[u] = 0;
    vv[u] = 0;
    h[u] = 0;
    key[u] = kzero<K>();
    if (j < total) {
      while (sPrefix[r + 1] <= j) ++r;
      const unsigned long long at = (unsigned long long)r * region_cap + (j - prefix[r]);
      key[u] = load_stream(&cand_key[at]);
      vv[u] = load_stream(&cand_v[at]);
      h[u] = core::home_slot(khash(key[u]), slots);
      st[u] = 1;
    }
  }
  K old[kItemsPerThread];
#pragma unroll
  for (int u = 0; u < kItemsPerThread; ++u)
    if (st[u] == 1) old[u] = kcas(&table[h[u]], empty, key[u]);
#pragma unroll
  for (int u = 0; u < kItemsPerThread; ++u) {
    if (st[u] != 1) continue;
    if (old[u] == empty) {
      st[u] = 2;
    } else if (old[u] == key[u]) {
      st[u] = 3;
    } else {
      for (int probe = 1;; ++probe) {
        if (probe >= max_probes) {
          atomicOr(&ctr->overflow, 2u);
          st[u] = 3;
          break;
        }
        h[u] = (h[u] + 1ull == slots) ? 0ull : h[u] + 1ull;
        const K o = kcas(&table[h[u]], empty, key[u]);
        if (o == empty) {
          st[u] = 2;
          break;
        }
        if (o == key[u]) {
          st[u] = 3;
          break;
        }
      }
    }
  }
  unsigned wm[kItemsPerThread];
  int wins = 0;
#pragma unroll
  for (int u = 0; u < kItemsPerThread; ++u) {
    wm[u] = __ballot_sync(kFull, st[u] == 2);
    wins += __popc(wm[u]);
  }
  // one output reservation per block (a single counter takes every block's
  // add, so fewer adds mean less serialisation at its L2 slice)
  __shared__ int sWins[8];
  __shared__ unsigned long long sBase;
  const int warp = threadIdx.x >> 5;
  if (lane == 0) sWins[warp] = wins;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) tot += sWins[w2];
    sBase = tot ? atomicAdd(&ctr->out_count, (unsigned long long)tot) : 0ull;
  }
  __syncthreads();
  if (wins) {
    unsigned long long b = sBase;
    for (int w2 = 0; w2 < warp; ++w2) b += (unsigned long long)sWins[w2];
#pragma unroll
    for (int u = 0; u < kItemsPerThread; ++u) {
      if (st[u] == 2) {
        const unsigned long long o = b + (unsigned long long)__popc(wm[u] & lanemask_lt);
        if (o < out_cap) {
          out_keys[o] = key[u];
          out_pred[o] = (uint8_t)vv[u];
        } else {
          atomicOr(&ctr->overflow, 1u);
        }
      }
      b += (unsigned long long)__popc(wm[u]);
    }
  }
}

// Sets slots [first, first + count) of a table of `total` slots (wrapping at
// the end) to the empty key.
template <class K>
__global__ void clear_slots_kernel(K* __restrict__ table, unsigned long long first, unsigned long long count,
                                   unsigned long long total) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    unsigned long long j = first + i;
    if (j >= total) j -= total;
    table[j] = kones<K>();
  }
}

// Drops the 128-byte lines of [lo, hi) from L2 without writing them back
// (PTX discard.global.L2): a table slice whose range is complete is never
// read again, and the next use of the table empties it first.
__global__ void discard_lines_kernel(char* base, unsigned long long first_line, unsigned long long lines) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < lines; i += stride) {
    char* line = base + (first_line + i) * 128ull;
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <class K>
cudaError_t emit_t(const ExpandLaunch& a, const PartitionBufs& pb, cudaStream_t s) {
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
  p.ranges = 1;
  p.range = 0;
  const unsigned long long blocks_needed = (a.n_in + kWarps * 32 - 1) / (kWarps * 32);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emit_kernel<K>, kWarps * 32, 0);
  unsigned long long grid = (unsigned long long)sm_count() * (per_sm > 0 ? per_sm : 1);
  if (grid > blocks_needed) grid = blocks_needed;
  if (grid < 1) grid = 1;
  emit_kernel<K><<<(int)grid, kWarps * 32, 0, s>>>(p, pb.ranges, static_cast<K*>(pb.cand_key), pb.cand_v,
                                                   pb.region_cap, pb.region_cnt, pb.overflow);
  return cudaGetLastError();
}

template <class K>
cudaError_t insert_t(const ExpandLaunch& a, const PartitionBufs& pb, unsigned long long first,
                     unsigned long long end, cudaStream_t s) {
  if (end <= first) return cudaSuccess;
  const unsigned long long per_block = 256ull * kItemsPerThread;
  const unsigned long long blocks = (end - first + per_block - 1) / per_block;
  insert_ranges_kernel<K><<<(unsigned)blocks, 256, 0, s>>>(
      static_cast<const K*>(pb.cand_key), pb.cand_v, pb.region_cap, pb.prefix, pb.ranges, first, end,
      static_cast<K*>(a.table), a.table_slots, a.max_probes, static_cast<K*>(a.out_keys), a.out_pred, a.out_cap,
      a.ctr);
  return cudaGetLastError();
}

template <class K>
cudaError_t clear_slots_t(void* table, unsigned long long first, unsigned long long count, unsigned long long total,
                          cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  unsigned long long g = (count + 1023) / 1024;
  const unsigned long long cap = (unsigned long long)sm_count() * 8ull;
  if (g > cap) g = cap;
  clear_slots_kernel<K><<<(int)g, 256, 0, s>>>(static_cast<K*>(table), first, count, total);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_emit(const ExpandLaunch& a, const PartitionBufs& pb, cudaStream_t s) {
  if (a.n_in == 0) return cudaSuccess;
  switch (a.kc) {
    case kKey32: return emit_t<uint32_t>(a, pb, s);
    case kKey64: return emit_t<unsigned long long>(a, pb, s);
    default: return emit_t<K128>(a, pb, s);
  }
}

cudaError_t launch_insert_ranges(const ExpandLaunch& a, const PartitionBufs& pb, unsigned long long first,
                                 unsigned long long end, cudaStream_t s) {
  switch (a.kc) {
    case kKey32: return insert_t<uint32_t>(a, pb, first, end, s);
    case kKey64: return insert_t<unsigned long long>(a, pb, first, end, s);
    default: return insert_t<K128>(a, pb, first, end, s);
  }
}

cudaError_t launch_clear_slots(KeyClass kc, void* table, unsigned long long first, unsigned long long count,
                               unsigned long long total, cudaStream_t s) {
  switch (kc) {
    case kKey32: return clear_slots_t<uint32_t>(table, first, count, total, s);
    case kKey64: return clear_slots_t<unsigned long long>(table, first, count, total, s);
    default: return clear_slots_t<K128>(table, first, count, total, s);
  }
}

cudaError_t launch_discard_l2(void* base, unsigned long long lo_bytes, unsigned long long hi_bytes, cudaStream_t s) {
  const unsigned long long first = (lo_bytes + 127) / 128, last = hi_bytes / 128;  // whole lines inside
  if (last <= first) return cudaSuccess;
  unsigned long long g = (last - first + 255) / 256;
  const unsigned long long cap = (unsigned long long)sm_count() * 8ull;
  if (g > cap) g = cap;
  discard_lines_kernel<<<(int)g, 256, 0, s>>>(static_cast<char*>(base), first, last - first);
  return cudaGetLastError();
}

}  // namespace tw
