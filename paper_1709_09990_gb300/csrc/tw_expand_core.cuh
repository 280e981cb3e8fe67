// Device building blocks of one wavefront level, shared by the single-graph
// and the batched expansion kernels.
//
// Level i -> i+1 of Listing 1 (arXiv 1709.09990, Section 3.1): every set S of
// L_i is extended by every vertex v outside S with |Q(S, v)| <= k, and the
// extensions are deduplicated (Section 3.2) in an exact hash table.
#pragma once

#include <cstdint>

#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace core {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxComps = 8;
#ifndef TW_INSERT_UNROLL
#define TW_INSERT_UNROLL 4  // compare-and-swaps in flight per lane (L2-resident tables)
#endif
// Tables larger than this many bytes (about twice the L2) miss in L2 on most
// probes; their levels run with twice as many compare-and-swaps in flight.
constexpr unsigned long long kDeepTableBytes = 256ull << 20;

// Resident warps per SM the register allocation must allow: 32 for the 32-
// and 64-bit kernels (at most 64 registers per thread, measured fastest on
// GB300), 16 for the 128-bit kernel.
template <class K>
struct ResidentWarps {
  static constexpr int value = KeyTraits<K>::kBits <= 64 ? 32 : 16;
};

// Home slot of a hash: the high word of hash * slots (uniform over [0, slots)
// for any table size, so the table can be sized to the level).
__device__ __forceinline__ unsigned long long home_slot(unsigned long long h, unsigned long long slots) {
  return __umul64hi(h, slots);
}

// Floods the component of G[S] that contains the vertices of todo (taken out
// of rem, the vertices of S not yet in a component) over the adjacency rows in
// shared memory; returns its outer boundary N(C) \ S and adds the component's
// vertices to *comp.
template <class K>
__device__ __forceinline__ K flood_component(K todo, K& rem, const K S, const K* __restrict__ sAdj, K* comp) {
  K bnd = kzero<K>();
  while (!kempty(todo)) {
    const K b = klsb(todo);
    todo ^= b;
    const K r = sAdj[kindex(b)];
    bnd |= r;
    const K nw = r & rem;  // unvisited vertices of S next to the component
    rem ^= nw;
    todo |= nw;
    if (comp) *comp |= nw;
  }
  return bnd & ~S;
}

// Adds the boundary of one more component of G[S] to the registers of
// feasible_extensions: a boundary with |B_C| >= k+2 rules out all of B_C;
// up to kMaxComps others are kept; beyond that the caller falls back to a
// flood fill per candidate.
template <class K>
__device__ __forceinline__ void keep_boundary(const K bnd, const int k, K (&comp_b)[kMaxComps], int& nc, bool& many,
                                              K& dead, K& bordered) {
  const int bs = kpopc(bnd);
  if (bs >= k + 2) {
    dead |= bnd;
  } else if (bs > 0) {
    if (nc < kMaxComps) {
#pragma unroll
      for (int c = 0; c < kMaxComps; ++c)
        if (c == nc) comp_b[c] = bnd;
      ++nc;
      bordered |= bnd;
    } else {
      many = true;
    }
  }
}

// |Q(S, v)| <= k for one candidate v (bit vb, row nv = N(v)), given the
// boundaries of the components of G[S] that v may border.
template <class K>
__device__ __forceinline__ bool q_within(const K S, const K vb, const K nv, K q, const K* __restrict__ sAdj,
                                         const int k, const K (&comp_b)[kMaxComps], const int nc, const bool many,
                                         const K bordered) {
  if (!many) {
    if (!kempty(bordered & vb)) {
#pragma unroll
      for (int c = 0; c < kMaxComps; ++c) {
        if (c >= nc) break;
        if (!kempty(comp_b[c] & vb)) q |= comp_b[c];
      }
    }
  } else {
    K vis = nv & S;
    K front = vis;
    while (!kempty(front)) {
      const K b = klsb(front);
      front ^= b;
      const K r = sAdj[kindex(b)];
      q |= r & ~S;
      const K nw = r & S & ~vis;
      vis |= nw;
      front |= nw;
    }
  }
  q &= ~vb;
  return kpopc(q) <= k;
}

// The set of vertices v outside S with |Q(S, v)| <= k (thread per state).
//
// The components of G[S] are found by a bitset flood fill over the adjacency
// rows in shared memory; each component C gives its outer boundary
// B_C = N(C) \ S.  A vertex outside S is reachable from v through S exactly
// when it borders a component that v borders, so
// Q(S, v) = (N(v) u U{B_C : v in B_C}) \ (S u {v}) - the bitset form of the
// search of Listing 1.  A boundary with |B_C| >= k+2 rules out all of B_C at
// once; up to kMaxComps other boundaries stay in registers, and a state with
// more falls back to a flood fill per candidate.
//
// With kCanonical only the canonical extensions are returned: the v that lie
// in the component of G[S u {v}] holding the lowest vertex of S u {v}, i.e.
// v below min(S) or v in the boundary of the component of min(S).  The level
// sets stay exactly those of Listing 1: Q(S, v) depends only on v's component
// of G[S u {v}] (a path from v whose interior lies in S never leaves it), so
// a set is feasible iff each of its components is, and a feasible set T is
// reached from T \ {u} with u the last vertex of a feasible ordering of T's
// lowest-vertex component.  Each new set is then produced by far fewer
// parents, which cuts the candidate tests and the table probes (on the
// geometric n=40 benchmark graph 3.3x fewer pairs).  The canonical search is
// also lazy: it floods the component of min(S) first, which fixes the
// candidates, and then only the components that border a candidate passing
// the |N(v) \ S| <= k test.
template <class K, bool kCanonical = true>
__device__ __forceinline__ K feasible_extensions(const K S, const K* __restrict__ sAdj, const K valid,
                                                 const K allowed, const int k) {
  K comp_b[kMaxComps];
#pragma unroll
  for (int c = 0; c < kMaxComps; ++c) comp_b[c] = kzero<K>();
  int nc = 0;
  bool many = false;
  K dead = kzero<K>();
  K bordered = kzero<K>();  // union of the kept boundaries
  K rem = S;                // vertices of S not yet in a component
  K cand;
  if (kCanonical) {
    K b0 = kzero<K>();  // boundary of the component of min(S)
    if (!kempty(S)) {
      const K first = klsb(S);
      rem ^= first;
      b0 = flood_component<K>(first, rem, S, sAdj, nullptr);
    }
    cand = valid & allowed & ~S & (kbelow_lowest(S) | b0);
    if (kpopc(b0) >= k + 2) {
      cand &= ~b0;
    } else if (!kempty(b0)) {
      comp_b[0] = b0;
      nc = 1;
      bordered = b0;
    }
    // keep the candidates that pass the cheap test; flood only the
    // components of S next to them
    K pre = kzero<K>(), need = kzero<K>();
    for (K c = cand; !kempty(c);) {
      const K vb = klsb(c);
      c ^= vb;
      const K nv = sAdj[kindex(vb)];
      if (kpopc(nv & ~S) > k) continue;
      pre |= vb;
      need |= nv;
    }
    need &= rem;
    while (!kempty(need)) {
      const K start = klsb(need);
      rem ^= start;
      K comp = start;
      const K bnd = flood_component<K>(start, rem, S, sAdj, &comp);
      need &= ~comp;
      keep_boundary<K>(bnd, k, comp_b, nc, many, dead, bordered);
    }
    cand = pre & ~dead;
  } else {
    while (!kempty(rem)) {
      const K start = klsb(rem);
      rem ^= start;
      const K bnd = flood_component<K>(start, rem, S, sAdj, nullptr);
      keep_boundary<K>(bnd, k, comp_b, nc, many, dead, bordered);
    }
    cand = valid & allowed & ~S & ~dead;
  }
  K feas = kzero<K>();
  while (!kempty(cand)) {
    const K vb = klsb(cand);
    cand ^= vb;
    const K nv = sAdj[kindex(vb)];
    const K q = nv & ~S;
    if (kpopc(q) > k) continue;
    if (q_within<K>(S, vb, nv, q, sAdj, k, comp_b, nc, many, bordered)) feas |= vb;
  }
  return feas;
}

// Warp-wide minimum of (d, v), lowest v on ties; v < 0 means none.
__device__ __forceinline__ void warp_min_pair(int& d, int& v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int od = __shfl_xor_sync(kFull, d, off);
    const int ov = __shfl_xor_sync(kFull, v, off);
    if (ov >= 0 && (v < 0 || od < d || (od == d && ov < v))) {
      d = od;
      v = ov;
    }
  }
}

// Does the minor-min-width bound of the graph H left after eliminating S
// exceed k (Section 3.3, with the second-smallest degree of each minor as the
// bound, which is also a treewidth lower bound)?  Warp-cooperative: every
// lane passes the same S; lane l owns the vertices l, l+32, ... and their rows
// of H (row of v = Q(S, v), found by a flood fill through S).  While H has
// more than k+1 vertices: take a minimum-degree vertex v (lowest index),
// record the second-smallest degree, delete v if isolated, else contract it
// into its minimum-degree neighbour (lowest index).  With at most k+1
// vertices left no degree can exceed k, so the answer is settled.
template <class K>
__device__ __forceinline__ bool mmw_exceeds(const K S, const K* __restrict__ sAdj, const int n, const int k,
                                            const int lane) {
  constexpr int NV = KeyTraits<K>::kBits / 32;  // vertices per lane
  constexpr int kNone = 1 << 30;
  K alive = kfirst_n<K>(n) & ~S;
  K row[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const int v = lane + 32 * t;
    row[t] = kzero<K>();
    if (v < n && ktest(alive, v)) {
      const K nv = sAdj[v];
      K q = nv & ~S;
      K vis = nv & S;
      K front = vis;
      while (!kempty(front)) {
        const K b = klsb(front);
        front ^= b;
        const K r = sAdj[kindex(b)];
        q |= r & ~S;
        const K nw = r & S & ~vis;
        vis |= nw;
        front |= nw;
      }
      row[t] = q & ~kbit<K>(v);
    }
  }
  int count = kpopc(alive);
  int lb = 0;
  while (count > k + 1) {
    int deg[NV];
    int dmin = kNone, vmin = -1;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int v = lane + 32 * t;
      deg[t] = (v < n && ktest(alive, v)) ? kpopc(row[t] & alive) : kNone;
      if (deg[t] < dmin) {
        dmin = deg[t];
        vmin = v;
      }
    }
    warp_min_pair(dmin, vmin);
    int d2 = kNone, v2 = -1;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int v = lane + 32 * t;
      if (v != vmin && deg[t] < d2) {
        d2 = deg[t];
        v2 = v;
      }
    }
    warp_min_pair(d2, v2);
    lb = max(lb, d2);
    if (lb > k) return true;
    const K bv = kbit<K>(vmin);
    alive &= ~bv;
    --count;
    if (dmin == 0) continue;
    K mine = kzero<K>();
#pragma unroll
    for (int t = 0; t < NV; ++t)
      if (t == (vmin >> 5)) mine = row[t];
    const K rv = kshfl(mine, vmin & 31) & alive;
    int du = kNone, u = -1;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int v = lane + 32 * t;
      if (v < n && ktest(rv, v) && deg[t] < du) {
        du = deg[t];
        u = v;
      }
    }
    warp_min_pair(du, u);
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int v = lane + 32 * t;
      if (v == u)
        row[t] |= rv & ~kbit<K>(u);
      else if (v < n && ktest(rv, v))
        row[t] |= kbit<K>(u);
    }
  }
  return false;
}

// Drops the extensions of every state of the warp whose remaining graph has
// a minor-min-width bound above k (the warp examines its states one by one).
template <class K>
__device__ __forceinline__ K mmw_filter(const K S, K feas, const K* __restrict__ sAdj, const int n, const int k,
                                        const int lane) {
  unsigned pending = __ballot_sync(kFull, !kempty(feas));
  while (pending) {
    const int j = __ffs(pending) - 1;
    pending &= pending - 1;
    const bool prune = mmw_exceeds<K>(kshfl(S, j), sAdj, n, k, lane);
    if (prune && lane == j) feas = kzero<K>();
  }
  return feas;
}

// Keeps the feasible extensions v of S whose new set S u {v} hashes into
// range `range` of `ranges` equal ranges of the hash space (the same split as
// the home slot: the high word of hash * ranges).
template <class K>
__device__ __forceinline__ K in_hash_range(const K S, K feas, const unsigned long long ranges,
                                           const unsigned long long range) {
  K keep = kzero<K>();
  while (!kempty(feas)) {
    const K vb = klsb(feas);
    feas ^= vb;
    if (__umul64hi(khash(S | vb), ranges) == range) keep |= vb;
  }
  return keep;
}

// Packs the feasible (S, v) pairs of the warp's 32 states into the warp's
// queue (entry = lane << 8 | v) and stores each lane's S; returns the number
// of pairs (warp uniform).
template <class K>
__device__ __forceinline__ int build_queue(const K S, K feas, const int lane, K* __restrict__ sS,
                                           uint16_t* __restrict__ sQ) {
  const int cnt = kpopc(feas);
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += t;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  int pos = incl - cnt;
  sS[lane] = S;
  while (!kempty(feas)) {
    const int v = klowest(feas);
    feas = kdrop_lowest(feas);
    sQ[pos++] = (uint16_t)((lane << 8) | v);
  }
  __syncwarp();
  return total;
}

// Where the winners of the inserts go.  With kParent the output records the
// index (parent_base + lane) of the parent state in its level; otherwise the
// added vertex.
template <class K, bool kParent>
struct LevelOut {
  K* keys;
  uint8_t* pred;       // used when !kParent
  uint32_t* parent;    // used when kParent
  uint32_t parent_base;
  unsigned long long cap;
  unsigned long long* count;
  unsigned int* overflow;  // bit 0: output full, bit 1: probe limit
};

// Inserts the queued pairs into the table, U per lane at a
// time: the first probe of every pair is issued before any result is
// inspected, so each lane has several compare-and-swaps in flight.  Linear
// probing from the home slot, at most max_probes slots.  Winners append
// (S u {v}, pred or parent) with one atomic add per round of the warp.
//
// With kRanged the table is the slice of one hash range (in_hash_range): the
// home slot spreads the range's hashes over the slice (the high word of
// (hash * ranges mod 2^64) * slots), no predecessor is stored, and output
// positions from split on go to tail[position - split] when tail is given (a
// list continued in a second buffer).
template <class K, bool kParent, int U = TW_INSERT_UNROLL, bool kRanged = false>
__device__ __forceinline__ void insert_queue(const uint16_t* __restrict__ sQ, const K* __restrict__ sS,
                                             const int total, const int lane, K* __restrict__ table,
                                             const unsigned long long slots, const int max_probes,
                                             const LevelOut<K, kParent>& out, const unsigned long long ranges = 1,
                                             K* tail = nullptr, const unsigned long long split = 0) {
  const K empty = kones<K>();
  const unsigned lanemask_lt = (1u << lane) - 1u;
  for (int base = 0; base < total; base += 32 * U) {
    K key[U];
    int vv[U];
    int src[U];
    unsigned long long h[U];
    int st[U];  // 0 idle, 1 probing, 2 inserted, 3 already present or given up
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = base + u * 32 + lane;
      st[u] = 0;
      vv[u] = 0;
      src[u] = 0;
      h[u] = 0;
      key[u] = kzero<K>();
      if (j < total) {
        const uint16_t e = sQ[j];
        vv[u] = e & 0xff;
        src[u] = e >> 8;
        key[u] = sS[src[u]] | kbit<K>(vv[u]);
        h[u] = kRanged ? home_slot(khash(key[u]) * ranges, slots) : home_slot(khash(key[u]), slots);
        st[u] = 1;
      }
    }
    K old[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (st[u] == 1) old[u] = kcas(&table[h[u]], empty, key[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (st[u] != 1) continue;
      if (old[u] == empty) {
        st[u] = 2;
      } else if (old[u] == key[u]) {
        st[u] = 3;
      } else {
        for (int probe = 1;; ++probe) {
          if (probe >= max_probes) {
            atomicOr(out.overflow, 2u);
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
    unsigned wm[U];
    int wins = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wm[u] = __ballot_sync(kFull, st[u] == 2);
      wins += __popc(wm[u]);
    }
    if (wins) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(out.count, (unsigned long long)wins);
      b = __shfl_sync(kFull, b, 0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (st[u] == 2) {
          const unsigned long long o = b + (unsigned long long)__popc(wm[u] & lanemask_lt);
          if (o < out.cap) {
            if (kRanged && tail != nullptr && o >= split)
              kstore_cs(&tail[o - split], key[u]);
            else
              kstore_cs(&out.keys[o], key[u]);
            if (kParent)
              __stcs(&out.parent[o], out.parent_base + (uint32_t)src[u]);
            else if (!kRanged)
              __stcs(reinterpret_cast<signed char*>(&out.pred[o]), (signed char)vv[u]);
          } else {
            atomicOr(out.overflow, 1u);
          }
        }
        b += (unsigned long long)__popc(wm[u]);
      }
    }
  }
}

// A key from two 64-bit words (low word first).
template <class K> __host__ __device__ __forceinline__ K kfrom_words(unsigned long long lo, unsigned long long hi);
template <> __host__ __device__ __forceinline__ uint32_t kfrom_words<uint32_t>(unsigned long long lo,
                                                                                unsigned long long) {
  return (uint32_t)lo;
}
template <> __host__ __device__ __forceinline__ unsigned long long kfrom_words<unsigned long long>(
    unsigned long long lo, unsigned long long) {
  return lo;
}
template <> __host__ __device__ __forceinline__ K128 kfrom_words<K128>(unsigned long long lo, unsigned long long hi) {
  return K128{lo, hi};
}

// Parameters of one level expansion.
template <class K>
struct ExpandParams {
  const K* in_keys;
  unsigned long long n_in;
  const K* adj;
  int n;
  int k;
  K* table;
  unsigned long long table_slots;
  int max_probes;
  K* out_keys;
  uint8_t* out_pred;
  unsigned long long out_cap;
  LevelCounters* ctr;
  K allowed;  // vertices that may be added (all by default)
  int mmw;    // 1: minor-min-width pruning of the states before they are extended
  unsigned long long ranges;  // ranged kernels: the hash space is split in this many ranges,
  unsigned long long range;   // and only pairs of this one are inserted (the table is its slice)
};

// C(n, r), or cap when it is at least cap.  The products run over
// min(r, n - r) steps, along which b = C(n - r + j, j) only grows and each
// division is exact, so with cap <= 2^40 nothing overflows.
__device__ __forceinline__ unsigned long long binom_capped(int n, int r, unsigned long long cap) {
  if (r < 0 || r > n) return 0ull;
  if (r > n - r) r = n - r;
  unsigned long long b = 1ull;
  for (int j = 1; j <= r; ++j) {
    b = b * (unsigned long long)(n - r + j) / (unsigned long long)j;
    if (b >= cap) return cap;
  }
  return b;
}

// The table of level i -> i+1 without FP64 (slow on this part; the result is
// the same in every thread): the expected size is cnt times the last growth
// ratio cnt / prev_cnt clamped to [1/4, n - i] (n at i = 0), plus 25% and
// 1024, at most the number of sets level i+1 can have; slots = that at
// load_pct percent, at least 64.  The ratio is exact integer arithmetic below
// 2^32 sets and single precision above.
__device__ __forceinline__ void plan_level(unsigned long long cnt, unsigned long long prev_cnt, int n, int i,
                                           int load_pct, unsigned long long* table_est, unsigned long long* slots) {
  const unsigned long long most = cnt * (unsigned long long)(n - i);
  const unsigned long long bound = min(most, binom_capped(n, i + 1, 1ull << 40)) + 1ull;
  unsigned long long est = (unsigned long long)n;
  if (i > 0) {
    if (prev_cnt == 0)
      est = cnt;
    else if (cnt < (1ull << 32))
      est = cnt * cnt / prev_cnt;
    else
      est = (unsigned long long)fminf((float)cnt * ((float)cnt / (float)prev_cnt), (float)most);
    est = max(est, cnt / 4ull);
    est = min(est, most);
  }
  *table_est = min(est + est / 4ull + 1024ull, bound);
  *slots = max(64ull, (*table_est * 100ull + (unsigned long long)load_pct - 1ull) / (unsigned long long)load_pct);
}

// One level i -> i+1 by the whole block: the adjacency rows go to shared
// memory, then each warp takes chunks of 32 consecutive states (coalesced key
// loads), finds their feasible extensions (thread per state), queues the
// pairs and inserts them cooperatively.  sState holds kWarps x 32 keys,
// sQueue kWarps x 32 x kBits entries.
//
// With kBlockLocal the block expands the whole level alone (its warps take the
// chunks in turn): a persistent kernel whose blocks work on different graphs.
// With kKeysL2 the input keys are read through L2 only: persistent kernels,
// whose arena other SMs rewrite while stale lines may sit in this SM's L1.
// With kGroup the level is expanded by a group of the grid's blocks (block
// group_block of group_blocks) instead of the whole grid.  Ranged kernels may
// continue the output list in out_tail from position out_split on.
template <class K, int kWarps, int U = TW_INSERT_UNROLL, bool kMMW = false, bool kRanged = false,
          bool kBlockLocal = false, bool kKeysL2 = false, bool kGroup = false>
__device__ __forceinline__ void expand_level(const ExpandParams<K>& p, K* sAdj, K* sState, uint16_t* sQueue,
                                             const unsigned group_block = 0, const unsigned group_blocks = 0,
                                             K* out_tail = nullptr, const unsigned long long out_split = 0) {
  constexpr int kBits = KeyTraits<K>::kBits;
  for (int i = threadIdx.x; i < p.n; i += blockDim.x) sAdj[i] = p.adj[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  K* sS = sState + warp * 32;
  uint16_t* sQ = sQueue + warp * 32 * kBits;
  const K valid = kfirst_n<K>(p.n);
  unsigned long long generated_total = 0;
  const unsigned long long n_chunks = (p.n_in + 31ull) / 32ull;
  const unsigned long long blk = kGroup ? (unsigned long long)group_block : (unsigned long long)blockIdx.x;
  const unsigned long long nblk = kGroup ? (unsigned long long)group_blocks : (unsigned long long)gridDim.x;
  const unsigned long long first = kBlockLocal ? (unsigned long long)warp : blk * kWarps + warp;
  const unsigned long long stride = kBlockLocal ? (unsigned long long)kWarps : nblk * kWarps;
  LevelOut<K, false> out;
  out.keys = p.out_keys;
  out.pred = p.out_pred;
  out.parent = nullptr;
  out.parent_base = 0;
  out.cap = p.out_cap;
  out.count = &p.ctr->out_count;
  out.overflow = &p.ctr->overflow;
  for (unsigned long long chunk = first; chunk < n_chunks; chunk += stride) {
    const unsigned long long idx = chunk * 32ull + lane;
    const bool active = idx < p.n_in;
    const K S = active ? (kKeysL2 ? kload_cg(&p.in_keys[idx]) : kload_cs(&p.in_keys[idx])) : valid;
    // (minor-min-width pruning drops some parents, so it extends by every
    // feasible vertex)
    K feas = active ? feasible_extensions<K, !kMMW>(S, sAdj, valid, p.allowed, p.k) : kzero<K>();
    if (kMMW) feas = mmw_filter<K>(S, feas, sAdj, p.n, p.k, lane);
    if (kRanged) feas = in_hash_range<K>(S, feas, p.ranges, p.range);
    const int total = build_queue<K>(S, feas, lane, sS, sQ);
    generated_total += (unsigned long long)total;
    insert_queue<K, false, U, kRanged>(sQ, sS, total, lane, p.table, p.table_slots, p.max_probes, out, p.ranges,
                                       out_tail, out_split);
    __syncwarp();
  }
  if (lane == 0 && generated_total) atomicAdd(&p.ctr->generated, generated_total);
}

// The backward walk by one block: from the first set of level `last`, find
// the current set in level j (keys [level_off[j], + level_cnt[j])), take its
// predecessor vertex as order[j-1] and drop it, down to level 1; then the
// vertices outside the final set in increasing order.  sWalk, sFound: shared.
template <class K>
__device__ __forceinline__ void walk_block(const K* __restrict__ keys, const uint8_t* __restrict__ pred,
                                          const unsigned long long* level_off, const unsigned long long* level_cnt,
                                          int last, int n, int32_t* order, K* sWalk, int* sFound) {
  if (threadIdx.x == 0) *sWalk = kload_cg(&keys[__ldcg(&level_off[last])]);
  __syncthreads();
  const K fin = *sWalk;
  for (int j = last; j >= 1; --j) {
    if (threadIdx.x == 0) *sFound = 0;
    __syncthreads();
    const K target = *sWalk;
    __syncthreads();  // every thread has the target before the finder replaces it
    const unsigned long long lo = __ldcg(&level_off[j]), cnt = __ldcg(&level_cnt[j]);
    // the scan issues kWalkU loads per thread before comparing (one L2
    // round trip per kWalkU keys, not per key) and stops at the batch that
    // found the set
    constexpr int kWalkU = 8;
    for (unsigned long long x0 = 0; x0 < cnt; x0 += (unsigned long long)blockDim.x * kWalkU) {
      K key[kWalkU];
#pragma unroll
      for (int u = 0; u < kWalkU; ++u) {
        const unsigned long long x = x0 + (unsigned long long)u * blockDim.x + threadIdx.x;
        key[u] = x < cnt ? kload_cg(&keys[lo + x]) : kzero<K>();
      }
      bool hit = false;
#pragma unroll
      for (int u = 0; u < kWalkU; ++u) {
        const unsigned long long x = x0 + (unsigned long long)u * blockDim.x + threadIdx.x;
        if (x < cnt && key[u] == target) {
          hit = true;
          if (atomicExch(sFound, 1) == 0) {
            const int v = __ldcg(&pred[lo + x]);
            order[j - 1] = v;
            *sWalk = target & ~kbit<K>(v);
          }
        }
      }
      if (__syncthreads_or(hit)) break;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int pos = last;
    for (int v = 0; v < n; ++v)
      if (!ktest(fin, v)) order[pos++] = v;
  }
  __syncthreads();
}

// Tree decomposition from an ordering, by one block (thread per vertex):
// bag(v) = {v} u Q(prefix(v), v) and parent(v) = the vertex of Q(prefix(v), v)
// eliminated first after v (the last vertex of the order when Q is empty; the
// last vertex is the root, -1).  adj64 / bags: n rows x words64 uint64;
// sAdj, sPos: shared arrays of 128 entries.
__device__ __forceinline__ void td_block(const unsigned long long* __restrict__ adj64, int n, int words64,
                                         const int32_t* __restrict__ order, int32_t* parent,
                                         unsigned long long* bags, K128* sAdj, int* sPos) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sAdj[i] = K128{adj64[(size_t)i * words64], words64 > 1 ? adj64[(size_t)i * words64 + 1] : 0ull};
    sPos[i] = n;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int o = order[i];
    if (o >= 0 && o < n) sPos[o] = i;  // a malformed order never indexes out of range
  }
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const int pv = sPos[v];
    K128 prefix = kzero<K128>();
    for (int u = 0; u < n; ++u)
      if (sPos[u] < pv) prefix |= kbit<K128>(u);
    K128 q = sAdj[v] & ~prefix;
    K128 vis = sAdj[v] & prefix;
    K128 front = vis;
    while (!kempty(front)) {
      const int u = klowest(front);
      front = kdrop_lowest(front);
      const K128 r = sAdj[u];
      q |= r & ~prefix;
      const K128 nw = r & prefix & ~vis;
      vis |= nw;
      front |= nw;
    }
    q &= ~kbit<K128>(v);
    const K128 bag = q | kbit<K128>(v);
    bags[(size_t)v * words64] = bag.lo;
    if (words64 > 1) bags[(size_t)v * words64 + 1] = bag.hi;
    int best = -1;
    K128 t = q;
    while (!kempty(t)) {
      const int u = klowest(t);
      t = kdrop_lowest(t);
      if (best < 0 || sPos[u] < sPos[best]) best = u;
    }
    if (best < 0) best = (pv >= n - 1) ? -1 : order[n - 1];
    parent[v] = best;
  }
}

}  // namespace core
}  // namespace tw
