// C ABI of libtw and the host drivers around the kernels.
//
// decide(k) follows Listing 1 of arXiv 1709.09990 (Section 3.1): L_0 = {{}},
// one expansion per level i = 0 .. n-k-2, stop early at an empty level, and
// answer yes iff L_{n-k-1} is not empty.  solve() is the iterative deepening
// of the same section, started at a lower bound instead of 0 (the first yes
// is the same k).
//
// Memory.  Every level's keys and predecessor bytes are kept in one growing
// device arena when an ordering is wanted (the backward walk reads them);
// otherwise only the current and the next level are live.  The hash table of
// the level being built is a second buffer.  Nothing exceeds the context's
// memory cap: a level that does not fit ends the call with TW_ERR_CAPACITY.
// A level whose table or output list turns out too small is cleared and run
// again with larger buffers, so no state is ever lost.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/tw.h"
#include "tw_internal.h"

using namespace tw;

namespace {

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct tw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t mem_cap = 0;
  tw_config cfg{};
  DevBuf keys, pred, table, small;  // small: adjacency, walk, order, td scratch
  DevBuf scratch;                    // staged batch inputs/outputs and network data
  DevBuf cand_key, cand_v, part_meta;  // regions of the partitioned insert
  LevelCounters* d_ctr = nullptr;
  LevelCounters* h_ctr = nullptr;
  int sms = 0;
  unsigned long long launches = 0;       // libtw kernels launched so far
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // expand timing (time_kernels)
  // graph-driven level loops, instantiated once per shape and buffer set
  struct GraphEntry {
    int kc, n, k, load, probes, bt;
    unsigned long long allowed0, allowed1;
    void *keys, *pred, *table;
    unsigned long long arena_cap, table_cap;
    cudaGraphExec_t exec;
    int nodes;
  };
  std::vector<GraphEntry> graphs;
  GraphState* d_gstate = nullptr;
  GraphState* h_gstate = nullptr;
  // autotuned (block threads, table load) per (key class, n / 8)
  struct Tuned {
    int kc, nb, block_threads, load_pct;
  };
  std::vector<Tuned> tuned;
  // options of Section 3.1 for the decide run being prepared
  unsigned long long allowed[2] = {~0ull, ~0ull};
  int skipped = 0;  // vertices excluded from the sets (|C| with the clique skip)
};

namespace {

constexpr size_t kSmallBytes = 1 << 20;

#define TW_CK(expr)                              \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) {                     \
      cudaGetLastError();                        \
      return TW_ERR_CUDA;                        \
    }                                            \
  } while (0)

// Launches a libtw kernel and counts it.
#define TW_LAUNCH(c, expr) \
  do {                     \
    TW_CK(expr);           \
    ++(c)->launches;       \
  } while (0)

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double seconds() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copies bytes from a host or device pointer into host memory.
int fetch(void* dst_host, const void* src, size_t bytes) {
  if (bytes == 0) return TW_OK;
  if (is_device_ptr(src)) {
    TW_CK(cudaMemcpy(dst_host, src, bytes, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst_host, src, bytes);
  }
  return TW_OK;
}

// Writes bytes from host memory to a host or device pointer.
int put(tw_ctx* c, void* dst, const void* src_host, size_t bytes) {
  if (bytes == 0 || dst == nullptr) return TW_OK;
  if (is_device_ptr(dst)) {
    TW_CK(cudaMemcpyAsync(dst, src_host, bytes, cudaMemcpyHostToDevice, c->stream));
    TW_CK(cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(dst, src_host, bytes);
  }
  return TW_OK;
}

// Copies bytes from device scratch to a host or device pointer.
int put_from_device(tw_ctx* c, void* dst, const void* src_dev, size_t bytes) {
  if (bytes == 0 || dst == nullptr) return TW_OK;
  TW_CK(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  return TW_OK;
}

size_t total_bytes(const tw_ctx* c) {
  return c->keys.bytes + c->pred.bytes + c->table.bytes + c->cand_key.bytes + c->cand_v.bytes;
}

// Grows b to at least need bytes, keeping its first keep bytes.  Growth is
// geometric while the cap allows it.
int grow(tw_ctx* c, DevBuf* b, size_t need, size_t keep) {
  if (need <= b->bytes) return TW_OK;
  const size_t others = total_bytes(c) - b->bytes;
  if (others + need > c->mem_cap) return TW_ERR_CAPACITY;
  size_t want = std::max(need, b->bytes * 2);
  if (others + want > c->mem_cap) want = need;
  want = (want + 255) & ~size_t(255);
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    if (want == need) return TW_ERR_CAPACITY;
    want = (need + 255) & ~size_t(255);
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return TW_ERR_CAPACITY;
    }
  }
  if (keep > 0 && b->ptr) {
    TW_CK(cudaMemcpyAsync(p, b->ptr, std::min(keep, b->bytes), cudaMemcpyDeviceToDevice, c->stream));
    TW_CK(cudaStreamSynchronize(c->stream));
  }
  if (b->ptr) {
    TW_CK(cudaStreamSynchronize(c->stream));
    cudaFree(b->ptr);
  }
  b->ptr = p;
  b->bytes = want;
  return TW_OK;
}

// A validated graph in the 64-bit-word row layout of the ABI.
struct HostGraph {
  int n = 0;
  int words = 1;
  std::vector<uint64_t> rows;  // n * words
};

int validate(const uint64_t* rows, int n, HostGraph* g) {
  if (n < 1 || n > TW_MAX_N) return TW_ERR_INVALID;
  const int W = (n + 63) / 64;
  g->n = n;
  g->words = W;
  g->rows.assign(rows, rows + (size_t)n * W);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < W * 64; ++c) {
      const bool bit = (g->rows[(size_t)r * W + (c >> 6)] >> (c & 63)) & 1ull;
      if (!bit) continue;
      if (c >= n || c == r) return TW_ERR_INVALID;
      if (!((g->rows[(size_t)c * W + (r >> 6)] >> (r & 63)) & 1ull)) return TW_ERR_INVALID;
    }
  return TW_OK;
}

int load_graph(const uint64_t* adj, int n, HostGraph* g) {
  if (adj == nullptr || n < 1 || n > TW_MAX_N) return TW_ERR_INVALID;
  const int W = (n + 63) / 64;
  std::vector<uint64_t> tmp((size_t)n * W);
  int rc = fetch(tmp.data(), adj, tmp.size() * sizeof(uint64_t));
  if (rc) return rc;
  return validate(tmp.data(), n, g);
}

// Layout of the small device buffer.
struct SmallLayout {
  size_t adj = 0;       // TW_MAX_N keys of 16 bytes
  size_t adj64 = 2048;  // TW_MAX_N * 2 uint64
  size_t walk = 4096;   // (TW_MAX_N + 1) keys of 16 bytes
  size_t order = 8192;  // TW_MAX_N int32
  size_t parent = 8704; // TW_MAX_N int32
  size_t bags = 9216;   // TW_MAX_N * 2 uint64
  size_t bounds = 11264;// 4 int32
};

char* small_at(tw_ctx* c, size_t off) { return static_cast<char*>(c->small.ptr) + off; }

// Uploads the adjacency in the key layout of class kc and in 64-bit rows.
int upload_graph(tw_ctx* c, const HostGraph& g, KeyClass kc) {
  SmallLayout L;
  std::vector<unsigned char> buf(TW_MAX_N * 16, 0);
  const size_t w = key_bytes(kc);
  for (int r = 0; r < g.n; ++r) {
    const uint64_t lo = g.rows[(size_t)r * g.words];
    const uint64_t hi = g.words > 1 ? g.rows[(size_t)r * g.words + 1] : 0;
    if (kc == kKey32) {
      const uint32_t x = (uint32_t)lo;
      std::memcpy(&buf[r * w], &x, 4);
    } else if (kc == kKey64) {
      std::memcpy(&buf[r * w], &lo, 8);
    } else {
      std::memcpy(&buf[r * w], &lo, 8);
      std::memcpy(&buf[r * w + 8], &hi, 8);
    }
  }
  TW_CK(cudaMemcpyAsync(small_at(c, L.adj), buf.data(), (size_t)g.n * w, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(small_at(c, L.adj64), g.rows.data(), g.rows.size() * 8, cudaMemcpyHostToDevice, c->stream));
  return TW_OK;
}

struct LevelRec {
  unsigned long long off = 0;
  unsigned long long count = 0;
};

unsigned long long next_pow2(unsigned long long x) {
  unsigned long long p = 64;
  while (p < x) p <<= 1;
  return p;
}

double binom(int n, int r) {
  if (r < 0 || r > n) return 0.0;
  double b = 1.0;
  for (int i = 1; i <= r; ++i) b = b * (n - r + i) / i;
  return b;
}

struct DecideResult {
  int yes = 0;
  std::vector<LevelRec> levels;
  unsigned long long states_expanded = 0, candidates = 0, feasible = 0, peak_bytes = 0, retries = 0;
  unsigned long long expand_launches = 0;
  double expand_seconds = 0.0, expand_bytes = 0.0;
  std::vector<unsigned long long> fp_sum, fp_xor;
};

// Table size above which a level takes the partitioned insert (opt-in: on
// the heavy levels measured on GB300 the direct kernel, which overlaps its
// DRAM compare-and-swaps with the search, was 30-40% faster).
unsigned long long partition_threshold_bytes(const tw_ctx* c) {
  if (c->cfg.partition_table_mb == -2) return 0ull;
  if (c->cfg.partition_table_mb <= 0) return ~0ull;
  return (unsigned long long)c->cfg.partition_table_mb << 20;
}

// One level through the partitioned insert (emit, then insert range by
// range), on a cleared table.  *fallback is set when a region overflowed
// (the caller then runs the direct kernel on a freshly cleared table).
int run_level_partitioned(tw_ctx* c, const ExpandLaunch& a, int cand_per_state, bool* fallback) {
  *fallback = false;
  const size_t w = key_bytes(a.kc);
  const unsigned long long table_bytes = a.table_slots * w;
#ifndef TW_PART_SLICE_MB
#define TW_PART_SLICE_MB 48  // table bytes per hash range: well inside the 126 MB L2
#endif
  const int P = (int)std::min<unsigned long long>(
      kMaxRanges, std::max<unsigned long long>(2, table_bytes / ((unsigned long long)TW_PART_SLICE_MB << 20) + 1));
  // input chunks whose candidate regions fit a budget of a quarter of the cap
  const double budget = std::min<double>(16e9, (double)c->mem_cap / 4.0);
  const double per_state = (double)std::max(1, cand_per_state) * (double)(w + 1);
  unsigned long long chunk = (unsigned long long)std::max(1024.0, budget / (per_state * 1.2));
  chunk = std::min<unsigned long long>(chunk, a.n_in);
  const unsigned long long region_cap =
      (unsigned long long)std::ceil((double)chunk * std::max(1, cand_per_state) / P * 1.15) + 4096ull;
  int rc = grow(c, &c->cand_key, (size_t)P * region_cap * w, 0);
  if (rc == TW_OK) rc = grow(c, &c->cand_v, (size_t)P * region_cap, 0);
  if (rc == TW_ERR_CAPACITY) {
    *fallback = true;
    return TW_OK;
  }
  if (rc) return rc;
  if (!c->part_meta.ptr) {
    TW_CK(cudaMalloc(&c->part_meta.ptr, 4096));
    c->part_meta.bytes = 4096;
  }
  PartitionBufs pb;
  pb.ranges = P;
  pb.cand_key = c->cand_key.ptr;
  pb.cand_v = static_cast<uint8_t*>(c->cand_v.ptr);
  pb.region_cap = region_cap;
  pb.region_cnt = static_cast<unsigned long long*>(c->part_meta.ptr);
  pb.prefix = pb.region_cnt + kMaxRanges;
  pb.overflow = reinterpret_cast<unsigned int*>(pb.prefix + kMaxRanges + 1);
  std::vector<unsigned long long> cnt(P), prefix(P + 1);
  const size_t kw = key_bytes(a.kc);
  for (unsigned long long lo = 0; lo < a.n_in; lo += chunk) {
    ExpandLaunch ca = a;
    ca.in_keys = static_cast<const char*>(a.in_keys) + lo * kw;
    ca.n_in = std::min<unsigned long long>(chunk, a.n_in - lo);
    TW_CK(cudaMemsetAsync(c->part_meta.ptr, 0, 4096, c->stream));
    TW_LAUNCH(c, launch_emit(ca, pb, c->stream));
    unsigned int ovf = 0;
    TW_CK(cudaMemcpyAsync(cnt.data(), pb.region_cnt, P * 8, cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaMemcpyAsync(&ovf, pb.overflow, 4, cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaStreamSynchronize(c->stream));
    if (ovf) {
      *fallback = true;
      return TW_OK;
    }
    prefix[0] = 0;
    for (int r = 0; r < P; ++r) prefix[r + 1] = prefix[r] + std::min(cnt[r], region_cap);
    TW_CK(cudaMemcpyAsync(pb.prefix, prefix.data(), (P + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    TW_LAUNCH(c, launch_insert_ranges(ca, pb, prefix[P], c->stream));
  }
  return TW_OK;
}

// One run of Listing 1 at bound k on the graph already uploaded.
int run_decide(tw_ctx* c, KeyClass kc, int n, int k, bool keep_levels, DecideResult* R) {
  const size_t w = key_bytes(kc);
  SmallLayout L;
  R->levels.clear();
  R->yes = 0;
  R->states_expanded = R->candidates = R->feasible = R->peak_bytes = R->retries = 0;
  R->expand_launches = 0;
  R->expand_seconds = R->expand_bytes = 0.0;
  R->fp_sum.assign(1, 0ull);  // fp of the empty set is 0
  R->fp_xor.assign(1, 0ull);
  int rc = grow(c, &c->keys, 64 * w, 0);
  if (rc) return rc;
  rc = grow(c, &c->pred, 64, 0);
  if (rc) return rc;
  TW_CK(cudaMemsetAsync(c->keys.ptr, 0, w, c->stream));
  R->levels.push_back({0, 1});
  R->peak_bytes = w + 1;
  if (k >= n - 1) {
    R->yes = 1;
    return TW_OK;
  }
  int load_pct = c->cfg.table_load_pct > 0 ? std::min(90, c->cfg.table_load_pct) : 50;
  int block_threads = c->cfg.block_threads;
  const int max_probes = c->cfg.max_probes > 0 ? c->cfg.max_probes : 256;
  const bool tune = c->cfg.autotune && c->cfg.table_load_pct == 0 && c->cfg.block_threads == 0;
  bool tuned_here = false;
  if (tune)
    for (const auto& t : c->tuned)
      if (t.kc == (int)kc && t.nb == n / 8) {
        load_pct = t.load_pct;
        block_threads = t.block_threads;
        tuned_here = true;
      }
  unsigned long long kept_states = 1;  // states of kept levels (keep mode)
  for (int i = 0; i <= n - k - 2; ++i) {
    const LevelRec cur = R->levels[i];
    // Upper bounds on |L_{i+1}|: every state has n-i extensions, and there
    // are C(n, i+1) sets of that size.
    const double bound = std::min((double)cur.count * (double)(n - i), binom(n, i + 1)) + 1.0;
    // Prediction from the previous level's growth; the table gets 25% slack
    // over the prediction at the target load, the output list room for the
    // worst case (clamped), so output overflow is rare.
    double est;
    if (i == 0) {
      est = n;
    } else {
      const double prev = (double)R->levels[i - 1].count;
      double r = prev > 0 ? (double)cur.count / prev : 1.0;
      r = std::min(std::max(r, 0.25), (double)(n - i));
      est = (double)cur.count * r;
    }
    double table_est = std::min(est * 1.25 + 1024.0, bound);
    const double mem_states = (double)c->mem_cap / (double)(w + 1);
    unsigned long long out_cap =
        (unsigned long long)std::ceil(std::min(bound, std::max(table_est * 3.0, std::min(bound, mem_states / 4))));
    unsigned long long slots = std::max<unsigned long long>(
        64ull, (unsigned long long)std::ceil(table_est * 100.0 / load_pct));
    // Autotune on the first large level: run it once per candidate
    // (identical results), keep the fastest choice for this shape.
    if (tune && !tuned_here && cur.count >= (1ull << 18)) {
      static const int kBt[2] = {128, 256};
      static const int kLoad[3] = {40, 50, 60};
      float best = 1e30f;
      int best_bt = 128, best_load = 50;
      for (int bt : kBt)
        for (int ld : kLoad) {
          const unsigned long long sl =
              std::max<unsigned long long>(64ull, (unsigned long long)std::ceil(table_est * 100.0 / ld));
          const size_t tb = (sl * w + 15) & ~size_t(15);
          const unsigned long long off = keep_levels ? cur.off + cur.count
                                                     : ((out_cap <= cur.off) ? 0ull : cur.off + cur.count);
          rc = grow(c, &c->table, tb, 0);
          if (rc) return rc;
          rc = grow(c, &c->keys, (size_t)(off + out_cap) * w, (size_t)(cur.off + cur.count) * w);
          if (rc) return rc;
          rc = grow(c, &c->pred, (size_t)(off + out_cap), (size_t)(cur.off + cur.count));
          if (rc) return rc;
          TW_LAUNCH(c, launch_clear(c->table.ptr, tb, c->d_ctr, c->stream));
          ExpandLaunch a;
          a.kc = kc;
          a.in_keys = static_cast<char*>(c->keys.ptr) + cur.off * w;
          a.n_in = cur.count;
          a.adj = small_at(c, L.adj);
          a.n = n;
          a.k = k;
          a.table = c->table.ptr;
          a.table_slots = sl;
          a.max_probes = max_probes;
          a.out_keys = static_cast<char*>(c->keys.ptr) + off * w;
          a.out_pred = static_cast<uint8_t*>(c->pred.ptr) + off;
          a.out_cap = out_cap;
          a.ctr = c->d_ctr;
          a.block_threads = bt;
          a.grid = 0;
          a.allowed[0] = c->allowed[0];
          a.allowed[1] = c->allowed[1];
          a.mmw = c->cfg.mmw_prune ? 1 : 0;
          TW_CK(cudaEventRecord(c->ev0, c->stream));
          TW_LAUNCH(c, launch_expand(a, c->stream));
          TW_CK(cudaEventRecord(c->ev1, c->stream));
          TW_CK(cudaStreamSynchronize(c->stream));
          float ms = 0.f;
          TW_CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
          if (ms < best) {
            best = ms;
            best_bt = bt;
            best_load = ld;
          }
        }
      c->tuned.push_back({(int)kc, n / 8, best_bt, best_load});
      load_pct = best_load;
      block_threads = best_bt;
      tuned_here = true;
      slots = std::max<unsigned long long>(64ull, (unsigned long long)std::ceil(table_est * 100.0 / load_pct));
    }
    LevelRec nxt;
    for (int attempt = 0;; ++attempt) {
      if (attempt > 40) return TW_ERR_CAPACITY;
      unsigned long long off;
      if (keep_levels) {
        off = cur.off + cur.count;
      } else {
        off = (out_cap <= cur.off) ? 0ull : cur.off + cur.count;
      }
      const unsigned long long live_end = cur.off + cur.count;  // data to keep on growth
      const size_t table_bytes = (slots * w + 15) & ~size_t(15);
      rc = grow(c, &c->table, table_bytes, 0);
      if (rc) return rc;
      rc = grow(c, &c->keys, (size_t)(off + out_cap) * w, (size_t)live_end * w);
      if (rc) return rc;
      rc = grow(c, &c->pred, (size_t)(off + out_cap), (size_t)live_end);
      if (rc) return rc;
      TW_LAUNCH(c, launch_clear(c->table.ptr, table_bytes, c->d_ctr, c->stream));
      ExpandLaunch a;
      a.kc = kc;
      a.in_keys = static_cast<char*>(c->keys.ptr) + cur.off * w;
      a.n_in = cur.count;
      a.adj = small_at(c, L.adj);
      a.n = n;
      a.k = k;
      a.table = c->table.ptr;
      a.table_slots = slots;
      a.max_probes = max_probes;
      a.out_keys = static_cast<char*>(c->keys.ptr) + off * w;
      a.out_pred = static_cast<uint8_t*>(c->pred.ptr) + off;
      a.out_cap = out_cap;
      a.ctr = c->d_ctr;
      a.block_threads = block_threads;
      a.grid = 0;
      a.allowed[0] = c->allowed[0];
      a.allowed[1] = c->allowed[1];
      a.mmw = c->cfg.mmw_prune ? 1 : 0;
      const bool timed = c->cfg.time_kernels != 0;
      if (timed) TW_CK(cudaEventRecord(c->ev0, c->stream));
      bool direct = true;
      if ((unsigned long long)table_bytes > partition_threshold_bytes(c)) {
        bool fallback = false;
        rc = run_level_partitioned(c, a, n - c->skipped - i, &fallback);
        if (rc) return rc;
        direct = fallback;
        if (fallback) TW_LAUNCH(c, launch_clear(c->table.ptr, table_bytes, c->d_ctr, c->stream));
      }
      if (direct) TW_LAUNCH(c, launch_expand(a, c->stream));
      if (timed) TW_CK(cudaEventRecord(c->ev1, c->stream));
      TW_CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      const LevelCounters h = *c->h_ctr;
      float ms = 0.f;
      if (timed) TW_CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      const bool table_full = (h.overflow & 2u) || h.out_count * 100ull > slots * 90ull;
      if (table_full) {
        table_est = std::max(table_est * 2.0, (double)h.out_count * 1.5);
        out_cap = std::max<unsigned long long>(out_cap, (unsigned long long)std::ceil(table_est));
        slots = (unsigned long long)std::ceil(table_est * 100.0 / load_pct);
        ++R->retries;
        continue;
      }
      if (h.overflow & 1u) {
        out_cap = h.out_count;  // exact: every insert that won was counted
        ++R->retries;
        continue;
      }
      nxt.off = off;
      nxt.count = h.out_count;
      R->feasible += h.feasible;
      R->expand_launches += 1;
      R->expand_seconds += (double)ms * 1e-3;
      R->expand_bytes += (double)(cur.count + h.feasible + 2ull * h.out_count) * (double)w + (double)h.out_count;
      const unsigned long long live_states = keep_levels ? kept_states + nxt.count : cur.count + nxt.count;
      R->peak_bytes = std::max<unsigned long long>(R->peak_bytes, live_states * (w + 1) + slots * w);
      break;
    }
    R->states_expanded += cur.count;
    R->candidates += cur.count * (unsigned long long)(n - c->skipped - i);
    if (keep_levels) kept_states += nxt.count;
    R->levels.push_back(nxt);
    if (c->cfg.fingerprints) {
      TW_LAUNCH(c, launch_fingerprint(kc, static_cast<char*>(c->keys.ptr) + nxt.off * w, nxt.count, c->d_ctr, c->stream));
      TW_CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      R->fp_sum.push_back(c->h_ctr->fp_sum);
      R->fp_xor.push_back(c->h_ctr->fp_xor);
    }
    if (nxt.count == 0) break;
  }
  const int last = (int)R->levels.size() - 1;
  R->yes = (last == n - k - 1 && R->levels[last].count > 0) ? 1 : 0;
  return TW_OK;
}

// decide(k) with the level loop as one captured CUDA graph (every level kept).
// *bailed is set when the graph gave up (a level did not fit the current
// buffers or its estimate); the caller then runs the host loop.
int run_decide_graph(tw_ctx* c, KeyClass kc, int n, int k, DecideResult* R, bool* bailed) {
  *bailed = true;
  const int w = (int)key_bytes(kc);
  if (k >= n - 1) return TW_OK;
  const unsigned long long arena_cap = std::min<unsigned long long>(c->keys.bytes / w, c->pred.bytes);
  const unsigned long long table_cap = c->table.bytes >= 16 ? (c->table.bytes - 16) / w : 0;
  if (arena_cap < 64 || table_cap < 64) return TW_OK;
  int load_pct = c->cfg.table_load_pct > 0 ? std::min(90, c->cfg.table_load_pct) : 50;
  if (c->cfg.autotune && c->cfg.table_load_pct == 0)
    for (const auto& t : c->tuned)
      if (t.kc == (int)kc && t.nb == n / 8) load_pct = t.load_pct;
  const int max_probes = c->cfg.max_probes > 0 ? c->cfg.max_probes : 256;
  tw_ctx::GraphEntry* e = nullptr;
  for (auto& g : c->graphs)
    if (g.kc == (int)kc && g.n == n && g.k == k && g.load == load_pct && g.probes == max_probes &&
        g.bt == c->cfg.block_threads && g.allowed0 == c->allowed[0] && g.allowed1 == c->allowed[1] &&
        g.keys == c->keys.ptr && g.pred == c->pred.ptr && g.table == c->table.ptr && g.arena_cap == arena_cap &&
        g.table_cap == table_cap)
      e = &g;
  if (e == nullptr) {
    if (c->graphs.size() >= 32) {
      TW_CK(cudaStreamSynchronize(c->stream));
      for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
      c->graphs.clear();
    }
    SmallLayout L;
    ExpandLaunch a;
    a.kc = kc;
    a.in_keys = c->keys.ptr;
    a.n_in = 0;
    a.adj = small_at(c, L.adj);
    a.n = n;
    a.k = k;
    a.table = c->table.ptr;
    a.table_slots = 0;
    a.max_probes = max_probes;
    a.out_keys = c->keys.ptr;
    a.out_pred = static_cast<uint8_t*>(c->pred.ptr);
    a.out_cap = 0;
    a.ctr = c->d_ctr;
    a.block_threads = 128;
    a.grid = 0;
    a.allowed[0] = c->allowed[0];
    a.allowed[1] = c->allowed[1];
    a.mmw = c->cfg.mmw_prune ? 1 : 0;
    cudaGraph_t graph = nullptr;
    TW_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    int nodes = 0;
    cudaError_t err = launch_graph_init(kc, c->d_gstate, c->keys.ptr, c->stream);
    ++nodes;
    if (err == cudaSuccess)
      err = launch_graph_plan(c->d_gstate, c->d_ctr, arena_cap, table_cap, partition_threshold_bytes(c), n, k,
                              load_pct, w, 1, c->stream);
    ++nodes;
    for (int i = 0; i <= n - k - 2 && err == cudaSuccess; ++i) {
      err = launch_graph_clear(kc, c->d_gstate, c->table.ptr, c->stream);
      if (err == cudaSuccess) err = launch_graph_expand(c->d_gstate, a, c->stream);
      if (err == cudaSuccess)
        err = launch_graph_plan(c->d_gstate, c->d_ctr, arena_cap, table_cap, partition_threshold_bytes(c), n, k,
                                load_pct, w, 0, c->stream);
      nodes += 3;
    }
    const cudaError_t end = cudaStreamEndCapture(c->stream, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return TW_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t inst = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    TW_CK(inst);
    c->graphs.push_back({(int)kc, n, k, load_pct, max_probes, c->cfg.block_threads, c->allowed[0], c->allowed[1],
                         c->keys.ptr, c->pred.ptr, c->table.ptr, arena_cap, table_cap, exec, nodes});
    e = &c->graphs.back();
  }
  TW_CK(cudaGraphLaunch(e->exec, c->stream));
  c->launches += (unsigned long long)e->nodes;
  TW_CK(cudaMemcpyAsync(c->h_gstate, c->d_gstate, sizeof(GraphState), cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  const GraphState& h = *c->h_gstate;
  if (h.bail || !h.done) return TW_OK;
  *bailed = false;
  R->levels.clear();
  R->fp_sum.assign(1, 0ull);
  R->fp_xor.assign(1, 0ull);
  R->states_expanded = R->candidates = R->retries = 0;
  R->expand_launches = 0;
  R->expand_seconds = R->expand_bytes = 0.0;
  for (int j = 0; j <= h.cur; ++j) R->levels.push_back({h.level_off[j], h.level_cnt[j]});
  for (int j = 0; j < h.cur; ++j) {
    R->states_expanded += h.level_cnt[j];
    R->candidates += h.level_cnt[j] * (unsigned long long)(n - c->skipped - j);
    R->expand_bytes += (double)(h.level_cnt[j] + 2ull * h.level_cnt[j + 1]) * (double)w + (double)h.level_cnt[j + 1];
  }
  R->feasible = h.feasible;
  R->expand_bytes += (double)h.feasible * (double)w;
  R->expand_launches = (unsigned long long)h.cur;
  R->peak_bytes = h.peak_bytes;
  R->yes = h.yes;
  if (c->cfg.fingerprints) {
    for (int j = 1; j <= h.cur; ++j) {
      TW_CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(LevelCounters), c->stream));
      TW_LAUNCH(c, launch_fingerprint(kc, static_cast<char*>(c->keys.ptr) + h.level_off[j] * w, h.level_cnt[j],
                                      c->d_ctr, c->stream));
      TW_CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      R->fp_sum.push_back(c->h_ctr->fp_sum);
      R->fp_xor.push_back(c->h_ctr->fp_xor);
    }
  }
  return TW_OK;
}

// Default of tw_config.graph_levels == 0.
constexpr bool kGraphLevelsByDefault = true;

bool graph_mode(const tw_ctx* c) {
  if (c->cfg.time_kernels || c->cfg.graph_levels < 0) return false;
  return c->cfg.graph_levels > 0 || kGraphLevelsByDefault;
}

// ---- options of Section 3.1 ------------------------------------------------
using Set128 = unsigned __int128;

Set128 row_set(const HostGraph& g, int v) {
  Set128 r = g.rows[(size_t)v * g.words];
  if (g.words > 1) r |= (Set128)g.rows[(size_t)v * g.words + 1] << 64;
  return r;
}
int popc128(Set128 a) { return __builtin_popcountll((uint64_t)a) + __builtin_popcountll((uint64_t)(a >> 64)); }
int lowest128(Set128 a) {
  const uint64_t lo = (uint64_t)a;
  return lo ? __builtin_ctzll(lo) : 64 + __builtin_ctzll((uint64_t)(a >> 64));
}
// Sorted vertex lists compare as: A < B iff the smallest vertex in exactly
// one of them belongs to A.
bool lex_less(Set128 a, Set128 b) {
  const Set128 d = a ^ b;
  return d != 0 && ((a >> lowest128(d)) & 1);
}

// Bron-Kerbosch with pivoting over bitsets: every maximal clique is visited,
// so every maximum one is; the lexicographically smallest maximum is kept.
void bron_kerbosch(const std::vector<Set128>& nb, Set128 r, Set128 p, Set128 x, int* best_size, Set128* best) {
  if (p == 0 && x == 0) {
    const int sz = popc128(r);
    if (sz > *best_size || (sz == *best_size && lex_less(r, *best))) {
      *best_size = sz;
      *best = r;
    }
    return;
  }
  if (popc128(r) + popc128(p) < *best_size) return;
  Set128 px = p | x;
  int pivot = lowest128(px), most = -1;
  for (Set128 t = px; t; t &= t - 1) {
    const int u = lowest128(t);
    const int c = popc128(p & nb[u]);
    if (c > most) {
      most = c;
      pivot = u;
    }
  }
  for (Set128 t = p & ~nb[pivot]; t; t &= t - 1) {
    const int v = lowest128(t);
    const Set128 bv = (Set128)1 << v;
    bron_kerbosch(nb, r | bv, p & nb[v], x & nb[v], best_size, best);
    p &= ~bv;
    x |= bv;
  }
}

Set128 max_clique(const HostGraph& g) {
  std::vector<Set128> nb(g.n);
  for (int v = 0; v < g.n; ++v) nb[v] = row_set(g, v);
  const Set128 all = g.n == 128 ? ~(Set128)0 : (((Set128)1 << g.n) - 1);
  int best_size = 0;
  Set128 best = 0;
  bron_kerbosch(nb, 0, all, 0, &best_size, &best);
  return best;
}

// At least t internally vertex-disjoint u-v paths (u, v not adjacent)?
// Unit vertex capacities by splitting x into x_in -> x_out; breadth-first
// augmenting paths in the residual network.
bool connected_at_least(const HostGraph& g, int u, int v, int t) {
  const int n = g.n, N = 2 * n;
  struct Arc {
    int to, cap, rev;
  };
  std::vector<std::vector<Arc>> adj(N);
  auto add = [&](int a, int b, int cap) {
    adj[a].push_back({b, cap, (int)adj[b].size()});
    adj[b].push_back({a, 0, (int)adj[a].size() - 1});
  };
  for (int x = 0; x < n; ++x) add(2 * x, 2 * x + 1, (x == u || x == v) ? n : 1);
  for (int a = 0; a < n; ++a)
    for (Set128 r = row_set(g, a); r; r &= r - 1) add(2 * a + 1, 2 * lowest128(r), n);
  const int src = 2 * u + 1, dst = 2 * v;
  int flow = 0;
  std::vector<int> pn(N), pa(N);
  while (flow < t) {
    std::fill(pn.begin(), pn.end(), -1);
    std::vector<int> queue{src};
    pn[src] = src;
    for (size_t h = 0; h < queue.size() && pn[dst] < 0; ++h) {
      const int a = queue[h];
      for (int e = 0; e < (int)adj[a].size(); ++e) {
        const Arc& arc = adj[a][e];
        if (arc.cap > 0 && pn[arc.to] < 0) {
          pn[arc.to] = a;
          pa[arc.to] = e;
          queue.push_back(arc.to);
        }
      }
    }
    if (pn[dst] < 0) break;
    for (int y = dst; y != src; y = pn[y]) {
      Arc& arc = adj[pn[y]][pa[y]];
      arc.cap -= 1;
      adj[y][arc.rev].cap += 1;
    }
    ++flow;
  }
  return flow >= t;
}

// Prepares decide(k) under the context's options: uploads the graph (with
// the disjoint-path edges for this k) and sets the allowed-vertex mask.
// *immediate_no is set when the skipped clique alone exceeds k+1 vertices.
int prepare_options(tw_ctx* c, const HostGraph& g, int k, KeyClass kc, bool* immediate_no) {
  *immediate_no = false;
  c->allowed[0] = c->allowed[1] = ~0ull;
  c->skipped = 0;
  if (!c->cfg.clique_skip && !c->cfg.disjoint_paths) return TW_OK;
  HostGraph gk = g;
  if (c->cfg.disjoint_paths) {
    for (int u = 0; u < g.n; ++u)
      for (int v = u + 1; v < g.n; ++v) {
        if ((row_set(g, u) >> v) & 1) continue;
        if (!connected_at_least(g, u, v, k + 1)) continue;
        gk.rows[(size_t)u * g.words + (v >> 6)] |= 1ull << (v & 63);
        gk.rows[(size_t)v * g.words + (u >> 6)] |= 1ull << (u & 63);
      }
  }
  int rc = upload_graph(c, gk, kc);
  if (rc) return rc;
  if (c->cfg.clique_skip) {
    const Set128 cl = max_clique(g);
    c->allowed[0] = ~(uint64_t)cl;
    c->allowed[1] = ~(uint64_t)(cl >> 64);
    c->skipped = popc128(cl);
    *immediate_no = c->skipped > k + 1;
  }
  return TW_OK;
}

// The run of a decide answered by the clique bound alone: only L_0.
void immediate_no_result(DecideResult* R) {
  R->levels.assign(1, LevelRec{0, 1});
  R->yes = 0;
  R->states_expanded = R->candidates = R->feasible = R->retries = 0;
  R->expand_launches = 0;
  R->expand_seconds = R->expand_bytes = 0.0;
  R->peak_bytes = 0;
  R->fp_sum.assign(1, 0ull);
  R->fp_xor.assign(1, 0ull);
}

// decide(k): the graph-driven loop when enabled, else (or when it gives up)
// the host loop.
int run_decide_any(tw_ctx* c, KeyClass kc, int n, int k, bool keep_levels, DecideResult* R) {
  if (graph_mode(c)) {
    bool bailed = true;
    int rc = run_decide_graph(c, kc, n, k, R, &bailed);
    if (rc) return rc;
    if (!bailed) return TW_OK;
  }
  return run_decide(c, kc, n, k, keep_levels, R);
}

// decide(k) under the context's options (Section 3.1's clique skip and
// disjoint-path edges when enabled).
int decide_with_options(tw_ctx* c, const HostGraph& g, KeyClass kc, int k, bool keep_levels, DecideResult* R) {
  bool no = false;
  int rc = prepare_options(c, g, k, kc, &no);
  if (rc) return rc;
  if (no) {
    immediate_no_result(R);
    return TW_OK;
  }
  return run_decide_any(c, kc, g.n, k, keep_levels, R);
}

// Backward walk through the kept levels into the device order buffer.
int reconstruct(tw_ctx* c, KeyClass kc, int n, const DecideResult& R) {
  SmallLayout L;
  const size_t w = key_bytes(kc);
  const int last = (int)R.levels.size() - 1;
  int32_t* d_order = reinterpret_cast<int32_t*>(small_at(c, L.order));
  void* walk = small_at(c, L.walk);
  char* keys = static_cast<char*>(c->keys.ptr);
  const uint8_t* pred = static_cast<const uint8_t*>(c->pred.ptr);
  TW_LAUNCH(c, launch_walk_init(kc, keys + R.levels[last].off * w, walk, last, c->stream));
  for (int j = last; j >= 1; --j) {
    const LevelRec& lr = R.levels[j];
    TW_LAUNCH(c, launch_walk_step(kc, keys + lr.off * w, pred + lr.off, lr.count, walk, j, d_order, c->stream));
  }
  TW_LAUNCH(c, launch_walk_finish(kc, walk, last, n, d_order, c->stream));
  return TW_OK;
}

void fill_stats(const DecideResult& R, int k, tw_stats* st, bool reset_totals) {
  if (!st) return;
  if (reset_totals) {
    st->states_expanded = st->candidates = st->feasible = st->peak_frontier_bytes = 0;
    st->decide_runs = st->level_retries = 0;
    st->expand_launches = 0;
    st->expand_seconds = st->expand_bytes = 0.0;
  }
  st->levels = (int)R.levels.size();
  st->k = k;
  for (int i = 0; i <= TW_MAX_N; ++i) {
    const bool in = i < (int)R.levels.size();
    st->level_size[i] = in ? R.levels[i].count : 0;
    st->level_fp_sum[i] = (in && i < (int)R.fp_sum.size()) ? R.fp_sum[i] : 0;
    st->level_fp_xor[i] = (in && i < (int)R.fp_xor.size()) ? R.fp_xor[i] : 0;
  }
  st->states_expanded += R.states_expanded;
  st->candidates += R.candidates;
  st->feasible += R.feasible;
  st->peak_frontier_bytes = std::max<uint64_t>(st->peak_frontier_bytes, R.peak_bytes);
  st->decide_runs += 1;
  st->level_retries += R.retries;
  st->expand_launches += R.expand_launches;
  st->expand_seconds += R.expand_seconds;
  st->expand_bytes += R.expand_bytes;
}

int decide_graph(tw_ctx* c, const HostGraph& g, int k, int* yes, int32_t* order, tw_stats* st) {
  Timer t;
  const unsigned long long launches0 = c->launches;
  if (k < 0 || yes == nullptr) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  const KeyClass kc = key_class_for(g.n);
  int rc = upload_graph(c, g, kc);
  if (rc) return rc;
  DecideResult R;
  rc = decide_with_options(c, g, kc, k, order != nullptr, &R);
  if (rc) {
    // the levels completed before the failure are still reported
    fill_stats(R, k, st, true);
    if (st) st->seconds = t.seconds();
    return rc;
  }
  if (R.yes && order) {
    rc = reconstruct(c, kc, g.n, R);
    if (rc) return rc;
    rc = put_from_device(c, order, small_at(c, SmallLayout().order), (size_t)g.n * 4);
    if (rc) return rc;
  }
  TW_CK(cudaStreamSynchronize(c->stream));
  fill_stats(R, k, st, true);
  int y = R.yes;
  rc = put(c, yes, &y, sizeof(int));
  if (rc) return rc;
  if (st) {
    st->seconds = t.seconds();
    st->kernel_launches = c->launches - launches0;
  }
  return TW_OK;
}

int bounds_graph(tw_ctx* c, const HostGraph& g, int32_t out[4]) {
  SmallLayout L;
  int32_t* d_out = reinterpret_cast<int32_t*>(small_at(c, L.bounds));
  int32_t* d_n = d_out + 4;
  int64_t* d_off = reinterpret_cast<int64_t*>(small_at(c, L.bounds + 64));
  const int32_t nn = g.n;
  const int64_t off = 0;
  TW_CK(cudaMemcpyAsync(d_n, &nn, 4, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_off, &off, 8, cudaMemcpyHostToDevice, c->stream));
  TW_LAUNCH(c, launch_bounds(reinterpret_cast<const unsigned long long*>(small_at(c, L.adj64)), d_n, d_off, 1, d_out,
                      nullptr, c->stream));
  TW_CK(cudaMemcpyAsync(out, d_out, 16, cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  return TW_OK;
}

int solve_graph(tw_ctx* c, const HostGraph& g, int* tw_out, int32_t* order, int32_t* td_parent, uint64_t* td_bags,
                tw_stats* st, int k_first) {
  Timer t;
  const unsigned long long launches0 = c->launches;
  TW_CK(cudaSetDevice(c->device));
  const KeyClass kc = key_class_for(g.n);
  int rc = upload_graph(c, g, kc);
  if (rc) return rc;
  int32_t b[4];
  rc = bounds_graph(c, g, b);
  if (rc) return rc;
  const int lb = std::max(b[0], b[1]);
  const int ub = std::min(b[2], b[3]);
  const bool want_walk = order || td_parent || td_bags;
  if (st) {
    st->states_expanded = st->candidates = st->feasible = st->peak_frontier_bytes = 0;
    st->decide_runs = st->level_retries = 0;
    st->expand_launches = 0;
    st->expand_seconds = st->expand_bytes = 0.0;
  }
  int tw = -1;
  DecideResult R;
  int k0 = std::max(lb, k_first);
  if (c->cfg.ub_shortcut && lb == ub && !want_walk) {
    tw = ub;
  } else {
    for (int k = k0; k < g.n; ++k) {
      rc = decide_with_options(c, g, kc, k, want_walk, &R);
      if (rc) return rc;
      fill_stats(R, k, st, false);
      if (R.yes) {
        tw = k;
        break;
      }
    }
  }
  if (tw < 0) return TW_ERR_CUDA;
  if (want_walk && R.yes) {
    SmallLayout L;
    rc = reconstruct(c, kc, g.n, R);
    if (rc) return rc;
    int32_t* d_order = reinterpret_cast<int32_t*>(small_at(c, L.order));
    if (c->cfg.disjoint_paths && (rc = upload_graph(c, g, kc))) return rc;  // bags of G itself
    if (td_parent || td_bags) {
      TW_LAUNCH(c, launch_td(reinterpret_cast<const unsigned long long*>(small_at(c, L.adj64)), g.n, g.words, d_order,
                      reinterpret_cast<int32_t*>(small_at(c, L.parent)),
                      reinterpret_cast<unsigned long long*>(small_at(c, L.bags)), c->stream));
    }
    rc = put_from_device(c, order, d_order, (size_t)g.n * 4);
    if (rc) return rc;
    rc = put_from_device(c, td_parent, small_at(c, L.parent), (size_t)g.n * 4);
    if (rc) return rc;
    rc = put_from_device(c, td_bags, small_at(c, L.bags), (size_t)g.n * g.words * 8);
    if (rc) return rc;
  }
  TW_CK(cudaStreamSynchronize(c->stream));
  rc = put(c, tw_out, &tw, sizeof(int));
  if (rc) return rc;
  if (st) {
    st->seconds = t.seconds();
    st->kernel_launches = c->launches - launches0;
  }
  return TW_OK;
}


// Scratch staging: a bump allocator over ctx->scratch (256-byte aligned
// pieces).  reserve() must be called with the total before any piece is taken.
struct Stager {
  tw_ctx* c;
  size_t used = 0;
  explicit Stager(tw_ctx* cc) : c(cc) {}
  int reserve(size_t total) {
    if (total > c->scratch.bytes) {
      if (c->scratch.ptr) {
        TW_CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->scratch.ptr);
        c->scratch.ptr = nullptr;
        c->scratch.bytes = 0;
      }
      const size_t want = (total + 4095) & ~size_t(4095);
      if (cudaMalloc(&c->scratch.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        return TW_ERR_CAPACITY;
      }
      c->scratch.bytes = want;
    }
    return TW_OK;
  }
  void* take(size_t bytes) {
    char* p = static_cast<char*>(c->scratch.ptr) + used;
    used += (bytes + 255) & ~size_t(255);
    return p;
  }
  // Device copy of a host or device array (device arrays are used in place).
  int in(const void* src, size_t bytes, const void** out) {
    if (is_device_ptr(src)) {
      *out = src;
      take(bytes);
      return TW_OK;
    }
    void* d = take(bytes);
    TW_CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, c->stream));
    *out = d;
    return TW_OK;
  }
};


// Decide runs of one graph guided by a proposed bound: decide(k0) and
// decide(k0-1) first, then walk up (on no) or down (on yes) until yes at tw
// and no at tw-1 (or tw = lower bound) certify the answer.  Returns the
// treewidth in *tw_out and the ordering of the yes run at tw in order_host.
int solve_hinted(tw_ctx* c, const HostGraph& g, float hint, int* tw_out, std::vector<int32_t>* order_host,
                 tw_stats* st) {
  const KeyClass kc = key_class_for(g.n);
  int rc = upload_graph(c, g, kc);
  if (rc) return rc;
  int32_t b[4];
  if ((rc = bounds_graph(c, g, b))) return rc;
  const int lb = std::max(b[0], b[1]);
  int k0 = (int)std::lround(hint);
  k0 = std::min(std::max(k0, lb), g.n - 1);
  DecideResult R;
  SmallLayout L;
  auto run = [&](int k, int* yes) -> int {
    int r = decide_with_options(c, g, kc, k, order_host != nullptr, &R);
    if (r) return r;
    fill_stats(R, k, st, false);
    *yes = R.yes;
    if (R.yes && order_host) {
      if ((r = reconstruct(c, kc, g.n, R))) return r;
      order_host->resize(g.n);
      TW_CK(cudaMemcpyAsync(order_host->data(), small_at(c, L.order), (size_t)g.n * 4, cudaMemcpyDeviceToHost,
                            c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
    }
    return TW_OK;
  };
  int yes = 0;
  if ((rc = run(k0, &yes))) return rc;
  if (yes) {
    int k = k0;
    while (k > lb) {
      int y2 = 0;
      if ((rc = run(k - 1, &y2))) return rc;
      if (!y2) break;
      --k;
    }
    *tw_out = k;
  } else {
    int k = k0 + 1;
    for (;; ++k) {
      int y2 = 0;
      if ((rc = run(k, &y2))) return rc;
      if (y2) break;
    }
    *tw_out = k;
  }
  return TW_OK;
}

size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }

// ---------------------------------------------------------------- batches
//
// Level-synchronous batched solve for graphs with n <= 64.  Every graph runs
// its own k sweep (Section 3.1) as a small state machine on the host; each
// step expands the current level of every running graph in one launch of
// expand_batch_kernel.  A graph whose level would exceed kEvictStates leaves
// the batch and is solved afterwards by the single-graph path, which sizes
// its buffers for large levels.
constexpr double kEvictStates = double(1 << 21);
constexpr unsigned long long kStepSlots = 1ull << 27;   // table slots per step
constexpr unsigned long long kStepOut = 1ull << 26;     // output states per step
constexpr int kBatchProbes = 256;

struct BGraph {
  int in_idx = 0;
  int n = 0;
  int lb = 0;
  int k0 = 0;
  int k = -1;
  int yes_min = 1 << 30;
  int no_max = -1;
  int state = 0;  // 0 running, 1 done, 2 evicted
  std::vector<LevelRec> levels;
  double table_mult = 1.0;
  unsigned long long ocap_retry = 0;
  int tw = -1;
  int64_t order_off = 0;
};

template <class T>
int dev_alloc(T** p, size_t count) {
  void* v = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&v, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return TW_ERR_CAPACITY;
  }
  *p = static_cast<T*>(v);
  return TW_OK;
}

struct BatchRun {
  tw_ctx* c;
  std::vector<BGraph> g;
  unsigned long long* adj = nullptr;
  unsigned long long* akeys = nullptr;
  uint32_t* apar = nullptr;
  unsigned long long acap = 0, atop = 0;
  unsigned long long* table = nullptr;
  unsigned long long tcap = 0;
  unsigned long long* okeys = nullptr;
  uint32_t* opar = nullptr;
  unsigned long long ocap = 0;
  BatchSeg* segs = nullptr;
  unsigned long long* cbeg = nullptr;
  BatchCounters* ctr = nullptr;
  CopySeg* copies = nullptr;
  WalkSeg* walks = nullptr;
  unsigned long long* lvl = nullptr;
  int32_t* orders = nullptr;
  size_t nslots_meta = 0;
  std::vector<void*> owned;

  explicit BatchRun(tw_ctx* cc) : c(cc) {}
  ~BatchRun() {
    cudaStreamSynchronize(c->stream);
    for (void* p : {(void*)adj, (void*)akeys, (void*)apar, (void*)table, (void*)okeys, (void*)opar, (void*)segs,
                    (void*)cbeg, (void*)ctr, (void*)copies, (void*)walks, (void*)lvl, (void*)orders})
      if (p) cudaFree(p);
    cudaGetLastError();
  }

  size_t live_states() const {
    size_t live = 0;
    for (const BGraph& x : g)
      if (x.state == 0)
        for (const LevelRec& l : x.levels) live += l.count;
    return live;
  }

  // Makes room for need more arena states, compacting the live levels of
  // running graphs into a fresh arena when the current one is full.
  int arena_room(unsigned long long need) {
    if (atop + need <= acap) return TW_OK;
    const unsigned long long live = live_states();
    const unsigned long long want = std::max<unsigned long long>({acap, 2 * (live + need), 1ull << 20});
    unsigned long long* nk = nullptr;
    uint32_t* np = nullptr;
    int rc = dev_alloc(&nk, want);
    if (rc == TW_OK) rc = dev_alloc(&np, want);
    if (rc != TW_OK) {
      if (nk) cudaFree(nk);
      return rc;
    }
    std::vector<CopySeg> cs;
    unsigned long long top = 0;
    for (BGraph& x : g) {
      if (x.state != 0) continue;
      for (LevelRec& l : x.levels) {
        if (l.count) cs.push_back({l.off, top, l.count});
        l.off = top;
        top += l.count;
      }
    }
    if (!cs.empty()) {
      CopySeg* d = nullptr;
      if ((rc = dev_alloc(&d, cs.size()))) return rc;
      TW_CK(cudaMemcpyAsync(d, cs.data(), cs.size() * sizeof(CopySeg), cudaMemcpyHostToDevice, c->stream));
      TW_LAUNCH(c, launch_copy_segments(d, (int)cs.size(), akeys, apar, nk, np, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      cudaFree(d);
    }
    TW_CK(cudaStreamSynchronize(c->stream));
    if (akeys) cudaFree(akeys);
    if (apar) cudaFree(apar);
    akeys = nk;
    apar = np;
    acap = want;
    atop = top;
    return TW_OK;
  }

  template <class T>
  int ensure(T** p, unsigned long long* cap, unsigned long long need) {
    if (need <= *cap && *p) return TW_OK;
    TW_CK(cudaStreamSynchronize(c->stream));
    if (*p) cudaFree(*p);
    *p = nullptr;
    const unsigned long long want = std::max<unsigned long long>(need, *cap * 2);
    int rc = dev_alloc(p, want);
    if (rc) return rc;
    *cap = want;
    return TW_OK;
  }
};

int next_k(const BGraph& x) {
  if (x.k < 0) return x.k0;
  if (x.yes_min >= (1 << 30)) return x.no_max + 1;
  return x.yes_min - 1;
}

// Records the answer of the run at x.k; returns true when tw is certified
// (yes at tw and no at tw-1, or tw equal to the lower bound).
bool record_answer(BGraph& x, bool yes) {
  if (yes)
    x.yes_min = std::min(x.yes_min, x.k);
  else
    x.no_max = std::max(x.no_max, x.k);
  if (x.yes_min == x.no_max + 1) {
    x.tw = x.yes_min;
    x.state = 1;
    return true;
  }
  return false;
}

// The batched part: every graph of idx either finishes here (state 1) or is
// returned in *evicted for the single-graph path.
int run_batch(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
              const std::vector<float>* hint, const std::vector<int64_t>& order_off, int* htw,
              std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st, std::vector<int>* evicted) {
  BatchRun B(c);
  const int G = (int)idx.size();
  if (G == 0) return TW_OK;
  int rc;
  // adjacency: 64 rows per graph; bounds input: the same rows
  {
    std::vector<unsigned long long> rows((size_t)G * 64, 0ull);
    std::vector<int32_t> ns(G);
    std::vector<int64_t> offs(G);
    for (int j = 0; j < G; ++j) {
      const HostGraph& hg = graphs[idx[j]];
      for (int r = 0; r < hg.n; ++r) rows[(size_t)j * 64 + r] = hg.rows[r];
      ns[j] = hg.n;
      offs[j] = (int64_t)j * 64;
    }
    if ((rc = dev_alloc(&B.adj, rows.size()))) return rc;
    TW_CK(cudaMemcpyAsync(B.adj, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice, c->stream));
    int32_t *d_n = nullptr, *d_b = nullptr;
    int64_t* d_off = nullptr;
    if ((rc = dev_alloc(&d_n, G)) || (rc = dev_alloc(&d_off, G)) || (rc = dev_alloc(&d_b, (size_t)G * 4))) return rc;
    TW_CK(cudaMemcpyAsync(d_n, ns.data(), G * 4, cudaMemcpyHostToDevice, c->stream));
    TW_CK(cudaMemcpyAsync(d_off, offs.data(), G * 8, cudaMemcpyHostToDevice, c->stream));
    TW_LAUNCH(c, launch_bounds(B.adj, d_n, d_off, G, d_b, nullptr, c->stream));
    std::vector<int32_t> b((size_t)G * 4);
    TW_CK(cudaMemcpyAsync(b.data(), d_b, b.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaStreamSynchronize(c->stream));
    cudaFree(d_n);
    cudaFree(d_off);
    cudaFree(d_b);
    B.g.resize(G);
    for (int j = 0; j < G; ++j) {
      BGraph& x = B.g[j];
      x.in_idx = idx[j];
      x.n = graphs[idx[j]].n;
      x.lb = std::max(b[4 * j], b[4 * j + 1]);
      x.no_max = x.lb - 1;
      int k0 = x.lb;
      if (hint) k0 = (int)std::lround((*hint)[idx[j]]);
      x.k0 = std::min(std::max(k0, x.lb), x.n - 1);
      x.order_off = order_off[idx[j]];
    }
  }
  int64_t total_n = 0;
  for (int j = 0; j < G; ++j) total_n = std::max<int64_t>(total_n, B.g[j].order_off + B.g[j].n);
  if ((rc = dev_alloc(&B.orders, (size_t)total_n))) return rc;
  if ((rc = dev_alloc(&B.segs, G)) || (rc = dev_alloc(&B.cbeg, (size_t)G + 1)) || (rc = dev_alloc(&B.ctr, G)) ||
      (rc = dev_alloc(&B.copies, G)) || (rc = dev_alloc(&B.walks, G)) ||
      (rc = dev_alloc(&B.lvl, (size_t)G * 65)))
    return rc;
  std::vector<BatchSeg> segs;
  std::vector<unsigned long long> cbeg;
  std::vector<BatchCounters> hc(G);
  std::vector<CopySeg> copies;
  std::vector<WalkSeg> walks;
  std::vector<unsigned long long> lvl;
  std::vector<int> seg_graph;
  size_t rr = 0;

  for (int step = 0;; ++step) {
    // 1. start a run (level 0 = {empty set}) for graphs without one
    copies.clear();
    {
      unsigned long long starting = 0;
      for (const BGraph& x : B.g)
        if (x.state == 0 && x.levels.empty()) ++starting;
      if (starting && (rc = B.arena_room(starting))) return rc;  // before any offset is handed out
    }
    for (BGraph& x : B.g) {
      if (x.state != 0 || !x.levels.empty()) continue;
      x.k = next_k(x);
      copies.push_back({~0ull, B.atop, 1});
      x.levels.push_back({B.atop, 1});
      B.atop += 1;
      if (st) st->decide_runs += 1;
    }
    if (!copies.empty()) {
      TW_CK(cudaMemcpyAsync(B.copies, copies.data(), copies.size() * sizeof(CopySeg), cudaMemcpyHostToDevice,
                            c->stream));
      TW_LAUNCH(c, launch_copy_segments(B.copies, (int)copies.size(), nullptr, nullptr, B.akeys, B.apar, c->stream));
    }
    // 2. finished runs: an empty level answers no; level n-k-1 answers yes
    walks.clear();
    lvl.clear();
    std::vector<int> walked;
    bool answered = false;
    for (int j = 0; j < G; ++j) {
      BGraph& x = B.g[j];
      if (x.state != 0) continue;
      const int last = (int)x.levels.size() - 1;
      if (x.levels.back().count == 0) {
        record_answer(x, false);
        x.levels.clear();
        answered = true;
      } else if (last == x.n - x.k - 1) {
        walks.push_back({(unsigned long long)lvl.size(), (unsigned long long)x.order_off, last, x.n});
        for (const LevelRec& l : x.levels) lvl.push_back(l.off);
        walked.push_back(j);
      }
    }
    if (!walks.empty()) {
      TW_CK(cudaMemcpyAsync(B.walks, walks.data(), walks.size() * sizeof(WalkSeg), cudaMemcpyHostToDevice,
                            c->stream));
      TW_CK(cudaMemcpyAsync(B.lvl, lvl.data(), lvl.size() * 8, cudaMemcpyHostToDevice, c->stream));
      TW_LAUNCH(c, launch_walk_batch(B.walks, (int)walks.size(), B.lvl, B.akeys, B.apar, B.orders, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      for (int j : walked) {
        record_answer(B.g[j], true);
        B.g[j].levels.clear();
      }
      answered = true;
    }
    if (answered) continue;  // graphs that answered need their next run started first
    // 3. build this step's segments (round robin under the step budgets)
    segs.clear();
    cbeg.clear();
    seg_graph.clear();
    unsigned long long tsum = 0, osum = 0, chunks = 0;
    int running = 0;
    for (int t = 0; t < G; ++t) {
      const int j = (int)((rr + t) % G);
      BGraph& x = B.g[j];
      if (x.state != 0) continue;
      ++running;
      const int i = (int)x.levels.size() - 1;
      const LevelRec cur = x.levels.back();
      const double bound = std::min((double)cur.count * (double)(x.n - i), binom(x.n, i + 1)) + 1.0;
      double est = x.n;
      if (i > 0) {
        const double prev = (double)x.levels[i - 1].count;
        double r = prev > 0 ? (double)cur.count / prev : 1.0;
        r = std::min(std::max(r, 0.25), (double)(x.n - i));
        est = (double)cur.count * r;
      }
      const double table_est = std::min(est * 1.25 * x.table_mult + 1024.0, bound);
      if (est > kEvictStates || (double)x.ocap_retry > kEvictStates) {
        x.state = 2;
        x.levels.clear();
        --running;
        continue;
      }
      const unsigned long long slots = std::max<unsigned long long>(64, (unsigned long long)std::ceil(table_est * 2.0));
      unsigned long long oc = x.ocap_retry ? x.ocap_retry
                                           : (unsigned long long)std::ceil(std::min(bound, std::max(table_est * 3.0, 1024.0)));
      if (!segs.empty() && (tsum + slots > kStepSlots || osum + oc > kStepOut)) continue;
      BatchSeg sg;
      sg.in_off = cur.off;
      sg.in_count = cur.count;
      sg.t_off = tsum;
      sg.t_slots = slots;
      sg.o_off = osum;
      sg.o_cap = oc;
      sg.graph = j;
      sg.n = x.n;
      sg.k = x.k;
      sg.pad = 0;
      segs.push_back(sg);
      seg_graph.push_back(j);
      cbeg.push_back(chunks);
      chunks += (cur.count + 31) / 32;
      tsum += slots;
      osum += oc;
    }
    rr = (rr + 1) % (size_t)G;
    if (running == 0) break;
    if (segs.empty()) continue;  // evictions only
    cbeg.push_back(chunks);
    if ((rc = B.ensure(&B.table, &B.tcap, tsum + 2))) return rc;
    {
      unsigned long long cap_o = B.ocap;
      if ((rc = B.ensure(&B.okeys, &cap_o, osum))) return rc;
      unsigned long long cap_p = B.ocap;
      if ((rc = B.ensure(&B.opar, &cap_p, osum))) return rc;
      B.ocap = std::min(cap_o, cap_p);
    }
    const int nseg = (int)segs.size();
    TW_CK(cudaMemcpyAsync(B.segs, segs.data(), nseg * sizeof(BatchSeg), cudaMemcpyHostToDevice, c->stream));
    TW_CK(cudaMemcpyAsync(B.cbeg, cbeg.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    TW_CK(cudaMemsetAsync(B.ctr, 0, nseg * sizeof(BatchCounters), c->stream));
    TW_LAUNCH(c, launch_clear(B.table, (size_t)((tsum * 8 + 15) & ~15ull), c->d_ctr, c->stream));
    TW_LAUNCH(c, launch_expand_batch(B.segs, B.cbeg, nseg, chunks, B.akeys, B.adj, B.table, B.okeys, B.opar, B.ctr,
                                     kBatchProbes, c->stream));
    if (st) st->expand_launches += 1;
    TW_CK(cudaMemcpyAsync(hc.data(), B.ctr, nseg * sizeof(BatchCounters), cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaStreamSynchronize(c->stream));
    // 4. results: retry, evict or commit into the arena
    unsigned long long need = 0;
    for (int s2 = 0; s2 < nseg; ++s2) {
      BGraph& x = B.g[seg_graph[s2]];
      const BatchCounters& h = hc[s2];
      const bool table_full = (h.overflow & 2u) || h.out_count * 100ull > segs[s2].t_slots * 90ull;
      if (table_full) {
        x.table_mult *= 2.0;
        if (st) st->level_retries += 1;
        continue;
      }
      if (h.out_count > segs[s2].o_cap) {
        x.ocap_retry = h.out_count;
        if (st) st->level_retries += 1;
        continue;
      }
      need += h.out_count;
    }
    if ((rc = B.arena_room(need))) return rc;
    copies.clear();
    for (int s2 = 0; s2 < nseg; ++s2) {
      BGraph& x = B.g[seg_graph[s2]];
      const BatchCounters& h = hc[s2];
      const bool table_full = (h.overflow & 2u) || h.out_count * 100ull > segs[s2].t_slots * 90ull;
      if (table_full || h.out_count > segs[s2].o_cap) continue;
      x.ocap_retry = 0;
      const int i = (int)x.levels.size() - 1;
      if (st) {
        st->states_expanded += segs[s2].in_count;
        st->candidates += segs[s2].in_count * (unsigned long long)(x.n - i);
        st->feasible += h.feasible;
      }
      if (h.out_count) copies.push_back({segs[s2].o_off, B.atop, h.out_count});
      x.levels.push_back({B.atop, h.out_count});
      B.atop += h.out_count;
    }
    if (!copies.empty()) {
      TW_CK(cudaMemcpyAsync(B.copies, copies.data(), copies.size() * sizeof(CopySeg), cudaMemcpyHostToDevice,
                            c->stream));
      TW_LAUNCH(c, launch_copy_segments(B.copies, (int)copies.size(), B.okeys, B.opar, B.akeys, B.apar, c->stream));
    }
  }
  // results of the batched graphs
  std::vector<int32_t> dord((size_t)total_n);
  TW_CK(cudaMemcpyAsync(dord.data(), B.orders, dord.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  for (BGraph& x : B.g) {
    if (x.state != 1) continue;
    htw[x.in_idx] = x.tw;
    (*hst)[x.in_idx] = TW_OK;
    if (hord)
      for (int v = 0; v < x.n; ++v) (*hord)[x.order_off + v] = dord[x.order_off + v];
  }
  for (BGraph& x : B.g)
    if (x.state == 2) evicted->push_back(x.in_idx);
  return TW_OK;
}

// Graphs with n <= 64 go through the batched kernel; graphs it evicts and
// graphs with n > 64 are solved one at a time by the single-graph path.
int solve_batch_gpu(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                    const std::vector<float>* hint, const std::vector<int64_t>& order_off, int* htw,
                    std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st) {
  std::vector<int> small, single;
  for (int i : idx) (graphs[i].n <= 64 ? small : single).push_back(i);
  int rc = run_batch(c, graphs, small, hint, order_off, htw, hord, hst, st, &single);
  if (rc) return rc;
  for (int gi : single) {
    const HostGraph& hg = graphs[gi];
    std::vector<int32_t> ord;
    int r2;
    tw_stats local;
    std::memset(&local, 0, sizeof(local));
    if (hint) {
      r2 = solve_hinted(c, hg, (*hint)[gi], &htw[gi], hord ? &ord : nullptr, &local);
    } else {
      ord.assign(hg.n, -1);
      r2 = solve_graph(c, hg, &htw[gi], hord ? ord.data() : nullptr, nullptr, nullptr, &local, 0);
    }
    if (st && r2 == TW_OK) {
      st->states_expanded += local.states_expanded;
      st->candidates += local.candidates;
      st->feasible += local.feasible;
      st->decide_runs += local.decide_runs;
      st->level_retries += local.level_retries;
      st->expand_launches += local.expand_launches;
    }
    if (r2 == TW_OK && hord)
      for (int v = 0; v < hg.n; ++v) (*hord)[order_off[gi] + v] = ord[v];
    if (r2 != TW_OK) htw[gi] = -1;
    (*hst)[gi] = r2;
  }
  return TW_OK;
}


// Batched per-graph validation into 64-bit rows.
int load_batch(const uint64_t* adj_concat, const int32_t* n, const int64_t* row_offset, int num_graphs,
               std::vector<int32_t>* hn, std::vector<int64_t>* hoff, std::vector<uint64_t>* hadj) {
  if (!adj_concat || !n || !row_offset || num_graphs < 0) return TW_ERR_INVALID;
  hn->resize(num_graphs);
  hoff->resize(num_graphs);
  int rc = fetch(hn->data(), n, (size_t)num_graphs * 4);
  if (rc) return rc;
  rc = fetch(hoff->data(), row_offset, (size_t)num_graphs * 8);
  if (rc) return rc;
  int64_t words = 0;
  for (int g = 0; g < num_graphs; ++g) {
    const int ng = (*hn)[g];
    if (ng < 1 || ng > TW_MAX_N || (*hoff)[g] < 0) return TW_ERR_INVALID;
    words = std::max<int64_t>(words, (*hoff)[g] + (int64_t)ng * ((ng + 63) / 64));
  }
  hadj->resize((size_t)words);
  return fetch(hadj->data(), adj_concat, (size_t)words * 8);
}

}  // namespace

extern "C" {

int tw_abi_version(void) { return TW_ABI_VERSION; }

const char* tw_strerror(int status) {
  switch (status) {
    case TW_OK: return "ok";
    case TW_ERR_INVALID: return "invalid argument (graph, n, k or a required pointer)";
    case TW_ERR_CAPACITY: return "frontier or table would exceed the memory cap; no answer given";
    case TW_ERR_TIMEOUT: return "a bounded device wait expired";
    case TW_ERR_CUDA: return "a CUDA runtime call failed";
    default: return "unknown status";
  }
}

int tw_create(tw_ctx** out, const tw_config* cfg) {
  if (out == nullptr) return TW_ERR_INVALID;
  *out = nullptr;
  tw_config cf{};
  if (cfg) cf = *cfg;
  for (int r : cf.reserved)
    if (r != 0) return TW_ERR_INVALID;
  if (cf.block_threads != 0 && cf.block_threads != 64 && cf.block_threads != 128 && cf.block_threads != 256)
    return TW_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cf.device < 0 || cf.device >= ndev) {
    cudaGetLastError();
    return TW_ERR_CUDA;
  }
  tw_ctx* c = new tw_ctx();
  c->device = cf.device;
  c->cfg = cf;
  auto fail = [&](int code) {
    tw_destroy(c);
    return code;
  };
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(TW_ERR_CUDA);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(TW_ERR_CUDA);
  const size_t dflt = std::min<size_t>(150ull << 30, (size_t)(0.9 * (double)free_b));
  c->mem_cap = cf.mem_cap_bytes ? cf.mem_cap_bytes : dflt;
  if (cf.stream) {
    c->stream = static_cast<cudaStream_t>(cf.stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(TW_ERR_CUDA);
    c->own_stream = true;
  }
  if (cudaMalloc(&c->small.ptr, kSmallBytes) != cudaSuccess) return fail(TW_ERR_CUDA);
  c->small.bytes = kSmallBytes;
  if (cudaMalloc(reinterpret_cast<void**>(&c->d_ctr), sizeof(LevelCounters)) != cudaSuccess) return fail(TW_ERR_CUDA);
  if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_ctr), sizeof(LevelCounters), cudaHostAllocDefault) != cudaSuccess)
    return fail(TW_ERR_CUDA);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return fail(TW_ERR_CUDA);
  if (cudaMalloc(reinterpret_cast<void**>(&c->d_gstate), sizeof(GraphState)) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&c->h_gstate), sizeof(GraphState), cudaHostAllocDefault) != cudaSuccess)
    return fail(TW_ERR_CUDA);
  *out = c;
  return TW_OK;
}

void tw_destroy(tw_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (DevBuf* b : {&c->keys, &c->pred, &c->table, &c->small, &c->scratch, &c->cand_key, &c->cand_v, &c->part_meta})
    if (b->ptr) cudaFree(b->ptr);
  if (c->d_ctr) cudaFree(c->d_ctr);
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  for (auto& e : c->graphs) cudaGraphExecDestroy(e.exec);
  if (c->d_gstate) cudaFree(c->d_gstate);
  if (c->h_gstate) cudaFreeHost(c->h_gstate);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
}

int tw_decide(tw_ctx* c, const uint64_t* adj, int n, int k, int* yes, int32_t* order, tw_stats* st) {
  if (!c || !yes || k < 0) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  HostGraph g;
  int rc = load_graph(adj, n, &g);
  if (rc) return rc;
  return decide_graph(c, g, k, yes, order, st);
}

int tw_decide_u32(tw_ctx* c, const uint32_t* adj_rows, int n, int k, int* yes, int32_t* order, tw_stats* st) {
  if (!c || !yes || !adj_rows || k < 0 || n < 1 || n > 32) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  std::vector<uint32_t> r32(n);
  int rc = fetch(r32.data(), adj_rows, (size_t)n * 4);
  if (rc) return rc;
  std::vector<uint64_t> r64(r32.begin(), r32.end());
  HostGraph g;
  rc = validate(r64.data(), n, &g);
  if (rc) return rc;
  return decide_graph(c, g, k, yes, order, st);
}

int tw_solve(tw_ctx* c, const uint64_t* adj, int n, int* tw, int32_t* order, int32_t* td_parent, uint64_t* td_bags,
             tw_stats* st) {
  if (!c || !tw) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  HostGraph g;
  int rc = load_graph(adj, n, &g);
  if (rc) return rc;
  return solve_graph(c, g, tw, order, td_parent, td_bags, st, 0);
}

int tw_bounds(tw_ctx* c, const uint64_t* adj, int n, int32_t out[4]) {
  if (!c || !out) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  HostGraph g;
  int rc = load_graph(adj, n, &g);
  if (rc) return rc;
  rc = upload_graph(c, g, key_class_for(g.n));
  if (rc) return rc;
  int32_t b[4];
  rc = bounds_graph(c, g, b);
  if (rc) return rc;
  return put(c, out, b, sizeof(b));
}

int tw_features_batch(tw_ctx* c, const uint64_t* adj_concat, const int32_t* n, const int64_t* row_offset,
                      int num_graphs, float* feats) {
  if (!c || !feats || num_graphs < 0) return TW_ERR_INVALID;
  if (num_graphs == 0) return TW_OK;
  TW_CK(cudaSetDevice(c->device));
  std::vector<int32_t> hn;
  std::vector<int64_t> hoff;
  std::vector<uint64_t> hadj;
  int rc = load_batch(adj_concat, n, row_offset, num_graphs, &hn, &hoff, &hadj);
  if (rc) return rc;
  for (int g = 0; g < num_graphs; ++g) {
    HostGraph tmp;
    rc = validate(hadj.data() + hoff[g], hn[g], &tmp);
    if (rc) return rc;
  }
  Stager S(c);
  const size_t fb = (size_t)num_graphs * 12 * 4;
  rc = S.reserve(pad256(hadj.size() * 8) + pad256(hn.size() * 4) + pad256(hoff.size() * 8) + pad256(fb) + 1024);
  if (rc) return rc;
  const void *d_adj, *d_n, *d_off;
  if ((rc = S.in(hadj.data(), hadj.size() * 8, &d_adj))) return rc;
  if ((rc = S.in(hn.data(), hn.size() * 4, &d_n))) return rc;
  if ((rc = S.in(hoff.data(), hoff.size() * 8, &d_off))) return rc;
  float* d_f = static_cast<float*>(S.take(fb));
  TW_CK(launch_bounds(static_cast<const unsigned long long*>(d_adj), static_cast<const int32_t*>(d_n),
                      static_cast<const int64_t*>(d_off), num_graphs, nullptr, d_f, c->stream));
  return put_from_device(c, feats, d_f, fb);
}

static const int kMlpParams = 32 * 12 + 32 + 32 + 1;

int tw_mlp_forward(tw_ctx* c, const float* params, const float* x, int batch, float* yhat) {
  if (!c || !params || !x || !yhat || batch < 0) return TW_ERR_INVALID;
  if (batch == 0) return TW_OK;
  TW_CK(cudaSetDevice(c->device));
  Stager S(c);
  int rc = S.reserve(pad256(kMlpParams * 4) + pad256((size_t)batch * 48) + pad256((size_t)batch * 4) + 1024);
  if (rc) return rc;
  const void *dp, *dx;
  if ((rc = S.in(params, kMlpParams * 4, &dp))) return rc;
  if ((rc = S.in(x, (size_t)batch * 48, &dx))) return rc;
  float* dy = static_cast<float*>(S.take((size_t)batch * 4));
  TW_CK(launch_mlp_forward(static_cast<const float*>(dp), static_cast<const float*>(dx), batch, dy, c->stream));
  return put_from_device(c, yhat, dy, (size_t)batch * 4);
}

int tw_mlp_grad(tw_ctx* c, const float* params, const float* x, const float* y, int batch, float* grad) {
  if (!c || !params || !x || !y || !grad || batch <= 0) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  const int blocks = std::max(1, std::min(c->sms * 2, (batch + 127) / 128));
  Stager S(c);
  int rc = S.reserve(pad256(kMlpParams * 4) * 2 + pad256((size_t)batch * 48) + pad256((size_t)batch * 4) +
                     pad256((size_t)blocks * kMlpParams * 4) + 1024);
  if (rc) return rc;
  const void *dp, *dx, *dyv;
  if ((rc = S.in(params, kMlpParams * 4, &dp))) return rc;
  if ((rc = S.in(x, (size_t)batch * 48, &dx))) return rc;
  if ((rc = S.in(y, (size_t)batch * 4, &dyv))) return rc;
  float* dg = static_cast<float*>(S.take(kMlpParams * 4));
  float* part = static_cast<float*>(S.take((size_t)blocks * kMlpParams * 4));
  TW_CK(launch_mlp_grad(static_cast<const float*>(dp), static_cast<const float*>(dx), static_cast<const float*>(dyv),
                        batch, dg, part, blocks, c->stream));
  return put_from_device(c, grad, dg, kMlpParams * 4);
}

int tw_mlp_adam(tw_ctx* c, float* params, const float* grad, float* m, float* v, int t, float lr, float beta1,
                float beta2, float eps) {
  if (!c || !params || !grad || !m || !v || t < 1) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  Stager S(c);
  int rc = S.reserve(pad256(kMlpParams * 4) * 4 + 1024);
  if (rc) return rc;
  const void *dp, *dg, *dm, *dv;
  if ((rc = S.in(params, kMlpParams * 4, &dp))) return rc;
  if ((rc = S.in(grad, kMlpParams * 4, &dg))) return rc;
  if ((rc = S.in(m, kMlpParams * 4, &dm))) return rc;
  if ((rc = S.in(v, kMlpParams * 4, &dv))) return rc;
  TW_CK(launch_mlp_adam(const_cast<float*>(static_cast<const float*>(dp)), static_cast<const float*>(dg),
                        const_cast<float*>(static_cast<const float*>(dm)), const_cast<float*>(static_cast<const float*>(dv)),
                        t, lr, beta1, beta2, eps, c->stream));
  if (dp != params && (rc = put_from_device(c, params, dp, kMlpParams * 4))) return rc;
  if (dm != m && (rc = put_from_device(c, m, dm, kMlpParams * 4))) return rc;
  if (dv != v && (rc = put_from_device(c, v, dv, kMlpParams * 4))) return rc;
  TW_CK(cudaStreamSynchronize(c->stream));
  return TW_OK;
}

int tw_mlp_train(tw_ctx* c, float* params, const float* x, const float* y, int batch_total, int minibatch, int epochs,
                 const int32_t* perm, float lr, float* loss_out) {
  if (!c || !params || !x || !y || !perm || batch_total <= 0 || minibatch <= 0 || epochs <= 0) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  const size_t pb = (size_t)epochs * batch_total * 4;
  {
    std::vector<int32_t> hp((size_t)epochs * batch_total);
    int r = fetch(hp.data(), perm, pb);
    if (r) return r;
    for (int32_t i : hp)
      if (i < 0 || i >= batch_total) return TW_ERR_INVALID;
  }
  Stager S(c);
  int rc = S.reserve(pad256(kMlpParams * 4) * 3 + pad256((size_t)batch_total * 48) + pad256((size_t)batch_total * 4) +
                     pad256(pb) + pad256((size_t)epochs * 4) + 2048);
  if (rc) return rc;
  const void *dp, *dx, *dy, *dperm;
  if ((rc = S.in(params, kMlpParams * 4, &dp))) return rc;
  if ((rc = S.in(x, (size_t)batch_total * 48, &dx))) return rc;
  if ((rc = S.in(y, (size_t)batch_total * 4, &dy))) return rc;
  if ((rc = S.in(perm, pb, &dperm))) return rc;
  float* dm = static_cast<float*>(S.take(kMlpParams * 4));
  float* dv = static_cast<float*>(S.take(kMlpParams * 4));
  float* dl = static_cast<float*>(S.take((size_t)epochs * 4));
  TW_CK(cudaMemsetAsync(dm, 0, kMlpParams * 4, c->stream));
  TW_CK(cudaMemsetAsync(dv, 0, kMlpParams * 4, c->stream));
  TW_CK(launch_mlp_train(const_cast<float*>(static_cast<const float*>(dp)), dm, dv, static_cast<const float*>(dx),
                         static_cast<const float*>(dy), batch_total, minibatch, epochs,
                         static_cast<const int32_t*>(dperm), lr, dl, c->stream));
  if (dp != params && (rc = put_from_device(c, params, dp, kMlpParams * 4))) return rc;
  if (loss_out && (rc = put_from_device(c, loss_out, dl, (size_t)epochs * 4))) return rc;
  TW_CK(cudaStreamSynchronize(c->stream));
  return TW_OK;
}

int tw_solve_batch(tw_ctx* c, const uint64_t* adj_concat, const int32_t* n, const int64_t* row_offset,
                   int num_graphs, int* tw, int32_t* orders, int* status, const float* k_hint, tw_stats* st) {
  if (!c || !tw || !status || num_graphs < 0) return TW_ERR_INVALID;
  Timer t;
  TW_CK(cudaSetDevice(c->device));
  std::vector<int32_t> hn;
  std::vector<int64_t> hoff;
  std::vector<uint64_t> hadj;
  int rc = load_batch(adj_concat, n, row_offset, num_graphs, &hn, &hoff, &hadj);
  if (rc) return rc;
  std::vector<float> hint;
  if (k_hint) {
    hint.resize(num_graphs);
    if ((rc = fetch(hint.data(), k_hint, (size_t)num_graphs * 4))) return rc;
  }
  const int G = num_graphs;
  std::vector<HostGraph> graphs(G);
  std::vector<int> hst(G, TW_OK), valid;
  std::vector<int> htw(G, -1);
  std::vector<int64_t> order_off(G, 0);
  int64_t total_n = 0;
  for (int g = 0; g < G; ++g) {
    order_off[g] = total_n;
    total_n += hn[g];
    hst[g] = validate(hadj.data() + hoff[g], hn[g], &graphs[g]);
    if (hst[g] == TW_OK) valid.push_back(g);
  }
  std::vector<int32_t> hord(orders ? (size_t)total_n : 0, -1);
  if (st) std::memset(st, 0, sizeof(*st));
  const unsigned long long launches0 = c->launches;
  rc = solve_batch_gpu(c, graphs, valid, k_hint ? &hint : nullptr, order_off, htw.data(), orders ? &hord : nullptr,
                       &hst, st);
  if (rc) return rc;
  int worst = TW_OK;
  for (int g = 0; g < G; ++g) worst = std::max(worst, hst[g]);
  if ((rc = put(c, tw, htw.data(), (size_t)G * sizeof(int)))) return rc;
  if ((rc = put(c, status, hst.data(), (size_t)G * sizeof(int)))) return rc;
  if (orders && (rc = put(c, orders, hord.data(), hord.size() * 4))) return rc;
  if (st) {
    st->seconds = t.seconds();
    st->kernel_launches = c->launches - launches0;
  }
  return worst;
}

}  // extern "C"
