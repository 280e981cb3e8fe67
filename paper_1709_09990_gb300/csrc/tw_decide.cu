// Host drivers of libtw: decide(k), the k sweep, reconstruction.
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
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tw_host.h"

namespace tw {
namespace host {

// Table size above which a level takes the partitioned insert: by default
// tables of more than 256 MB (about twice the L2), where the direct kernel's
// compare-and-swaps go to DRAM.
unsigned long long partition_threshold_bytes(const tw_ctx* c) {
  if (c->cfg.partition_table_mb == -2) return 0ull;
  if (c->cfg.partition_table_mb < 0) return ~0ull;
  if (c->cfg.partition_table_mb == 0) return 256ull << 20;
  return (unsigned long long)c->cfg.partition_table_mb << 20;
}

// One level through the partitioned insert (emit, then insert range by
// range); the caller has zeroed the counters but not the table.  When the
// whole level is emitted in one chunk, each range's slice of the table
// (plus the slots its probes can run into) is emptied just before the
// range's inserts and dropped from L2 afterwards without a write-back, so
// the table never travels to DRAM; with several chunks the whole table is
// emptied first and kept.  *fallback is set when a region overflowed (the
// caller then runs the direct kernel on a freshly cleared table).
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
  const bool one_chunk = chunk >= a.n_in;
  if (!one_chunk) TW_LAUNCH(c, launch_clear(a.table, (size_t)((a.table_slots * kw + 15) & ~15ull), nullptr, c->stream));
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
    if (!one_chunk) {
      TW_LAUNCH(c, launch_insert_ranges(ca, pb, 0, prefix[P], c->stream));
      continue;
    }
    // range r's home slots are [r S / P, (r+1) S / P); its probes may run up
    // to max_probes slots further (wrapping at the end of the table)
    const unsigned long long S = a.table_slots;
    for (int r = 0; r < P; ++r) {
      const unsigned long long s_lo = (unsigned long long)(((unsigned __int128)S * r) / P);
      const unsigned long long s_hi = (unsigned long long)(((unsigned __int128)S * (r + 1)) / P);
      const unsigned long long span = std::min<unsigned long long>(S, s_hi - s_lo + (unsigned long long)a.max_probes);
      TW_LAUNCH(c, launch_clear_slots(a.kc, a.table, s_lo, span, S, c->stream));
      TW_LAUNCH(c, launch_insert_ranges(ca, pb, prefix[r], prefix[r + 1], c->stream));
      TW_LAUNCH(c, launch_discard_l2(a.table, s_lo * kw, s_hi * kw, c->stream));
    }
  }
  return TW_OK;
}

// ---- out-of-core levels (tw_config.out_of_core) ------------------------------
//
// A decide run without ordering keeps only two levels: the one being expanded
// and the one being built.  When they and the level's hash table would not
// fit the memory cap, the run goes on here:
//  * a level may be split: a device part (in one of two device buffers) and a
//    host part (in one of two pinned, device-mapped host buffers, Grace memory
//    on GB300, read and written by the kernels over NVLink-C2C).  The new
//    level fills the host buffer the input does not use first, up to the host
//    limit, and the rest goes to the device, so that the device keeps as much
//    room as possible for the table;
//  * the level's table is split into P hash ranges: each pass empties a slice
//    that fits what the cap leaves, expands the whole input level (each of its
//    parts) and inserts only the pairs whose hash falls in its range (the
//    ranged kernel), so the passes together insert every pair once.  A pass
//    writes its new sets to the host part while that has room for it, else to
//    the device part; a pass whose output overflows its part is redone on its
//    own into the other part.
// Level sets, sizes and counters are those of the in-memory run; the input is
// read and searched once per pass.

// Pinned host bytes that out-of-core levels may occupy.
size_t ooc_host_limit(const tw_ctx* c) {
  if (c->cfg.host_cap_mb > 0) return (size_t)c->cfg.host_cap_mb << 20;
  const size_t phys = (size_t)sysconf(_SC_PHYS_PAGES) * (size_t)sysconf(_SC_PAGESIZE);
  return phys / 20 * 17;
}

// Frees host buffer hb (its level is no longer needed).
void release_host(tw_ctx* c, int hb) {
  tw_ctx::HostChunk& ch = c->ooc_host[hb];
  if (!ch.ptr) return;
  cudaStreamSynchronize(c->stream);
  cudaFreeHost(ch.ptr);
  ch = {nullptr, nullptr, 0};
}

// Host buffer hb of the context, grown to at least bytes (whole MiB); *dptr
// is its device-side address.  Both buffers together stay within the host
// limit.
int ooc_host_buffer(tw_ctx* c, int hb, size_t bytes, char** dptr) {
  tw_ctx::HostChunk& ch = c->ooc_host[hb];
  if (ch.bytes < bytes) {
    const size_t mib = size_t(1) << 20;
    const size_t want = (bytes + mib - 1) / mib * mib;
    if (want + c->ooc_host[1 - hb].bytes > ooc_host_limit(c)) return TW_ERR_CAPACITY;
    release_host(c, hb);
    void* p = nullptr;
    if (cudaHostAlloc(&p, want, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return TW_ERR_CAPACITY;
    }
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(p);
      return TW_ERR_CUDA;
    }
    ch = {static_cast<char*>(p), static_cast<char*>(d), want};
  }
  *dptr = ch.dptr;
  return TW_OK;
}

void release(tw_ctx* c, DevBuf* b) {
  if (!b->ptr) return;
  cudaStreamSynchronize(c->stream);
  cudaFree(b->ptr);
  b->ptr = nullptr;
  b->bytes = 0;
}

// Allocates b with exactly bytes (rounded up to 256); false when the cap or
// the device refuses.
bool alloc_exact(tw_ctx* c, DevBuf* b, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (total_bytes(c) - b->bytes + bytes > c->mem_cap) return false;
  release(c, b);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b->ptr = p;
  b->bytes = bytes;
  return true;
}

// Where one out-of-core level lives: dcount keys in device buffer db from
// offset off, then hcount keys at the start of host buffer hb.
struct OocLevel {
  int db = 0;
  unsigned long long off = 0, dcount = 0;
  int hb = -1;
  unsigned long long hcount = 0;
};

// Continues decide(k) out of core from the last level of R (on the device in
// the level arena at its offset).  stop_level as in run_decide.
int run_decide_ooc(tw_ctx* c, KeyClass kc, int n, int k, DecideResult* R, int stop_level) {
  NvtxRange range("tw decide out of core n=%d k=%d", n, k);
  const size_t w = key_bytes(kc);
  SmallLayout L;
  release(c, &c->pred);
  release(c, &c->cand_key);
  release(c, &c->cand_v);
  DevBuf* dev[2] = {&c->keys, &c->ooc_keys};
  const int load_pct = c->cfg.table_load_pct > 0 ? std::min(90, c->cfg.table_load_pct) : 75;
  const int max_probes = c->cfg.max_probes > 0 ? c->cfg.max_probes : 256;
  const size_t margin = std::min<size_t>(64ull << 20, c->mem_cap / 16);
  const size_t host_limit = ooc_host_limit(c);
  const bool timed = c->cfg.time_kernels != 0;
  OocLevel in;
  in.off = R->levels.back().off;
  in.dcount = R->levels.back().count;
  for (int i = (int)R->levels.size() - 1; i <= n - k - 2; ++i) {
    if (stop_level >= 0 && i >= stop_level) break;
    const unsigned long long cur_count = R->levels[i].count;
    if (cur_count == 0) break;
    // size estimate of the new level: the last growth ratio, lowered by half
    // of its last fall (geometric mean) while the ratios fall
    const double bound = std::min((double)cur_count * (double)(n - i), binom(n, i + 1)) + 1.0;
    double est = (double)cur_count;
    if (i > 0 && R->levels[i - 1].count > 0) {
      double r = (double)cur_count / (double)R->levels[i - 1].count;
      if (i > 1 && R->levels[i - 2].count > 0) {
        const double r_prev = (double)R->levels[i - 1].count / (double)R->levels[i - 2].count;
        if (r < r_prev) r *= std::sqrt(std::max(0.25, r / r_prev));
      }
      r = std::min(std::max(r, 0.25), (double)(n - i));
      est = (double)cur_count * r;
    }
    double out_est = std::min(bound, est * 1.04 + 4096.0);
    // the parts of the input
    const char* in_part[2] = {
        in.dcount ? static_cast<const char*>(dev[in.db]->ptr) + in.off * w : nullptr,
        in.hcount ? c->ooc_host[in.hb].dptr : nullptr};
    const unsigned long long in_cnt[2] = {in.dcount, in.hcount};
    // buffers the new level may use: those the input does not hold
    const int od = in.dcount ? 1 - in.db : 0;
    if (!in.dcount) release(c, dev[1]);
    const int oh = in.hcount ? 1 - in.hb : (c->ooc_host[1].bytes > c->ooc_host[0].bytes ? 1 : 0);
    if (!in.hcount) release_host(c, 1 - oh);
    OocLevel nxt;
    unsigned long long generated = 0, launches = 0;
    float ms_total = 0.f;
    for (int attempt = 0;; ++attempt) {
      if (attempt > 16) return TW_ERR_CAPACITY;
      if (attempt > 0) ++R->retries;
      const unsigned long long out_cap = (unsigned long long)std::ceil(out_est);
      release(c, &c->table);
      release(c, dev[od]);
      const unsigned long long total_slots =
          std::max<unsigned long long>(1024ull, (unsigned long long)std::ceil(out_est * 100.0 / load_pct));
      const size_t table_bytes = (size_t)total_slots * w;
      const size_t small_slice = std::max<size_t>(std::min<size_t>(256ull << 20, c->mem_cap / 8), table_bytes / 512);
      if (total_bytes(c) + margin + small_slice > c->mem_cap) return TW_ERR_CAPACITY;
      const size_t dev_room = c->mem_cap - total_bytes(c) - margin;
      // placement: all on the device when the level and its whole table fit
      // there; else as much of it as the host limit allows in host memory
      unsigned long long cap_part[2] = {out_cap, 0};
      if ((size_t)out_cap * w + table_bytes + 16384 > dev_room) {
        const size_t in_host_bytes = in.hcount ? c->ooc_host[in.hb].bytes : 0;
        const size_t host_room = host_limit > in_host_bytes ? (host_limit - in_host_bytes) & ~((size_t(1) << 20) - 1) : 0;
        // (the host part also takes up to 10% more than the estimate, which
        // costs the device nothing)
        const unsigned long long on_host = std::min<unsigned long long>(out_cap, host_room / w);
        cap_part[0] = out_cap - on_host;
        cap_part[1] = std::min<unsigned long long>(host_room / w, on_host + out_cap / 10);
        if ((size_t)cap_part[0] * w + small_slice > dev_room) return TW_ERR_CAPACITY;
      }
      char* out_part[2] = {nullptr, nullptr};
      if (cap_part[0]) {
        if (!alloc_exact(c, dev[od], (size_t)cap_part[0] * w)) return TW_ERR_CAPACITY;
        out_part[0] = static_cast<char*>(dev[od]->ptr);
      }
      if (cap_part[1]) {
        int rc = ooc_host_buffer(c, oh, (size_t)cap_part[1] * w, &out_part[1]);
        if (rc) return rc;
      }
      // the table: as many hash-range passes as the cap needs
      if (total_bytes(c) + margin + 16384 > c->mem_cap) return TW_ERR_CAPACITY;
      const size_t slice_budget = c->mem_cap - total_bytes(c) - margin;
      unsigned long long P = std::max<unsigned long long>(1ull, (table_bytes + slice_budget - 1) / slice_budget);
      unsigned long long slice_slots = 0;
      size_t slice_bytes = 0;
      for (;; P *= 2) {  // (more, smaller slices when the device refuses one)
        if (P > 1024) return TW_ERR_CAPACITY;
        slice_slots = (total_slots + P - 1) / P + 1024ull;
        slice_bytes = (size_t)((slice_slots * w + 15) & ~15ull);
        if (alloc_exact(c, &c->table, slice_bytes)) break;
      }
      // the passes append to one list that fills the device part first and
      // goes on in the host part (the ranged kernel's split output)
      char* out_first = cap_part[0] ? out_part[0] : out_part[1];
      char* out_tail = cap_part[0] && cap_part[1] ? out_part[1] : nullptr;
      TW_CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(LevelCounters), c->stream));
      LevelCounters h{};
      bool replan = false;
      ms_total = 0.f;
      launches = 0;
      for (unsigned long long r = 0; r < P; ++r) {
        const unsigned long long before = h.out_count;
        TW_LAUNCH(c, launch_clear(c->table.ptr, slice_bytes, nullptr, c->stream));
        if (timed) TW_CK(cudaEventRecord(c->ev0, c->stream));
        for (int ip = 0; ip < 2; ++ip) {
          if (!in_cnt[ip]) continue;
          ExpandLaunch a;
          a.kc = kc;
          a.in_keys = in_part[ip];
          a.n_in = in_cnt[ip];
          a.adj = small_at(c, L.adj);
          a.n = n;
          a.k = k;
          a.table = c->table.ptr;
          a.table_slots = slice_slots;
          a.max_probes = max_probes;
          a.out_keys = out_first;
          a.out_pred = nullptr;
          a.out_cap = cap_part[0] + cap_part[1];
          a.out_tail = out_tail;
          a.out_split = cap_part[0];
          a.ctr = c->d_ctr;
          a.block_threads = 128;
          a.grid = 0;
          a.allowed[0] = c->allowed[0];
          a.allowed[1] = c->allowed[1];
          a.mmw = 0;
          a.ranges = P;
          a.range = r;
          TW_LAUNCH(c, launch_expand(a, c->stream));
          ++launches;
        }
        if (timed) TW_CK(cudaEventRecord(c->ev1, c->stream));
        TW_CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, c->stream));
        TW_CK(cudaStreamSynchronize(c->stream));
        h = *c->h_ctr;
        if (timed) {
          float ms = 0.f;
          TW_CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
          ms_total += ms;
        }
        const unsigned long long got = h.out_count - before;
        if ((h.overflow & 2u) || got * 100ull > slice_slots * 90ull) {
          // this range held more than its slice: more states than estimated
          const double projected = (double)h.out_count / (double)(r + 1) * (double)P;
          out_est = std::max(out_est * 1.25, projected * 1.1);
          replan = true;
          break;
        }
      }
      // more new sets than the two parts hold: every range was inserted
      // completely, so the count is exact
      if (!replan && (h.overflow & 1u)) {
        out_est = (double)h.out_count * 1.01 + 1024.0;
        replan = true;
      }
      if (replan) continue;
      nxt.db = od;
      nxt.off = 0;
      nxt.dcount = std::min<unsigned long long>(h.out_count, cap_part[0]);
      nxt.hb = oh;
      nxt.hcount = h.out_count - nxt.dcount;
      generated = h.generated;
      R->peak_bytes = std::max<unsigned long long>(R->peak_bytes, total_bytes(c));
      break;
    }
    const unsigned long long nxt_count = nxt.dcount + nxt.hcount;
    R->states_expanded += cur_count;
    R->candidates += cur_count * (unsigned long long)(n - c->skipped - i);
    R->generated += generated;
    R->expand_launches += launches;
    R->expand_seconds += (double)ms_total * 1e-3;
    R->expand_bytes += (double)(cur_count + generated + 2ull * nxt_count) * (double)w;
    LevelRec rec;
    rec.off = 0;
    rec.count = nxt_count;
    if (nxt.dcount == 0 && nxt.hcount > 0) {
      rec.hkeys = c->ooc_host[nxt.hb].dptr;
    } else if (nxt.hcount > 0) {
      rec.htail = c->ooc_host[nxt.hb].dptr;
      rec.tail = nxt.hcount;
    }
    R->levels.push_back(rec);
    if (c->cfg.fingerprints) {
      TW_CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(LevelCounters), c->stream));
      if (nxt.dcount) TW_LAUNCH(c, launch_fingerprint(kc, dev[nxt.db]->ptr, nxt.dcount, c->d_ctr, c->stream));
      if (nxt.hcount)
        TW_LAUNCH(c, launch_fingerprint(kc, c->ooc_host[nxt.hb].dptr, nxt.hcount, c->d_ctr, c->stream));
      TW_CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      R->fp_sum.push_back(c->h_ctr->fp_sum);
      R->fp_xor.push_back(c->h_ctr->fp_xor);
    }
    // the input's buffers are free now; drop an empty device part's buffer
    in = nxt;
    if (!in.dcount) release(c, dev[in.db]);
    if (nxt_count == 0) break;
  }
  const int last = (int)R->levels.size() - 1;
  R->yes = (last == n - k - 1 && R->levels[last].count > 0) ? 1 : 0;
  // device level records refer to the level arena (callers read the last
  // level only): make the buffer that holds the last level's device part the
  // arena
  if (in.dcount && in.db == 1) std::swap(c->keys, c->ooc_keys);
  return TW_OK;
}

// One run of Listing 1 at bound k on the graph already uploaded.  With
// stop_level >= 0 the run ends once that level is built (its answer is then
// only meaningful when the run reached level n-k-1).
int run_decide(tw_ctx* c, KeyClass kc, int n, int k, bool keep_levels, DecideResult* R, int stop_level) {
  const size_t w = key_bytes(kc);
  // With spill_levels the finished levels go to pinned host memory and the
  // device arena only alternates between the input and the output level.
  const bool spill = keep_levels && c->cfg.spill_levels != 0;
  // levels or tables beyond the cap continue out of core (no ordering only)
  const bool ooc = c->cfg.out_of_core != 0 && !keep_levels && !spill && !c->cfg.mmw_prune;
  if (spill) {
    c->host_chunk = 0;
    c->host_used = 0;
    keep_levels = false;
  }
  SmallLayout L;
  R->levels.clear();
  R->yes = 0;
  R->states_expanded = R->candidates = R->generated = R->peak_bytes = R->retries = 0;
  R->expand_launches = 0;
  R->expand_seconds = R->expand_bytes = 0.0;
  R->fp_sum.assign(1, 0ull);  // fp of the empty set is 0
  R->fp_xor.assign(1, 0ull);
  int rc = grow(c, &c->keys, 64 * w, 0);
  if (rc == TW_OK) rc = grow(c, &c->pred, 64, 0);
  if (rc == TW_ERR_CAPACITY) {
    // the buffers of an earlier run fill the cap: its table and its second
    // level buffer are scratch now
    release(c, &c->table);
    release(c, &c->ooc_keys);
    rc = grow(c, &c->keys, 64 * w, 0);
    if (rc == TW_OK) rc = grow(c, &c->pred, 64, 0);
  }
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
  double gen_per_state = 0.0;          // generated pairs per input state of the last level
  for (int i = 0; i <= n - k - 2; ++i) {
    if (stop_level >= 0 && i >= stop_level) break;
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
    // More than 90% of the slots filled re-runs the level with a larger table,
    // so the output never needs more room than that.
    out_cap = std::min(out_cap, slots / 10ull * 9ull + 64ull);
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
      if (rc == TW_OK) rc = grow(c, &c->keys, (size_t)(off + out_cap) * w, (size_t)live_end * w);
      if (rc == TW_OK) rc = grow(c, &c->pred, (size_t)(off + out_cap), (size_t)live_end);
      if (rc == TW_ERR_CAPACITY && ooc) return run_decide_ooc(c, kc, n, k, R, stop_level);
      if (rc) return rc;
      // (the partitioned insert empties the table itself, range by range)
      const bool partitioned = (unsigned long long)table_bytes > partition_threshold_bytes(c);
      if (partitioned)
        TW_CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(LevelCounters), c->stream));
      else
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
      if (partitioned) {
        bool fallback = false;
        // Regions are sized by the pairs per state of the previous level
        // (with slack), not by the n-i candidates: with canonical parents a
        // state submits a few pairs, and oversized regions would split the
        // level into many passes over the table.  A region that still
        // overflows sends the level to the direct kernel.
        const int cand_bound = n - c->skipped - i;
        const int cand_est = gen_per_state > 0.0
                                 ? std::min(cand_bound, (int)std::ceil(gen_per_state * 2.0) + 2)
                                 : cand_bound;
        rc = run_level_partitioned(c, a, cand_est, &fallback);
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
      R->generated += h.generated;
      gen_per_state = cur.count ? (double)h.generated / (double)cur.count : 0.0;
      R->expand_launches += 1;
      R->expand_seconds += (double)ms * 1e-3;
      R->expand_bytes += (double)(cur.count + h.generated + 2ull * h.out_count) * (double)w + (double)h.out_count;
      const unsigned long long live_states = keep_levels ? kept_states + nxt.count : cur.count + nxt.count;
      R->peak_bytes = std::max<unsigned long long>(R->peak_bytes, live_states * (w + 1) + slots * w);
      break;
    }
    R->states_expanded += cur.count;
    R->candidates += cur.count * (unsigned long long)(n - c->skipped - i);
    if (keep_levels) kept_states += nxt.count;
    R->levels.push_back(nxt);
    if (spill && nxt.count > 0) {
      char* hk = nullptr;
      char* hp = nullptr;
      rc = host_take(c, (size_t)nxt.count * w, &hk);
      if (rc) return rc;
      rc = host_take(c, (size_t)nxt.count, &hp);
      if (rc) return rc;
      TW_CK(cudaMemcpyAsync(hk, static_cast<char*>(c->keys.ptr) + nxt.off * w, (size_t)nxt.count * w,
                            cudaMemcpyDefault, c->stream));
      TW_CK(cudaMemcpyAsync(hp, static_cast<uint8_t*>(c->pred.ptr) + nxt.off, (size_t)nxt.count, cudaMemcpyDefault,
                            c->stream));
      R->levels.back().hkeys = hk;
      R->levels.back().hpred = reinterpret_cast<const uint8_t*>(hp);
    }
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
  const bool timed = c->cfg.time_kernels != 0;
  tw_ctx::GraphEntry* e = nullptr;
  for (auto& g : c->graphs)
    if (g.kc == (int)kc && g.n == n && g.k == k && g.load == load_pct && g.probes == max_probes &&
        g.bt == c->cfg.block_threads && g.allowed0 == c->allowed[0] && g.allowed1 == c->allowed[1] &&
        g.keys == c->keys.ptr && g.pred == c->pred.ptr && g.table == c->table.ptr && g.arena_cap == arena_cap &&
        g.table_cap == table_cap && g.ev.empty() == !timed)
      e = &g;
  if (e == nullptr) {
    if (c->graphs.size() >= 32) {
      TW_CK(cudaStreamSynchronize(c->stream));
      for (auto& g : c->graphs) {
        cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t v : g.ev) cudaEventDestroy(v);
      }
      c->graphs.clear();
    }
    // With time_kernels every level's expand launch is bracketed by two
    // event-record nodes, read after the replay.
    std::vector<cudaEvent_t> ev;
    if (timed) {
      ev.resize(2 * (size_t)(n - k - 1), nullptr);
      for (cudaEvent_t& v : ev)
        if (cudaEventCreate(&v) != cudaSuccess) {
          cudaGetLastError();
          for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
          return TW_ERR_CUDA;
        }
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
      if (err == cudaSuccess && timed) err = cudaEventRecordWithFlags(ev[2 * i], c->stream, cudaEventRecordExternal);
      if (err == cudaSuccess) err = launch_graph_expand(c->d_gstate, a, c->stream);
      if (err == cudaSuccess && timed)
        err = cudaEventRecordWithFlags(ev[2 * i + 1], c->stream, cudaEventRecordExternal);
      if (err == cudaSuccess)
        err = launch_graph_plan(c->d_gstate, c->d_ctr, arena_cap, table_cap, partition_threshold_bytes(c), n, k,
                                load_pct, w, 0, c->stream);
      nodes += 3;
    }
    const cudaError_t end = cudaStreamEndCapture(c->stream, &graph);
    auto drop_events = [&]() {
      for (cudaEvent_t x : ev) cudaEventDestroy(x);
    };
    if (err != cudaSuccess || end != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      drop_events();
      return TW_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t inst = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
      cudaGetLastError();
      drop_events();
      return TW_ERR_CUDA;
    }
    c->graphs.push_back({(int)kc, n, k, load_pct, max_probes, c->cfg.block_threads, c->allowed[0], c->allowed[1],
                         c->keys.ptr, c->pred.ptr, c->table.ptr, arena_cap, table_cap, exec, nodes, ev});
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
  R->generated = h.generated;
  R->expand_bytes += (double)h.generated * (double)w;
  R->expand_launches = (unsigned long long)h.cur;
  if (!e->ev.empty())
    for (int j = 0; j < h.cur; ++j) {
      float ms = 0.f;
      TW_CK(cudaEventElapsedTime(&ms, e->ev[2 * j], e->ev[2 * j + 1]));
      R->expand_seconds += (double)ms * 1e-3;
    }
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
  if (c->cfg.spill_levels || c->cfg.graph_levels < 0) return false;
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
  R->states_expanded = R->candidates = R->generated = R->retries = 0;
  R->expand_launches = 0;
  R->expand_seconds = R->expand_bytes = 0.0;
  R->peak_bytes = 0;
  R->fp_sum.assign(1, 0ull);
  R->fp_xor.assign(1, 0ull);
}

// decide(k): the graph-driven loop when enabled, else (or when it gives up)
// the host loop.
int run_decide_any(tw_ctx* c, KeyClass kc, int n, int k, bool keep_levels, DecideResult* R) {
  NvtxRange range("tw decide n=%d k=%d", n, k);
  if (graph_mode(c)) {
    bool bailed = true;
    int rc = run_decide_graph(c, kc, n, k, R, &bailed);
    if (rc) return rc;
    if (!bailed) return TW_OK;
  }
  return run_decide(c, kc, n, k, keep_levels, R, -1);
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

// ---- fused small solve (tw_fused.cu) -----------------------------------------
void fill_stats(const DecideResult& R, int k, tw_stats* st, bool reset_totals);

unsigned long long graph_hash(const HostGraph& g) {
  unsigned long long h = 0x9e3779b97f4a7c15ull ^ (unsigned long long)g.n;
  for (uint64_t r : g.rows) {
    h ^= r + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h *= 0xff51afd7ed558ccdull;
  }
  return h;
}

bool fused_eligible(const tw_ctx* c, const HostGraph& g) {
  if (g.n > 64 || c->cfg.fused_states < 0 || c->cfg.clique_skip || c->cfg.disjoint_paths || c->cfg.mmw_prune ||
      c->cfg.spill_levels)
    return false;
  const unsigned long long h = graph_hash(g);
  for (unsigned long long x : c->fused_skip)
    if (x == h) return false;
  return true;
}

// decide(k) for k = k0 .. k_last in one fused launch on the graph already
// uploaded.  *status: 1 = finished - R describes the last run (the yes run
// when *answer_k >= 0, with the ordering and tree decomposition in the small
// buffer); 2 = gave up at k = *bail_k (the runs before it answered no), and
// the graph is remembered so that later solves skip the fused attempt; 0 =
// not run (its buffers do not fit the memory cap).
// Totals of every run go into st.
int run_fused(tw_ctx* c, const HostGraph& g, KeyClass kc, int k0, int k_last, DecideResult* R, int* status,
              int* answer_k, int* bail_k, tw_stats* st, const int32_t* lb_dev) {
  NvtxRange range("tw fused solve n=%d k0=%d", g.n, k0);
  const size_t w = key_bytes(kc);
  // decide runs in flight at once: k0, k0+1, k0+2 (the sweep from a lower
  // bound usually ends within a few k)
  constexpr int kGroups = 3;
  static_assert(kGroups <= kFusedMaxGroups, "the fused launch holds at most kFusedMaxGroups groups");
  const int G = std::max(1, std::min(kGroups, k_last - k0 + 1));
  const unsigned long long A =
      c->cfg.fused_states > 0 ? (unsigned long long)c->cfg.fused_states : (1ull << 20);
  const unsigned long long T = 2 * A + 1024;
  const size_t st_bytes = (sizeof(FusedState) + 255) & ~size_t(255);
  const size_t tb = ((size_t)T * 8 + 255) & ~size_t(255);  // sized for 64-bit states
  const size_t kb = ((size_t)A * 8 + 255) & ~size_t(255);
  const size_t pb = ((size_t)A + 255) & ~size_t(255);
  const size_t group_bytes = st_bytes + 2 * tb + kb + pb;
  const size_t need = (size_t)kGroups * group_bytes;
  *status = 0;
  if (c->fused.bytes < need) {
    c->fused_clean = false;
    int rc = grow(c, &c->fused, need, 0);
    if (rc == TW_ERR_CAPACITY) return TW_OK;  // no room under the cap: the level loop runs instead
    if (rc) return rc;
  }
  if (!c->h_fused) {
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_fused), kFusedMaxGroups * sizeof(FusedState),
                      cudaHostAllocDefault) != cudaSuccess) {
      c->h_fused = nullptr;
      cudaGetLastError();
      return TW_ERR_CUDA;
    }
  }
  char* base = static_cast<char*>(c->fused.ptr);
  SmallLayout L;
  FusedLaunch f;
  f.kc = kc;
  f.adj = small_at(c, L.adj);
  f.adj64 = reinterpret_cast<const unsigned long long*>(small_at(c, L.adj64));
  f.n = g.n;
  f.words64 = g.words;
  f.k0 = k0;
  f.k_last = k_last;
  f.max_probes = c->cfg.max_probes > 0 ? c->cfg.max_probes : 256;
  f.load_pct = c->cfg.table_load_pct > 0 ? std::min(90, c->cfg.table_load_pct) : 50;
  f.groups = G;
  f.lb_dev = lb_dev;
  for (int j = 0; j < kFusedMaxGroups; ++j) {
    char* gbase = base + (size_t)std::min(j, kGroups - 1) * group_bytes;
    f.st[j] = reinterpret_cast<FusedState*>(gbase);
    f.table0[j] = gbase + st_bytes;
    f.table1[j] = gbase + st_bytes + tb;
    f.keys[j] = gbase + st_bytes + 2 * tb;
    f.pred[j] = reinterpret_cast<uint8_t*>(gbase + st_bytes + 2 * tb + kb);
  }
  f.arena_cap = A;
  f.table_cap = T;
  f.order = reinterpret_cast<int32_t*>(small_at(c, L.order));
  f.parent = reinterpret_cast<int32_t*>(small_at(c, L.parent));
  f.bags = reinterpret_cast<unsigned long long*>(small_at(c, L.bags));
  if (!c->fused_clean) {
    // a new buffer, or one a launch left early: empty every group's tables
    // (all ones) once; launches that run to their end leave them empty
    for (int j = 0; j < kGroups; ++j) TW_CK(cudaMemsetAsync(f.table0[j], 0xff, 2 * tb, c->stream));
    c->fused_clean = true;
  }
  f.tables_clean = 1;
  for (int j = 0; j < G; ++j) TW_CK(cudaMemsetAsync(f.st[j], 0, sizeof(FusedState), c->stream));
  const bool timed = c->cfg.time_kernels != 0;
  if (timed) TW_CK(cudaEventRecord(c->ev0, c->stream));
  TW_LAUNCH(c, launch_fused_solve(f, c->stream));
  if (timed) TW_CK(cudaEventRecord(c->ev1, c->stream));
  TW_CK(cudaMemcpyAsync(c->h_fused, f.st[0], sizeof(FusedState), cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  const FusedState& h = *c->h_fused;
  c->fused_clean = h.error == 0u;  // a launch that ran to its end empties the tables it used
  if (h.error) return TW_ERR_TIMEOUT;  // a barrier wait gave up
  *status = h.status;
  k0 = h.k_start;  // (raised by the device lower bounds when given)
  if (h.status != 1) {
    *bail_k = h.last;
    if (c->fused_skip.size() >= 4096) c->fused_skip.clear();
    c->fused_skip.push_back(graph_hash(g));
    if (st) {
      st->states_expanded += h.states_expanded;
      st->candidates += h.candidates;
      st->generated += h.generated;
      st->decide_runs += (unsigned long long)std::max(0, h.last - k0);
    }
    return TW_OK;
  }
  // the levels of the deciding run are in its group's state and arena
  const int grp = std::min(std::max(h.group, 0), G - 1);
  const FusedState* hl = &h;
  if (grp != 0) {
    TW_CK(cudaMemcpyAsync(c->h_fused + 1, f.st[grp], sizeof(FusedState), cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaStreamSynchronize(c->stream));
    hl = c->h_fused + 1;
  }
  *answer_k = h.tw;
  const int last_k = h.tw >= 0 ? h.tw : k_last;
  R->levels.clear();
  for (int j = 0; j <= h.last; ++j) R->levels.push_back({hl->level_off[j], hl->level_cnt[j]});
  R->yes = h.tw >= 0 ? 1 : 0;
  R->states_expanded = h.states_expanded;
  R->candidates = h.candidates;
  R->generated = h.generated;
  R->retries = 0;
  R->peak_bytes = c->fused.bytes;
  R->expand_launches = 1;
  R->expand_seconds = 0.0;
  if (timed) {
    float ms = 0.f;
    TW_CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    R->expand_seconds = (double)ms * 1e-3;
  }
  unsigned long long out_states = 0;
  for (int j = 1; j <= h.last; ++j) out_states += hl->level_cnt[j];
  R->expand_bytes = (double)(h.states_expanded + h.generated + 2ull * out_states) * (double)w + (double)out_states;
  R->fp_sum.assign(1, 0ull);
  R->fp_xor.assign(1, 0ull);
  if (c->cfg.fingerprints) {
    for (int j = 1; j <= h.last; ++j) {
      TW_CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(LevelCounters), c->stream));
      TW_LAUNCH(c, launch_fingerprint(kc, static_cast<char*>(f.keys[grp]) + hl->level_off[j] * w, hl->level_cnt[j],
                                      c->d_ctr, c->stream));
      TW_CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, c->stream));
      TW_CK(cudaStreamSynchronize(c->stream));
      R->fp_sum.push_back(c->h_ctr->fp_sum);
      R->fp_xor.push_back(c->h_ctr->fp_xor);
    }
  }
  fill_stats(*R, last_k, st, false);
  if (st) st->decide_runs += (unsigned long long)(last_k - k0);  // fill_stats counted one run
  return TW_OK;
}

// Backward walk through the kept levels into the device order buffer.
int reconstruct(tw_ctx* c, KeyClass kc, int n, const DecideResult& R) {
  NvtxRange range("tw walk n=%d levels=%d", n, (int)R.levels.size());
  SmallLayout L;
  const size_t w = key_bytes(kc);
  const int last = (int)R.levels.size() - 1;
  int32_t* d_order = reinterpret_cast<int32_t*>(small_at(c, L.order));
  void* walk = small_at(c, L.walk);
  char* keys = static_cast<char*>(c->keys.ptr);
  const uint8_t* pred = static_cast<const uint8_t*>(c->pred.ptr);
  // (levels kept in host memory by spill_levels are read there in place)
  auto level_keys = [&](const LevelRec& lr) -> const char* { return lr.hkeys ? lr.hkeys : keys + lr.off * w; };
  auto level_pred = [&](const LevelRec& lr) -> const uint8_t* { return lr.hpred ? lr.hpred : pred + lr.off; };
  TW_LAUNCH(c, launch_walk_init(kc, level_keys(R.levels[last]), walk, last, c->stream));
  for (int j = last; j >= 1; --j) {
    const LevelRec& lr = R.levels[j];
    TW_LAUNCH(c, launch_walk_step(kc, level_keys(lr), level_pred(lr), lr.count, walk, j, d_order, c->stream));
  }
  TW_LAUNCH(c, launch_walk_finish(kc, walk, last, n, d_order, c->stream));
  return TW_OK;
}

void fill_stats(const DecideResult& R, int k, tw_stats* st, bool reset_totals) {
  if (!st) return;
  if (reset_totals) {
    st->states_expanded = st->candidates = st->generated = st->peak_frontier_bytes = 0;
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
  st->generated += R.generated;
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
  if (fused_eligible(c, g)) {
    int status = 0, ans = -1, bail_k = -1;
    tw_stats tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    rc = run_fused(c, g, kc, k, k, &R, &status, &ans, &bail_k, &tmp, nullptr);
    if (rc) return rc;
    if (status == 1) {
      if (R.yes && order) {
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
  }
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

// The sets of one level of decide(k) (run with the context's options and
// stopped after that level, so that it is the live output level), as
// ceil(n/64) words each.
int level_keys_graph(tw_ctx* c, const HostGraph& g, int k, int level, uint64_t* keys, uint64_t cap, uint64_t* count,
                     tw_stats* st) {
  Timer t;
  const unsigned long long launches0 = c->launches;
  if (k < 0 || level < 0 || count == nullptr) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  const KeyClass kc = key_class_for(g.n);
  int rc = upload_graph(c, g, kc);
  if (rc) return rc;
  DecideResult R;
  bool no = false;
  if ((rc = prepare_options(c, g, k, kc, &no))) return rc;
  if (no)
    immediate_no_result(&R);
  else if ((rc = run_decide(c, kc, g.n, k, false, &R, level))) {  // the level asked for is the last one built
    fill_stats(R, k, st, true);  // the levels completed before the failure
    return rc;
  }
  fill_stats(R, k, st, true);
  const unsigned long long cnt = level < (int)R.levels.size() ? R.levels[level].count : 0ull;
  if ((rc = put(c, count, &cnt, sizeof(cnt)))) return rc;
  if (cnt > cap) return TW_ERR_CAPACITY;
  if (cnt > 0) {
    if (keys == nullptr) return TW_ERR_INVALID;
    const LevelRec& lr = R.levels[level];
    const size_t w = key_bytes(kc);
    // the level's keys: one run, or (an out-of-core level split between
    // device and host memory) a device run followed by a host run
    const char* src[2] = {lr.hkeys ? lr.hkeys : static_cast<const char*>(c->keys.ptr) + lr.off * w, lr.htail};
    const unsigned long long run[2] = {cnt - lr.tail, lr.tail};
    const bool dev_out = is_device_ptr(keys);
    unsigned long long at = 0;
    for (int p = 0; p < 2; ++p) {
      if (run[p] == 0) continue;
      if (kc == kKey32) {
        // 32-bit states widen to the ABI's 64-bit words: by a kernel into a
        // device buffer of the caller, or on the host side of the copy
        if (dev_out) {
          TW_LAUNCH(c, launch_widen32(reinterpret_cast<const uint32_t*>(src[p]),
                                      reinterpret_cast<unsigned long long*>(keys) + at, run[p], c->stream));
        } else {
          std::vector<uint32_t> narrow((size_t)run[p]);
          TW_CK(cudaMemcpyAsync(narrow.data(), src[p], (size_t)run[p] * 4, cudaMemcpyDefault, c->stream));
          TW_CK(cudaStreamSynchronize(c->stream));
          for (unsigned long long x = 0; x < run[p]; ++x) keys[at + x] = narrow[x];
        }
      } else if ((rc = put_from_device(c, keys + at * (size_t)g.words, src[p], (size_t)run[p] * (size_t)g.words * 8))) {
        return rc;
      }
      at += run[p];
    }
  }
  TW_CK(cudaStreamSynchronize(c->stream));
  if (st) {
    st->seconds = t.seconds();
    st->kernel_launches = c->launches - launches0;
  }
  return TW_OK;
}

int bounds_graph(tw_ctx* c, const HostGraph& g, int32_t out[4], bool lower_only) {
  SmallLayout L;
  int32_t* d_out = reinterpret_cast<int32_t*>(small_at(c, L.bounds));
  int32_t* d_n = d_out + 4;
  int64_t* d_off = reinterpret_cast<int64_t*>(small_at(c, L.bounds + 64));
  const int32_t nn = g.n;
  const int64_t off = 0;
  TW_CK(cudaMemcpyAsync(d_n, &nn, 4, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_off, &off, 8, cudaMemcpyHostToDevice, c->stream));
  TW_LAUNCH(c, launch_bounds(reinterpret_cast<const unsigned long long*>(small_at(c, L.adj64)), d_n, d_off, 1, d_out,
                      nullptr, c->stream, lower_only ? 1 : 0));
  TW_CK(cudaMemcpyAsync(out, d_out, 16, cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  return TW_OK;
}

// Launches the lower bounds (MMD, MMD+) of the uploaded graph into the small
// buffer's bounds slot without waiting for them; returns their device
// address.
int launch_lower_bounds(tw_ctx* c, const HostGraph& g, const int32_t** d_bounds) {
  SmallLayout L;
  int32_t* d_out = reinterpret_cast<int32_t*>(small_at(c, L.bounds));
  int32_t* d_n = d_out + 4;
  int64_t* d_off = reinterpret_cast<int64_t*>(small_at(c, L.bounds + 64));
  // (n and the row offset go through the context's pinned counter block)
  c->h_ctr->out_count = (unsigned long long)(unsigned)g.n;
  c->h_ctr->generated = 0ull;
  TW_CK(cudaMemcpyAsync(d_n, &c->h_ctr->out_count, 4, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_off, &c->h_ctr->generated, 8, cudaMemcpyHostToDevice, c->stream));
  TW_LAUNCH(c, launch_bounds(reinterpret_cast<const unsigned long long*>(small_at(c, L.adj64)), d_n, d_off, 1, d_out,
                             nullptr, c->stream, 1));
  *d_bounds = d_out;
  return TW_OK;
}

int solve_graph(tw_ctx* c, const HostGraph& g, int* tw_out, int32_t* order, int32_t* td_parent, uint64_t* td_bags,
                tw_stats* st, int k_first) {
  NvtxRange range("tw solve n=%d", g.n);
  Timer t;
  const unsigned long long launches0 = c->launches;
  TW_CK(cudaSetDevice(c->device));
  const KeyClass kc = key_class_for(g.n);
  int rc = upload_graph(c, g, kc);
  if (rc) return rc;
  const bool want_walk = order || td_parent || td_bags;
  if (st) {
    st->states_expanded = st->candidates = st->generated = st->peak_frontier_bytes = 0;
    st->decide_runs = st->level_retries = 0;
    st->expand_launches = 0;
    st->expand_seconds = st->expand_bytes = 0.0;
  }
  int tw = -1;
  DecideResult R;
  int k0 = k_first;
  bool fused_done = false;
  bool have_bounds = false;
  if (!c->cfg.ub_shortcut && fused_eligible(c, g)) {
    // the fused solve reads the lower bounds on the device: no host round
    // trip between the bounds and the sweep
    const int32_t* d_bounds = nullptr;
    if ((rc = launch_lower_bounds(c, g, &d_bounds))) return rc;
    int status = 0, ans = -1, bail_k = -1;
    rc = run_fused(c, g, kc, k_first, g.n - 1, &R, &status, &ans, &bail_k, st, d_bounds);
    if (rc) return rc;
    if (status == 1) {
      tw = ans;
      fused_done = true;
    } else if (status == 2) {
      k0 = bail_k;
      have_bounds = true;  // (bail_k is at least the lower bound)
    }
  }
  if (!fused_done && !have_bounds) {
    int32_t b[4];
    rc = bounds_graph(c, g, b, !c->cfg.ub_shortcut);  // the widths only for the shortcut
    if (rc) return rc;
    const int lb = std::max(b[0], b[1]);
    const int ub = std::min(b[2], b[3]);
    k0 = std::max(lb, k_first);
    if (c->cfg.ub_shortcut && lb == ub && !want_walk) {
      tw = ub;
      fused_done = true;  // (no decide run and no walk)
    } else if (c->cfg.ub_shortcut && fused_eligible(c, g)) {
      int status = 0, ans = -1, bail_k = -1;
      rc = run_fused(c, g, kc, k0, g.n - 1, &R, &status, &ans, &bail_k, st, nullptr);
      if (rc) return rc;
      if (status == 1) {
        tw = ans;
        fused_done = true;
      } else if (status == 2) {
        k0 = bail_k;
      }
    }
  }
  {
    for (int k = k0; k < g.n && !fused_done; ++k) {
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
    // (the fused solve has already walked back and built the decomposition)
    if (!fused_done && (rc = reconstruct(c, kc, g.n, R))) return rc;
    int32_t* d_order = reinterpret_cast<int32_t*>(small_at(c, L.order));
    if (c->cfg.disjoint_paths && (rc = upload_graph(c, g, kc))) return rc;  // bags of G itself
    if (!fused_done && (td_parent || td_bags)) {
      TW_LAUNCH(c, launch_td(reinterpret_cast<const unsigned long long*>(small_at(c, L.adj64)), g.n, g.words, d_order,
                      reinterpret_cast<int32_t*>(small_at(c, L.parent)),
                      reinterpret_cast<unsigned long long*>(small_at(c, L.bags)), c->stream));
    }
    (void)d_order;
    rc = put_solution(c, g.n, g.words, order, td_parent, td_bags);
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
  if ((rc = bounds_graph(c, g, b, true))) return rc;
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

}  // namespace host
}  // namespace tw
