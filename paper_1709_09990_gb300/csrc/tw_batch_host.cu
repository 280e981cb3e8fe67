// Host driver of tw_solve_batch (see the section comment below and
// tw_batch.cu for the kernels).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tw_host.h"

namespace tw {
namespace host {

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

// Decide-only mode of run_batch (tw_decide_batch): every graph runs one
// decide at its own k and reports its answer, level sizes and fingerprints.
struct BatchDecide {
  const std::vector<int>* k = nullptr;                             // by graph index
  std::vector<int>* yes = nullptr;                                 // by graph index
  std::vector<std::vector<unsigned long long>>* size = nullptr;    // by graph index
  std::vector<std::vector<unsigned long long>>* fp_sum = nullptr;  // (or nullptr)
  std::vector<std::vector<unsigned long long>>* fp_xor = nullptr;
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
              std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st, std::vector<int>* evicted,
              const BatchDecide* dm) {
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
    TW_LAUNCH(c, launch_bounds(B.adj, d_n, d_off, G, d_b, nullptr, c->stream, 1));
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
      if (dm) x.k0 = (*dm->k)[idx[j]];  // 0 <= k < n-1 (the caller answers larger k)
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
    if (dm) {
      // decide-only: record the run's levels (sizes and fingerprints) and stop
      std::vector<int> fin;
      std::vector<CopySeg> fseg;
      for (int j = 0; j < G; ++j) {
        BGraph& x = B.g[j];
        if (x.state != 0) continue;
        const int last = (int)x.levels.size() - 1;
        if (x.levels.back().count != 0 && last != x.n - x.k - 1) continue;
        fin.push_back(j);
        for (const LevelRec& l : x.levels) fseg.push_back({l.off, 0ull, l.count});
      }
      if (!fin.empty()) {
        std::vector<unsigned long long> fp(2 * fseg.size(), 0ull);
        if (dm->fp_sum) {
          CopySeg* d_seg = nullptr;
          unsigned long long* d_fp = nullptr;
          if ((rc = dev_alloc(&d_seg, fseg.size())) || (rc = dev_alloc(&d_fp, fp.size()))) return rc;
          TW_CK(cudaMemcpyAsync(d_seg, fseg.data(), fseg.size() * sizeof(CopySeg), cudaMemcpyHostToDevice,
                                c->stream));
          TW_CK(cudaMemsetAsync(d_fp, 0, fp.size() * 8, c->stream));
          TW_LAUNCH(c, launch_fingerprint_segments(d_seg, (int)fseg.size(), B.akeys, d_fp, c->stream));
          TW_CK(cudaMemcpyAsync(fp.data(), d_fp, fp.size() * 8, cudaMemcpyDeviceToHost, c->stream));
          TW_CK(cudaStreamSynchronize(c->stream));
          cudaFree(d_seg);
          cudaFree(d_fp);
        }
        size_t q = 0;
        for (int j : fin) {
          BGraph& x = B.g[j];
          const int gi = x.in_idx;
          (*dm->yes)[gi] = x.levels.back().count != 0 ? 1 : 0;
          (*dm->size)[gi].clear();
          if (dm->fp_sum) (*dm->fp_sum)[gi].clear();
          if (dm->fp_xor) (*dm->fp_xor)[gi].clear();
          for (const LevelRec& l : x.levels) {
            (*dm->size)[gi].push_back(l.count);
            if (dm->fp_sum) (*dm->fp_sum)[gi].push_back(fp[2 * q]);
            if (dm->fp_xor) (*dm->fp_xor)[gi].push_back(fp[2 * q + 1]);
            ++q;
          }
          x.tw = x.k;
          x.state = 1;
          x.levels.clear();
        }
        answered = true;
      }
    } else {
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
      // (more than 90% of the slots filled re-runs the level with a larger
      // table, so the output never needs more room than that)
      unsigned long long oc =
          x.ocap_retry ? x.ocap_retry
                       : std::min<unsigned long long>(
                             (unsigned long long)std::ceil(std::min(bound, std::max(table_est * 3.0, 1024.0))),
                             slots / 10ull * 9ull + 64ull);
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
        st->generated += h.generated;
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
    if (dm) {
      (*hst)[x.in_idx] = TW_OK;
      continue;
    }
    htw[x.in_idx] = x.tw;
    (*hst)[x.in_idx] = TW_OK;
    if (hord)
      for (int v = 0; v < x.n; ++v) (*hord)[x.order_off + v] = dord[x.order_off + v];
  }
  for (BGraph& x : B.g)
    if (x.state == 2) evicted->push_back(x.in_idx);
  return TW_OK;
}

// ---------------------------------------------------------------- persistent
//
// The default batched path: one launch of batch_solve_kernel (tw_batch_solve.cu)
// for all graphs with n <= 64; each block solves one graph at a time from a
// device queue.  Graphs are queued largest n first so that long solves start
// early.  A graph whose levels outgrow a block's workspace is returned in
// *evicted for the single-graph path.
// Device allocations of one call, freed (after the stream) on return.
struct DevMem {
  tw_ctx* c;
  std::vector<void*> p;
  explicit DevMem(tw_ctx* cc) : c(cc) {}
  ~DevMem() {
    cudaStreamSynchronize(c->stream);
    for (void* x : p) cudaFree(x);
    cudaGetLastError();
  }
  template <class X>
  int get(X** out, size_t count) {
    void* v = nullptr;
    if (cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(X)) != cudaSuccess) {
      cudaGetLastError();
      return TW_ERR_CAPACITY;
    }
    p.push_back(v);
    *out = static_cast<X*>(v);
    return TW_OK;
  }
};

int run_batch_persistent(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                         const std::vector<float>* hint, const std::vector<int64_t>& order_off, int* htw,
                         std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st, std::vector<int>* evicted,
                         const BatchDecide* dm, int warps);

// With tw_config.autotune, the first batch of at least 512 graphs times the
// persistent kernel with 4 and with 8 warps per block on a sample of 256 of
// its graphs (every G/256-th) and keeps the faster choice for the context.
int batch_warps(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                const std::vector<float>* hint, const std::vector<int64_t>& order_off, const BatchDecide* dm) {
  if (c->batch_warps > 0) return c->batch_warps;
  if (!c->cfg.autotune || idx.size() < 512) return 4;
  std::vector<int> sample;
  const size_t step = idx.size() / 256;
  for (size_t j = 0; j < idx.size() && sample.size() < 256; j += step) sample.push_back(idx[j]);
  std::vector<int> tw_tmp(graphs.size(), -1), st_tmp(graphs.size(), 0), ev;
  double best = 1e30;
  int best_w = 4;
  for (int w : {4, 8}) {
    ev.clear();
    Timer t;
    int rc = run_batch_persistent(c, graphs, sample, hint, order_off, tw_tmp.data(), nullptr, &st_tmp, nullptr, &ev,
                                  dm, w);
    if (rc) return 4;
    const double secs = t.seconds();
    if (secs < best) {
      best = secs;
      best_w = w;
    }
  }
  c->batch_warps = best_w;
  return best_w;
}

int run_batch_persistent(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                         const std::vector<float>* hint, const std::vector<int64_t>& order_off, int* htw,
                         std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st, std::vector<int>* evicted,
                         const BatchDecide* dm, int warps) {
  const int G = (int)idx.size();
  if (G == 0) return TW_OK;
  if (warps == 0) warps = batch_warps(c, graphs, idx, hint, order_off, dm);
  NvtxRange range("tw batch persistent graphs=%d", G);
  std::vector<int> q(idx);
  std::stable_sort(q.begin(), q.end(), [&](int a, int b) { return graphs[a].n > graphs[b].n; });
  std::vector<unsigned long long> rows((size_t)G * 64, 0ull);
  std::vector<int32_t> ns(G), kst(G), lbv(G);
  std::vector<int64_t> offs(G), ooff(G);
  int64_t total_n = 0;
  for (int j = 0; j < G; ++j) {
    const HostGraph& hg = graphs[q[j]];
    for (int r = 0; r < hg.n; ++r) rows[(size_t)j * 64 + r] = hg.rows[r];
    ns[j] = hg.n;
    offs[j] = (int64_t)j * 64;
    ooff[j] = order_off[q[j]];
    total_n = std::max<int64_t>(total_n, ooff[j] + hg.n);
  }
  const int blocks = batch_solve_blocks(warps);
  // workspace: per block A keys and predecessor bytes, two tables of 2A slots
  const size_t room = c->mem_cap > total_bytes(c) ? c->mem_cap - total_bytes(c) : 0;
  const size_t budget = std::min<size_t>(room / 4, 32ull << 30);
  // 2^16 states by default: a graph whose decide runs outgrow that is better
  // served by the level-synchronous kernel, which spreads each level over the
  // whole GPU, than by one block (measured on the batch workload's light
  // graphs: 2^19 1.09 s, 2^17 0.67 s, 2^15 0.56 s, 2^13 0.54 s)
  unsigned long long A = 1ull << 16;
  if (c->cfg.batch_arena_states > 0) {
    A = 1ull << 19;
    while (A > 4096 && A > (unsigned long long)c->cfg.batch_arena_states) A >>= 1;
  }
  while (A > 4096 && (size_t)blocks * (A * 41 + 4096) > budget) A >>= 1;
  const unsigned long long T = 2 * A;
  DevMem mem(c);
  BatchSolveArgs a{};
  unsigned long long* d_adj = nullptr;
  int32_t *d_n = nullptr, *d_lb = nullptr, *d_k = nullptr, *d_b = nullptr;
  int64_t *d_off = nullptr, *d_ooff = nullptr;
  int rc;
  if ((rc = mem.get(&d_adj, rows.size())) || (rc = mem.get(&d_n, G)) || (rc = mem.get(&d_lb, G)) ||
      (rc = mem.get(&d_k, G)) || (rc = mem.get(&d_b, (size_t)G * 4)) || (rc = mem.get(&d_off, G)) ||
      (rc = mem.get(&d_ooff, G)))
    return rc;
  TW_CK(cudaMemcpyAsync(d_adj, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_n, ns.data(), (size_t)G * 4, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_off, offs.data(), (size_t)G * 8, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_ooff, ooff.data(), (size_t)G * 8, cudaMemcpyHostToDevice, c->stream));
  TW_LAUNCH(c, launch_bounds(d_adj, d_n, d_off, G, d_b, nullptr, c->stream, 1));
  std::vector<int32_t> b((size_t)G * 4);
  TW_CK(cudaMemcpyAsync(b.data(), d_b, b.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaStreamSynchronize(c->stream));
  for (int j = 0; j < G; ++j) {
    const int gi = q[j], n = ns[j];
    lbv[j] = std::max(b[4 * j], b[4 * j + 1]);
    int k0 = lbv[j];
    if (hint) k0 = (int)std::lround((*hint)[gi]);
    kst[j] = std::min(std::max(k0, lbv[j]), n - 1);
    if (dm) kst[j] = (*dm->k)[gi];
  }
  TW_CK(cudaMemcpyAsync(d_lb, lbv.data(), (size_t)G * 4, cudaMemcpyHostToDevice, c->stream));
  TW_CK(cudaMemcpyAsync(d_k, kst.data(), (size_t)G * 4, cudaMemcpyHostToDevice, c->stream));
  a.adj = d_adj;
  a.n = d_n;
  a.lb = d_lb;
  a.k_start = d_k;
  a.num_graphs = G;
  a.decide_mode = dm ? 1 : 0;
  a.max_probes = kBatchProbes;
  a.load_pct = 50;
  a.A = A;
  a.T = T;
  unsigned int* d_next = nullptr;
  unsigned long long* d_tot = nullptr;
  if ((rc = mem.get(&d_next, 1)) || (rc = mem.get(&d_tot, 4)) || (rc = mem.get(&a.arena, (size_t)blocks * A)) ||
      (rc = mem.get(&a.pred, (size_t)blocks * A)) || (rc = mem.get(&a.tables, (size_t)blocks * 2 * T)) ||
      (rc = mem.get(&a.ctr, (size_t)blocks)) || (rc = mem.get(&a.level_off, (size_t)blocks * 130)) ||
      (rc = mem.get(&a.level_cnt, (size_t)blocks * 130)) || (rc = mem.get(&a.tw, G)) || (rc = mem.get(&a.status, G)))
    return rc;
  TW_CK(cudaMemsetAsync(d_next, 0, 4, c->stream));
  TW_CK(cudaMemsetAsync(d_tot, 0, 32, c->stream));
  a.next_graph = d_next;
  a.totals = d_tot;
  a.order_off = d_ooff;
  if (hord && !dm && (rc = mem.get(&a.orders, (size_t)std::max<int64_t>(total_n, 1)))) return rc;
  if (dm) {
    if ((rc = mem.get(&a.yes, G)) || (rc = mem.get(&a.last, G)) || (rc = mem.get(&a.level_size, (size_t)G * 129)))
      return rc;
    TW_CK(cudaMemsetAsync(a.level_size, 0, (size_t)G * 129 * 8, c->stream));
    if (dm->fp_sum) {
      if ((rc = mem.get(&a.fp_sum, (size_t)G * 129)) || (rc = mem.get(&a.fp_xor, (size_t)G * 129))) return rc;
      TW_CK(cudaMemsetAsync(a.fp_sum, 0, (size_t)G * 129 * 8, c->stream));
      TW_CK(cudaMemsetAsync(a.fp_xor, 0, (size_t)G * 129 * 8, c->stream));
    }
  }
  TW_LAUNCH(c, launch_batch_solve(a, blocks, warps, c->stream));
  if (st) st->expand_launches += 1;
  std::vector<int32_t> htw_p(G), hst_p(G);
  unsigned long long tot[4];
  TW_CK(cudaMemcpyAsync(hst_p.data(), a.status, (size_t)G * 4, cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaMemcpyAsync(htw_p.data(), a.tw, (size_t)G * 4, cudaMemcpyDeviceToHost, c->stream));
  TW_CK(cudaMemcpyAsync(tot, d_tot, 32, cudaMemcpyDeviceToHost, c->stream));
  std::vector<int32_t> dord;
  if (a.orders) {
    dord.resize((size_t)total_n);
    TW_CK(cudaMemcpyAsync(dord.data(), a.orders, dord.size() * 4, cudaMemcpyDeviceToHost, c->stream));
  }
  std::vector<int32_t> hy, hl;
  std::vector<unsigned long long> hls, hfs, hfx;
  if (dm) {
    hy.resize(G);
    hl.resize(G);
    hls.resize((size_t)G * 129);
    TW_CK(cudaMemcpyAsync(hy.data(), a.yes, (size_t)G * 4, cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaMemcpyAsync(hl.data(), a.last, (size_t)G * 4, cudaMemcpyDeviceToHost, c->stream));
    TW_CK(cudaMemcpyAsync(hls.data(), a.level_size, hls.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    if (a.fp_sum) {
      hfs.resize((size_t)G * 129);
      hfx.resize((size_t)G * 129);
      TW_CK(cudaMemcpyAsync(hfs.data(), a.fp_sum, hfs.size() * 8, cudaMemcpyDeviceToHost, c->stream));
      TW_CK(cudaMemcpyAsync(hfx.data(), a.fp_xor, hfx.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  TW_CK(cudaStreamSynchronize(c->stream));
  if (st) {
    st->states_expanded += tot[0];
    st->candidates += tot[1];
    st->generated += tot[2];
    st->decide_runs += tot[3];
  }
  for (int j = 0; j < G; ++j) {
    const int gi = q[j];
    if (hst_p[j] != 0) {
      evicted->push_back(gi);
      continue;
    }
    (*hst)[gi] = TW_OK;
    if (dm) {
      (*dm->yes)[gi] = hy[j];
      const int L = hl[j] + 1;
      (*dm->size)[gi].assign(hls.begin() + (size_t)j * 129, hls.begin() + (size_t)j * 129 + L);
      if (dm->fp_sum) {
        (*dm->fp_sum)[gi].assign(hfs.begin() + (size_t)j * 129, hfs.begin() + (size_t)j * 129 + L);
        (*dm->fp_xor)[gi].assign(hfx.begin() + (size_t)j * 129, hfx.begin() + (size_t)j * 129 + L);
      }
      continue;
    }
    htw[gi] = htw_p[j];
    if (hord && a.orders)
      for (int v = 0; v < ns[j]; ++v) (*hord)[ooff[j] + v] = dord[ooff[j] + v];
  }
  return TW_OK;
}

// Graphs with n <= 64 go through the batched kernels: the persistent one
// first (by default), then the level-synchronous one for the graphs that
// outgrew a block's workspace (it holds levels of up to 2^21 sets per graph);
// graphs it evicts in turn and graphs with n > 64 are solved one at a time by
// the single-graph path.
int solve_batch_gpu(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                    const std::vector<float>* hint, const std::vector<int64_t>& order_off, int* htw,
                    std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st) {
  NvtxRange range("tw solve_batch graphs=%d", (int)idx.size());
  std::vector<int> small, single;
  for (int i : idx) (graphs[i].n <= 64 ? small : single).push_back(i);
  int rc;
  if (c->cfg.batch_kernel == 1) {
    rc = run_batch(c, graphs, small, hint, order_off, htw, hord, hst, st, &single, nullptr);
  } else {
    std::vector<int> outgrown;
    rc = run_batch_persistent(c, graphs, small, hint, order_off, htw, hord, hst, st, &outgrown, nullptr, 0);
    if (rc == TW_OK && !outgrown.empty())
      rc = run_batch(c, graphs, outgrown, hint, order_off, htw, hord, hst, st, &single, nullptr);
  }
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
      st->generated += local.generated;
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

// Decide runs of many graphs at their own k: graphs with n <= 64 through the
// batched kernel, the others (and any the batch evicts) one at a time through
// the single-graph path, with the Section 3.1 options and pruning turned off
// so that every graph reports the plain method's level sets.
int decide_batch_gpu(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                     const std::vector<int>& kk, std::vector<int>* yes, std::vector<int>* hst,
                     std::vector<std::vector<unsigned long long>>* size,
                     std::vector<std::vector<unsigned long long>>* fp_sum,
                     std::vector<std::vector<unsigned long long>>* fp_xor, tw_stats* st) {
  NvtxRange range("tw decide_batch graphs=%d", (int)idx.size());
  std::vector<int> small, single;
  for (int i : idx) {
    const int n = graphs[i].n;
    if (kk[i] >= n - 1) {
      // the listing's loop is empty: yes with the single level {empty set}
      (*yes)[i] = 1;
      (*size)[i].assign(1, 1ull);
      if (fp_sum) (*fp_sum)[i].assign(1, 0ull);
      if (fp_xor) (*fp_xor)[i].assign(1, 0ull);
      (*hst)[i] = TW_OK;
      continue;
    }
    (n <= 64 ? small : single).push_back(i);
  }
  BatchDecide dm;
  dm.k = &kk;
  dm.yes = yes;
  dm.size = size;
  dm.fp_sum = fp_sum;
  dm.fp_xor = fp_xor;
  std::vector<int64_t> order_off(graphs.size(), 0);
  std::vector<int> htw(graphs.size(), -1);
  int rc = c->cfg.batch_kernel == 1
               ? run_batch(c, graphs, small, nullptr, order_off, htw.data(), nullptr, hst, st, &single, &dm)
               : run_batch_persistent(c, graphs, small, nullptr, order_off, htw.data(), nullptr, hst, st, &single, &dm,
                                      0);
  if (rc) return rc;
  const tw_config saved = c->cfg;
  c->cfg.clique_skip = c->cfg.disjoint_paths = c->cfg.mmw_prune = 0;
  c->cfg.fingerprints = fp_sum || fp_xor ? 1 : 0;
  for (int gi : single) {
    tw_stats local;
    std::memset(&local, 0, sizeof(local));
    int y = 0;
    const int r2 = decide_graph(c, graphs[gi], kk[gi], &y, nullptr, &local);
    (*hst)[gi] = r2;
    if (r2 != TW_OK) continue;
    (*yes)[gi] = y;
    (*size)[gi].assign(local.level_size, local.level_size + local.levels);
    if (fp_sum) (*fp_sum)[gi].assign(local.level_fp_sum, local.level_fp_sum + local.levels);
    if (fp_xor) (*fp_xor)[gi].assign(local.level_fp_xor, local.level_fp_xor + local.levels);
    if (st) {
      st->states_expanded += local.states_expanded;
      st->candidates += local.candidates;
      st->generated += local.generated;
      st->decide_runs += local.decide_runs;
      st->level_retries += local.level_retries;
      st->expand_launches += local.expand_launches;
    }
  }
  c->cfg = saved;
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

}  // namespace host
}  // namespace tw
