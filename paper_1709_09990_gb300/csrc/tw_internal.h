// Interfaces between the translation units of libtw (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace tw {

// Width class of the state bitsets.
enum KeyClass : int { kKey32 = 0, kKey64 = 1, kKey128 = 2 };

inline KeyClass key_class_for(int n) { return n <= 32 ? kKey32 : (n <= 64 ? kKey64 : kKey128); }
inline size_t key_bytes(KeyClass c) { return c == kKey32 ? 4 : (c == kKey64 ? 8 : 16); }

// Device-side counters of one level expansion (one per context, 64-byte
// aligned in device memory and mirrored in pinned host memory).
struct LevelCounters {
  unsigned long long out_count;  // states appended to L_{i+1} (counts past capacity too)
  unsigned long long generated;  // pairs (S, v) submitted to the table
  unsigned long long fp_sum;     // sum of fingerprints of L_{i+1}
  unsigned long long fp_xor;     // xor of fingerprints of L_{i+1}
  unsigned int overflow;         // bit 0: output list full, bit 1: probe limit reached
  unsigned int pad[7];
};

// One level i -> i+1 of Listing 1 (arXiv 1709.09990, Section 3.1).
struct ExpandLaunch {
  KeyClass kc;
  const void* in_keys;           // |L_i| keys
  unsigned long long n_in;
  const void* adj;               // n rows, one key each
  int n;
  int k;
  void* table;                   // power-of-two slots, all set to the empty key
  unsigned long long table_slots;
  int max_probes;
  void* out_keys;                // L_{i+1} keys (capacity out_cap)
  uint8_t* out_pred;             // predecessor vertex of each L_{i+1} state
  unsigned long long out_cap;
  LevelCounters* ctr;
  int block_threads;             // 64, 128 or 256
  int grid;                      // 0 = derived from the occupancy of this device
  unsigned long long allowed[2]; // vertices that may be added (low word first)
  int mmw;                       // 1: minor-min-width pruning (Section 3.3)
  unsigned long long ranges = 0; // > 0: ranged launch - only the pairs whose hash lies in
  unsigned long long range = 0;  // range `range` of `ranges` are inserted, into a table that
                                 // is that range's slice; out_pred is not written
  void* out_tail = nullptr;      // ranged launch: output positions from out_split on go to
  unsigned long long out_split = 0;  // out_tail (a second buffer, e.g. in host memory)
};

cudaError_t launch_expand(const ExpandLaunch& a, cudaStream_t s);

// Sets every slot of a table to the empty key (all ones) and zeroes ctr
// (unless ctr is null).
cudaError_t launch_clear(void* table, size_t table_bytes, LevelCounters* ctr, cudaStream_t s);

// dst[i] = src[i] zero-extended, i < count (32-bit states in 64-bit words).
cudaError_t launch_widen32(const uint32_t* src, unsigned long long* dst, unsigned long long count, cudaStream_t s);

// Adds the fingerprints of count keys into ctr->fp_sum / fp_xor.
cudaError_t launch_fingerprint(KeyClass kc, const void* keys, unsigned long long count,
                               LevelCounters* ctr, cudaStream_t s);

// One step of the backward walk: finds walk[j] among the count keys of level
// j, writes its predecessor vertex v to order[j-1] and walk[j-1] = walk[j]
// minus v.  walk holds one key per level.
cudaError_t launch_walk_step(KeyClass kc, const void* keys, const uint8_t* pred,
                             unsigned long long count, void* walk, int j, int32_t* order,
                             cudaStream_t s);

// walk[last] = keys[0] (first state of the final level).
cudaError_t launch_walk_init(KeyClass kc, const void* keys, void* walk, int last, cudaStream_t s);

// order[last..n-1] = the vertices outside walk[last], in increasing order.
cudaError_t launch_walk_finish(KeyClass kc, const void* walk, int last, int n, int32_t* order,
                               cudaStream_t s);

// Tree decomposition from an ordering (one thread per vertex):
// bag(v) = {v} u Q(prefix(v), v), parent(v) = first vertex of Q after v in
// the order (or the last vertex; the last vertex is the root).
// adj64 / bags: n rows x words64 uint64.
cudaError_t launch_td(const unsigned long long* adj64, int n, int words64, const int32_t* order,
                      int32_t* parent, unsigned long long* bags, cudaStream_t s);

// Bounds (one warp per graph): out[4*g + 0..3] = MMD, MMD+, min-degree width,
// min-fill width (-1 for the widths with lower_only, unless feats is given).  Graph g: n[g] rows of ceil(n[g]/64) words at row_offset[g].
cudaError_t launch_bounds(const unsigned long long* adj, const int32_t* n, const int64_t* row_offset,
                          int num_graphs, int32_t* out, float* feats, cudaStream_t s,
                          int lower_only = 0);

// ---- partitioned insert (tw_partition.cu) ----------------------------------
constexpr int kMaxRanges = 64;

// Candidate regions of a partitioned level: range r owns entries
// [r * region_cap, (r + 1) * region_cap) of cand_key / cand_v.
struct PartitionBufs {
  int ranges;                         // P <= kMaxRanges
  void* cand_key;                     // P * region_cap keys
  uint8_t* cand_v;                    // P * region_cap added vertices
  unsigned long long region_cap;
  unsigned long long* region_cnt;     // P counters (zeroed before emit)
  unsigned long long* prefix;         // P + 1 prefix sums of the clamped counts (for insert)
  unsigned int* overflow;             // set when a region overflows
};

// Launch A: search + per-block counting sort of the pairs into the regions
// (adds the count of generated pairs to a.ctr).
cudaError_t launch_emit(const ExpandLaunch& a, const PartitionBufs& pb, cudaStream_t s);
// Launch B: insert entries [first, end) of the concatenated regions (range-
// major) into a.table, appending winners to a.out_keys / a.out_pred.
cudaError_t launch_insert_ranges(const ExpandLaunch& a, const PartitionBufs& pb, unsigned long long first,
                                 unsigned long long end, cudaStream_t s);
// Empties slots [first, first + count) of a table of total slots (wrapping).
cudaError_t launch_clear_slots(KeyClass kc, void* table, unsigned long long first, unsigned long long count,
                               unsigned long long total, cudaStream_t s);
// Drops the whole 128-byte lines of bytes [lo, hi) of base from L2 without
// writing them back (their contents become undefined).
cudaError_t launch_discard_l2(void* base, unsigned long long lo_bytes, unsigned long long hi_bytes, cudaStream_t s);

// ---- graph-driven levels (tw_graph.cu) ---------------------------------------
// Device state of a decide run whose level loop is a captured CUDA graph: a
// one-thread plan kernel between levels records the level just built, sizes
// the next one and stops the run (done) or gives up (bail: the host re-runs
// the decide with its own loop, which can grow buffers).
struct GraphState {
  unsigned long long level_off[130];  // arena index of level j
  unsigned long long level_cnt[130];  // |L_j|
  unsigned long long table_slots;     // table size of the level being built
  unsigned long long out_off;         // arena index where it is written
  unsigned long long out_cap;
  unsigned long long generated;       // pairs submitted to the table, summed
  unsigned long long peak_bytes;      // max kept-level + table bytes
  int cur;                            // newest level
  int done;
  int bail;
  int yes;
};

cudaError_t launch_graph_init(KeyClass kc, GraphState* st, void* keys, cudaStream_t s);
cudaError_t launch_graph_plan(GraphState* st, LevelCounters* ctr, unsigned long long arena_cap,
                              unsigned long long table_cap, unsigned long long direct_table_bytes, int n, int k,
                              int load_pct, int key_bytes, int first, cudaStream_t s);
cudaError_t launch_graph_clear(KeyClass kc, const GraphState* st, void* table, cudaStream_t s);
// base: in_keys/out_keys = the arena, out_pred = the predecessor arena; the
// level fields come from st.
cudaError_t launch_graph_expand(const GraphState* st, const ExpandLaunch& base, cudaStream_t s);

// ---- fused small solve (tw_fused.cu) -----------------------------------------
constexpr int kFusedMaxGroups = 4;  // decide runs of the sweep in flight at once

// Device state of one group of a fused solve (zeroed by the host before the
// launch).  Group 0's state also holds the solve's summary and the window
// barrier of the whole grid.
struct FusedState {
  unsigned long long level_off[130];  // arena index of level j of the group's run
  unsigned long long level_cnt[130];  // |L_j|
  LevelCounters ctr[130];             // counters of the expansion that built level j
  unsigned long long states_expanded, candidates, generated;  // group 0: over the counted runs
  unsigned long long run_states, run_candidates, run_generated;  // the group's current run
  unsigned int arrive, gen, error;    // the group's barrier; error (group 0): a wait gave up
  unsigned int w_arrive, w_gen;       // group 0: barrier of all blocks at the end of a window
  int result, run_last;               // the group's run: 0 no, 1 yes, 2 gave up, -1 not run;
                                      // index of its final level
  int status;                         // group 0: 1 finished, 2 gave up at k = last
  int tw, last, group;                // group 0: the first yes k (-1: none up to k_last), the
                                      // index of the final level of the deciding run and
                                      // the group that ran it
  int k_start;                        // group 0: the first k of the sweep
};

struct FusedLaunch {
  KeyClass kc;                        // kKey32 or kKey64
  const void* adj;                    // n rows in the state layout
  const unsigned long long* adj64;    // n rows of words64 words
  int n, words64, k0, k_last, max_probes, load_pct;  // decide runs at k0 .. k_last
  int groups;                         // runs in flight at once: k, k+1, .. (1 .. kFusedMaxGroups)
  int tables_clean;                   // 1: every table slot is empty (the last launch emptied them)
  const int32_t* lb_dev;              // or null: the sweep starts at max(k0, lb_dev[0], lb_dev[1])
                                      // (lower bounds written by a kernel earlier on the stream)
  void* keys[kFusedMaxGroups];        // per group: arena of arena_cap states
  uint8_t* pred[kFusedMaxGroups];
  unsigned long long arena_cap;
  void* table0[kFusedMaxGroups];      // per group: two tables of table_cap slots
  void* table1[kFusedMaxGroups];
  unsigned long long table_cap;       // slots of each table
  FusedState* st[kFusedMaxGroups];
  int32_t* order;
  int32_t* parent;
  unsigned long long* bags;
};

// The k sweep from k0, the walk and the tree decomposition of one graph
// (n <= 64) in one cooperative launch; see tw_fused.cu.
cudaError_t launch_fused_solve(const FusedLaunch& f, cudaStream_t s);

// ---- persistent batched solve (tw_batch_solve.cu) ----------------------------
struct BatchSolveArgs {
  const unsigned long long* adj;      // 64 rows per graph
  const int32_t* n;
  const int32_t* lb;                  // lower bound of each graph (certification)
  const int32_t* k_start;             // first k of each graph (decide mode: its k)
  int num_graphs;
  int decide_mode;                    // 1: one decide per graph, level sizes and fingerprints
  int max_probes, load_pct;
  unsigned int* next_graph;           // the work queue (zero before the launch)
  // workspace of each block (blockIdx.x): A keys + A predecessor bytes, two
  // tables of T slots, counters, level offsets and sizes (130 each)
  unsigned long long* arena;
  uint8_t* pred;
  unsigned long long* tables;
  LevelCounters* ctr;
  unsigned long long* level_off;
  unsigned long long* level_cnt;
  unsigned long long A, T;
  // results
  int32_t* tw;                        // solve mode (-1 when the graph was left to the host)
  int32_t* orders;                    // solve mode, or null
  const int64_t* order_off;
  int32_t* status;                    // 0 done, 2 outgrew the workspace
  int32_t* yes;                       // decide mode
  int32_t* last;                      // decide mode: index of the final level
  unsigned long long* level_size;     // decide mode: 129 per graph
  unsigned long long* fp_sum;         // decide mode (or null): 129 per graph
  unsigned long long* fp_xor;
  unsigned long long* totals;         // states expanded, candidates, generated pairs, decide runs
};

// Resident blocks of the kernel with `warps` warps per block (4 or 8).
int batch_solve_blocks(int warps);
cudaError_t launch_batch_solve(const BatchSolveArgs& a, int blocks, int warps, cudaStream_t s);

// ---- batched expansion (tw_batch.cu) ---------------------------------------
// One graph's share of a batched level step (64-bit states, n <= 64).
struct BatchSeg {
  unsigned long long in_off;    // arena index of the graph's L_i
  unsigned long long in_count;  // |L_i|
  unsigned long long t_off;     // first slot of the graph's table segment
  unsigned long long t_slots;   // slots of that segment
  unsigned long long o_off;     // first entry of the graph's output segment
  unsigned long long o_cap;     // capacity of that segment
  int graph;                    // row block of the graph in the adjacency array (64 rows each)
  int n;
  int k;
  int pad;
};

struct BatchCounters {
  unsigned long long out_count;
  unsigned long long generated;
  unsigned int overflow;  // bit 0: output full, bit 1: probe limit
  unsigned int pad;
  unsigned long long pad2;
};

struct CopySeg {
  unsigned long long src_off;  // ~0 = write the empty set
  unsigned long long dst_off;
  unsigned long long count;
};

struct WalkSeg {
  unsigned long long level_base;  // index of the graph's level offsets in level_off
  unsigned long long order_off;   // first entry of the graph's ordering
  int last;                       // index of the final level
  int n;
};

// chunk_begin has nseg+1 entries (the last one = total_chunks); segments
// must be non-empty.  Keys are u64, parents u32.
cudaError_t launch_expand_batch(const BatchSeg* segs, const unsigned long long* chunk_begin, int nseg,
                                unsigned long long total_chunks, const unsigned long long* keys,
                                const unsigned long long* adj_all, unsigned long long* table,
                                unsigned long long* out_keys, uint32_t* out_parent, BatchCounters* ctr, int max_probes,
                                cudaStream_t s);
cudaError_t launch_copy_segments(const CopySeg* segs, int nseg, const unsigned long long* src_keys,
                                 const uint32_t* src_par, unsigned long long* dst_keys, uint32_t* dst_par,
                                 cudaStream_t s);
// out[2s], out[2s+1] += sum and xor of the fingerprints of keys
// [segs[s].src_off, segs[s].src_off + segs[s].count) (u64 keys); out zeroed
// by the caller.
cudaError_t launch_fingerprint_segments(const CopySeg* segs, int nseg, const unsigned long long* keys,
                                        unsigned long long* out, cudaStream_t s);
cudaError_t launch_walk_batch(const WalkSeg* walks, int nwalk, const unsigned long long* level_off,
                              const unsigned long long* keys, const uint32_t* par, int32_t* orders, cudaStream_t s);

// Network kernels.
cudaError_t launch_mlp_forward(const float* params, const float* x, int batch, float* yhat, cudaStream_t s);
cudaError_t launch_mlp_grad(const float* params, const float* x, const float* y, int batch,
                            float* grad, float* partial, int partial_blocks, cudaStream_t s);
cudaError_t launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr,
                            float beta1, float beta2, float eps, cudaStream_t s);
cudaError_t launch_mlp_train(float* params, float* m, float* v, const float* x, const float* y,
                             int batch_total, int minibatch, int epochs, const int32_t* perm,
                             float lr, float* loss_out, cudaStream_t s);

}  // namespace tw
