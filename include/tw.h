/*
 * tw.h - C ABI of libtw, exact treewidth on one GB300 GPU (sm_103a).
 *
 * Method: van der Zanden & Bodlaender, "Computing Treewidth on the GPU"
 * (arXiv 1709.09990).
 *   Section 2: tw(G) = min over elimination orderings pi of
 *     max_v |Q({u : pi(u) < pi(v)}, v)|, where Q(S, v) is the set of vertices
 *     outside S u {v} reachable from v by a path whose interior lies in S.
 *   Section 3.1, Listing 1: decide(k) grows the wavefront level by level:
 *     L_0 = {empty set}; L_{i+1} = { S u {v} : S in L_i, v not in S,
 *     |Q(S,v)| <= k }, for i = 0 .. n-k-2; tw <= k iff L_{n-k-1} is not empty
 *     (the last k+1 vertices can be eliminated in any order).  The treewidth
 *     is the first k that answers yes.
 *   Section 3.2: duplicate sets are removed; here with an exact device hash
 *     table (the paper's Bloom filter can lose states and is not used).
 *   Section 3.1, last paragraph: the paper does not reconstruct orderings;
 *     libtw keeps one predecessor vertex per state and walks back.
 *
 * Conventions shared by every entry point
 *   Adjacency ("adj"): n rows, each W = ceil(n/64) little-endian uint64
 *     words; bit c of row r is set iff rc is an edge.  The graph must be
 *     simple and undirected: symmetric rows, zero diagonal, no bit >= n.
 *     1 <= n <= TW_MAX_N.  Anything else returns TW_ERR_INVALID.
 *   Pointers: every array argument may be host memory or device memory of
 *     the context's device (libtw asks the driver which one it is).  The
 *     caller owns all memory; libtw copies inputs before working and writes
 *     outputs before returning; it keeps no pointer after a call returns.
 *   Results are exact.  When the frontier or table would exceed the memory
 *     cap the call returns TW_ERR_CAPACITY and gives no answer; no state is
 *     ever dropped.
 *   A context is bound to one device and one stream and is not thread safe:
 *     use one context per host thread.
 */
#ifndef TW_H
#define TW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TW_MAX_N 128
#define TW_ABI_VERSION 3

/* Status codes. */
#define TW_OK 0
#define TW_ERR_INVALID 1  /* bad graph, n, k or NULL required pointer        */
#define TW_ERR_CAPACITY 2 /* frontier or table would exceed the memory cap   */
#define TW_ERR_TIMEOUT 3  /* a bounded device wait expired                   */
#define TW_ERR_CUDA 4     /* a CUDA runtime call failed                      */

typedef struct tw_ctx tw_ctx;

/* Context configuration; an all-zero struct selects every default. */
typedef struct {
  int device;             /* CUDA device ordinal                                  */
  int fingerprints;       /* 1: fill level_fp_sum / level_fp_xor in tw_stats     */
  size_t mem_cap_bytes;   /* device bytes libtw may hold; 0 = 150 GB or 90% free  */
  void* stream;           /* cudaStream_t to run on; NULL = a stream of libtw's  */
  int block_threads;      /* expand kernel block size; 0 = autotuned/default     */
  int table_load_pct;     /* hash table target load in percent; 0 = default (50) */
  int max_probes;         /* probe limit per insert; 0 = default (cap of table)  */
  int ub_shortcut;        /* tw_solve: accept the heuristic upper bound when the
                             lower bound meets it, without a decide run (0 = off) */
  int graph_levels;       /* 1: run each decide's level loop as one captured CUDA
                             graph when the context's buffers can hold it (else
                             the host loop); -1: host-driven loop, one host round
                             trip per level; 0: the library default.
                             spill_levels forces the host loop.                  */
  int time_kernels;       /* 1 = time every expand launch with CUDA events on the
                             context's stream (fills expand_seconds); in a
                             graph-driven level loop the events are event-record
                             nodes of the graph around each expand launch        */
  int clique_skip;        /* 1 = Section 3.1, first optimisation: a maximum clique
                             C (the one with the lexicographically smallest
                             sorted vertex list) is eliminated last, so decide
                             never adds a vertex of C and answers no at once when
                             |C| > k+1.  Answers are unchanged, level sets shrink.
                             tw_solve_batch ignores it.                          */
  int disjoint_paths;     /* 1 = Section 3.1, second optimisation: decide(k) adds
                             the edge uv for every non-adjacent pair joined by at
                             least k+1 internally vertex-disjoint paths in G.
                             Answers are unchanged; orderings are valid for G.
                             tw_solve_batch ignores it.                          */
  int autotune;           /* 1 = pick the expand block size and table load by
                             timing the first level of >= 2^18 states once per
                             (state width, n/8) and reuse the choice; the level
                             is recomputed per candidate, results are unchanged.
                             Explicit block_threads / table_load_pct win.        */
  int partition_table_mb; /* levels whose hash table exceeds this many MB insert
                             in two steps: the search writes the pairs grouped
                             by hash range, then the ranges are inserted one by
                             one into their slice of the table, which is emptied
                             in L2 just before and dropped from L2 without a
                             write-back after, so the table stays out of DRAM.
                             0 = 256 MB (the default), -1 = never, -2 = every
                             level.  Results are unchanged.                     */
  int mmw_prune;          /* 1 = Section 3.3: a state whose remaining graph has a
                             minor-min-width bound (second-smallest degree of each
                             contraction step) above k is not extended.  Answers
                             are unchanged, level sets shrink.  Ignored by
                             tw_solve_batch's batched kernel.                     */
  int spill_levels;       /* 1 = keep the finished levels, which only the ordering
                             walk reads, in pinned host memory instead of device
                             memory: the device then holds just the level being
                             expanded, the level being built and the table, so
                             frontiers that would not fit mem_cap_bytes with every
                             level resident can still be solved (Section 4.2: the
                             list capacity behind Table 1's starred rows).  Each level
                             is copied out once on the context's stream; the walk
                             reads the host copies in place.  Forces the host-
                             driven level loop.  Results are unchanged.  A failed
                             host allocation is TW_ERR_CAPACITY.                  */
  int out_of_core;        /* 1 = a decide run that needs no ordering goes on when a
                             level or its table would exceed mem_cap_bytes
                             (Section 4.2's list capacity; the Conclusions' future
                             work), instead of returning TW_ERR_CAPACITY: the
                             table is built in slices, one hash range at a time,
                             each slice small enough for the cap (the level's
                             search repeats once per slice), and a level that
                             does not fit the device next to its input and table
                             is written, wholly or in part, to pinned host
                             memory (Grace memory over NVLink-C2C on GB300; up
                             to host_cap_mb) and read from there by the next
                             level.  Results are unchanged.  tw_decide without
                             order, tw_decide_level and the decide runs of
                             tw_solve without outputs use it; a failed host
                             allocation is TW_ERR_CAPACITY.                      */
  int fused_states;       /* tw_solve / tw_decide on graphs with n <= 64 first run
                             the whole k sweep, walk and tree decomposition in one
                             cooperative launch (barriers between levels; the
                             decide runs k, k+1, k+2 of the sweep run at once in
                             three groups of blocks, and the first of them that
                             does not answer no decides, as in the sequential
                             sweep) whose level arenas hold this many states; a run
                             whose levels outgrow it goes on with the level loop
                             from the k it reached.  0 = 2^20 states (the
                             default), -1 = never.  Not used with clique_skip,
                             disjoint_paths, mmw_prune or spill_levels.  Results
                             are unchanged.                                      */
  int batch_kernel;       /* tw_solve_batch / tw_decide_batch: 0 = one persistent
                             launch for the whole batch, each block solving one
                             graph at a time from a device queue (the default);
                             1 = level-synchronous steps, one launch per step for
                             the current level of every running graph.  Results
                             are unchanged.                                      */
  int host_cap_mb;        /* out_of_core: pinned host memory, in MB, that levels
                             may occupy; 0 = 85% of the host's physical memory  */
  int batch_arena_states; /* persistent batched kernel: states each block's arena
                             holds (a power of two, 4096 .. 2^19; 0 = 2^16, less
                             when the cap is tight).  A graph whose decide run
                             outgrows it continues in the level-synchronous
                             batched kernel.                                     */
  int reserved[1];        /* must be zero                                         */
} tw_config;

/* Per-call statistics.  Level arrays describe the last decide run. */
typedef struct {
  int levels;                               /* levels computed (incl. L_0)     */
  int k;                                    /* bound of the last decide run    */
  uint64_t level_size[TW_MAX_N + 1];        /* |L_i|                            */
  uint64_t level_fp_sum[TW_MAX_N + 1];      /* sum of fp(S) over L_i (mod 2^64) */
  uint64_t level_fp_xor[TW_MAX_N + 1];      /* xor of fp(S) over L_i            */
  uint64_t states_expanded;                 /* sum of |L_i| over expanded levels,
                                               summed over every decide run    */
  uint64_t candidates;                      /* sum of |L_i| * (n - i), likewise */
  uint64_t generated;                       /* pairs (S, v) with |Q(S, v)| <= k
                                               submitted to the duplicate-removal
                                               table: only v in the component of
                                               G[S u {v}] holding its lowest
                                               vertex (every such pair with
                                               mmw_prune), see tw_decide        */
  uint64_t peak_frontier_bytes;             /* max over levels of the device
                                               bytes of kept lists + live table
                                               (levels spilled to host memory
                                               are not counted)                 */
  uint64_t decide_runs;                     /* decide runs in this call         */
  uint64_t level_retries;                   /* levels re-run after growing      */
  double seconds;                           /* wall time of the call            */
  uint64_t kernel_launches;                 /* libtw kernels launched by the call */
  uint64_t expand_launches;                 /* expand+insert launches           */
  double expand_seconds;                    /* summed CUDA-event time of those
                                               launches (time_kernels only)     */
  double expand_bytes;                      /* algorithmic bytes of those launches:
                                               sum over levels of (|L_i| + F_i +
                                               2|L_{i+1}|) * w + |L_{i+1}|, with
                                               w the key bytes and F_i the
                                               generated pairs of level i      */
} tw_stats;

/* fp(S) = mix(w0 ^ mix(w1)), mix = the splitmix64 output function, over the
 * two low words of S (zero-extended).  Used only for the level fingerprints. */

/* Creates a context on cfg->device.  cfg may be NULL (defaults).
 * Errors: TW_ERR_INVALID (out NULL, nonzero reserved), TW_ERR_CUDA. */
int tw_create(tw_ctx** out, const tw_config* cfg);

/* Frees every device buffer of the context.  NULL is ignored. */
void tw_destroy(tw_ctx* ctx);

/* Listing 1 at bound k (arXiv 1709.09990, Section 3.1).  The level sets are
 * exactly Listing 1's; each set is generated only from the parents that drop
 * a vertex of its lowest-vertex component (Q(S, v) depends only on v's
 * component of G[S u {v}], so no set is lost), which st->generated counts.
 *   adj   : n x ceil(n/64) uint64 rows (see conventions).
 *   k     : the bound, k >= 0.  k >= n-1 answers yes without expansion.
 *   yes   : out, 1 if tw <= k, else 0.
 *   order : out, n int32 (or NULL): on yes, an elimination ordering of width
 *           <= k (order[j] = the j-th vertex eliminated); untouched on no.
 *   st    : out statistics (or NULL).
 * Returns TW_OK or an error status; on error nothing is written to yes/order. */
int tw_decide(tw_ctx* ctx, const uint64_t* adj, int n, int k, int* yes, int32_t* order,
              tw_stats* st);

/* The wavefront itself: the sets of level `level` of decide(k) (Section 3.1,
 * Listing 1; the same run as tw_decide with the context's options, stopped
 * once that level is built).
 *   level : 0 .. n; a level after the run's last one (the run ended at an
 *           empty level, or level > n-k-1) has no sets.
 *   keys  : out, cap sets of W = ceil(n/64) uint64 words each (bit v of word
 *           v/64 = vertex v), in no particular order.  May be NULL when cap
 *           is 0.
 *   cap   : room in keys, in sets.
 *   count : out (required), |L_level|, also when it exceeds cap.
 *   st    : out statistics of the run (or NULL).
 * Returns TW_OK, or TW_ERR_CAPACITY when |L_level| > cap (nothing is written
 * to keys; *count tells the caller how much room to pass), or the errors of
 * tw_decide. */
int tw_decide_level(tw_ctx* ctx, const uint64_t* adj, int n, int k, int level, uint64_t* keys, uint64_t cap,
                    uint64_t* count, tw_stats* st);

/* As tw_decide for n <= 32 with one uint32 word per row (bit c of row r =
 * edge rc).  Runs the 32-bit state kernel. */
int tw_decide_u32(tw_ctx* ctx, const uint32_t* adj_rows, int n, int k, int* yes,
                  int32_t* order, tw_stats* st);

/* Exact treewidth: decide(k) for k = LB, LB+1, ... where LB = max(minimum-
 * degree bound, minor-min-width bound); the first yes is tw (Section 3.1,
 * iterative deepening).
 *   tw        : out, the treewidth.
 *   order     : out, n int32 (or NULL), an ordering of width tw.
 *   td_parent : out, n int32 (or NULL): bag of vertex v hangs below the bag of
 *               td_parent[v]; exactly one root has -1.
 *   td_bags   : out, n rows x ceil(n/64) uint64 (or NULL): bag of v =
 *               {v} u Q(prefix(v), v).  td_* need order's walk, so they are
 *               filled only when order or the td arrays are requested.
 *   st        : out (or NULL); level arrays describe the final (yes) run.   */
int tw_solve(tw_ctx* ctx, const uint64_t* adj, int n, int* tw, int32_t* order,
             int32_t* td_parent, uint64_t* td_bags, tw_stats* st);

/* Many graphs of uneven size in one batched run (the Section 3.1 sweep for
 * each graph).  By default one persistent launch
 * solves the graphs from a device queue, a block per graph (the whole k sweep,
 * certification and walk on the device); graphs whose decide runs outgrow a
 * block's arena (batch_arena_states) continue in level-synchronous steps that
 * expand the current level of every such graph over the whole GPU, and graphs
 * that outgrow those, or have n > 64, are solved one at a time
 * (batch_kernel = 1 uses the level-synchronous steps for every graph).
 *   adj_concat : the graphs' rows concatenated; graph g starts at word
 *                row_offset[g] and has n[g] rows of ceil(n[g]/64) words.
 *   n          : num_graphs vertex counts (1 .. 64 for the batched kernel;
 *                larger graphs are solved one at a time).
 *   tw         : out, num_graphs treewidths (-1 where status != TW_OK).
 *   orders     : out (or NULL), concatenated orderings; graph g's starts at
 *                the prefix sum of n[0..g-1].
 *   status     : out, num_graphs per-graph status.
 *   k_hint     : NULL for the plain sweep from the lower bound, else
 *                num_graphs proposed starting bounds: decide runs at
 *                round(k_hint) and round(k_hint)-1 and walks up or down from
 *                there until the answer is certified (yes at tw, no at tw-1).
 *   st         : out (or NULL): totals over all graphs.
 * Returns the worst per-graph status. */
int tw_solve_batch(tw_ctx* ctx, const uint64_t* adj_concat, const int32_t* n,
                   const int64_t* row_offset, int num_graphs, int* tw, int32_t* orders,
                   int* status, const float* k_hint, tw_stats* st);

/* decide(k[g]) for many graphs of uneven size (Section 3.1, Listing 1 per
 * graph), through the same batched kernel as tw_solve_batch (graphs with
 * n > 64, and graphs whose levels outgrow the batch, run one at a time).
 * The level sets are those of the plain method: clique_skip, disjoint_paths
 * and mmw_prune are not applied.
 *   adj_concat, n, row_offset : as tw_solve_batch.
 *   k          : num_graphs bounds, k[g] >= 0.
 *   yes        : out, num_graphs answers (1 iff tw(G_g) <= k[g]).
 *   status     : out, num_graphs per-graph status.
 *   level_size : out (or NULL), num_graphs rows of TW_MAX_N+1 uint64: row g
 *                holds |L_0|, |L_1|, ... of graph g's run (up to and
 *                including its first empty level), then zeros.
 *   level_fp_sum, level_fp_xor : out (or NULL), the same layout: the sum and
 *                xor of fp(S) over each level (see tw_stats).
 *   st         : out (or NULL): totals over all graphs.
 * Returns the worst per-graph status. */
int tw_decide_batch(tw_ctx* ctx, const uint64_t* adj_concat, const int32_t* n, const int64_t* row_offset,
                    int num_graphs, const int32_t* k, int* yes, int* status, uint64_t* level_size,
                    uint64_t* level_fp_sum, uint64_t* level_fp_xor, tw_stats* st);

/* Lower and upper bounds on the device (one warp per graph):
 * out[0] = minimum-degree (degeneracy) bound, out[1] = minor-min-width
 * (MMD+, Section 3.3), out[2] = width of the greedy minimum-degree ordering,
 * out[3] = width of the greedy minimum-fill ordering.  Ties: lowest index. */
int tw_bounds(tw_ctx* ctx, const uint64_t* adj, int n, int32_t out[4]);

/* The 12 features of the learned starting bound for many graphs (same
 * concatenated layout as tw_solve_batch), one warp per graph, fp32:
 * 0 n/64; 1 density; 2-5 min/max/mean/std degree over n; 6-9 fraction of
 * vertices with degree/n in [0,.25), [.25,.5), [.5,.75), [.75,1];
 * 10 MMD+/n; 11 (min-degree width + min-fill width)/(2n).
 *   feats : out, num_graphs x 12 float (row-major). */
int tw_features_batch(tw_ctx* ctx, const uint64_t* adj_concat, const int32_t* n,
                      const int64_t* row_offset, int num_graphs, float* feats);

/* The 12-32-1 ReLU network that proposes a starting bound (no counterpart in
 * the paper; every answer it leads to is still certified by decide runs).
 * Parameters: 449 float, W1 [32][12] row-major, b1[32], W2[32], b2.
 *   tw_mlp_forward : yhat[b] = W2 . relu(W1 x_b + b1) + b2 for b < batch.
 *   tw_mlp_grad    : grad (449 float) of (1/B) sum_b (yhat_b - y_b)^2.
 *   tw_mlp_adam    : one Adam step (Kingma & Ba) in place on params, m, v at
 *                    step t >= 1 with the given hyper-parameters.
 *   tw_mlp_train   : epochs of minibatch Adam over (x, y); perm holds
 *                    epochs x batch_total sample indices (the random order is
 *                    drawn by the caller); loss_out (epochs floats, or NULL)
 *                    gets the mean training loss of each epoch. */
int tw_mlp_forward(tw_ctx* ctx, const float* params, const float* x, int batch, float* yhat);
int tw_mlp_grad(tw_ctx* ctx, const float* params, const float* x, const float* y, int batch,
                float* grad);
int tw_mlp_adam(tw_ctx* ctx, float* params, const float* grad, float* m, float* v, int t,
                float lr, float beta1, float beta2, float eps);
int tw_mlp_train(tw_ctx* ctx, float* params, const float* x, const float* y, int batch_total,
                 int minibatch, int epochs, const int32_t* perm, float lr, float* loss_out);

/* One wavefront level that allocates nothing (the paper has no counterpart;
 * this exists for callers that cannot let a library call cudaMalloc, e.g. a
 * host that has already given the device's memory to its own pool, or a
 * latency-critical loop that cannot take the device-wide synchronisation of
 * cudaMalloc/cudaFree).
 * It runs the expand+insert kernel of tw_decide for one level i -> i+1 on the
 * current device and the given stream (NULL = the legacy default stream).
 * Its hash table and counters live in a fixed static device array of 16 MiB
 * + 256 bytes inside libtw, held by every GPU that loads the library until
 * the process exits.
 *   d_in_keys  : device, n_in 64-bit keys of level i (bit v = vertex v).
 *                The output is level i+1 when the input is the whole of
 *                level i: like tw_decide, each set is extended only by the
 *                vertices of the component of S u {v} that holds its lowest
 *                vertex, so from part of a level the output holds just those
 *                canonical extensions of the given sets.
 *   d_adj      : device, n 64-bit adjacency rows, n <= 64.
 *   k          : the bound.
 *   d_out_keys : device, out_cap keys of level i+1 (written in any order).
 *   d_out_pred : device, out_cap bytes: the vertex added to each output key.
 *   out_cap    : at most TW_STATIC_MAX_STATES; larger values return
 *                TW_ERR_INVALID without running.
 *   out_count  : host, receives |L_{i+1}|, also when it exceeds out_cap,
 *                as long as the level fits the fixed table (about 2^21
 *                states).  A level that fills the whole table yields
 *                TW_ERR_CAPACITY with *out_count set above
 *                TW_STATIC_MAX_STATES; the value is then only a lower bound,
 *                and no call of this entry point can build that level.
 * Returns TW_OK; TW_ERR_CAPACITY when level i+1 has more than out_cap states
 * (or the fixed table overflows) - the output is then incomplete;
 * TW_ERR_INVALID for host pointers, n > 64, out_cap too large, or, when
 * n = 64, an input set of 63 or 64 vertices (its extension would be the
 * all-ones set, which the table uses as its empty marker); TW_ERR_CUDA.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress).  Every call reads its counters back and
 * synchronises the stream, so it must not be called while the stream is
 * being captured into a CUDA graph.  Every call reuses the same array: calls
 * that overlap on the GPU (other streams, other host threads) race and
 * corrupt each other. */
#define TW_STATIC_MAX_STATES (1ull << 20)
int tw_expand_level_static(const uint64_t* d_in_keys, uint64_t n_in, const uint64_t* d_adj, int n, int k,
                           uint64_t* d_out_keys, uint8_t* d_out_pred, uint64_t out_cap,
                           uint64_t* out_count, void* stream);

/* Human-readable name of a status code (static storage). */
const char* tw_strerror(int status);

/* ABI version (TW_ABI_VERSION of the library that was loaded). */
int tw_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TW_H */
