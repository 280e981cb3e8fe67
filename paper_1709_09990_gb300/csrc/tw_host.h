// Host-side internals of libtw shared by its translation units (not part of
// the ABI): the context, the validated-graph and level records, the small
// device buffer layout, and the helpers between the C entry points
// (tw_api.cu), the decide/solve drivers (tw_decide.cu), the batched driver
// (tw_batch_host.cu) and the common host utilities (tw_host.cu).
#pragma once

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/tw.h"
#include "tw_internal.h"

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

namespace tw {
namespace host {

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace host
}  // namespace tw

using tw::FusedState;
using tw::GraphState;
using tw::LevelCounters;
using tw::host::DevBuf;

struct tw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t mem_cap = 0;
  tw_config cfg{};
  DevBuf keys, pred, table, small;  // small: adjacency, walk, order, td scratch
  DevBuf scratch;                    // staged batch inputs/outputs and network data
  DevBuf cand_key, cand_v, part_meta;  // regions of the partitioned insert
  DevBuf ooc_keys;                   // second level buffer of out-of-core decide runs
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
    std::vector<cudaEvent_t> ev;  // with time_kernels: start and end of every level's expand
  };
  std::vector<GraphEntry> graphs;
  GraphState* d_gstate = nullptr;
  GraphState* h_gstate = nullptr;
  // autotuned (block threads, table load) per (key class, n / 8)
  struct Tuned {
    int kc, nb, block_threads, load_pct;
  };
  std::vector<Tuned> tuned;
  int batch_warps = 0;  // warps per block of the persistent batch kernel (autotuned once)
  // pinned host chunks that hold finished levels with spill_levels; reused
  // from the start by every decide run
  struct HostChunk {
    char* ptr;   // host address
    char* dptr;  // device-side address of the same bytes
    size_t bytes;
  };
  std::vector<HostChunk> host_chunks;
  size_t host_chunk = 0, host_used = 0;  // allocation cursor of the current run
  // out-of-core decide runs: two pinned, device-mapped host buffers that hold
  // the levels that do not fit the device (reused from run to run)
  HostChunk ooc_host[2] = {{nullptr, nullptr, 0}, {nullptr, nullptr, 0}};
  // fused small solves: state, two tables and the level arena in one buffer,
  // a pinned mirror of the state, and the graphs whose fused run gave up
  DevBuf fused;
  bool fused_clean = false;  // every table slot of the fused buffer is empty
  FusedState* h_fused = nullptr;
  unsigned char* h_out = nullptr;  // pinned mirror of the small buffer's order .. bags region
  std::vector<unsigned long long> fused_skip;
  // options of Section 3.1 for the decide run being prepared
  unsigned long long allowed[2] = {~0ull, ~0ull};
  int skipped = 0;  // vertices excluded from the sets (|C| with the clique skip)
};

namespace tw {
namespace host {

constexpr size_t kSmallBytes = 1 << 20;

// A named NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* fmt, int a = 0, int b = 0) {
    char name[64];
    std::snprintf(name, sizeof(name), fmt, a, b);
    nvtxRangePushA(name);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double seconds() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

// A validated graph in the 64-bit-word row layout of the ABI.
struct HostGraph {
  int n = 0;
  int words = 1;
  std::vector<uint64_t> rows;  // n * words
};

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

struct LevelRec {
  unsigned long long off = 0;
  unsigned long long count = 0;
  const char* hkeys = nullptr;     // host copy (spill_levels), else in c->keys at off
  const char* htail = nullptr;     // out of core: the last `tail` keys, in host memory
  unsigned long long tail = 0;
  const uint8_t* hpred = nullptr;  // host copy of the predecessors, else in c->pred
};

struct DecideResult {
  int yes = 0;
  std::vector<LevelRec> levels;
  unsigned long long states_expanded = 0, candidates = 0, generated = 0, peak_bytes = 0, retries = 0;
  unsigned long long expand_launches = 0;
  double expand_seconds = 0.0, expand_bytes = 0.0;
  std::vector<unsigned long long> fp_sum, fp_xor;
};

// ---- tw_host.cu: pointers, buffers, graphs
bool is_device_ptr(const void* p);
int fetch(void* dst_host, const void* src, size_t bytes);
int put(tw_ctx* c, void* dst, const void* src_host, size_t bytes);
int put_from_device(tw_ctx* c, void* dst, const void* src_dev, size_t bytes);
// The ordering, tree-decomposition parents and bags of a solve from the small
// buffer into the caller's pointers (each host, device or NULL) with one
// stream synchronisation.
int put_solution(tw_ctx* c, int n, int words, int32_t* order, int32_t* td_parent, uint64_t* td_bags);
size_t total_bytes(const tw_ctx* c);
int grow(tw_ctx* c, DevBuf* b, size_t need, size_t keep);
int host_take(tw_ctx* c, size_t bytes, char** out);
int validate(const uint64_t* rows, int n, HostGraph* g);
int load_graph(const uint64_t* adj, int n, HostGraph* g);
char* small_at(tw_ctx* c, size_t off);
int upload_graph(tw_ctx* c, const HostGraph& g, KeyClass kc);
unsigned long long next_pow2(unsigned long long x);
double binom(int n, int r);

// ---- tw_decide.cu: decide runs, the k sweep, reconstruction
int decide_graph(tw_ctx* c, const HostGraph& g, int k, int* yes, int32_t* order, tw_stats* st);
int level_keys_graph(tw_ctx* c, const HostGraph& g, int k, int level, uint64_t* keys, uint64_t cap, uint64_t* count,
                     tw_stats* st);
int bounds_graph(tw_ctx* c, const HostGraph& g, int32_t out[4], bool lower_only = false);
int solve_graph(tw_ctx* c, const HostGraph& g, int* tw_out, int32_t* order, int32_t* td_parent, uint64_t* td_bags,
                tw_stats* st, int k_first);
int solve_hinted(tw_ctx* c, const HostGraph& g, float hint, int* tw_out, std::vector<int32_t>* order_host,
                 tw_stats* st);

// ---- tw_batch_host.cu: many graphs
int solve_batch_gpu(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                    const std::vector<float>* hint, const std::vector<int64_t>& order_off, int* htw,
                    std::vector<int32_t>* hord, std::vector<int>* hst, tw_stats* st);
int decide_batch_gpu(tw_ctx* c, const std::vector<HostGraph>& graphs, const std::vector<int>& idx,
                     const std::vector<int>& kk, std::vector<int>* yes, std::vector<int>* hst,
                     std::vector<std::vector<unsigned long long>>* size,
                     std::vector<std::vector<unsigned long long>>* fp_sum,
                     std::vector<std::vector<unsigned long long>>* fp_xor, tw_stats* st);
int load_batch(const uint64_t* adj_concat, const int32_t* n, const int64_t* row_offset, int num_graphs,
               std::vector<int32_t>* hn, std::vector<int64_t>* hoff, std::vector<uint64_t>* hadj);

}  // namespace host
}  // namespace tw
