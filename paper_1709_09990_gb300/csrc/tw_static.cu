// One wavefront level without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host application that
// has already handed the device's memory to its own pool (a cudaMalloc would
// fail or fragment that pool), or a latency-critical loop that cannot afford
// the implicit device-wide synchronisation of cudaMalloc/cudaFree.  For them,
// tw_expand_level_static runs the same expand+insert kernel as tw_decide on
// buffers the caller owns, with the kernel's hash table and counters placed in
// a fixed scratch array that lives in this file as a static __device__
// variable.  Every GPU that loads the library holds that array until the
// process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/tw.h"
#include "tw_internal.h"

using namespace tw;

namespace {

constexpr unsigned long long kStaticSlots = 1ull << 21;  // 16 MiB of 64-bit slots
constexpr size_t kStaticTableBytes = kStaticSlots * sizeof(unsigned long long);
constexpr size_t kStaticCounterBytes = 256;  // one LevelCounters, padded
constexpr int kMaxDevices = 64;

static_assert(sizeof(LevelCounters) <= kStaticCounterBytes, "counters must fit their slot");

}  // namespace

// The scratch of tw_expand_level_static: the hash table followed by the level
// counters.  In host code this name is only a stand-in for the device
// variable; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char tw_static_scratch[kStaticTableBytes + kStaticCounterBytes];

namespace {

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, resolved once
// per device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TW_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, tw_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TW_ERR_CUDA;
    }
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return TW_OK;
}

// Sets *flag when an input set has 63 or more of the 64 vertices: its
// extensions would include the all-ones set, which is the table's empty
// marker (a 64-vertex graph only).
__global__ void wide_input_kernel(const unsigned long long* __restrict__ keys, unsigned long long n_in,
                                  unsigned int* flag) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += stride)
    if (__popcll(keys[i]) >= 63) *flag = 1u;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (p == nullptr || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int tw_expand_level_static(const uint64_t* d_in_keys, uint64_t n_in, const uint64_t* d_adj, int n, int k,
                                      uint64_t* d_out_keys, uint8_t* d_out_pred, uint64_t out_cap,
                                      uint64_t* out_count, void* stream) {
  if (out_count == nullptr || n < 1 || n > 64 || k < 0) return TW_ERR_INVALID;
  if (out_cap > TW_STATIC_MAX_STATES) return TW_ERR_INVALID;  // beyond the fixed scratch table
  if (n_in == 0) {
    *out_count = 0;
    return TW_OK;
  }
  if (!on_device(d_in_keys) || !on_device(d_adj) || !on_device(d_out_keys) || !on_device(d_out_pred))
    return TW_ERR_INVALID;
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != TW_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* table = scratch;
  LevelCounters* ctr = reinterpret_cast<LevelCounters*>(static_cast<unsigned char*>(scratch) + kStaticTableBytes);
  // Only the slots this call needs are emptied: twice the output capacity
  // (at most 50% load while the level fits out_cap).  If that smaller table
  // fills up (a level far above out_cap), the level runs once more over the
  // whole array so that the count it reports is still exact.
  unsigned long long slots = 1024;
  while (slots < 2 * out_cap && slots < kStaticSlots) slots <<= 1;
  LevelCounters h;
  for (;;) {
    // The array keeps the previous call's contents: empty the slots and zero
    // the counters before this call's inserts.
    if (launch_clear(table, slots * sizeof(unsigned long long), ctr, s) != cudaSuccess) {
      cudaGetLastError();
      return TW_ERR_CUDA;
    }
    if (n == 64) {
      wide_input_kernel<<<(int)std::min<unsigned long long>((n_in + 255) / 256, 1024), 256, 0, s>>>(
          reinterpret_cast<const unsigned long long*>(d_in_keys), n_in, &ctr->pad[0]);
      if (cudaGetLastError() != cudaSuccess) return TW_ERR_CUDA;
    }
    ExpandLaunch a;
    a.kc = kKey64;
    a.in_keys = d_in_keys;
    a.n_in = n_in;
    a.adj = d_adj;
    a.n = n;
    a.k = k;
    a.table = table;
    a.table_slots = slots;
    a.max_probes = 256;
    a.out_keys = d_out_keys;
    a.out_pred = d_out_pred;
    a.out_cap = out_cap;
    a.ctr = ctr;
    a.block_threads = 128;
    a.grid = 0;
    a.allowed[0] = ~0ull;
    a.allowed[1] = ~0ull;
    a.mmw = 0;
    if (launch_expand(a, s) != cudaSuccess) {
      cudaGetLastError();
      return TW_ERR_CUDA;
    }
    if (cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return TW_ERR_CUDA;
    }
    if (h.pad[0] != 0u) return TW_ERR_INVALID;  // a 63- or 64-vertex input set, n = 64
    if (!(h.overflow & 2u) || slots == kStaticSlots) break;
    slots = kStaticSlots;
  }
  if (h.overflow & 2u) {
    // the whole array filled before every pair was placed: the count is only
    // a lower bound, reported above the limit of this entry point
    *out_count = std::max<unsigned long long>(h.out_count, TW_STATIC_MAX_STATES + 1);
    return TW_ERR_CAPACITY;
  }
  *out_count = h.out_count;
  if (h.overflow != 0 || h.out_count > out_cap) return TW_ERR_CAPACITY;
  return TW_OK;
}
