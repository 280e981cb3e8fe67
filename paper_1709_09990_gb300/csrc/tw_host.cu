// Host utilities of libtw: host/device pointers, growing device buffers within
// the context's memory cap, graph validation and upload.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tw_host.h"

namespace tw {
namespace host {

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

int put_solution(tw_ctx* c, int n, int words, int32_t* order, int32_t* td_parent, uint64_t* td_bags) {
  SmallLayout L;
  struct Part {
    void* dst;
    size_t off, bytes;
  } parts[3] = {{order, L.order, (size_t)n * 4},
                {td_parent, L.parent, (size_t)n * 4},
                {td_bags, L.bags, (size_t)n * (size_t)words * 8}};
  bool any_host = false;
  for (const Part& p : parts) {
    if (!p.dst) continue;
    if (is_device_ptr(p.dst))
      TW_CK(cudaMemcpyAsync(p.dst, small_at(c, p.off), p.bytes, cudaMemcpyDeviceToDevice, c->stream));
    else
      any_host = true;
  }
  if (any_host) {
    // the region order .. bags in one copy into the pinned mirror
    constexpr size_t kRegion = SmallLayout().bounds - SmallLayout().order;
    if (!c->h_out) {
      if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_out), kRegion, cudaHostAllocDefault) != cudaSuccess) {
        c->h_out = nullptr;
        cudaGetLastError();
        return TW_ERR_CUDA;
      }
    }
    TW_CK(cudaMemcpyAsync(c->h_out, small_at(c, L.order), kRegion, cudaMemcpyDeviceToHost, c->stream));
  }
  TW_CK(cudaStreamSynchronize(c->stream));
  if (any_host)
    for (const Part& p : parts)
      if (p.dst && !is_device_ptr(p.dst)) std::memcpy(p.dst, c->h_out + (p.off - L.order), p.bytes);
  return TW_OK;
}

size_t total_bytes(const tw_ctx* c) {
  return c->keys.bytes + c->pred.bytes + c->table.bytes + c->cand_key.bytes + c->cand_v.bytes + c->ooc_keys.bytes;
}

// Takes bytes (rounded up to 256) of pinned, device-mapped host memory from
// the context's chunks, allocating a chunk of at least kHostChunkBytes when
// the current ones are full; *out is the device-side address of the bytes.
// A failed allocation is TW_ERR_CAPACITY.
int host_take(tw_ctx* c, size_t bytes, char** out) {
  constexpr size_t kHostChunkBytes = 256ull << 20;
  bytes = (bytes + 255) & ~size_t(255);
  while (c->host_chunk < c->host_chunks.size()) {
    const tw_ctx::HostChunk& ch = c->host_chunks[c->host_chunk];
    if (c->host_used + bytes <= ch.bytes) {
      *out = ch.dptr + c->host_used;
      c->host_used += bytes;
      return TW_OK;
    }
    ++c->host_chunk;
    c->host_used = 0;
  }
  const size_t want = std::max(bytes, kHostChunkBytes);
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
  c->host_chunks.push_back({static_cast<char*>(p), static_cast<char*>(d), want});
  c->host_chunk = c->host_chunks.size() - 1;
  c->host_used = bytes;
  *out = static_cast<char*>(d);
  return TW_OK;
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

}  // namespace host
}  // namespace tw
