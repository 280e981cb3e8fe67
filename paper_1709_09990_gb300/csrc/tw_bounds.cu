// Treewidth bounds and graph features, one warp per graph.
//
// Lower bounds (start of the k sweep):
//   MMD  - degeneracy: repeatedly delete a minimum-degree vertex; the largest
//          minimum degree seen.
//   MMD+ - minor-min-width (arXiv 1709.09990, Section 3.3): repeatedly take a
//          minimum-degree vertex v, record its degree, and contract it into
//          its minimum-degree neighbour u; an isolated v is deleted.  Minors
//          do not raise treewidth, so the largest degree recorded is a bound.
// Upper bounds: widths of the greedy minimum-degree and minimum-fill
// elimination orderings.  Ties go to the lowest vertex index everywhere.
//
// Each lane owns the vertices lane, lane+32, lane+64, lane+96; the rows of
// the graph being reduced live in shared memory and the argmin of a step is a
// warp shuffle reduction.
#include <cuda_runtime.h>

#include "tw_internal.h"
#include "tw_keys.cuh"

namespace tw {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;

// Warp-wide minimum of (val, idx), lowest idx on ties; idx < 0 means none.
// One warp reduction of the packed value val << 8 | idx (0 <= val < 2^24,
// idx < 128) replaces a chain of shuffles: the selection loops of the bounds
// are sequences of these argmins, so their latency is the kernel's time.
__device__ __forceinline__ void warp_argmin(int& val, int& idx) {
  const unsigned packed = idx < 0 ? 0xffffffffu : ((unsigned)val << 8) | (unsigned)idx;
  const unsigned m = __reduce_min_sync(kFull, packed);
  if (m == 0xffffffffu) {
    val = 1 << 30;
    idx = -1;
  } else {
    val = (int)(m >> 8);
    idx = (int)(m & 0xffu);
  }
}

__device__ __forceinline__ void load_rows(K128* rows, const unsigned long long* adj, int n, int W, int lane) {
  for (int u = lane; u < n; u += 32)
    rows[u] = K128{adj[(size_t)u * W], W > 1 ? adj[(size_t)u * W + 1] : 0ull};
  __syncwarp();
}

// Minimum degree among alive vertices of `among` (lowest index on ties).
__device__ __forceinline__ void min_degree(const K128* rows, K128 alive, K128 among, int n, int lane, int& d,
                                           int& v) {
  d = 1 << 30;
  v = -1;
  for (int u = lane; u < n; u += 32) {
    if (!ktest(among, u)) continue;
    const int du = kpopc(rows[u] & alive);
    if (v < 0 || du < d) {
      d = du;
      v = u;
    }
  }
  warp_argmin(d, v);
}

__device__ int bound_mmd(K128* rows, const unsigned long long* adj, int n, int W, int lane) {
  load_rows(rows, adj, n, W, lane);
  K128 alive = kfirst_n<K128>(n);
  int lb = 0;
  for (int step = 0; step < n; ++step) {
    int d, v;
    min_degree(rows, alive, alive, n, lane, d, v);
    lb = max(lb, d);
    alive &= ~kbit<K128>(v);
  }
  return lb;
}

__device__ int bound_mmd_plus(K128* rows, const unsigned long long* adj, int n, int W, int lane) {
  load_rows(rows, adj, n, W, lane);
  K128 alive = kfirst_n<K128>(n);
  int lb = 0;
  while (kpopc(alive) >= 2) {
    int d, v;
    min_degree(rows, alive, alive, n, lane, d, v);
    lb = max(lb, d);
    if (d == 0) {
      alive &= ~kbit<K128>(v);
      continue;
    }
    const K128 nv = rows[v] & alive;
    int du, u;
    min_degree(rows, alive, nv, n, lane, du, u);
    __syncwarp();
    for (int w = lane; w < n; w += 32) {
      if (w == u) rows[w] |= nv & ~kbit<K128>(u);
      else if (ktest(nv, w)) rows[w] |= kbit<K128>(u);
    }
    __syncwarp();
    alive &= ~kbit<K128>(v);
  }
  return lb;
}

// Eliminates v: its alive neighbourhood becomes a clique.
__device__ __forceinline__ void eliminate(K128* rows, K128& alive, int v, int n, int lane) {
  const K128 nv = rows[v] & alive;
  __syncwarp();
  for (int w = lane; w < n; w += 32)
    if (ktest(nv, w)) rows[w] |= nv & ~kbit<K128>(w);
  __syncwarp();
  alive &= ~kbit<K128>(v);
}

__device__ int ub_min_degree(K128* rows, const unsigned long long* adj, int n, int W, int lane) {
  load_rows(rows, adj, n, W, lane);
  K128 alive = kfirst_n<K128>(n);
  int width = 0;
  for (int step = 0; step < n; ++step) {
    int d, v;
    min_degree(rows, alive, alive, n, lane, d, v);
    width = max(width, d);
    eliminate(rows, alive, v, n, lane);
  }
  return width;
}

__device__ int ub_min_fill(K128* rows, const unsigned long long* adj, int n, int W, int lane) {
  load_rows(rows, adj, n, W, lane);
  K128 alive = kfirst_n<K128>(n);
  int width = 0;
  for (int step = 0; step < n; ++step) {
    int f = 1 << 30, v = -1;
    for (int u = lane; u < n; u += 32) {
      if (!ktest(alive, u)) continue;
      const K128 nu = rows[u] & alive;
      int missing2 = 0;
      K128 t = nu;
      while (!kempty(t)) {
        const int a = klowest(t);
        t = kdrop_lowest(t);
        missing2 += kpopc(nu & ~rows[a] & ~kbit<K128>(a));
      }
      const int fu = missing2 / 2;
      if (v < 0 || fu < f) {
        f = fu;
        v = u;
      }
    }
    warp_argmin(f, v);
    width = max(width, kpopc(rows[v] & alive));
    eliminate(rows, alive, v, n, lane);
  }
  return width;
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    bounds_kernel(const unsigned long long* __restrict__ adj, const int32_t* __restrict__ ns,
                  const int64_t* __restrict__ offs, int num_graphs, int32_t* out, float* feats, int lower_only) {
  __shared__ K128 sRows[kWarpsPerBlock][128];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * kWarpsPerBlock + warp;
  if (g >= num_graphs) return;
  const int n = ns[g];
  const int W = (n + 63) / 64;
  const unsigned long long* a = adj + offs[g];
  K128* rows = sRows[warp];
  const int mmd = bound_mmd(rows, a, n, W, lane);
  const int mmdp = bound_mmd_plus(rows, a, n, W, lane);
  // (the greedy widths take most of the time; a k sweep needs only the lower bounds)
  const bool ub = !lower_only || feats;
  const int ubd = ub ? ub_min_degree(rows, a, n, W, lane) : -1;
  const int ubf = ub ? ub_min_fill(rows, a, n, W, lane) : -1;
  if (out && lane == 0) {
    out[4 * g + 0] = mmd;
    out[4 * g + 1] = mmdp;
    out[4 * g + 2] = ubd;
    out[4 * g + 3] = ubf;
  }
  if (feats) {
    // degree statistics of the input graph
    load_rows(rows, a, n, W, lane);
    long long sum = 0, sum2 = 0;
    int dmin = 1 << 30, dmax = 0;
    int h0 = 0, h1 = 0, h2 = 0, h3 = 0;
    for (int u = lane; u < n; u += 32) {
      const int d = kpopc(rows[u]);
      sum += d;
      sum2 += (long long)d * d;
      dmin = min(dmin, d);
      dmax = max(dmax, d);
      // bins d/n in [0,1/4), [1/4,1/2), [1/2,3/4), [3/4,1], compared in integers
      if (4 * d < n) ++h0;
      else if (2 * d < n) ++h1;
      else if (4 * d < 3 * n) ++h2;
      else ++h3;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      sum += __shfl_xor_sync(kFull, sum, d);
      sum2 += __shfl_xor_sync(kFull, sum2, d);
      dmin = min(dmin, __shfl_xor_sync(kFull, dmin, d));
      dmax = max(dmax, __shfl_xor_sync(kFull, dmax, d));
      h0 += __shfl_xor_sync(kFull, h0, d);
      h1 += __shfl_xor_sync(kFull, h1, d);
      h2 += __shfl_xor_sync(kFull, h2, d);
      h3 += __shfl_xor_sync(kFull, h3, d);
    }
    if (lane == 0) {
      const double dn = (double)n;
      float* f = feats + (size_t)g * 12;
      f[0] = (float)(dn / 64.0);
      f[1] = n > 1 ? (float)((double)sum / (dn * (dn - 1.0))) : 0.0f;
      f[2] = (float)((double)dmin / dn);
      f[3] = (float)((double)dmax / dn);
      f[4] = (float)((double)sum / (dn * dn));
      const long long num = (long long)n * sum2 - sum * sum;  // n^2 * variance
      f[5] = (float)(sqrt((double)num) / (dn * dn));
      f[6] = (float)(h0 / dn);
      f[7] = (float)(h1 / dn);
      f[8] = (float)(h2 / dn);
      f[9] = (float)(h3 / dn);
      f[10] = (float)(mmdp / dn);
      f[11] = (float)((double)(ubd + ubf) / (2.0 * dn));
    }
  }
}

}  // namespace

cudaError_t launch_bounds(const unsigned long long* adj, const int32_t* n, const int64_t* row_offset, int num_graphs,
                          int32_t* out, float* feats, cudaStream_t s, int lower_only) {
  if (num_graphs <= 0) return cudaSuccess;
  const int blocks = (num_graphs + kWarpsPerBlock - 1) / kWarpsPerBlock;
  bounds_kernel<<<blocks, kWarpsPerBlock * 32, 0, s>>>(adj, n, row_offset, num_graphs, out, feats, lower_only);
  return cudaGetLastError();
}

}  // namespace tw
