// C ABI of libtw (include/tw.h): argument checks, contexts, staging of host or
// device arrays, and dispatch to the drivers in tw_decide.cu and
// tw_batch_host.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tw_host.h"

using namespace tw;
using namespace tw::host;

namespace {

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

size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }

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
  for (DevBuf* b : {&c->keys, &c->pred, &c->table, &c->small, &c->scratch, &c->cand_key, &c->cand_v, &c->part_meta,
                    &c->ooc_keys, &c->fused})
    if (b->ptr) cudaFree(b->ptr);
  for (const tw_ctx::HostChunk& ch : c->host_chunks) cudaFreeHost(ch.ptr);
  for (const tw_ctx::HostChunk& ch : c->ooc_host)
    if (ch.ptr) cudaFreeHost(ch.ptr);
  if (c->d_ctr) cudaFree(c->d_ctr);
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_fused) cudaFreeHost(c->h_fused);
  for (auto& e : c->graphs) {
    cudaGraphExecDestroy(e.exec);
    for (cudaEvent_t v : e.ev) cudaEventDestroy(v);
  }
  if (c->d_gstate) cudaFree(c->d_gstate);
  if (c->h_gstate) cudaFreeHost(c->h_gstate);
  if (c->h_out) cudaFreeHost(c->h_out);
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

int tw_decide_level(tw_ctx* c, const uint64_t* adj, int n, int k, int level, uint64_t* keys, uint64_t cap,
                    uint64_t* count, tw_stats* st) {
  if (!c || !count || k < 0 || level < 0) return TW_ERR_INVALID;
  TW_CK(cudaSetDevice(c->device));
  HostGraph g;
  int rc = load_graph(adj, n, &g);
  if (rc) return rc;
  return level_keys_graph(c, g, k, level, keys, cap, count, st);
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

int tw_decide_batch(tw_ctx* c, const uint64_t* adj_concat, const int32_t* n, const int64_t* row_offset,
                    int num_graphs, const int32_t* k, int* yes, int* status, uint64_t* level_size,
                    uint64_t* level_fp_sum, uint64_t* level_fp_xor, tw_stats* st) {
  if (!c || !k || !yes || !status || num_graphs < 0) return TW_ERR_INVALID;
  Timer t;
  TW_CK(cudaSetDevice(c->device));
  std::vector<int32_t> hn;
  std::vector<int64_t> hoff;
  std::vector<uint64_t> hadj;
  int rc = load_batch(adj_concat, n, row_offset, num_graphs, &hn, &hoff, &hadj);
  if (rc) return rc;
  const int G = num_graphs;
  std::vector<int32_t> hk(G);
  if ((rc = fetch(hk.data(), k, (size_t)G * 4))) return rc;
  std::vector<HostGraph> graphs(G);
  std::vector<int> hst(G, TW_OK), valid, hyes(G, 0), kk(G, 0);
  for (int g = 0; g < G; ++g) {
    hst[g] = validate(hadj.data() + hoff[g], hn[g], &graphs[g]);
    if (hst[g] == TW_OK && hk[g] < 0) hst[g] = TW_ERR_INVALID;
    if (hst[g] == TW_OK) valid.push_back(g);
    kk[g] = hk[g];
  }
  std::vector<std::vector<unsigned long long>> sizes(G), fs(G), fx(G);
  if (st) std::memset(st, 0, sizeof(*st));
  const unsigned long long launches0 = c->launches;
  rc = decide_batch_gpu(c, graphs, valid, kk, &hyes, &hst, &sizes, level_fp_sum ? &fs : nullptr,
                        level_fp_xor ? &fx : nullptr, st);
  if (rc) return rc;
  int worst = TW_OK;
  for (int g = 0; g < G; ++g) worst = std::max(worst, hst[g]);
  if ((rc = put(c, yes, hyes.data(), (size_t)G * sizeof(int)))) return rc;
  if ((rc = put(c, status, hst.data(), (size_t)G * sizeof(int)))) return rc;
  const size_t L = TW_MAX_N + 1;
  auto flat = [&](const std::vector<std::vector<unsigned long long>>& v, uint64_t* dst) -> int {
    if (!dst) return TW_OK;
    std::vector<uint64_t> h((size_t)G * L, 0ull);
    for (int g = 0; g < G; ++g)
      for (size_t i = 0; i < v[g].size() && i < L; ++i) h[(size_t)g * L + i] = v[g][i];
    return put(c, dst, h.data(), h.size() * 8);
  };
  if ((rc = flat(sizes, level_size)) || (rc = flat(fs, level_fp_sum)) || (rc = flat(fx, level_fp_xor))) return rc;
  if (st) {
    st->seconds = t.seconds();
    st->kernel_launches = c->launches - launches0;
  }
  return worst;
}

}  // extern "C"
