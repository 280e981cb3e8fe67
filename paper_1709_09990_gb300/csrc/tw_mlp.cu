// The 12-32-1 ReLU network that proposes a starting bound for the k sweep.
// The paper has no learned component; the proposal only changes which decide
// runs are made first, and the answer is always certified by decide runs.
//
// Parameters (449 fp32): W1 [32][12] row-major, b1[32], W2[32], b2.
//   z = W1 x + b1, h = relu(z), yhat = W2 . h + b2
//   loss = (1/B) sum_b (yhat_b - y_b)^2, g_b = 2 (yhat_b - y_b) / B
//   dW2 = sum_b g_b h_b, db2 = sum_b g_b, dz_b = g_b W2 * [z_b > 0],
//   dW1 = sum_b dz_b x_b^T, db1 = sum_b dz_b
// Gradients are reduced in a fixed order (per 128-sample tile, then per block,
// then over blocks), so results are deterministic.  Adam: Kingma & Ba (2015).
#include <cuda_runtime.h>

#include "tw_internal.h"

namespace tw {
namespace {

constexpr int kIn = 12;
constexpr int kHid = 32;
constexpr int kParams = kHid * kIn + kHid + kHid + 1;  // 449
constexpr int kTile = 128;

struct TileScratch {
  float x[kTile][kIn];
  float h[kTile][kHid];
  float dz[kTile][kHid];
  float g[kTile];
  float sq[kTile];
};

// Forward + backward of samples [s0, s0 + cnt) (cnt <= kTile) into the tile
// scratch; idx (or nullptr = identity) maps tile rows to sample indices.
__device__ void tile_forward_backward(const float* __restrict__ P, const float* __restrict__ x,
                                      const float* __restrict__ y, const int32_t* idx, int s0, int cnt,
                                      float inv_b, TileScratch& T) {
  for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
    if (t >= cnt) {
      T.g[t] = 0.f;
      T.sq[t] = 0.f;
      for (int j = 0; j < kHid; ++j) {
        T.h[t][j] = 0.f;
        T.dz[t][j] = 0.f;
      }
      for (int i = 0; i < kIn; ++i) T.x[t][i] = 0.f;
      continue;
    }
    const int s = idx ? idx[s0 + t] : (s0 + t);
    float xi[kIn];
    for (int i = 0; i < kIn; ++i) {
      xi[i] = x[(size_t)s * kIn + i];
      T.x[t][i] = xi[i];
    }
    const float* W1 = P;
    const float* b1 = P + kHid * kIn;
    const float* W2 = b1 + kHid;
    const float b2 = W2[kHid];
    float out = b2;
    float z[kHid];
    for (int j = 0; j < kHid; ++j) {
      float a = b1[j];
      for (int i = 0; i < kIn; ++i) a = fmaf(W1[j * kIn + i], xi[i], a);
      z[j] = a;
      const float hj = a > 0.f ? a : 0.f;
      T.h[t][j] = hj;
      out = fmaf(W2[j], hj, out);
    }
    const float diff = out - y[s];
    const float g = 2.f * diff * inv_b;
    T.g[t] = g;
    T.sq[t] = diff * diff;
    for (int j = 0; j < kHid; ++j) T.dz[t][j] = z[j] > 0.f ? g * W2[j] : 0.f;
  }
  __syncthreads();
}

// acc[p] += gradient contribution of the tile for parameter p (fixed order).
__device__ void tile_accumulate(const TileScratch& T, float* acc) {
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    float a = 0.f;
    if (p < kHid * kIn) {
      const int j = p / kIn, i = p % kIn;
      for (int t = 0; t < kTile; ++t) a = fmaf(T.dz[t][j], T.x[t][i], a);
    } else if (p < kHid * kIn + kHid) {
      const int j = p - kHid * kIn;
      for (int t = 0; t < kTile; ++t) a += T.dz[t][j];
    } else if (p < kHid * kIn + 2 * kHid) {
      const int j = p - kHid * kIn - kHid;
      for (int t = 0; t < kTile; ++t) a = fmaf(T.g[t], T.h[t][j], a);
    } else {
      for (int t = 0; t < kTile; ++t) a += T.g[t];
    }
    acc[p] += a;
  }
  __syncthreads();
}

__global__ void mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ x, int batch,
                                   float* __restrict__ yhat) {
  __shared__ float sP[kParams];
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) sP[p] = P[p];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  float xi[kIn];
  for (int i = 0; i < kIn; ++i) xi[i] = x[(size_t)b * kIn + i];
  const float* b1 = sP + kHid * kIn;
  const float* W2 = b1 + kHid;
  float out = W2[kHid];
  for (int j = 0; j < kHid; ++j) {
    float a = b1[j];
    for (int i = 0; i < kIn; ++i) a = fmaf(sP[j * kIn + i], xi[i], a);
    out = fmaf(W2[j], a > 0.f ? a : 0.f, out);
  }
  yhat[b] = out;
}

// Stage 1: block blk reduces samples [blk*per, (blk+1)*per) into partial[blk].
__global__ void mlp_grad_partial_kernel(const float* __restrict__ P, const float* __restrict__ x,
                                        const float* __restrict__ y, int batch, int per, float* partial) {
  __shared__ float sP[kParams];
  __shared__ float sAcc[kParams];
  __shared__ TileScratch T;
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    sP[p] = P[p];
    sAcc[p] = 0.f;
  }
  __syncthreads();
  const float inv_b = 1.f / (float)batch;
  const int lo = blockIdx.x * per;
  const int hi = min(batch, lo + per);
  for (int s0 = lo; s0 < hi; s0 += kTile) {
    tile_forward_backward(sP, x, y, nullptr, s0, min(kTile, hi - s0), inv_b, T);
    tile_accumulate(T, sAcc);
  }
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) partial[(size_t)blockIdx.x * kParams + p] = sAcc[p];
}

// Stage 2: grad[p] = sum over blocks of partial[blk][p], in block order.
__global__ void mlp_grad_final_kernel(const float* __restrict__ partial, int blocks, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float a = 0.f;
  for (int b = 0; b < blocks; ++b) a += partial[(size_t)b * kParams + p];
  grad[p] = a;
}

__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, float lr, float beta1, float beta2,
                                            float eps, float c1, float c2) {
  m = beta1 * m + (1.f - beta1) * g;
  v = beta2 * v + (1.f - beta2) * g * g;
  const float mhat = m / c1;
  const float vhat = v / c2;
  p -= lr * mhat / (sqrtf(vhat) + eps);
}

__global__ void mlp_adam_kernel(float* P, const float* __restrict__ G, float* M, float* V, float lr, float beta1,
                                float beta2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float pp = P[p], m = M[p], v = V[p];
  adam_update(pp, G[p], m, v, lr, beta1, beta2, eps, c1, c2);
  P[p] = pp;
  M[p] = m;
  V[p] = v;
}

// The whole training run in one CTA: for each epoch and minibatch, forward,
// backward (fixed-order reduction) and an Adam step, all on chip.
__global__ void __launch_bounds__(256) mlp_train_kernel(float* P, float* M, float* V, const float* __restrict__ x,
                                                        const float* __restrict__ y, int batch_total, int minibatch,
                                                        int epochs, const int32_t* __restrict__ perm, float lr,
                                                        float* loss_out) {
  __shared__ float sP[kParams], sM[kParams], sV[kParams], sAcc[kParams];
  __shared__ TileScratch T;
  __shared__ float sLoss;
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    sP[p] = P[p];
    sM[p] = M[p];
    sV[p] = V[p];
  }
  __syncthreads();
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  int t = 0;
  float b1t = 1.f, b2t = 1.f;
  for (int e = 0; e < epochs; ++e) {
    const int32_t* idx = perm + (size_t)e * batch_total;
    if (threadIdx.x == 0) sLoss = 0.f;
    for (int mb0 = 0; mb0 < batch_total; mb0 += minibatch) {
      const int mb = min(minibatch, batch_total - mb0);
      for (int p = threadIdx.x; p < kParams; p += blockDim.x) sAcc[p] = 0.f;
      __syncthreads();
      const float inv_b = 1.f / (float)mb;
      for (int s0 = 0; s0 < mb; s0 += kTile) {
        tile_forward_backward(sP, x, y, idx + mb0, s0, min(kTile, mb - s0), inv_b, T);
        if (threadIdx.x == 0) {
          float l = 0.f;
          for (int q = 0; q < kTile; ++q) l += T.sq[q];
          sLoss += l;
        }
        tile_accumulate(T, sAcc);
      }
      ++t;
      b1t *= beta1;
      b2t *= beta2;
      for (int p = threadIdx.x; p < kParams; p += blockDim.x)
        adam_update(sP[p], sAcc[p], sM[p], sV[p], lr, beta1, beta2, eps, 1.f - b1t, 1.f - b2t);
      __syncthreads();
    }
    if (threadIdx.x == 0 && loss_out) loss_out[e] = sLoss / (float)batch_total;
    __syncthreads();
  }
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    P[p] = sP[p];
    M[p] = sM[p];
    V[p] = sV[p];
  }
}

}  // namespace

cudaError_t launch_mlp_forward(const float* params, const float* x, int batch, float* yhat, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  mlp_forward_kernel<<<(batch + 255) / 256, 256, 0, s>>>(params, x, batch, yhat);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* params, const float* x, const float* y, int batch, float* grad,
                            float* partial, int partial_blocks, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const int per = ((batch + partial_blocks - 1) / partial_blocks + kTile - 1) / kTile * kTile;
  const int blocks = (batch + per - 1) / per;
  mlp_grad_partial_kernel<<<blocks, 256, 0, s>>>(params, x, y, batch, per, partial);
  mlp_grad_final_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(partial, blocks, grad);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, float beta1,
                            float beta2, float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(beta1, (float)t);
  const float c2 = 1.f - powf(beta2, (float)t);
  mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_train(float* params, float* m, float* v, const float* x, const float* y, int batch_total,
                             int minibatch, int epochs, const int32_t* perm, float lr, float* loss_out,
                             cudaStream_t s) {
  if (batch_total <= 0 || epochs <= 0) return cudaSuccess;
  mlp_train_kernel<<<1, 256, 0, s>>>(params, m, v, x, y, batch_total, minibatch, epochs, perm, lr, loss_out);
  return cudaGetLastError();
}

}  // namespace tw
