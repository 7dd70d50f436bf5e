// MLP of the learned wall model: 40 -> 128 -> 128 -> 128 -> 128 -> 5, erf-based
// GELU on the hidden layers, linear output.  The GEMMs run on the tensor cores
// (k_mlp_tc.cu: BF16 weights and activation operands, FP32 accumulation);
// training keeps FP32 master weights, forms the gradients of the mean-squared
// error of the normalised outputs with the same BF16-operand GEMMs, and
// applies Adam (Kingma & Ba 2015).  Batch reductions (weight gradients, loss)
// go through per-block partials summed in a fixed order: deterministic.
// (No counterpart in the paper.)
#include <cuda_bf16.h>

#include "pnp_common.cuh"
#include "pnp_wall.cuh"

namespace pnp {

MlpDims mlp_dims() {
  MlpDims d{};
  const int ins[kMlpLayers] = {kMlpIn, kMlpHidden, kMlpHidden, kMlpHidden, kMlpHidden};
  const int outs[kMlpLayers] = {kMlpHidden, kMlpHidden, kMlpHidden, kMlpHidden, kMlpOut};
  size_t off = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    d.in[l] = ins[l];
    d.out[l] = outs[l];
    d.woff[l] = off;
    off += (size_t)ins[l] * outs[l];
    d.boff[l] = off;
    off += outs[l];
  }
  d.nparam = off;
  return d;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Sum of the per-CTA partial gradients in a fixed order: four interleaved running
// sums (partials b = 4q .. 4q + 3), combined as (s0 + s1) + (s2 + s3).
__global__ void k_mlp_reduce_partial(const float* __restrict__ partial, int nblk, int len, float* __restrict__ gw,
                                     float* __restrict__ gb, int nk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int b = 0;
  for (; b + 3 < nblk; b += 4) {
    s0 += partial[(size_t)b * len + e];
    s1 += partial[(size_t)(b + 1) * len + e];
    s2 += partial[(size_t)(b + 2) * len + e];
    s3 += partial[(size_t)(b + 3) * len + e];
  }
  for (; b < nblk; ++b) s0 += partial[(size_t)b * len + e];
  const float s = (s0 + s1) + (s2 + s3);
  if (e < nk) gw[e] = s;
  else gb[e - nk] = s;
}

// Normalised input x_n = (x - shift) * scale.
__global__ void k_mlp_norm_in(const float* __restrict__ X, int B, const float* __restrict__ shift,
                              const float* __restrict__ scale, float* __restrict__ out) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)B * kMlpIn) return;
  const int f = (int)(t % kMlpIn);
  out[t] = (X[t] - shift[f]) * scale[f];
}

// dz of the output layer for L = mean((y_n - t_n)^2), with per-block partial losses;
// with a residual output the network's target in column skip_out is t - x[skip_in].
__global__ void __launch_bounds__(256) k_mlp_loss(const float* __restrict__ yn, const float* __restrict__ T, int B,
                                                  const float* __restrict__ shift, const float* __restrict__ scale,
                                                  const float* __restrict__ X, int skip_out, int skip_in,
                                                  float* __restrict__ dz, float* __restrict__ loss_partial) {
  __shared__ float sh[256];
  const size_t n = (size_t)B * kMlpOut;
  const float inv = 1.0f / (float)n;
  float acc = 0.f;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(t % kMlpOut);
    const float tf = f == skip_out ? T[t] - X[(t / kMlpOut) * kMlpIn + skip_in] : T[t];
    const float e = yn[t] - (tf - shift[f]) * scale[f];
    dz[t] = 2.0f * e * inv;
    acc += e * e;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_partial[blockIdx.x] = sh[0] * inv;
}

__global__ void k_mlp_loss_final(float* loss_partial, int nblk) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += loss_partial[b];
    loss_partial[nblk] = s;
  }
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// ---------------------------------------------------------------------------
cudaError_t mlp_sync_bf16(const MlpBufs& b, size_t nparam, cudaStream_t s) {
  (void)nparam;
  return mlp_make_images(b.param, b.wimg, s);
}

cudaError_t mlp_forward(const MlpBufs& b, const float* X, int B, float* Y, cudaStream_t s) {
  // outputs only: the fused kernel; the layer-by-layer path keeps the activations
  // the backward pass needs
  if (Y)
    return mlp_infer_tc(X, B, b.wimg, b.param, b.in_shift, b.in_scale, b.out_shift, b.out_scale, b.skip_out,
                        b.skip_in, Y, b.err, s);
  const MlpDims d = mlp_dims();
  const MlpImg im = mlp_images();
  const size_t ni = (size_t)B * kMlpIn;
  k_mlp_norm_in<<<(unsigned)((ni + 255) / 256), 256, 0, s>>>(X, B, b.in_shift, b.in_scale, b.act[0]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l < kMlpLayers; ++l) {
    e = mlp_fwd_layer_tc(b.act[l], d.in[l], l > 0, b.wimg + im.fwd[l], b.param + d.boff[l], d.out[l], B,
                         b.act[l + 1], b.err, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// Gradient of the loss for the activations left by mlp_forward on the same batch.
cudaError_t mlp_backward(const MlpBufs& b, const float* X, const float* T, int B, int max_partial, cudaStream_t s) {
  const MlpDims d = mlp_dims();
  const MlpImg im = mlp_images();
  const int nloss = 120;
  k_mlp_loss<<<nloss, 256, 0, s>>>(b.act[kMlpLayers], T, B, b.out_shift, b.out_scale, X, b.skip_out, b.skip_in,
                                   b.dact, b.loss);
  k_mlp_loss_final<<<1, 32, 0, s>>>(b.loss, nloss);
  // rows per weight-gradient CTA: a multiple of the tensor-core chunk (64 rows)
  int rows_per_block = (B + max_partial - 1) / max_partial;
  rows_per_block = (rows_per_block + 63) / 64 * 64;
  const int nblk = (B + rows_per_block - 1) / rows_per_block;
  float* dz = b.dact;
  float* other = b.dact2;
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const int N = d.out[l], K = d.in[l];
    cudaError_t e = mlp_wgrad_tc(dz, N, b.act[l], K, l > 0, B, rows_per_block, nblk, b.partial, b.err, s);
    if (e != cudaSuccess) return e;
    const int len = N * K + N;
    k_mlp_reduce_partial<<<(len + 255) / 256, 256, 0, s>>>(b.partial, nblk, len, b.grad + d.woff[l],
                                                           b.grad + d.boff[l], N * K);
    if (l > 0) {
      e = mlp_bwd_data_tc(dz, N, b.wimg + im.bwd[l], K, B, b.act[l], other, b.err, s);
      if (e != cudaSuccess) return e;
      float* t = dz;
      dz = other;
      other = t;
    }
  }
  return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpBufs& b, size_t nparam, float lr, float beta1, float beta2, float eps, int t,
                     cudaStream_t s) {
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  k_mlp_adam<<<(unsigned)((nparam + 255) / 256), 256, 0, s>>>(b.param, b.grad, b.m, b.v, nparam, lr, beta1, beta2,
                                                              eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return mlp_sync_bf16(b, nparam, s);
}

}  // namespace pnp
