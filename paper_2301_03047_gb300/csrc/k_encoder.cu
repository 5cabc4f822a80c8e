// Learned matching proposal: the patch encoder f(p) = W2 relu(W1 p + b1) + b2
// (64 -> 64 -> 16), its training step on pairs produced by the matcher, and
// the embeddings that replace patches in the proposal contraction.
//
// Parameter buffer (FP32 master, 5200 floats): W1[64][64] (row = hidden unit),
// b1[64], W2[16][64] (row = output), b2[16].
//
//  k_encode_positions  embedding of every patch position (mean-shifted patch),
//                      weights rounded to FP16 in shared memory, FP32 math
//  k_encode_vectors    embedding of given 64-vectors (the shifted key patches)
//  k_enc_train         one block per 64 pairs: FP32 forward of both patches,
//                      loss w (||f(p)-f(q)||^2 - d)^2 with w = 1/(d + 0.05)^2
//                      and d the exact squared patch distance, backward with
//                      the per-parameter sums over the block's 128 rows done in
//                      shared memory, one atomic add per parameter per block
//  k_adamw             AdamW update (decay on W1 and W2 only)
#include <cuda_fp16.h>

#include "glr_kernels.cuh"

namespace glr {

namespace {

constexpr int EI = 64, EH = 64, EO = 16;
constexpr int OFF_W1 = 0, OFF_B1 = EH * EI, OFF_W2 = OFF_B1 + EH, OFF_B2 = OFF_W2 + EO * EH;
constexpr int NPARAM = OFF_B2 + EO;  // 5200
static_assert(NPARAM == GLR_ENCODER_PARAMS, "parameter count");
constexpr float kD0 = 0.05f;

// weights (optionally FP16-rounded) into shared memory
__device__ __forceinline__ void load_weights(const float* __restrict__ params, float* w, bool round16) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    const float v = params[i];
    w[i] = round16 ? __half2float(__float2half_rn(v)) : v;
  }
}

__device__ __forceinline__ void enc_forward(const float* w, const float (&p)[EI], float (&e)[EO]) {
  float h[EH];
#pragma unroll 4
  for (int j = 0; j < EH; ++j) {
    float z = w[OFF_B1 + j];
    const float4* row = reinterpret_cast<const float4*>(w + OFF_W1 + j * EI);
#pragma unroll
    for (int i = 0; i < EI / 4; ++i) {
      const float4 a = row[i];
      z = fmaf(a.x, p[4 * i], z);
      z = fmaf(a.y, p[4 * i + 1], z);
      z = fmaf(a.z, p[4 * i + 2], z);
      z = fmaf(a.w, p[4 * i + 3], z);
    }
    h[j] = fmaxf(z, 0.f);
  }
#pragma unroll
  for (int o = 0; o < EO; ++o) {
    float z = w[OFF_B2 + o];
    const float4* row = reinterpret_cast<const float4*>(w + OFF_W2 + o * EH);
#pragma unroll
    for (int j = 0; j < EH / 4; ++j) {
      const float4 a = row[j];
      z = fmaf(a.x, h[4 * j], z);
      z = fmaf(a.y, h[4 * j + 1], z);
      z = fmaf(a.z, h[4 * j + 2], z);
      z = fmaf(a.w, h[4 * j + 3], z);
    }
    e[o] = z;
  }
}

__global__ void __launch_bounds__(128) k_encode_positions(const float* __restrict__ x, const float* __restrict__ mean,
                                                          int n_img, int C, int H, int W, int P,
                                                          const float* __restrict__ params, float* __restrict__ emb) {
  extern __shared__ __align__(16) float wsm[];
  load_weights(params, wsm, true);
  __syncthreads();
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const long long total = (long long)n_img * npos;
  const int d = C * P * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / npos;
    const int q = (int)(i - f * npos);
    const int r = q / Wq, c = q - (q / Wq) * Wq;
    const float mu = mean[f];
    float p[EI];
#pragma unroll
    for (int e = 0; e < EI; ++e) {
      float v = 0.f;
      if (e < d) {
        const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
        v = __ldg(x + (((long long)f * C + ch) * H + r + dr) * W + c + dc) - mu;
      }
      p[e] = v;
    }
    float out[EO];
    enc_forward(wsm, p, out);
    float4* dst = reinterpret_cast<float4*>(emb + i * EO);
#pragma unroll
    for (int k = 0; k < EO / 4; ++k) dst[k] = make_float4(out[4 * k], out[4 * k + 1], out[4 * k + 2], out[4 * k + 3]);
  }
}

__global__ void __launch_bounds__(128) k_encode_vectors(const float* __restrict__ vecs, long long n, int d,
                                                        const float* __restrict__ params, float* __restrict__ emb) {
  extern __shared__ __align__(16) float wsm[];
  load_weights(params, wsm, true);
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float p[EI];
#pragma unroll
    for (int e = 0; e < EI; ++e) p[e] = e < d ? vecs[i * d + e] : 0.f;
    float out[EO];
    enc_forward(wsm, p, out);
#pragma unroll
    for (int o = 0; o < EO; ++o) emb[i * EO + o] = out[o];
  }
}

// ---- training
constexpr int TB = 64;  // pairs per block; 128 rows (p and q of each pair)

__global__ void __launch_bounds__(256) k_enc_train(const float* __restrict__ x, const float* __restrict__ mean, int C,
                                                   int H, int W, int P, const int32_t* __restrict__ pairs, int n_pairs,
                                                   const float* __restrict__ params, float* __restrict__ grad,
                                                   float* __restrict__ loss) {
  extern __shared__ __align__(16) float sm[];
  float* w = sm;                       // NPARAM (FP32 master weights)
  float* X = w + NPARAM;               // [128][64] inputs
  float* Z = X + 2 * TB * EI;          // [128][64] hidden pre-activations, later hidden gradients
  float* G = Z + 2 * TB * EH;          // [128][16] output gradients
  float* red = G + 2 * TB * EO;        // [8] warp partial losses
  load_weights(params, w, false);
  const int tid = threadIdx.x;
  const int base = blockIdx.x * TB;
  const int Wq = W - P + 1;
  const int d = C * P * P;
  // gather the 128 mean-shifted patches (row 2 t = p of pair t, row 2 t + 1 = q)
  for (int i = tid; i < 2 * TB * EI; i += 256) {
    const int row = i / EI, e = i - (i / EI) * EI;
    const int t = base + row / 2;
    float v = 0.f;
    if (t < n_pairs && e < d) {
      const int f = pairs[3 * t], q = pairs[3 * t + 1 + (row & 1)];
      const int r = q / Wq, c = q - (q / Wq) * Wq;
      const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
      v = __ldg(x + (((long long)f * C + ch) * H + r + dr) * W + c + dc) - mean[f];
    }
    X[i] = v;
  }
  __syncthreads();
  // forward of the 128 rows, one thread each; keep Z and E
  float e_out[EO];
  if (tid < 2 * TB) {
    const float* xr = X + tid * EI;
    float h[EH];
    for (int j = 0; j < EH; ++j) {
      float z = w[OFF_B1 + j];
      for (int i = 0; i < EI; ++i) z = fmaf(w[OFF_W1 + j * EI + i], xr[i], z);
      Z[tid * EH + j] = z;
      h[j] = fmaxf(z, 0.f);
    }
    for (int o = 0; o < EO; ++o) {
      float z = w[OFF_B2 + o];
      for (int j = 0; j < EH; ++j) z = fmaf(w[OFF_W2 + o * EH + j], h[j], z);
      e_out[o] = z;
      G[tid * EO + o] = z;  // holds E for now
    }
  }
  __syncthreads();
  // per pair: s, d, loss and dL/dE
  float lsum = 0.f;
  if (tid < TB) {
    const int t = base + tid;
    if (t < n_pairs) {
      const float* xp = X + (2 * tid) * EI;
      const float* xq = X + (2 * tid + 1) * EI;
      float dd = 0.f;
      for (int e = 0; e < EI; ++e) {
        const float df = xp[e] - xq[e];
        dd = fmaf(df, df, dd);
      }
      float* gp = G + (2 * tid) * EO;
      float* gq = G + (2 * tid + 1) * EO;
      float diff[EO], s = 0.f;
      for (int o = 0; o < EO; ++o) {
        diff[o] = gp[o] - gq[o];
        s = fmaf(diff[o], diff[o], s);
      }
      const float wt = 1.f / ((dd + kD0) * (dd + kD0));
      lsum = wt * (s - dd) * (s - dd);
      const float coef = 4.f / (float)n_pairs * wt * (s - dd);
      for (int o = 0; o < EO; ++o) {
        gp[o] = coef * diff[o];
        gq[o] = -coef * diff[o];
      }
    } else {
      for (int o = 0; o < EO; ++o) {
        G[(2 * tid) * EO + o] = 0.f;
        G[(2 * tid + 1) * EO + o] = 0.f;
      }
    }
  }
  // block loss
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((tid & 31) == 0) red[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += red[k];
    atomicAdd(loss, t / (float)n_pairs);
  }
  // dW2[o][j] = sum_rows G[row][o] relu(Z[row][j]); db2[o] = sum_rows G[row][o]
  for (int k = tid; k < EO * EH + EO; k += 256) {
    float acc = 0.f;
    if (k < EO * EH) {
      const int o = k / EH, j = k - (k / EH) * EH;
      for (int row = 0; row < 2 * TB; ++row) acc = fmaf(G[row * EO + o], fmaxf(Z[row * EH + j], 0.f), acc);
      atomicAdd(grad + OFF_W2 + k, acc);
    } else {
      const int o = k - EO * EH;
      for (int row = 0; row < 2 * TB; ++row) acc += G[row * EO + o];
      atomicAdd(grad + OFF_B2 + o, acc);
    }
  }
  __syncthreads();
  // hidden gradients gH[row][j] = (sum_o G[row][o] W2[o][j]) [Z > 0], written over Z
  for (int i = tid; i < 2 * TB * EH; i += 256) {
    const int row = i / EH, j = i - (i / EH) * EH;
    float acc = 0.f;
    for (int o = 0; o < EO; ++o) acc = fmaf(G[row * EO + o], w[OFF_W2 + o * EH + j], acc);
    Z[i] = Z[i] > 0.f ? acc : 0.f;
  }
  __syncthreads();
  // dW1[j][i] = sum_rows gH[row][j] X[row][i]; db1[j] = sum_rows gH[row][j]
  for (int k = tid; k < EH * EI + EH; k += 256) {
    float acc = 0.f;
    if (k < EH * EI) {
      const int j = k / EI, i = k - (k / EI) * EI;
      for (int row = 0; row < 2 * TB; ++row) acc = fmaf(Z[row * EH + j], X[row * EI + i], acc);
      atomicAdd(grad + OFF_W1 + k, acc);
    } else {
      const int j = k - EH * EI;
      for (int row = 0; row < 2 * TB; ++row) acc += Z[row * EH + j];
      atomicAdd(grad + OFF_B1 + j, acc);
    }
  }
  (void)e_out;
}

__global__ void k_adamw(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                        float* __restrict__ v, float lr, float wd, float b1, float b2, float eps, float bc1,
                        float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  float p = params[i];
  const bool decay = (i < OFF_B1) || (i >= OFF_W2 && i < OFF_B2);
  if (decay) p -= lr * wd * p;
  params[i] = p - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

}  // namespace

glr_status launch_encode_positions(const float* x, const glr_images& im, const float* mean, const float* params,
                                   float* emb, cudaStream_t s) {
  const long long total = (long long)im.n_img * (im.H - im.P + 1) * (im.W - im.P + 1);
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 128), (long long)num_sms() * 16));
  const size_t smem = NPARAM * 4;
  GLR_LAUNCH("k_encode_positions", s,
             k_encode_positions<<<blocks, 128, smem, s>>>(x, mean, im.n_img, im.C, im.H, im.W, im.P, params, emb));
  return GLR_OK;
}

glr_status launch_encode_vectors(const float* vecs, long long n, int d, const float* params, float* emb,
                                 cudaStream_t s) {
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(n, 128), (long long)num_sms() * 16));
  GLR_LAUNCH("k_encode_vectors", s, k_encode_vectors<<<blocks, 128, NPARAM * 4, s>>>(vecs, n, d, params, emb));
  return GLR_OK;
}

glr_status launch_encoder_train(const float* x, const glr_images& im, const float* mean, const int32_t* pairs,
                                int n_pairs, float* params, float* m, float* v, int step, float lr, float wd,
                                float* grad, float* loss, cudaStream_t s) {
  if (cudaMemsetAsync(grad, 0, NPARAM * 4, s) != cudaSuccess) return GLR_ECUDA;
  if (cudaMemsetAsync(loss, 0, 4, s) != cudaSuccess) return GLR_ECUDA;
  const size_t smem = (size_t)(NPARAM + 2 * TB * EI + 2 * TB * EH + 2 * TB * EO + 8) * 4;
  if (cudaFuncSetAttribute(k_enc_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GLR_ECUDA;
  const int blocks = (int)ceil_div(n_pairs, TB);
  GLR_LAUNCH("k_enc_train", s,
             k_enc_train<<<blocks, 256, smem, s>>>(x, mean, im.C, im.H, im.W, im.P, pairs, n_pairs, params, grad,
                                                    loss));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  GLR_LAUNCH("k_adamw", s,
             k_adamw<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, grad, m, v, lr, wd, b1, b2, eps, bc1, bc2));
  return GLR_OK;
}

}  // namespace glr
