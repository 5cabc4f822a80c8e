// Learned matching proposal: the patch encoder f(p) = W2 relu(W1 p + b1) + b2
// (64 -> 64 -> 16), its training step on pairs produced by the matcher, and
// the embeddings that replace patches in the proposal contraction.
//
// Parameter buffer (FP32 master, 5200 floats): W1[64][64] (row = hidden unit),
// b1[64], W2[16][64] (row = output), b2[16].
//
//  k_encode_tc         embedding of every patch position (mean-shifted patch) on the
//                      tensor cores: FP16 patches, weights and hidden activations,
//                      FP32 accumulation
//  k_encode_vectors    embedding of given 64-vectors (the shifted key patches)
//  k_enc_train         one block per 64 pairs: FP32 forward of both patches,
//                      loss w (||f(p)-f(q)||^2 - d)^2 with w = 1/(d + 0.05)^2
//                      and d the exact squared patch distance, backward with
//                      the per-parameter sums over the block's 128 rows done in
//                      shared memory, one atomic add per parameter per block
//  k_adamw             AdamW update (decay on W1 and W2 only)
#include <cuda_fp16.h>

#include "glr_kernels.cuh"
#include "tc_ptx.cuh"

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

// ---- inference on the tensor cores: 128 positions per tile, two tcgen05.mma (kind::f16,
// FP16 operands, FP32 accumulators in tensor memory).  A = the tile's mean-shifted patches
// [128][64] and H = its hidden activations, both FP16 in the 128-byte swizzled K-major
// layout; W1 [64][64] and W2 [16][64] (FP16) are the B operands.  Per tile:
//   threads write their patch rows -> MMA1 (128 x 64 x 64) -> threads read their row of
//   D1, add b1, apply the ReLU, write their FP16 row of H -> MMA2 (128 x 16 x 64) ->
//   threads read D2, add b2 and store the FP32 embedding.
// 128 threads (thread t owns row t, i.e. tensor-memory lane t); 128 tensor-memory columns
// (D1: 0..63, D2: 64..79); at most four CTAs per SM (shared memory), so the columns of
// all resident CTAs fit.  The largest squared embedding norm goes to *n2max (the scale of
// the 8-bit proposal operand).
constexpr int ENC_M = 128;
constexpr uint32_t ENC_A = 0, ENC_H = 16384, ENC_W1 = 32768, ENC_W2 = 40960, ENC_B = 43008, ENC_BAR = 43520;
constexpr uint32_t ENC_SMEM = 50 * 1024;  // > 228 KB / 5: at most four resident CTAs

// Byte offset of 16-byte chunk c of row r in a [rows][128 B] tile with the 128-byte swizzle.
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}
__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int PT>
__global__ void __launch_bounds__(ENC_M) k_encode_tc(const float* __restrict__ x, const float* __restrict__ mean,
                                                     int n_img, int C, int H, int W, int P_,
                                                     const float* __restrict__ params, float* __restrict__ emb,
                                                     unsigned* __restrict__ n2max, StatusBlock* st) {
  extern __shared__ uint8_t enc_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(enc_raw) + 1023) & ~(uintptr_t)1023);
  const int P = PT ? PT : P_;
  const int tid = threadIdx.x, warp = tid >> 5;
  float* bias = reinterpret_cast<float*>(sm + ENC_B);  // b1[64], b2[16]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + ENC_BAR);
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(sm + ENC_BAR + 32);
  volatile int* abort_s = reinterpret_cast<volatile int*>(sm + ENC_BAR + 36);
  // FP16 weights into the swizzled B tiles; biases stay FP32
  for (int i = tid; i < (EH + EO) * 8; i += ENC_M) {
    const int row = i >> 3, c = i & 7;
    const float* src = params + (row < EH ? OFF_W1 + row * EI : OFF_W2 + (row - EH) * EH) + 8 * c;
    const uint4 v = make_uint4(pack_h2(src[0], src[1]), pack_h2(src[2], src[3]), pack_h2(src[4], src[5]),
                               pack_h2(src[6], src[7]));
    *reinterpret_cast<uint4*>(sm + (row < EH ? ENC_W1 + sw128(row, c) : ENC_W2 + sw128(row - EH, c))) = v;
  }
  for (int i = tid; i < EH + EO; i += ENC_M) bias[i] = params[i < EH ? OFF_B1 + i : OFF_B2 + i - EH];
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    mbar_init(bar + 2, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(tmem_s, 128);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_s;
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const long long tiles_per_img = (npos + ENC_M - 1) / ENC_M;
  const int d = C * P * P;
  const uint32_t sA = smem_u32(sm + ENC_A), sH = smem_u32(sm + ENC_H);
  const uint32_t sW1 = smem_u32(sm + ENC_W1), sW2 = smem_u32(sm + ENC_W2);
  float wmax = 0.f;
  uint32_t phase = 0;
  for (long long t = blockIdx.x; t < (long long)n_img * tiles_per_img; t += gridDim.x) {
    const long long f = t / tiles_per_img;
    const long long q = (t - f * tiles_per_img) * ENC_M + tid;
    const bool valid = q < npos;
    // this thread's mean-shifted patch (zeros past d and past the last position), FP16
    {
      const int r = valid ? (int)(q / Wq) : 0, c = valid ? (int)(q - (q / Wq) * Wq) : 0;
      const float mu = mean[f];
      const float* xf = x + (long long)f * C * H * W + (long long)r * W + c;
      uint32_t w[32];
#pragma unroll
      for (int e2 = 0; e2 < 32; ++e2) {
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int e = 2 * e2 + u;
          float val = 0.f;
          if constexpr (PT > 0) {
            const int ch = e / (PT * PT), dr = (e / PT) % PT, dc = e % PT;
            if (valid && ch < C) val = __ldg(xf + ((long long)ch * H + dr) * W + dc) - mu;
          } else if (valid && e < d) {
            const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
            val = __ldg(xf + ((long long)ch * H + dr) * W + dc) - mu;
          }
          v[u] = val;
        }
        w[e2] = pack_h2(v[0], v[1]);
      }
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8)
        *reinterpret_cast<uint4*>(sm + ENC_A + sw128(tid, c8)) =
            make_uint4(w[4 * c8], w[4 * c8 + 1], w[4 * c8 + 2], w[4 * c8 + 3]);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < EI / 16; ++k)
        mma_f16(tmem, smem_desc(sA + 32 * k, 1024, LAYOUT_SW128), smem_desc(sW1 + 32 * k, 1024, LAYOUT_SW128),
                 idesc_f16(ENC_M, EH), k > 0 ? 1u : 0u);
      mma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait(bar, phase, abort_s, st))) break;
    tc_fence_after();
    {
      float z[2][32];
      tmem_ld_32x32_nowait(lane_addr, z[0]);
      tmem_ld_32x32_nowait(lane_addr + 32, z[1]);
      tmem_ld_wait();
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        uint32_t w4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = 8 * c8 + 2 * u;
          w4[u] = pack_h2(fmaxf(z[j >> 5][j & 31] + bias[j], 0.f), fmaxf(z[(j + 1) >> 5][(j + 1) & 31] + bias[j + 1], 0.f));
        }
        *reinterpret_cast<uint4*>(sm + ENC_H + sw128(tid, c8)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < EH / 16; ++k)
        mma_f16(tmem + 64, smem_desc(sH + 32 * k, 1024, LAYOUT_SW128), smem_desc(sW2 + 32 * k, 1024, LAYOUT_SW128),
                 idesc_f16(ENC_M, EO), k > 0 ? 1u : 0u);
      mma_commit(bar + 1);
    }
    if (__syncthreads_or(!mbar_wait(bar + 1, phase, abort_s, st))) break;
    tc_fence_after();
    {
      float o[32];
      tmem_ld_32x32_nowait(lane_addr + 64, o);
      tmem_ld_wait();
      float n2 = 0.f;
#pragma unroll
      for (int j = 0; j < EO; ++j) {
        o[j] += bias[EH + j];
        n2 = fmaf(o[j], o[j], n2);
      }
      if (valid) {
        float4* dst = reinterpret_cast<float4*>(emb + (f * npos + q) * EO);
#pragma unroll
        for (int k = 0; k < EO / 4; ++k) dst[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
        wmax = fmaxf(wmax, n2);
      }
    }
    tc_fence_before();
    phase ^= 1u;
  }
  // teardown: every MMA issued has completed before tensor memory is freed
  if (tid == 0) {
    mma_commit(bar + 2);
    mbar_wait(bar + 2, 0, abort_s, st, false);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if (n2max != nullptr && (tid & 31) == 0) atomicMax(n2max, __float_as_uint(wmax));
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
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
                                   float* emb, unsigned* n2max, StatusBlock* st, cudaStream_t s) {
  if (im.C * im.P * im.P > EI) return GLR_ENOTSUP;
  const long long npos = (long long)(im.H - im.P + 1) * (im.W - im.P + 1);
  const long long tiles = (long long)im.n_img * ceil_div(npos, (long long)ENC_M);
  const int blocks = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)num_sms() * 4));
  if (n2max != nullptr && cudaMemsetAsync(n2max, 0, 4, s) != cudaSuccess) return GLR_ECUDA;
#define GLR_ENC_CASE(PP)                                                                                       \
  {                                                                                                            \
    if (cudaFuncSetAttribute(k_encode_tc<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ENC_SMEM) !=   \
        cudaSuccess)                                                                                           \
      return GLR_ECUDA;                                                                                        \
    GLR_LAUNCH("k_encode_tc", s,                                                                               \
               k_encode_tc<PP><<<blocks, ENC_M, ENC_SMEM, s>>>(x, mean, im.n_img, im.C, im.H, im.W, im.P, params, \
                                                               emb, n2max, st));                               \
  }
  switch (im.P) {
    case 4: GLR_ENC_CASE(4); break;
    case 6: GLR_ENC_CASE(6); break;
    case 8: GLR_ENC_CASE(8); break;
    default: GLR_ENC_CASE(0); break;
  }
#undef GLR_ENC_CASE
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
