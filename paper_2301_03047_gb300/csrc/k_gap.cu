// GAP projection for y = sum_t A_t x_t (Eq. 6; Eq. 8 with orthogonal masks, Eq. 9).
//   R = sum_t A_t^2 (0 -> 1), x_t = v_t + A_t (y - sum_s A_s v_s) / R
// One thread per pixel (4 pixels with float4 when the plane size allows);
// HBM-bound: reads y, T masks, T estimates and writes T outputs.
#include "glr_kernels.cuh"

namespace glr {

template <bool VEC>
__global__ void __launch_bounds__(256) k_gap_step(const float* __restrict__ y, const float* __restrict__ masks,
                                                  long long mstride, const float* v, int G, int T,
                                                  long long HW, int accelerate, float* y_acc, float* x_out) {
  using V = typename std::conditional<VEC, float4, float>::type;
  constexpr int L = VEC ? 4 : 1;
  const long long nvec = HW / L;
  const long long total = (long long)G * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long g = i / nvec, p = i - g * nvec;
    const V* yv = reinterpret_cast<const V*>(y + g * HW) + p;
    const float* mg = masks + g * mstride;
    float R[L], phi[L], yy[L];
    {
      V t = __ldg(yv);
      const float* tp = reinterpret_cast<const float*>(&t);
#pragma unroll
      for (int l = 0; l < L; ++l) { yy[l] = tp[l]; R[l] = 0.f; phi[l] = 0.f; }
    }
    for (int t = 0; t < T; ++t) {
      V a = __ldg(reinterpret_cast<const V*>(mg + (long long)t * HW) + p);
      const float* ap = reinterpret_cast<const float*>(&a);
      V vv;
      float* vp = reinterpret_cast<float*>(&vv);
      if (v) vv = *(reinterpret_cast<const V*>(v + (g * T + t) * HW) + p);
#pragma unroll
      for (int l = 0; l < L; ++l) {
        R[l] = fmaf(ap[l], ap[l], R[l]);
        if (v) phi[l] = fmaf(ap[l], vp[l], phi[l]);
      }
    }
    float coef[L];
    if (accelerate) {
      V* yap = reinterpret_cast<V*>(y_acc + g * HW) + p;
      V ya = *yap;
      float* yp = reinterpret_cast<float*>(&ya);
#pragma unroll
      for (int l = 0; l < L; ++l) {
        yp[l] = yp[l] + (yy[l] - phi[l]);
        yy[l] = yp[l];
      }
      *yap = ya;
    }
#pragma unroll
    for (int l = 0; l < L; ++l) coef[l] = (yy[l] - phi[l]) / (R[l] == 0.f ? 1.f : R[l]);
    for (int t = 0; t < T; ++t) {
      V a = __ldg(reinterpret_cast<const V*>(mg + (long long)t * HW) + p);
      const float* ap = reinterpret_cast<const float*>(&a);
      V vv;
      float* vp = reinterpret_cast<float*>(&vv);
      if (v) vv = *(reinterpret_cast<const V*>(v + (g * T + t) * HW) + p);
      V o;
      float* op = reinterpret_cast<float*>(&o);
#pragma unroll
      for (int l = 0; l < L; ++l) op[l] = fmaf(ap[l], coef[l], v ? vp[l] : 0.f);
      *(reinterpret_cast<V*>(x_out + (g * T + t) * HW) + p) = o;
    }
  }
}

glr_status launch_gap_step(const float* y, const float* masks, long long mstride, const float* v, int G, int T,
                           long long HW, int accelerate, float* y_acc, float* x_out, cudaStream_t s) {
  const bool vec = (HW % 4 == 0) && ((uintptr_t)y % 16 == 0) && ((uintptr_t)masks % 16 == 0) &&
                   (mstride % 4 == 0) && (!v || (uintptr_t)v % 16 == 0) && ((uintptr_t)x_out % 16 == 0) &&
                   (!y_acc || (uintptr_t)y_acc % 16 == 0);
  const long long work = (long long)G * (vec ? HW / 4 : HW);
  int blocks = (int)std::min<long long>(ceil_div(work, 256), (long long)num_sms() * 16);
  if (blocks < 1) blocks = 1;
  if (vec)
    GLR_LAUNCH("k_gap_step", s, k_gap_step<true><<<blocks, 256, 0, s>>>(y, masks, mstride, v, G, T, HW, accelerate, y_acc, x_out));
  else
    GLR_LAUNCH("k_gap_step", s, k_gap_step<false><<<blocks, 256, 0, s>>>(y, masks, mstride, v, G, T, HW, accelerate, y_acc, x_out));
  return GLR_OK;
}

}  // namespace glr

// Start of MSFA demosaicing: per band, normalised convolution of the sampled
// values with a separable tent of half-width s (bilinear interpolation when
// the mosaic period is s):
//   x_t(p) = sum_q w(q - p) A_t(q) y(q) / sum_q w(q - p) A_t(q),
//   w(dr, dc) = (1 - |dr| / s)(1 - |dc| / s), |dr|, |dc| < s, q inside the image;
// 0 where no sample of band t lies in the window.  One thread per output value.
namespace glr {

__global__ void __launch_bounds__(256) k_mosaic_init(const float* __restrict__ y, const float* __restrict__ masks,
                                                     long long mstride, int G, int T, int H, int W, int s,
                                                     float* __restrict__ x_out) {
  const long long HW = (long long)H * W;
  const long long total = (long long)G * T * HW;
  const float inv_s = 1.f / (float)s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long gt = i / HW, p = i - gt * HW;
    const int g = (int)(gt / T), t = (int)(gt - (long long)g * T);
    const int r = (int)(p / W), c = (int)(p - (p / W) * W);
    const float* yg = y + g * HW;
    const float* a = masks + g * mstride + (long long)t * HW;
    float num = 0.f, den = 0.f;
    for (int dr = -(s - 1); dr <= s - 1; ++dr) {
      const int rr = r + dr;
      if (rr < 0 || rr >= H) continue;
      const float wr = 1.f - fabsf((float)dr) * inv_s;
      for (int dc = -(s - 1); dc <= s - 1; ++dc) {
        const int cc = c + dc;
        if (cc < 0 || cc >= W) continue;
        const float w = wr * (1.f - fabsf((float)dc) * inv_s) * __ldg(a + (long long)rr * W + cc);
        num = fmaf(w, __ldg(yg + (long long)rr * W + cc), num);
        den += w;
      }
    }
    x_out[i] = den > 0.f ? num / den : 0.f;
  }
}

glr_status launch_mosaic_init(const float* y, const float* masks, long long mstride, int G, int T, int H, int W, int s,
                              float* x_out, cudaStream_t st) {
  const long long total = (long long)G * T * H * W;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
  GLR_LAUNCH("k_mosaic_init", st, k_mosaic_init<<<blocks, 256, 0, st>>>(y, masks, mstride, G, T, H, W, s, x_out));
  return GLR_OK;
}

}  // namespace glr

// ADMM step for y = sum_t A_t x_t after the denoiser (scaled form): u += x - z,
// w = z - u, x' = w + A (y - Phi w) / (R + rho), next denoiser input x' + u.
// One thread per pixel over all T frames (x_out may alias x, w_out may alias z:
// each element is read before it is written by the same thread).
namespace glr {

__global__ void __launch_bounds__(256) k_admm_sci(const float* __restrict__ y, const float* __restrict__ masks,
                                                  long long mstride, const float* z, const float* x, float* u, int G,
                                                  int T, long long HW, float rho, float* x_out, float* w_out) {
  const long long total = (long long)G * HW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long g = i / HW, p = i - g * HW;
    const float* mg = masks + g * mstride;
    float R = 0.f, phi = 0.f;
    for (int t = 0; t < T; ++t) {
      const long long o = (g * T + t) * HW + p;
      const float a = __ldg(mg + (long long)t * HW + p);
      const float un = u[o] + x[o] - z[o];
      u[o] = un;
      const float w = z[o] - un;
      R = fmaf(a, a, R);
      phi = fmaf(a, w, phi);
    }
    const float coef = (__ldg(y + g * HW + p) - phi) / (R + rho);
    for (int t = 0; t < T; ++t) {
      const long long o = (g * T + t) * HW + p;
      const float a = __ldg(mg + (long long)t * HW + p);
      const float un = u[o];
      const float xn = fmaf(a, coef, z[o] - un);
      x_out[o] = xn;
      w_out[o] = xn + un;
    }
  }
}

glr_status launch_admm_sci(const float* y, const float* masks, long long mstride, const float* z, const float* x,
                           float* u, int G, int T, long long HW, float rho, float* x_out, float* w_out, cudaStream_t s) {
  const long long total = (long long)G * HW;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 16));
  GLR_LAUNCH("k_admm_sci", s, k_admm_sci<<<blocks, 256, 0, s>>>(y, masks, mstride, z, x, u, G, T, HW, rho, x_out, w_out));
  return GLR_OK;
}

}  // namespace glr
