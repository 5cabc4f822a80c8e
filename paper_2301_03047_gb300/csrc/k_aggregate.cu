// Aggregation: the low-rank patch estimates go back to their positions and
// overlapping estimates are averaged (weight 1); uncovered pixels keep x_in.
//
//  k_scatter    one warp per group (its rows one after the other) for short rows, one warp
//               per row for d > 128; lanes add a row's d values
//               into the numerator planes as 64-bit fixed point (value x 2^32,
//               rounded to an integer: exact for |value| >= 2^-9, else within
//               2^-33) with integer atomics, so the sums do not depend on the
//               order in which the atomics land; lane 0 adds 1 to the integer
//               count of that patch position.
//  k_normalise  32x32 pixel tiles: den = P x P box sum of the position counts
//               (separable, in shared memory), v = num 2^-32 / den (FP64) or x_in.
#include "glr_kernels.cuh"

namespace glr {

namespace {

// Adds one group row (a patch estimate at position q) into the fixed-point sums.
template <int PT>
__device__ __forceinline__ void scatter_row(const float* __restrict__ src, int q, unsigned long long* __restrict__ nf,
                                            int* __restrict__ cnt_f, int C, int H, int W, int P, int lane) {
  const int PP = P * P, d = C * PP, Wq = W - P + 1;
  const int r = q / Wq, c = q - (q / Wq) * Wq;
  unsigned long long* dst = nf + (long long)r * W + c;
  for (int e = lane; e < d; e += 32) {
    const int ch = e / PP, rem = e - ch * PP, rr = rem / P, cc = rem - rr * P;
    // |value| < 2^30 keeps every partial sum of up to 2^32 terms inside int64
    const float v = fminf(fmaxf(__ldg(src + e), -1073741824.f), 1073741824.f);
    const long long fx = __float2ll_rn(v * 4294967296.f);  // exact scaling by 2^32
    atomicAdd(dst + ((long long)ch * H + rr) * W + cc, (unsigned long long)fx);
  }
  if (lane == 0) atomicAdd(cnt_f + q, 1);
}

// PT = P (compile-time patch side; 0: the runtime value).  PER_ROW = false: one
// warp per group (the image and key decoded once, the K rows one after the
// other; short rows); true: one warp per row (long rows, d > 128).
template <int PT, bool PER_ROW>
__global__ void __launch_bounds__(256) k_scatter(const float* __restrict__ groups, const int32_t* __restrict__ idx,
                                                 const int32_t* __restrict__ n_found, int n_img, int C, int H, int W,
                                                 int Prt, int N, int K, unsigned long long* __restrict__ num,
                                                 int* __restrict__ cnt, StatusBlock* st) {
  const int P = PT ? PT : Prt;
  const int d = C * P * P;
  const int Wq = W - P + 1, Hq = H - P + 1;
  const int lane = threadIdx.x & 31;
  const long long units = (long long)n_img * N * (PER_ROW ? K : 1);
  for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < units;
       u += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long g = PER_ROW ? u / K : u;
    const int f = (int)(g / N), k = (int)(g - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    unsigned long long* nf = num + (long long)f * C * H * W;
    int* cnt_f = cnt + (long long)f * Hq * Wq;
    const int j0 = PER_ROW ? (int)(u - g * K) : 0, j1 = PER_ROW ? j0 + 1 : K;
    for (int j = j0; j < j1; ++j) {
      const long long row = g * K + j;
      const int q = idx[row];
      if ((unsigned)q >= (unsigned)(Wq * Hq)) {
        if (lane == 0) status_set(st, GLR_DEV_BAD_INDEX);
        continue;
      }
      scatter_row<PT>(groups + row * d, q, nf, cnt_f, C, H, W, P, lane);
    }
  }
}

constexpr int AT = 32;

__global__ void __launch_bounds__(256) k_normalise(const long long* __restrict__ num, const int* __restrict__ cnt,
                                                   const float* x_in, float* v_out, int C, int H, int W, int P) {
  // counts of positions that cover the tile: rows r0-P+1 .. r0+AT-1
  __shared__ int cs[AT + 16][AT + 16];
  __shared__ int hs[AT + 16][AT];
  const int Hq = H - P + 1, Wq = W - P + 1;
  const int f = blockIdx.z;
  const int r0 = blockIdx.y * AT, c0 = blockIdx.x * AT;
  const int tid = threadIdx.x;
  const int ext = AT + P - 1;
  const int* cf = cnt + (long long)f * Hq * Wq;
  for (int i = tid; i < ext * ext; i += 256) {
    const int a = i / ext, b = i % ext;
    const int pr = r0 - (P - 1) + a, pc = c0 - (P - 1) + b;
    cs[a][b] = (pr >= 0 && pr < Hq && pc >= 0 && pc < Wq) ? cf[(long long)pr * Wq + pc] : 0;
  }
  __syncthreads();
  for (int i = tid; i < ext * AT; i += 256) {
    const int a = i / AT, b = i % AT;
    int s = 0;
    for (int t = 0; t < P; ++t) s += cs[a][b + t];
    hs[a][b] = s;
  }
  __syncthreads();
  for (int i = tid; i < AT * AT; i += 256) {
    const int a = i / AT, b = i % AT;
    const int rr = r0 + a, cc = c0 + b;
    if (rr >= H || cc >= W) continue;
    int den = 0;
    for (int t = 0; t < P; ++t) den += hs[a + t][b];
    for (int ch = 0; ch < C; ++ch) {
      const long long o = (((long long)f * C + ch) * H + rr) * W + cc;
      v_out[o] = den > 0 ? (float)((double)num[o] * 2.3283064365386963e-10 / (double)den) : x_in[o];
    }
  }
}

}  // namespace

AggWs agg_ws_layout(const glr_images& im) {
  WsLayout L;
  AggWs w;
  w.num_off = L.take((size_t)im.n_img * im.C * im.H * im.W * 8);
  w.cnt_off = L.take((size_t)im.n_img * (im.H - im.P + 1) * (im.W - im.P + 1) * 4);
  w.total = L.off;
  return w;
}

glr_status launch_fused_lowrank_aggregate(const float* x, const glr_images& im, const int32_t* idx,
                                         const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                                         float* v_out, int32_t* rank, char* ws, const AggWs& L, cudaStream_t s) {
  unsigned long long* num = reinterpret_cast<unsigned long long*>(ws + L.num_off);
  int* cnt = reinterpret_cast<int*>(ws + L.cnt_off);
  const size_t num_b = (size_t)im.n_img * im.C * im.H * im.W * 8;
  const size_t cnt_b = (size_t)im.n_img * (im.H - im.P + 1) * (im.W - im.P + 1) * 4;
  if (cudaMemsetAsync(num, 0, num_b, s) != cudaSuccess) return GLR_ECUDA;
  if (cudaMemsetAsync(cnt, 0, cnt_b, s) != cudaSuccess) return GLR_ECUDA;
  const glr_status st = launch_wnnm_fused(x, im, idx, n_found, N, K, sigma_w, c_wnnm, num, cnt, rank,
                                          reinterpret_cast<StatusBlock*>(ws), s);
  if (st != GLR_OK) return st;
  dim3 g((unsigned)ceil_div(im.W, AT), (unsigned)ceil_div(im.H, AT), (unsigned)im.n_img);
  GLR_LAUNCH("k_normalise", s, k_normalise<<<g, 256, 0, s>>>(reinterpret_cast<const long long*>(num), cnt, x, v_out, im.C, im.H, im.W, im.P));
  return GLR_OK;
}

glr_status launch_aggregate(const float* groups, const int32_t* idx, const int32_t* n_found, const glr_images& im,
                            int N, int K, const float* x_in, float* v_out, char* ws, const AggWs& L,
                            cudaStream_t s) {
  unsigned long long* num = reinterpret_cast<unsigned long long*>(ws + L.num_off);
  int* cnt = reinterpret_cast<int*>(ws + L.cnt_off);
  const size_t num_b = (size_t)im.n_img * im.C * im.H * im.W * 8;
  const size_t cnt_b = (size_t)im.n_img * (im.H - im.P + 1) * (im.W - im.P + 1) * 4;
  if (cudaMemsetAsync(num, 0, num_b, s) != cudaSuccess) return GLR_ECUDA;
  if (cudaMemsetAsync(cnt, 0, cnt_b, s) != cudaSuccess) return GLR_ECUDA;
  const bool per_row = im.C * im.P * im.P > 128;
  const long long units = (long long)im.n_img * N * (per_row ? K : 1);
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(units * 32, 256), (long long)num_sms() * 32));
#define GLR_SCATTER_CASE(PP, ROW)                                                                            \
  GLR_LAUNCH("k_scatter", s,                                                                                 \
             (k_scatter<PP, ROW><<<blocks, 256, 0, s>>>(groups, idx, n_found, im.n_img, im.C, im.H, im.W, im.P, N, \
                                                        K, num, cnt, reinterpret_cast<StatusBlock*>(ws))))
  switch (im.P * 2 + (per_row ? 1 : 0)) {
    case 8: GLR_SCATTER_CASE(4, false); break;
    case 12: GLR_SCATTER_CASE(6, false); break;
    case 13: GLR_SCATTER_CASE(6, true); break;
    case 16: GLR_SCATTER_CASE(8, false); break;
    case 17: GLR_SCATTER_CASE(8, true); break;
    default:
      if (per_row) GLR_SCATTER_CASE(0, true);
      else GLR_SCATTER_CASE(0, false);
      break;
  }
#undef GLR_SCATTER_CASE
  dim3 g((unsigned)ceil_div(im.W, AT), (unsigned)ceil_div(im.H, AT), (unsigned)im.n_img);
  GLR_LAUNCH("k_normalise", s, k_normalise<<<g, 256, 0, s>>>(reinterpret_cast<const long long*>(num), cnt, x_in, v_out, im.C, im.H, im.W, im.P));
  return GLR_OK;
}

}  // namespace glr
