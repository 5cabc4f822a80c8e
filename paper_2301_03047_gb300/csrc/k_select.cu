// Key (exemplar) patch selection -- Section 2 of the paper: exemplar patches are
// centred on corner points of the averaged edge map, the edge maps being the
// four signed binary Sobel maps of Eq. 2 thresholded by Eq. 3.
//
//  k_edge_sum     Sobel (replicated border) per channel in FP32, the four maps
//                 T(max(g,0)), T(max(-g,0)) for g in {g_h, g_v}, OR-ed over
//                 channels and summed: S in 0..4 (uint8).
//  k_harris       integer Harris response R = 25 (A B - C^2) - (A + B)^2 of S
//                 (k = 1/25; Sobel of S with replicated border, 5x5 box sums
//                 with zero outside the image), 32x32 output tiles in smem.
//  k_nms_collect  3x3 non-maximum suppression (strict against lower pixel ids,
//                 >= against higher ones), R > 0; survivors are appended as the
//                 64-bit rank key ((2^31-1-R) << 32 | pixel id).
//  k_topn         one CTA per image: radix-select of the N smallest rank keys,
//                 bitonic sort, centre -> clamped top-left, rank-ordered
//                 removal of duplicates, uniform-grid fill.
// Everything after the edge maps is integer arithmetic, so the keys are
// bit-exact given the edge maps.
#include "glr_kernels.cuh"

namespace glr {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Sobel gradients (replicated border) at (r, c) of one channel, in a fixed FP32
// order (exact for 8-bit-quantised images): gh = right - left columns, gv =
// bottom - top rows, weights 1 2 1.
__device__ __forceinline__ void sobel_at(const float* __restrict__ im, int H, int W, int r, int c, float& gh,
                                         float& gv) {
  const int rm = max(r - 1, 0), rp = min(r + 1, H - 1), cm = max(c - 1, 0), cp = min(c + 1, W - 1);
  const float a00 = __ldg(im + rm * W + cm), a01 = __ldg(im + rm * W + c), a02 = __ldg(im + rm * W + cp);
  const float a10 = __ldg(im + r * W + cm), a12 = __ldg(im + r * W + cp);
  const float a20 = __ldg(im + rp * W + cm), a21 = __ldg(im + rp * W + c), a22 = __ldg(im + rp * W + cp);
  gh = ((a02 - a00) + 2.f * (a12 - a10)) + (a22 - a20);
  gv = ((a20 - a00) + 2.f * (a21 - a01)) + (a22 - a02);
}

// The four binary edge maps of Eq. 2 for every channel (the operands of the
// heat map of Eq. 4): planes[f][m * C + ch][r][c] = 0 / 1 for m = h+, h-, v+, v-.
__global__ void __launch_bounds__(256) k_edge_planes(const float* __restrict__ x, int n_img, int C, int H, int W,
                                                     float th, float* __restrict__ planes) {
  const long long HW = (long long)H * W;
  const long long total = (long long)n_img * C * HW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long fc = i / HW;
    const int p = (int)(i - fc * HW);
    const int f = (int)(fc / C), ch = (int)(fc - (long long)f * C);
    const int r = p / W, c = p - (p / W) * W;
    float gh, gv;
    sobel_at(x + fc * HW, H, W, r, c, gh, gv);
    float* o = planes + ((long long)f * 4 * C + ch) * HW + p;
    o[0] = gh > th ? 1.f : 0.f;
    o[(long long)C * HW] = -gh > th ? 1.f : 0.f;
    o[2LL * C * HW] = gv > th ? 1.f : 0.f;
    o[3LL * C * HW] = -gv > th ? 1.f : 0.f;
  }
}

__global__ void __launch_bounds__(256) k_edge_sum(const float* __restrict__ x, int n_img, int C, int H, int W,
                                                  float th, uint8_t* __restrict__ S) {
  const long long HW = (long long)H * W;
  const long long total = (long long)n_img * HW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / HW;
    const int p = (int)(i - f * HW);
    const int r = p / W, c = p - (p / W) * W;
    unsigned bits = 0;
    for (int ch = 0; ch < C; ++ch) {
      float gh, gv;
      sobel_at(x + (f * C + ch) * HW, H, W, r, c, gh, gv);
      bits |= (gh > th ? 1u : 0u) | (-gh > th ? 2u : 0u) | (gv > th ? 4u : 0u) | (-gv > th ? 8u : 0u);
    }
    S[i] = (uint8_t)__popc(bits);
  }
}

constexpr int HT = 32;  // Harris output tile

__global__ void __launch_bounds__(256) k_harris(const uint8_t* __restrict__ S, int H, int W, int32_t* __restrict__ R) {
  __shared__ int Ss[HT + 6][HT + 7];
  __shared__ int Pxx[HT + 4][HT + 4], Pyy[HT + 4][HT + 4], Pxy[HT + 4][HT + 4];
  __shared__ int Hxx[HT + 4][HT], Hyy[HT + 4][HT], Hxy[HT + 4][HT];
  const int f = blockIdx.z;
  const int r0 = blockIdx.y * HT, c0 = blockIdx.x * HT;
  const uint8_t* Sf = S + (long long)f * H * W;
  const int tid = threadIdx.x;
  for (int i = tid; i < (HT + 6) * (HT + 6); i += 256) {
    const int a = i / (HT + 6), b = i % (HT + 6);
    const int rr = clampi(r0 - 3 + a, 0, H - 1), cc = clampi(c0 - 3 + b, 0, W - 1);
    Ss[a][b] = Sf[(long long)rr * W + cc];
  }
  __syncthreads();
  for (int i = tid; i < (HT + 4) * (HT + 4); i += 256) {
    const int a = i / (HT + 4), b = i % (HT + 4);
    const int rr = r0 - 2 + a, cc = c0 - 2 + b;
    int xx = 0, yy = 0, xy = 0;
    if (rr >= 0 && rr < H && cc >= 0 && cc < W) {
      const int ix = (Ss[a][b + 2] - Ss[a][b]) + 2 * (Ss[a + 1][b + 2] - Ss[a + 1][b]) + (Ss[a + 2][b + 2] - Ss[a + 2][b]);
      const int iy = (Ss[a + 2][b] - Ss[a][b]) + 2 * (Ss[a + 2][b + 1] - Ss[a][b + 1]) + (Ss[a + 2][b + 2] - Ss[a][b + 2]);
      xx = ix * ix;
      yy = iy * iy;
      xy = ix * iy;
    }
    Pxx[a][b] = xx;
    Pyy[a][b] = yy;
    Pxy[a][b] = xy;
  }
  __syncthreads();
  for (int i = tid; i < (HT + 4) * HT; i += 256) {
    const int a = i / HT, b = i % HT;
    int sx = 0, sy = 0, sxy = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      sx += Pxx[a][b + k];
      sy += Pyy[a][b + k];
      sxy += Pxy[a][b + k];
    }
    Hxx[a][b] = sx;
    Hyy[a][b] = sy;
    Hxy[a][b] = sxy;
  }
  __syncthreads();
  for (int i = tid; i < HT * HT; i += 256) {
    const int a = i / HT, b = i % HT;
    const int rr = r0 + a, cc = c0 + b;
    if (rr >= H || cc >= W) continue;
    long long A = 0, B = 0, Cc = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      A += Hxx[a + k][b];
      B += Hyy[a + k][b];
      Cc += Hxy[a + k][b];
    }
    const long long resp = 25 * (A * B - Cc * Cc) - (A + B) * (A + B);
    R[(long long)f * H * W + (long long)rr * W + cc] = (int32_t)resp;
  }
}

__global__ void __launch_bounds__(256) k_nms_collect(const int32_t* __restrict__ R, int n_img, int H, int W,
                                                     unsigned long long* __restrict__ cand, long long cap,
                                                     unsigned int* __restrict__ cnt) {
  const long long HW = (long long)H * W;
  const long long total = (long long)n_img * HW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / HW;
    const int p = (int)(i - f * HW);
    const int r = p / W, c = p - (p / W) * W;
    const int32_t* Rf = R + f * HW;
    const int32_t v = Rf[p];
    if (v <= 0) continue;
    bool keep = true;
#pragma unroll
    for (int dr = -1; dr <= 1; ++dr) {
#pragma unroll
      for (int dc = -1; dc <= 1; ++dc) {
        if (dr == 0 && dc == 0) continue;
        const int rr = r + dr, cc = c + dc;
        if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
        const int32_t n = Rf[rr * W + cc];
        const bool lower = (dr < 0) || (dr == 0 && dc < 0);
        keep = keep && (lower ? (v > n) : (v >= n));
      }
    }
    if (!keep) continue;
    const unsigned slot = atomicAdd(cnt + f, 1u);
    if (slot < cap)
      cand[f * cap + slot] = ((unsigned long long)(0x7fffffffu - (uint32_t)v) << 32) | (unsigned)p;
  }
}

// ---- block helpers (blockDim.x == 1024)
__device__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;  // inclusive
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const int base = wid ? warp_sums[wid - 1] : 0;
  const int res = base + x - v;
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(1024) k_topn(const unsigned long long* __restrict__ cand,
                                               const unsigned int* __restrict__ cnt, long long cap, int H, int W,
                                               int P, int N, int n_uniform, int pow2, uint32_t* __restrict__ bitmap,
                                               int32_t* __restrict__ keys, int32_t* __restrict__ n_found,
                                               int32_t* __restrict__ n_corner) {
  extern __shared__ unsigned long long sb[];  // [pow2]
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix, s_mask;
  __shared__ long long s_k;
  __shared__ int s_nsel, s_total;
  __shared__ int warp_sums[32];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long M = min((long long)cnt[f], cap);
  const unsigned long long* cf = cand + (long long)f * cap;
  const int Nc = N - n_uniform;  // corners allowed (the rest are uniform keys)

  // 1. radix-select the Nc-th smallest rank key when there are more than Nc corners
  unsigned long long T = ~0ull;
  if (Nc == 0) T = 0;  // no corner is taken (rank keys of corners are never 0: R > 0)
  if (Nc > 0 && M > Nc) {
    if (tid == 0) {
      s_prefix = 0;
      s_mask = 0;
      s_k = Nc;
    }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      for (int i = tid; i < 256; i += 1024) hist[i] = 0;
      __syncthreads();
      const unsigned long long pre = s_prefix, msk = s_mask;
      // warp-aggregated counts: the leading bytes of the rank keys are nearly constant,
      // so lanes of a warp mostly share one bin; one atomic per distinct bin per warp
      for (long long i0 = 0; i0 < M; i0 += 1024) {
        const long long i = i0 + tid;
        unsigned bin = 256u;
        if (i < M) {
          const unsigned long long k = cf[i];
          if ((k & msk) == pre) bin = (unsigned)((k >> shift) & 255u);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (bin < 256u && (tid & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
      }
      __syncthreads();
      if (tid == 0) {
        long long cum = 0;
        int sel = 255;
        for (int b = 0; b < 256; ++b) {
          if (cum + hist[b] >= s_k) {
            sel = b;
            break;
          }
          cum += hist[b];
        }
        s_k -= cum;
        s_prefix = pre | ((unsigned long long)sel << shift);
        s_mask = msk | (255ull << shift);
      }
      __syncthreads();
    }
    T = s_prefix;
  }
  // 2. collect the selected rank keys and sort them
  if (tid == 0) s_nsel = 0;
  for (int i = tid; i < pow2; i += 1024) sb[i] = ~0ull;
  __syncthreads();
  for (long long i = tid; Nc > 0 && i < M; i += 1024) {
    const unsigned long long k = cf[i];
    if (k <= T) {
      const int slot = atomicAdd(&s_nsel, 1);
      if (slot < pow2) sb[slot] = k;
    }
  }
  __syncthreads();
  const int nsel = min(s_nsel, Nc);
  for (int k = 2; k <= pow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < pow2; i += 1024) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const unsigned long long a = sb[i], b = sb[ixj];
          if ((a > b) == up) {
            sb[i] = b;
            sb[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // 3. centre -> clamped top-left position id (rank order is the array order)
  for (int i = tid; i < nsel; i += 1024) {
    const unsigned pix = (unsigned)(sb[i] & 0xffffffffull);
    const int r = (int)(pix / (unsigned)W), c = (int)(pix % (unsigned)W);
    const int tr = clampi(r - P / 2, 0, Hq - 1), tc = clampi(c - P / 2, 0, Wq - 1);
    sb[i] = (unsigned long long)(tr * Wq + tc);
  }
  __syncthreads();
  // 4. duplicates: only top-lefts on the border of the position grid can collide
  //    (an unclamped coordinate is one-to-one); drop later ranks of a repeated id:
  //    each border position records its first rank (atomicMin over the ranks).
  const int per = (nsel + 1023) / 1024;
  int* first = reinterpret_cast<int*>(sb + pow2);  // [2 (Hq + Wq)] border slots
  for (int i = tid; i < 2 * (Hq + Wq); i += 1024) first[i] = 0x7fffffff;
  __syncthreads();
  // slot of a border position: top row, bottom row, left column, right column
  auto border_slot = [&](int q) -> int {
    const int tr = q / Wq, tc = q - (q / Wq) * Wq;
    if (tr == 0) return tc;
    if (tr == Hq - 1) return Wq + tc;
    if (tc == 0) return 2 * Wq + tr;
    if (tc == Wq - 1) return 2 * Wq + Hq + tr;
    return -1;
  };
  for (int t = 0; t < per; ++t) {
    const int i = tid * per + t;
    if (i >= nsel) break;
    const int b = border_slot((int)sb[i]);
    if (b >= 0) atomicMin(first + b, i);
  }
  __syncthreads();
  int keepbits = 0;  // bit t: entry tid*per + t is kept
  for (int t = 0; t < per; ++t) {
    const int i = tid * per + t;
    if (i >= nsel) break;
    const int b = border_slot((int)sb[i]);
    if (b < 0 || first[b] == i) keepbits |= 1 << t;
  }
  const int nk_local = __popc(keepbits);
  const int base = block_exclusive_scan(nk_local, warp_sums, &s_total);
  const int n_kept = s_total;
  int32_t* kf = keys + (long long)f * N;
  {
    int o = base;
    for (int t = 0; t < per; ++t)
      if (keepbits & (1 << t)) kf[o++] = (int32_t)sb[tid * per + t];
  }
  // 5. uniform grid fill in row-major order, skipping positions already chosen:
  //    first the grid of stride isqrt(npos / n_uniform) (mixed selections), then the
  //    grid of stride isqrt(npos / N) while keys are still missing
  if (n_kept < N) {
    const long long npos = (long long)Hq * Wq;
    const long long words = (npos + 31) / 32;
    uint32_t* bm = bitmap + (long long)f * words;
    for (long long i = tid; i < words; i += 1024) bm[i] = 0;
    __syncthreads();
    for (int t = 0; t < per; ++t)
      if (keepbits & (1 << t)) {
        const int q = (int)sb[tid * per + t];
        atomicOr(bm + (q >> 5), 1u << (q & 31));
      }
    __syncthreads();
    int filled = n_kept;
    for (int pass = (n_uniform > 0 ? 0 : 1); pass < 2 && filled < N; ++pass) {
      long long s;
      if (pass == 0) {  // the smallest stride whose grid has at most n_uniform points
        s = 1;
        while (((Hq + s - 1) / s) * ((Wq + s - 1) / s) > n_uniform) ++s;
      } else {
        const long long ratio = npos / N;
        s = (long long)sqrt((double)ratio);
        while (s * s > ratio) --s;
        while ((s + 1) * (s + 1) <= ratio) ++s;
        if (s < 1) s = 1;
      }
      const long long ncol = (Wq + s - 1) / s, nrow = (Hq + s - 1) / s;
      const long long G = ncol * nrow;
      for (long long g0 = 0; g0 < G && filled < N; g0 += 1024) {
        const long long g = g0 + tid;
        int freeq = 0;
        long long q = 0;
        if (g < G) {
          q = (g / ncol) * s * Wq + (g % ncol) * s;
          freeq = ((bm[q >> 5] >> (q & 31)) & 1u) ? 0 : 1;
        }
        const int off = block_exclusive_scan(freeq, warp_sums, &s_total);
        if (freeq && filled + off < N) {
          kf[filled + off] = (int32_t)q;
          atomicOr(bm + (q >> 5), 1u << (q & 31));  // the second grid skips it
        }
        filled += s_total;  // every thread sees the same s_total
        __syncthreads();
      }
      filled = min(filled, N);
    }
  }
  if (tid == 0) {
    n_found[f] = N;
    if (n_corner) n_corner[f] = n_kept;
  }
}

}  // namespace

SelectWs select_ws_layout(const glr_images& im, int N) {
  WsLayout L;
  SelectWs w;
  const long long HW = (long long)im.H * im.W;
  const long long cap = (long long)((im.H + 1) / 2) * ((im.W + 1) / 2);
  const long long npos = (long long)(im.H - im.P + 1) * (im.W - im.P + 1);
  w.S_off = L.take((size_t)im.n_img * HW);
  w.R_off = L.take((size_t)im.n_img * HW * 4);
  w.cand_off = L.take((size_t)im.n_img * cap * 8);
  w.cnt_off = L.take((size_t)im.n_img * 4);
  w.bitmap_off = L.take((size_t)im.n_img * ((npos + 31) / 32) * 4);
  w.total = L.off;
  (void)N;
  return w;
}

glr_status launch_select(const float* x, const glr_images& im, float th, int N, int n_uniform, int32_t* keys,
                         int32_t* n_found, int32_t* n_corner, char* ws, const SelectWs& L, cudaStream_t s) {
  const long long HW = (long long)im.H * im.W;
  const long long cap = (long long)((im.H + 1) / 2) * ((im.W + 1) / 2);
  uint8_t* S = reinterpret_cast<uint8_t*>(ws + L.S_off);
  int32_t* R = reinterpret_cast<int32_t*>(ws + L.R_off);
  auto* cand = reinterpret_cast<unsigned long long*>(ws + L.cand_off);
  auto* cnt = reinterpret_cast<unsigned int*>(ws + L.cnt_off);
  auto* bm = reinterpret_cast<uint32_t*>(ws + L.bitmap_off);
  if (cudaMemsetAsync(cnt, 0, (size_t)im.n_img * 4, s) != cudaSuccess) return GLR_ECUDA;
  const long long total = (long long)im.n_img * HW;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
  GLR_LAUNCH("k_edge_sum", s, k_edge_sum<<<blocks, 256, 0, s>>>(x, im.n_img, im.C, im.H, im.W, th, S));
  dim3 hg((unsigned)ceil_div(im.W, HT), (unsigned)ceil_div(im.H, HT), (unsigned)im.n_img);
  GLR_LAUNCH("k_harris", s, k_harris<<<hg, 256, 0, s>>>(S, im.H, im.W, R));
  GLR_LAUNCH("k_nms_collect", s, k_nms_collect<<<blocks, 256, 0, s>>>(R, im.n_img, im.H, im.W, cand, cap, cnt));
  int pow2 = 1;
  while (pow2 < N) pow2 <<= 1;
  const int Hq = im.H - im.P + 1, Wq = im.W - im.P + 1;
  const size_t smem = (size_t)pow2 * 8 + (size_t)2 * (Hq + Wq) * 4;  // sort buffer + border slots
  if (smem > 200 * 1024) return GLR_ENOTSUP;
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(k_topn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
      return GLR_ECUDA;
    attr_done = true;
  }
  GLR_LAUNCH("k_topn", s, k_topn<<<im.n_img, 1024, smem, s>>>(cand, cnt, cap, im.H, im.W, im.P, N, n_uniform, pow2, bm, keys, n_found, n_corner));
  return GLR_OK;
}

glr_status launch_edge_planes(const float* x, const glr_images& im, float th, float* planes, cudaStream_t s) {
  const long long total = (long long)im.n_img * im.C * im.H * im.W;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
  GLR_LAUNCH("k_edge_planes", s, k_edge_planes<<<blocks, 256, 0, s>>>(x, im.n_img, im.C, im.H, im.W, th, planes));
  return GLR_OK;
}

}  // namespace glr
