// Global patch matching (Section 2: the search covers every position of the
// image; the similarity is the squared L2 distance of Eq. 1, evaluated as
// ||p||^2 - 2<p,q> + ||q||^2 for all key/position pairs, i.e. the Conv2d
// heat map of Eq. 4 on intensities) fused with a running per-key top-K.
//
// Pipeline of glr_match_topk:
//   k_image_mean   mean of each image (values are shifted by it before the
//                  expanded form; distances are unchanged, cancellation shrinks)
//   k_patch_norms  ||q - mu||^2 for every position
//   k_key_vectors  shifted key patches, [img][key][d]
//   scorer         FP32 (k_match_fp32, below) or BF16 tcgen05 (k_match_tc.cu):
//                  scores of 128 keys x all positions of a split, pushed
//                  through the running top-K' streams (topk_stream.cuh)
//   k_rerank       per key: the K' best stream scores over all the key's
//                  streams (ties to smaller ids), their exact FP32
//                  sum((p-q)^2), sort by (distance, id), emit the K best.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "glr_kernels.cuh"
#include "topk_stream.cuh"

namespace glr {

namespace {

// Image mean in two passes: S CTAs per image each sum a contiguous slice in FP64
// (float4 loads when aligned) into part[f][slice]; then one thread per image adds
// the S partial sums in slice order, so the result does not depend on scheduling.
// S depends only on the shape (about two CTAs per SM over the batch).
__global__ void __launch_bounds__(512)
    k_image_mean_part(const float* __restrict__ x, long long n_per_img, int S, double* __restrict__ part, ImgMap imap) {
  __shared__ double red[16];
  const long long f = blockIdx.x / S;
  const int sl = (int)(blockIdx.x - f * S);
  const float* xf = x + imap.pix((int)f, n_per_img);
  const long long per = (n_per_img + S - 1) / S;
  const long long lo = min(n_per_img, per * sl), hi = min(n_per_img, lo + per);
  double s = 0.0;
  long long i = lo + threadIdx.x;
  // aligned float4 body (slice boundaries rounded to 4 elements)
  const long long a0 = min(hi, (lo + 3) & ~3LL), a1 = max(a0, hi & ~3LL);
  if ((reinterpret_cast<uintptr_t>(xf) & 15u) == 0) {
    for (i = lo + threadIdx.x; i < a0; i += 512) s += (double)xf[i];
    const float4* v4 = reinterpret_cast<const float4*>(xf);
    for (long long j = a0 / 4 + threadIdx.x; j < a1 / 4; j += 512) {
      const float4 v = __ldg(v4 + j);
      s += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
    }
    for (i = a1 + threadIdx.x; i < hi; i += 512) s += (double)xf[i];
  } else {
    for (; i < hi; i += 512) s += (double)xf[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 16; ++w) t += red[w];
    part[f * S + sl] = t;
  }
}

__global__ void k_image_mean_final(const double* __restrict__ part, int n_img, int S, long long n_per_img,
                                   float* __restrict__ mean) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_img) return;
  double t = 0.0;
  for (int sl = 0; sl < S; ++sl) t += part[(long long)f * S + sl];
  mean[f] = (float)(t / (double)n_per_img);
}

__global__ void __launch_bounds__(256) k_patch_norms(const float* __restrict__ x, const float* __restrict__ mean,
                                                     int n_img, int C, int H, int W, int P, float* __restrict__ qn) {
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const long long total = (long long)n_img * npos;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / npos;
    const int q = (int)(i - f * npos);
    const int r = q / Wq, c = q - (q / Wq) * Wq;
    const float mu = mean[f];
    float s = 0.f;
    for (int ch = 0; ch < C; ++ch)
      for (int dr = 0; dr < P; ++dr) {
        const float* row = x + (((long long)f * C + ch) * H + r + dr) * W + c;
        for (int dc = 0; dc < P; ++dc) {
          const float v = __ldg(row + dc) - mu;
          s = fmaf(v, v, s);
        }
      }
    qn[i] = s;
  }
}

__global__ void __launch_bounds__(256) k_key_vectors(const float* __restrict__ x, const float* __restrict__ mean,
                                                     const int32_t* __restrict__ keys,
                                                     const int32_t* __restrict__ n_found, int n_img, int C, int H,
                                                     int W, int P, int N, int Npad, float* __restrict__ keyv,
                                                     StatusBlock* st, ImgMap imap) {
  const int d = C * P * P;
  const int Wq = W - P + 1;
  const long long total = (long long)n_img * Npad * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long fk = i / d;
    const int e = (int)(i - fk * d);
    const int f = (int)(fk / Npad), k = (int)(fk - (long long)f * Npad);
    float v = 0.f;
    const int q = k < min(n_found[imap.id(f)], N) ? keys[imap.key(f, N) + k] : -1;
    if ((unsigned)q >= (unsigned)(Wq * (H - P + 1))) {
      if (q != -1 && e == 0) status_set(st, GLR_DEV_BAD_INDEX);
    } else {
      const int r = q / Wq, c = q - (q / Wq) * Wq;
      const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
      v = __ldg(x + imap.pix(f, (long long)C * H * W) + ((long long)ch * H + r + dr) * W + c + dc) - mean[f];
    }
    keyv[i] = v;
  }
}

// ---------------------------------------------------------------------------
// FP32 scorer: 128 keys x 128 positions per tile, 256 threads, 8x8 per thread.
// A position tile is one row r of the position grid, columns c0..c0+127; its
// patches are read from a C x P x (128+P-1) strip of the image, so no patch
// matrix is materialised.  Thread (ty, tx) owns keys 8ty..8ty+7 and positions
// 8tx..8tx+7; for each (channel, patch row) it loads a 16-float window of the
// strip once and reuses it for the P column offsets.
// ---------------------------------------------------------------------------
constexpr int FT = 128;     // keys and positions per tile
constexpr int SC_LD = 132;  // score tile row stride (conflict-free LDS.128 by row owners)

template <int P>
__global__ void __launch_bounds__(256, 2)
    k_match_fp32(const float* __restrict__ x, const float* __restrict__ mean, const float* __restrict__ qn,
                 const float* __restrict__ keyv, const int32_t* __restrict__ n_found, int C, int H, int W, int Npad,
                 int splits, int tiles_per_split, int cc, StreamCfg cfg, uint2* __restrict__ bufs,
                 int* __restrict__ buf_cnt, uint32_t* __restrict__ tau_gl, StatusBlock* st) {
  extern __shared__ __align__(16) float smem[];
  // channels are processed in chunks of cc (all of them at once when the key tile fits)
  const int d = C * P * P;
  const int dc_ = cc * P * P;                // key values per chunk
  const bool one_chunk = cc >= C;
  float* As = smem;                          // [cc P^2][FT]
  float* strip = As + dc_ * FT;              // [cc][P][FT + 8]
  float* Sc = strip + cc * P * (FT + 8);     // [FT][SC_LD]
  float* pn = Sc + FT * SC_LD;              // [FT]
  unsigned* hist = reinterpret_cast<unsigned*>(pn + FT);  // [8][256]
  uint32_t* tau_sh = hist + 8 * 256;                        // [FT] published thresholds of the tile's rows
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int kt = blockIdx.x, f = blockIdx.y, split = blockIdx.z;
  const int Hq = H - P + 1, Wq = W - P + 1;
  const int tpr = (Wq + FT - 1) / FT;
  const int ntiles = Hq * tpr;
  const int nf = min(n_found[f], Npad);
  const float mu = mean[f];

  // key tile, transposed: As[e][i] (channels ch0 .. ch0 + n of every key)
  const float* kv = keyv + ((long long)f * Npad + (long long)kt * FT) * d;
  auto load_keys = [&](int ch0, int n) {
    const int dn = n * P * P;
    for (int i = tid; i < dn * FT; i += 256) {
      const int key = i / dn, e = i - (i / dn) * dn;
      As[e * FT + key] = kv[(long long)key * d + ch0 * P * P + e];
    }
  };
  if (one_chunk) load_keys(0, C);
  if (tid < FT) {
    float s = 0.f;
    for (int e = 0; e < d; ++e) {
      const float v = kv[(long long)tid * d + e];
      s = fmaf(v, v, s);
    }
    pn[tid] = s;
    tau_sh[tid] = 0xffffffffu;
  }
  __syncthreads();
  // stream owned by this thread: row = 32 (wid % 4) + lane, column half h = wid / 4
  const int row = 32 * (wid & 3) + lane;
  const int h = wid >> 2;
  const int key = kt * FT + row;
  const long long stream = (((long long)f * Npad + key) * splits + split) * 2 + h;
  uint2* mybuf = bufs + stream * (cfg.cap + 32);
  float tau = (key < nf) ? INFINITY : -INFINITY;
  int cnt = 0;
  uint2 stats = make_uint2(0u, 0u);
  unsigned* whist = hist + wid * 256;
  uint32_t* pub_sh = tau_sh + 32 * (wid & 3);
  uint32_t* pub_gl = tau_gl + (long long)f * Npad + (long long)kt * FT + 32 * (wid & 3);

  const int ty = tid >> 4, tx = tid & 15;
  const int t_begin = split * tiles_per_split;
  const int t_end = min(ntiles, t_begin + tiles_per_split);
  for (int t = t_begin; t < t_end; ++t) {
    const int r = t / tpr, c0 = (t - (t / tpr) * tpr) * FT;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 1
    for (int ch0 = 0; ch0 < C; ch0 += cc) {
    const int nch = min(cc, C - ch0);
    __syncthreads();  // previous chunk / tile fully consumed
    if (!one_chunk) load_keys(ch0, nch);
    for (int i = tid; i < nch * P * (FT + 8); i += 256) {
      const int cr = i / (FT + 8), j = i - (i / (FT + 8)) * (FT + 8);
      const int ch = ch0 + cr / P, dr = cr - (cr / P) * P;
      const int col = c0 + j;
      strip[i] = (col < W) ? __ldg(x + (((long long)f * C + ch) * H + r + dr) * W + col) - mu : 0.f;
    }
    __syncthreads();
    for (int ch = 0; ch < nch; ++ch) {
#pragma unroll
      for (int dr = 0; dr < P; ++dr) {
        float w[16];
        const float4* sp = reinterpret_cast<const float4*>(strip + (ch * P + dr) * (FT + 8) + tx * 8);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float4 t4 = sp[v];
          w[4 * v] = t4.x;
          w[4 * v + 1] = t4.y;
          w[4 * v + 2] = t4.z;
          w[4 * v + 3] = t4.w;
        }
#pragma unroll
        for (int dc = 0; dc < P; ++dc) {
          const float4* ap = reinterpret_cast<const float4*>(As + ((ch * P + dr) * P + dc) * FT + ty * 8);
          const float4 a0 = ap[0], a1 = ap[1];
          const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], w[j + dc], acc[i][j]);
        }
      }
    }
    }  // channel chunks
    // scores s = ||p||^2 + ||q||^2 - 2 <p,q>; missing positions -> +inf
    {
      float qv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int cc = c0 + tx * 8 + j;
        qv[j] = (cc < Wq) ? __ldg(qn + (long long)f * Hq * Wq + (long long)r * Wq + cc) : INFINITY;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float pi = pn[ty * 8 + i];
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = fmaf(-2.f, acc[i][j], pi + qv[j]);
        float4* dst = reinterpret_cast<float4*>(Sc + (ty * 8 + i) * SC_LD + tx * 8);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
      }
    }
    __syncthreads();
    // row owners push their half row in two 32-column chunks
    const int qbase = r * Wq + c0;
    const uint32_t gl = *reinterpret_cast<volatile uint32_t*>(pub_gl + lane);
#pragma unroll 1
    for (int ch2 = 0; ch2 < 2; ++ch2) {
      const int col0 = h * 64 + ch2 * 32;
      const int nvalid = max(0, min(32, Wq - (c0 + col0)));
      float s[32];
      const float4* src = reinterpret_cast<const float4*>(Sc + row * SC_LD + col0);
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const float4 t4 = src[v];
        s[4 * v] = t4.x;
        s[4 * v + 1] = t4.y;
        s[4 * v + 2] = t4.z;
        s[4 * v + 3] = t4.w;
      }
      const float te = stream_tau_eff(tau, *reinterpret_cast<volatile uint32_t*>(pub_sh + lane), gl);
      const unsigned rows = stream_filter(s, nvalid, te);
      if (rows)
        stream_append(rows, Sc + (32 * (wid & 3)) * SC_LD + col0, SC_LD, qbase + col0, nvalid, te, tau, cnt, mybuf,
                      cfg, whist, pub_sh, pub_gl, stats);
    }
  }
  if (cfg.finish) stream_finish(tau, cnt, mybuf, cfg, whist);
  stream_stats_flush(stats, st);
  buf_cnt[stream] = (key < nf) ? cnt : 0;
}

// ---------------------------------------------------------------------------
// Exact re-rank: one warp per key.  The K' candidates with the best stream
// scores over every stream of the key are scored with the direct FP32
// sum((p - q)^2) (fixed order over the vector index), then sorted by
// (distance, position id) with a bitonic sort in shared memory; the first K are
// written.
// ---------------------------------------------------------------------------
constexpr int RR_WARPS = 4;
constexpr int kRerankMaxList = 2048;  // candidates of one key held by the re-rank (pow2)

// A threshold T with exactly `rank` of the n distinct 64-bit keys <= T: the
// rank-th smallest key, or the upper end of its radix bin when that key is the
// largest of the bin (MSB radix select, 8 bits per pass, stopping early; one
// warp, 256 shared counters).
__device__ unsigned long long warp_select_kth(const unsigned long long* list, int n, int rank, unsigned* hist,
                                              int lane) {
  // leading bytes that every entry shares need no pass (nearby scores share their exponent byte,
  // and a pass over one bin would put every entry's atomic on the same counter)
  unsigned long long all_and = ~0ull, all_or = 0ull;
  for (int i = lane; i < n; i += 32) {
    const unsigned long long e = list[i];
    all_and &= e;
    all_or |= e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    all_and &= __shfl_xor_sync(0xffffffffu, all_and, o);
    all_or |= __shfl_xor_sync(0xffffffffu, all_or, o);
  }
  const unsigned long long diff = all_and ^ all_or;  // bits that vary over the list
  if (diff == 0) return all_and;                    // every entry equal (n == 1)
  const int first = 63 - __clzll((long long)diff);  // highest varying bit
  const int pass0 = (63 - first) / 8;                // first byte with a varying bit
  unsigned long long pmask = pass0 > 0 ? ~0ull << (64 - 8 * pass0) : 0ull;
  unsigned long long prefix = all_and & pmask;
  for (int pass = pass0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int i = lane; i < 256; i += 32) hist[i] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const unsigned long long e = list[i];
      if ((e & pmask) == prefix) atomicAdd(&hist[(e >> shift) & 255u], 1u);
    }
    __syncwarp();
    int loc[8], sum = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      loc[t] = (int)hist[lane * 8 + t];
      sum += loc[t];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int yv = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += yv;
    }
    const int excl = incl - sum;
    const int owner = __ffs(__ballot_sync(0xffffffffu, excl < rank && rank <= incl)) - 1;
    int sel = 0, before = 0, in_bin = 0;
    if (lane == owner) {
      int c = excl;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (c + loc[t] >= rank) {
          sel = lane * 8 + t;
          before = c;
          in_bin = loc[t];
          break;
        }
        c += loc[t];
      }
    }
    sel = __shfl_sync(0xffffffffu, sel, owner);
    before = __shfl_sync(0xffffffffu, before, owner);
    in_bin = __shfl_sync(0xffffffffu, in_bin, owner);
    rank -= before;
    prefix |= (unsigned long long)sel << shift;
    pmask |= 255ull << shift;
    __syncwarp();
    // the wanted key is the largest of its bin: every key of the bin is kept, so
    // the bin's upper end is the answer (exactly rank keys lie below it)
    if (rank == in_bin) return prefix | ((1ull << shift) - 1ull);
  }
  return prefix;
}

// Keep the k smallest of n distinct keys (k < n), compacted to the front of the
// list in their current order; returns k.
__device__ int warp_keep_smallest(unsigned long long* list, int n, int k, unsigned* hist, int lane) {
  const unsigned long long T = warp_select_kth(list, n, k, hist, lane);
  int out = 0;
  const unsigned ltm = (1u << lane) - 1u;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const unsigned long long e = i < n ? list[i] : ~0ull;
    const bool keep = i < n && e <= T;
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) list[out + __popc(km & ltm)] = e;
    out += __popc(km);
    __syncwarp();
  }
  return out;
}

__global__ void __launch_bounds__(RR_WARPS * 32)
    k_rerank(const float* __restrict__ x, const int32_t* __restrict__ keys, const int32_t* __restrict__ n_found,
             int n_img, int C, int H, int W, int P, int N, int Npad, int K, int streams_per_key, int cap_slots,
             int kp, int pow2, const uint2* __restrict__ bufs, const int* __restrict__ buf_cnt,
             int exact_scores, float dist_scale, int window, int32_t* __restrict__ idx, float* __restrict__ dist,
             ImgMap imap) {
  // window > 0: the candidates are every position within `window` rows and columns
  // of the key (block matching in a local window) instead of the stream buffers
  // exact_scores != 0: the stream scores are already exact (the heat map of Eq. 4 on
  // 0/1 operands); they are sorted as they are and dist = dist_scale * score
  extern __shared__ unsigned long long rr_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int d = C * P * P;
  const int Wq = W - P + 1;
  unsigned long long* list = rr_smem + (size_t)wid * pow2;
  const int dpad = (d + 31) & ~31;
  float* pv = reinterpret_cast<float*>(rr_smem + (size_t)RR_WARPS * pow2) + wid * (dpad + 256);  // key patch + 256 counters
  const long long nkeys = (long long)n_img * N;
  for (long long gk = blockIdx.x * (long long)RR_WARPS + wid; gk < nkeys; gk += (long long)gridDim.x * RR_WARPS) {
    const int f = (int)(gk / N), k = (int)(gk - (long long)f * N);
    if (k >= min(n_found[imap.id(f)], N)) continue;
    const long long krow = imap.key(f, N) + k;  // row of this key in keys, idx and dist
    const float* xf = x + imap.pix(f, (long long)C * H * W);
    const int kq = keys[krow];
    if ((unsigned)kq >= (unsigned)(Wq * (H - P + 1))) continue;  // flagged by k_key_vectors
    const int kr = kq / Wq, kc = kq - (kq / Wq) * Wq;
    for (int e = lane; !exact_scores && e < d; e += 32) {
      const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
      pv[e] = __ldg(xf + ((long long)ch * H + kr + dr) * W + kc + dc);
    }
    // gather candidate ids
    int total = 0;
    if (window > 0) {
      // a (2w+1)^2 window centred on the key, shifted inside the position grid at its borders
      const int Hq = H - P + 1, wl = 2 * window + 1;
      const int r0 = min(max(kr - window, 0), Hq - wl), c0 = min(max(kc - window, 0), Wq - wl);
      total = wl * wl;
      for (int i = lane; i < total; i += 32) list[i] = (unsigned)((r0 + i / wl) * Wq + c0 + i % wl);
    }
    const long long s0 = ((long long)f * Npad + k) * streams_per_key;
    for (int sidx = 0; window == 0 && sidx < streams_per_key; ++sidx) {
      const int n = min(buf_cnt[s0 + sidx], cap_slots);
      const uint2* b = bufs + (s0 + sidx) * cap_slots;
      for (int i = lane; i < n; i += 32) {
        const uint2 e = b[i];
        list[total + i] = ((unsigned long long)e.x << 32) | e.y;  // (stream score, id)
      }
      total += n;
    }
    __syncwarp();
    unsigned* hist = reinterpret_cast<unsigned*>(pv + dpad);  // 256 counters after the key patch
    // the kp best stream scores over all streams of the key (ties to smaller ids):
    // which extra candidates the streams kept depends on when bounds were
    // published, so only these kp are re-ranked
    if (window == 0 && !exact_scores && total > kp) total = warp_keep_smallest(list, total, kp, hist, lane);
    // exact FP32 distances, summed in a fixed order over the vector index
    for (int i = lane; !exact_scores && i < total; i += 32) {
      const int q = (int)(unsigned)(list[i] & 0xffffffffull);
      const int r = q / Wq, c = q - (q / Wq) * Wq;
      float acc = 0.f;
      for (int ch = 0; ch < C; ++ch)
        for (int dr = 0; dr < P; ++dr) {
          const float* rowp = xf + ((long long)ch * H + r + dr) * W + c;
          const float* pp = pv + (ch * P + dr) * P;
          for (int dc = 0; dc < P; ++dc) {
            const float df = pp[dc] - __ldg(rowp + dc);
            acc = fmaf(df, df, acc);
          }
        }
      list[i] = ((unsigned long long)float_order_key(acc) << 32) | (unsigned)q;
    }
    __syncwarp();
    // select the K smallest (distance, id) pairs with an MSB radix select over the
    // 64-bit keys, then sort those K (bitonic); ties in distance go to smaller ids
    if (total > K) total = warp_keep_smallest(list, total, K, hist, lane);
    int p2 = 32;
    while (p2 < total) p2 <<= 1;
    for (int i = total + lane; i < p2; i += 32) list[i] = ~0ull;
    __syncwarp();
    for (int kk = 2; kk <= p2; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < p2; i += 32) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const bool up = (i & kk) == 0;
            const unsigned long long a = list[i], b = list[ixj];
            if ((a > b) == up) {
              list[i] = b;
              list[ixj] = a;
            }
          }
        }
        __syncwarp();
      }
    }
    for (int i = lane; i < K; i += 32) {
      const unsigned long long e = list[i];
      if (idx) idx[krow * K + i] = (int32_t)(e & 0xffffffffu);
      if (dist) dist[krow * K + i] = dist_scale * float_from_order_key((uint32_t)(e >> 32));
    }
    __syncwarp();
  }
}

// Keep the k smallest of n distinct keys (k < n) like warp_keep_smallest and return the
// largest kept key (the k-th smallest) in *kth.
__device__ int warp_keep_smallest_kth(unsigned long long* list, int n, int k, unsigned* hist, int lane,
                                      unsigned long long* kth) {
  const int out = warp_keep_smallest(list, n, k, hist, lane);
  unsigned long long m = 0;
  for (int i = lane; i < out; i += 32) m = max(m, list[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  *kth = m;
  return out;
}

// Bound and candidate chunks of every key for the exact evaluation (one warp per key, many
// warps per SM to hide the memory latency).
//  * Each lane keeps the L smallest of its share of the key's 16-bit chunk minima (the upper
//    half of each minimum's order key; runs of 8 chunks, interleaved over the lanes) in
//    registers; the K'-th smallest of those 32 L values is tau16.  It bounds the K'-th smallest
//    of all the 16-bit minima from above (the K'-th smallest of a subset is never smaller).  If
//    M is the K'-th smallest chunk minimum, K' chunks have minima <= M, so at least K' scores
//    are <= M and every chunk holding one of the key's K' smallest scores has its minimum <= M;
//    truncating the keys keeps that order, so those chunks are at or below tau16, and M lies at
//    or below the upper end of tau16's 2^16-key bucket.  tau16 equals the exact K'-th smallest
//    unless a lane's share holds more than L of the K' smallest.
//  * Then the ids of every chunk at or below tau16, ascending (the first clcap of them; ccount
//    receives the full count).
constexpr int CT_CL = 256;   // listed candidate chunks per key (exact matching)
constexpr int CT_CL_EMB = 512;  // listed candidate chunks per key (learned proposal, K' up to 256)

// L = values each lane keeps (8 for K' <= 96; 24 for the learned proposal's K' up to 256)
template <int L>
__global__ void __launch_bounds__(256) k_tau_chunk(const uint16_t* __restrict__ mins16, const int32_t* __restrict__ n_found,
                                                   int n_img, int N, int Npad, int nchunks, int kp, int clcap,
                                                   uint32_t* __restrict__ tau16, int32_t* __restrict__ ccount,
                                                   uint32_t* __restrict__ clist, StatusBlock* st,
                                                   int* __restrict__ ticket = nullptr) {
  __shared__ unsigned hist_s[8][256];
  __shared__ uint16_t vals_s[8][32 * L];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* hist = hist_s[wid];
  uint16_t* vals = vals_s[wid];
  const long long nkeys = (long long)n_img * N;
  const int n8 = nchunks / 8;  // nchunks is a multiple of 8
  if (ticket != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;  // for k_chunk_topk
  for (long long gk = blockIdx.x * 8LL + wid; gk < nkeys; gk += gridDim.x * 8LL) {
    const int f = (int)(gk / N), k = (int)(gk - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    const long long row = (long long)f * Npad + k;
    uint32_t prefix = 0xffffu;
    if (nchunks > kp) {
      // per-lane 8 smallest (sorted ascending)
      // 8 minima (16 bytes) per lane and step, the next two steps' loads in flight; a step
      // whose smallest value does not beat the lane's L-th is skipped after one compare
      const uint4* m8r = reinterpret_cast<const uint4*>(mins16 + row * nchunks);
      const uint4 none = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
      uint32_t t[L];
#pragma unroll
      for (int j = 0; j < L; ++j) t[j] = 0xffffu;
      uint4 nx1 = lane < n8 ? __ldg(m8r + lane) : none;
      uint4 nx2 = lane + 32 < n8 ? __ldg(m8r + lane + 32) : none;
      for (int i = lane; i < n8; i += 32) {
        const uint4 cur = nx1;
        nx1 = nx2;
        nx2 = i + 64 < n8 ? __ldg(m8r + i + 64) : none;
        const uint32_t m2 = __vminu2(__vminu2(cur.x, cur.y), __vminu2(cur.z, cur.w));
        if (min(m2 & 0xffffu, m2 >> 16) >= t[L - 1]) continue;
        const uint32_t w4[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          uint32_t v = (w4[h >> 1] >> (16 * (h & 1))) & 0xffffu;
          if (v < t[L - 1]) {
#pragma unroll
            for (int j = 0; j < L; ++j) {  // insertion: t stays sorted, the largest drops out
              const uint32_t lo = min(t[j], v);
              v = max(t[j], v);
              t[j] = lo;
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < L; ++j) vals[lane * L + j] = (uint16_t)t[j];
      __syncwarp();
      // the kp-th smallest of the 256 kept values: two 8-bit radix passes
      int rank = kp;
      prefix = 0;
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        const int shift = 8 - 8 * pass;
#pragma unroll
        for (int j = 0; j < 8; ++j) hist[lane * 8 + j] = 0;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < L; ++j) {
          const uint32_t e = vals[j * 32 + lane];
          if (pass == 0 || (e >> 8) == prefix) atomicAdd(&hist[(e >> shift) & 255u], 1u);
        }
        __syncwarp();
        int loc[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          loc[j] = (int)hist[lane * 8 + j];
          sum += loc[j];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int yv = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += yv;
        }
        const int excl = incl - sum;
        const int owner = __ffs(__ballot_sync(0xffffffffu, excl < rank && rank <= incl)) - 1;
        int sel = 0, before = 0;
        if (lane == owner) {
          int c = excl;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (c + loc[j] >= rank) {
              sel = lane * 8 + j;
              before = c;
              break;
            }
            c += loc[j];
          }
        }
        sel = __shfl_sync(0xffffffffu, sel, owner);
        before = __shfl_sync(0xffffffffu, before, owner);
        rank -= before;
        prefix = (prefix << 8) | (uint32_t)sel;
        __syncwarp();
      }
    }
    // candidate chunks in ascending order
    const uint4* m8 = reinterpret_cast<const uint4*>(mins16 + row * nchunks);
    int total = 0;
    uint4 nxt = lane < n8 ? __ldg(m8 + lane) : make_uint4(0u, 0u, 0u, 0u);
    for (int base = 0; base < n8; base += 32) {
      const int i = base + lane;
      uint32_t bits = 0;
      const uint4 v = nxt;
      if (i + 32 < n8) nxt = __ldg(m8 + i + 32);
      // most steps hold no candidate: the smallest of each lane's 8 minima decides that
      const uint32_t m2 = __vminu2(__vminu2(v.x, v.y), __vminu2(v.z, v.w));
      if (!__any_sync(0xffffffffu, i < n8 && min(m2 & 0xffffu, m2 >> 16) <= prefix)) continue;
      if (i < n8) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (((w[j >> 1] >> (16 * (j & 1))) & 0xffffu) <= prefix) bits |= 1u << j;
      }
      const int c = __popc(bits);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int yv = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += yv;
      }
      int pos = total + incl - c;
      while (bits) {
        const int j = __ffs(bits) - 1;
        bits &= bits - 1;
        if (pos < clcap) clist[row * clcap + pos] = (uint32_t)(8 * i + j);
        ++pos;
      }
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      tau16[row] = prefix;
      ccount[row] = total;
      atomicAdd(&st->cand_appends, (unsigned long long)total);  // candidate chunks (status counter 4)
    }
  }
}

// Exact distances sum((p - q)^2) of the cnt (score, position) entries of a warp's list (pv =
// the key's raw patch, xf = its image; the re-rank's order of summation), then the K smallest
// (distance, id) pairs written sorted to row gk of idx / dist.  list holds at least the next
// power of two above max(cnt, K) entries.
template <int PT>
__device__ void exact_topk_finish(unsigned long long* list, int cnt, const float* pv, const float* xf, int C, int H,
                                  int W, int P_, int Wq, int K, unsigned* hist, int lane, long long gk,
                                  int32_t* __restrict__ idx, float* __restrict__ dist) {
  const int P = PT ? PT : P_;
  for (int i = lane; i < cnt; i += 32) {
    const int q = (int)(unsigned)(list[i] & 0xffffffffull);
    const int r = q / Wq, c = q - (q / Wq) * Wq;
    float acc = 0.f;
    for (int ch = 0; ch < C; ++ch)
      for (int dr = 0; dr < P; ++dr) {
        const float* rowp = xf + ((long long)ch * H + r + dr) * W + c;
        const float* pp = pv + (ch * P + dr) * P;
        for (int dc = 0; dc < P; ++dc) {
          const float df = pp[dc] - __ldg(rowp + dc);
          acc = fmaf(df, df, acc);
        }
      }
    list[i] = ((unsigned long long)float_order_key(acc) << 32) | (unsigned)q;
  }
  __syncwarp();
  int total = cnt;
  if (total > K) total = warp_keep_smallest(list, total, K, hist, lane);
  int p2 = 32;
  while (p2 < total) p2 <<= 1;
  for (int i = total + lane; i < p2; i += 32) list[i] = ~0ull;
  __syncwarp();
  for (int kk = 2; kk <= p2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < p2; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & kk) == 0;
          const unsigned long long a = list[i], b = list[ixj];
          if ((a > b) == up) {
            list[i] = b;
            list[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < K; i += 32) {
    const unsigned long long e = list[i];
    if (idx) idx[gk * K + i] = (int32_t)(e & 0xffffffffu);
    if (dist) dist[gk * K + i] = float_from_order_key((uint32_t)(e >> 32));
  }
  __syncwarp();
}

// Candidate chunks of the chunk-minima scan, evaluated exactly.  One warp per key:
//  1. tau = the upper end of the bucket of the key's K'-th smallest 16-bit chunk minimum (every
//     chunk holding one of the key's K' smallest BF16 scores has its minimum at or below tau);
//  2. every chunk with minimum <= tau (in position order, 4 chunks at a time: the image strips
//     of the 4 chunks staged in shared memory, each lane scoring 4 adjacent positions from
//     registers) gets the FP32 score ||q - mu||^2 - 2 <p - mu, q> (the squared distance of the
//     mean-shifted patches minus a constant of the key), and a running list keeps the K' best
//     (score, id) pairs;
//  3. those K' get their exact distance sum((p - q)^2) (the re-rank's arithmetic), and the K
//     smallest (distance, id) pairs are written sorted.
// Chunks whose 32 positions wrap to the next row of the position grid are scored position by
// position from global memory.
constexpr int CT_WARPS = 4;
constexpr int CT_LCAP = 512;  // running top-K' list of a warp (entries)
constexpr int CT_CCAP = 512;  // candidate chunk ids gathered before they are scored

constexpr int CT_SROW = 48;   // strip row stride (floats; 16-byte aligned rows)

template <int PT, int CMAX>
__host__ __device__ constexpr size_t chunk_topk_warp_bytes() {
  return (size_t)CT_LCAP * 8 + CT_CCAP * 4 + 256 * 4 + (size_t)4 * CMAX * PT * CT_SROW * 4 + 2 * 96 * 4;
}

template <int PT, int CMAX>
__global__ void __launch_bounds__(CT_WARPS * 32, 4)
    k_chunk_topk(const float* __restrict__ x, const float* __restrict__ mean, const float* __restrict__ qn,
                 const float* __restrict__ keyv,
                 const int32_t* __restrict__ keys, const int32_t* __restrict__ n_found,
                 const uint16_t* __restrict__ mins16, const uint32_t* __restrict__ tau16s,
                 const int32_t* __restrict__ ccount, const uint32_t* __restrict__ clist_g, int n_img, int C, int H,
                 int W, int N, int Npad, int nchunks, int K, int Kp, int32_t* __restrict__ idx,
                 float* __restrict__ dist, int* __restrict__ ticket) {
  constexpr int P = PT, PP = P * P, CP = CMAX * P, DM = CMAX * PP, SW = 32 + P - 1;
  extern __shared__ unsigned long long ct_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* wbase = reinterpret_cast<uint8_t*>(ct_smem) + (size_t)wid * chunk_topk_warp_bytes<PT, CMAX>();
  unsigned long long* list = reinterpret_cast<unsigned long long*>(wbase);
  uint32_t* clist = reinterpret_cast<uint32_t*>(wbase + CT_LCAP * 8);
  unsigned* hist = reinterpret_cast<unsigned*>(wbase + CT_LCAP * 8 + CT_CCAP * 4);
  float* strip = reinterpret_cast<float*>(wbase + CT_LCAP * 8 + CT_CCAP * 4 + 256 * 4);  // [4][CP][CT_SROW]
  float* pv = strip + 4 * CP * CT_SROW;  // raw key patch (exact distances)
  float* pk = pv + 96;                   // mean-shifted key patch
  const int d = C * PP;
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const int g = lane >> 3, l8 = lane & 7;
  const unsigned ltm = (1u << lane) - 1u;
  const long long nkeys = (long long)n_img * N;
  // keys are taken one at a time from a shared ticket (zeroed by k_tau_chunk): the candidate
  // counts differ from key to key, and every resident warp stays busy until the last key
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    const long long gk = __shfl_sync(0xffffffffu, t, 0);
    if (gk >= nkeys) break;
    const int f = (int)(gk / N), k = (int)(gk - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    const int kq = keys[gk];
    if ((unsigned)kq >= (unsigned)npos) continue;  // flagged by k_key_vectors
    const int kr = kq / Wq, kc = kq - (kq / Wq) * Wq;
    const float* xf = x + (long long)f * C * H * W;
    for (int e = lane; e < d; e += 32) {
      const int ch = e / PP, dr = (e / P) % P, dc = e % P;
      pv[e] = __ldg(xf + ((long long)ch * H + kr + dr) * W + kc + dc);
      pk[e] = keyv[((long long)f * Npad + k) * d + e];
    }
    __syncwarp();
    float kreg[DM];
#pragma unroll
    for (int e = 0; e < DM; ++e) kreg[e] = e < d ? pk[e] : 0.f;
    // the FP32 score sc = ||q'||^2 - 2 <p', q> is the squared distance of the mean-shifted
    // patches minus c_k = ||p'||^2 + 2 mu sum(p'); a position can only hold one of the key's K'
    // smallest BF16 scores if its distance is at most tau plus the BF16 error of that score,
    // |s~ - d| <= 2 sqrt(d) delta + delta^2 + 2.02e-6 (||p'||^2 + ||q'||^2), delta = 2^-9 S,
    // S = ||p'|| + ||q'|| (BF16 rounds within 2^-9 per value; the last term is the FP32
    // accumulation of the scan), so only positions within that bound (and a margin for the
    // FP32 rounding of the score here) enter the list
    float pn2 = 0.f, psum = 0.f;
#pragma unroll
    for (int e = 0; e < DM; ++e) {
      pn2 = fmaf(kreg[e], kreg[e], pn2);
      psum += kreg[e];
    }
    const float pn = sqrtf(pn2);
    const float c_k = pn2 + 2.f * mean[f] * psum;
    // 1. the bound and the candidate chunks (k_tau_chunk); a key with more candidates than the
    //    list holds scans its chunk minima here
    const long long row = (long long)f * Npad + k;
    const uint32_t tau16 = tau16s[row];
    const int ctot = ccount[row];
    const bool listed = ctot <= CT_CL;
    const uint16_t* mk = mins16 + row * nchunks;
    const float* qf = qn + (long long)f * npos;
    const float tau_f = tau16 < 0xff80u ? float_from_order_key((tau16 << 16) | 0xffffu) : INFINITY;
    const float inv_wq = 1.f / (float)Wq;
    // 2. candidate chunks, scored in groups of four
    int cnt = 0, scan = 0;
    unsigned long long kth = ~0ull;
    for (;;) {
      const uint32_t* ids;
      int ncl = 0;
      if (listed) {
        for (int i = lane; i < ctot; i += 32) clist[i] = clist_g[row * CT_CL + i];
        __syncwarp();
        ids = clist;
        ncl = ctot;
      } else {
        while (scan < nchunks && ncl < CT_CCAP - 32) {
          const int c = scan + lane;
          const bool cand = c < nchunks && (uint32_t)__ldg(mk + c) <= tau16;
          const unsigned m = __ballot_sync(0xffffffffu, cand);
          if (cand) clist[ncl + __popc(m & ltm)] = (uint32_t)c;
          ncl += __popc(m);
          scan += 32;
        }
        __syncwarp();
        ids = clist;
      }
      for (int i0 = 0; i0 < ncl; i0 += 4) {
        // the four chunks of this group; slot g of the warp scores chunk i0 + g.  Positions fit
        // in 24 bits, so the row of a position id comes from a float reciprocal plus one fix-up.
        const int cid = i0 + g < ncl ? (int)ids[i0 + g] : -1;
        const int q0c = 32 * max(cid, 0);
        int ra = (int)((float)q0c * inv_wq);
        int ca = q0c - ra * Wq;
        if (ca < 0) { --ra; ca += Wq; } else if (ca >= Wq) { ++ra; ca -= Wq; }
        const bool simple = cid >= 0 && q0c < npos && ca + 31 < Wq;
        // stage the strips of the slots' chunks: row by row, lanes along the row (coalesced)
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
          const int rs = __shfl_sync(0xffffffffu, ra, 8 * s4), cs = __shfl_sync(0xffffffffu, ca, 8 * s4);
          if (__shfl_sync(0xffffffffu, (int)simple, 8 * s4)) {
            const float* src = xf + (long long)rs * W + cs;
            float* dst = strip + s4 * CP * CT_SROW;
#pragma unroll
            for (int row = 0; row < CP; ++row) {
              if (row < C * P) {
                const int ch = row / P, dr = row - (row / P) * P;
                const float* sr = src + ((long long)ch * H + dr) * W;
                dst[row * CT_SROW + lane] = __ldg(sr + lane);
                if (lane < SW - 32) dst[row * CT_SROW + 32 + lane] = __ldg(sr + 32 + lane);
              }
            }
          }
        }
        __syncwarp();
        const int q0 = q0c + 4 * l8;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (simple) {
#pragma unroll
          for (int ch = 0; ch < CMAX; ++ch) {
            if (ch < C) {
#pragma unroll
              for (int dr = 0; dr < P; ++dr) {
                const float4* srow = reinterpret_cast<const float4*>(strip + (g * CP + ch * P + dr) * CT_SROW + 4 * l8);
                float v[12];
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                  const float4 t = srow[u];
                  v[4 * u] = t.x;
                  v[4 * u + 1] = t.y;
                  v[4 * u + 2] = t.z;
                  v[4 * u + 3] = t.w;
                }
#pragma unroll
                for (int dc = 0; dc < P; ++dc)
#pragma unroll
                  for (int i = 0; i < 4; ++i) acc[i] = fmaf(kreg[(ch * P + dr) * P + dc], v[i + dc], acc[i]);
              }
            }
          }
        } else if (cid >= 0) {
          // the chunk wraps to the next row of positions (or ends the grid): position by position,
          // the key patch read back from shared memory (a short loop keeps the code small)
#pragma unroll 1
          for (int i = 0; i < 4; ++i) {
            const int q = q0 + i;
            float a = 0.f;
            if (q < npos) {
              int r = (int)((float)q * inv_wq);
              int c = q - r * Wq;
              if (c < 0) { --r; c += Wq; } else if (c >= Wq) { ++r; c -= Wq; }
#pragma unroll 1
              for (int ch = 0; ch < C; ++ch)
#pragma unroll 1
                for (int dr = 0; dr < P; ++dr) {
                  const float* xr = xf + ((long long)ch * H + r + dr) * W + c;
                  const float* kp = pk + (ch * P + dr) * P;
#pragma unroll
                  for (int dc = 0; dc < P; ++dc) a = fmaf(kp[dc], __ldg(xr + dc), a);
                }
            }
            acc[i] = a;
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const bool valid = cid >= 0 && q < npos;
          unsigned long long e = ~0ull;
          bool near = false;
          if (valid) {
            const float qq = __ldg(qf + q);
            const float sc = fmaf(-2.f, acc[i], qq);
            const float S = pn + sqrtf(qq);
            const float dl = 0.001953125f * S;  // 2^-9 (||p'|| + ||q'||)
            const float dq = sc + c_k;           // the FP32 distance
            const float thr = tau_f + fmaf(2.f * sqrtf(fmaxf(dq, 0.f)), dl, dl * dl) + 2.02e-6f * (pn2 + qq) +
                              1e-4f * (1.f + fabsf(sc) + fabsf(c_k) + qq + pn2);
            near = dq <= thr;
            e = ((unsigned long long)float_order_key(sc) << 32) | (unsigned)q;
          }
          const bool keep = valid && near && e < kth;
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (keep) list[cnt + __popc(m & ltm)] = e;
          cnt += __popc(m);
        }
        __syncwarp();
        if (cnt > CT_LCAP - 128 && cnt > Kp) cnt = warp_keep_smallest_kth(list, cnt, Kp, hist, lane, &kth);
      }
      __syncwarp();
      if (listed || scan >= nchunks) break;
    }
    if (cnt > Kp) cnt = warp_keep_smallest_kth(list, cnt, Kp, hist, lane, &kth);
    // 3. exact distances of the K' best, the K smallest written sorted
    exact_topk_finish<PT>(list, cnt, pv, xf, C, H, W, P, Wq, K, hist, lane, gk, idx, dist);
  }
}

// Learned proposal, after the embedding scan: every chunk whose 16-bit minimum is at or
// below the key's K'-th smallest (k_tau_chunk<24>; they hold the key's K' smallest scan
// scores) is scored again in FP32 from the same operand values,
//   sc = sum_j a_q,j (a_q,j + b_p,j) = ||a_p - a_q||^2 - ||a_p||^2   (the scan's score up to
//                                                                    a constant of the key),
// a running warp list keeps the K' smallest (score, id), and those K' get their exact
// distance and the K smallest are written sorted (exact_topk_finish).  One warp per key,
// four chunks per step (lane = position within each), their operand rows loaded together.
constexpr int ET_WARPS = 4;
constexpr size_t ET_WARP_BYTES = (size_t)CT_LCAP * 8 + CT_CCAP * 4 + 256 * 4 + 96 * 4;

template <bool FP8>
__device__ __forceinline__ void emb_row_values(const uint8_t* row, float (&a)[16]) {
  if constexpr (FP8) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(row));
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __half2_raw hr =
            __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((u[k] >> (16 * h)) & 0xffffu), __NV_E4M3);
        const float2 v = __half22float2(__half2(hr));
        a[4 * k + 2 * h] = v.x;
        a[4 * k + 2 * h + 1] = v.y;
      }
    }
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(row);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint4 w = __ldg(p + k);
      const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a[8 * k + 2 * t] = __uint_as_float(u[t] << 16);
        a[8 * k + 2 * t + 1] = __uint_as_float(u[t] & 0xffff0000u);
      }
    }
  }
}

template <bool FP8>
__global__ void __launch_bounds__(ET_WARPS * 32)
    k_emb_topk(const float* __restrict__ x, const int32_t* __restrict__ keys, const int32_t* __restrict__ n_found,
               const uint8_t* __restrict__ qop, const uint8_t* __restrict__ kop, const uint16_t* __restrict__ mins16,
               const uint32_t* __restrict__ tau16s, const int32_t* __restrict__ ccount,
               const uint32_t* __restrict__ clist_g, int clcap, int n_img, int C, int H, int W, int P, int N, int Npad,
               long long npos_pad, int nchunks, int K, int Kp, int32_t* __restrict__ idx, float* __restrict__ dist) {
  constexpr int RB = FP8 ? 32 : 64;  // operand row bytes
  extern __shared__ unsigned long long et_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* wbase = reinterpret_cast<uint8_t*>(et_smem) + (size_t)wid * ET_WARP_BYTES;
  unsigned long long* list = reinterpret_cast<unsigned long long*>(wbase);
  uint32_t* clist = reinterpret_cast<uint32_t*>(wbase + CT_LCAP * 8);
  unsigned* hist = reinterpret_cast<unsigned*>(wbase + CT_LCAP * 8 + CT_CCAP * 4);
  float* pv = reinterpret_cast<float*>(wbase + CT_LCAP * 8 + CT_CCAP * 4 + 256 * 4);  // raw key patch
  const int d = C * P * P;
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const unsigned ltm = (1u << lane) - 1u;
  const long long nkeys = (long long)n_img * N;
  for (long long gk = blockIdx.x * (long long)ET_WARPS + wid; gk < nkeys; gk += (long long)gridDim.x * ET_WARPS) {
    const int f = (int)(gk / N), k = (int)(gk - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    const int kq = keys[gk];
    if ((unsigned)kq >= (unsigned)npos) continue;  // flagged by k_key_vectors
    const int kr = kq / Wq, kc = kq - (kq / Wq) * Wq;
    const float* xf = x + (long long)f * C * H * W;
    for (int e = lane; e < d; e += 32) {
      const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
      pv[e] = __ldg(xf + ((long long)ch * H + kr + dr) * W + kc + dc);
    }
    const long long row = (long long)f * Npad + k;
    float b[16];
    emb_row_values<FP8>(kop + row * RB, b);
    const uint32_t tau16 = tau16s[row];
    const int ctot = ccount[row];
    const bool listed = ctot <= clcap;
    const uint16_t* mk = mins16 + row * nchunks;
    const uint8_t* qf = qop + (long long)f * npos_pad * RB;
    int cnt = 0, scan = 0;
    unsigned long long kth = ~0ull;
    for (;;) {
      int ncl = 0;
      if (listed) {
        for (int i = lane; i < ctot; i += 32) clist[i] = clist_g[row * clcap + i];
        ncl = ctot;
      } else {
        // more candidates than the list holds: gather them from the minima, a batch at a time
        while (scan < nchunks && ncl < CT_CCAP - 32) {
          const int c = scan + lane;
          const bool cand = c < nchunks && (uint32_t)__ldg(mk + c) <= tau16;
          const unsigned m = __ballot_sync(0xffffffffu, cand);
          if (cand) clist[ncl + __popc(m & ltm)] = (uint32_t)c;
          ncl += __popc(m);
          scan += 32;
        }
      }
      __syncwarp();
      for (int i0 = 0; i0 < ncl; i0 += 4) {
        float a[4][16];
        int q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int cid = i0 + u < ncl ? (int)clist[i0 + u] : -1;
          q[u] = cid >= 0 && 32LL * cid + lane < npos ? 32 * cid + lane : -1;
          if (q[u] >= 0) {
            emb_row_values<FP8>(qf + (long long)q[u] * RB, a[u]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) a[u][j] = 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float sc = 0.f;
#pragma unroll
          for (int j = 0; j < 16; ++j) sc = fmaf(a[u][j], a[u][j] + b[j], sc);
          const unsigned long long e =
              q[u] >= 0 ? (((unsigned long long)float_order_key(sc) << 32) | (unsigned)q[u]) : ~0ull;
          const bool keep = e < kth;
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (keep) list[cnt + __popc(m & ltm)] = e;
          cnt += __popc(m);
        }
        __syncwarp();
        if (cnt > CT_LCAP - 128 && cnt > Kp) cnt = warp_keep_smallest_kth(list, cnt, Kp, hist, lane, &kth);
      }
      __syncwarp();
      if (listed || scan >= nchunks) break;
    }
    if (cnt > Kp) cnt = warp_keep_smallest_kth(list, cnt, Kp, hist, lane, &kth);
    exact_topk_finish<0>(list, cnt, pv, xf, C, H, W, P, Wq, K, hist, lane, gk, idx, dist);
  }
}

}  // namespace

int image_mean_slices(const glr_images& im) {
  const long long n = (long long)im.C * im.H * im.W;
  long long S = ceil_div(2LL * num_sms(), (long long)im.n_img);
  S = std::min<long long>(S, ceil_div(n, 4096));
  return (int)std::max<long long>(1, std::min<long long>(S, kMeanMaxSlices));
}

glr_status launch_image_mean(const float* x, const glr_images& im, float* mean, double* part, cudaStream_t s,
                             ImgMap imap) {
  const long long n = (long long)im.C * im.H * im.W;
  const int S = image_mean_slices(im);
  GLR_LAUNCH("k_image_mean", s, k_image_mean_part<<<(unsigned)(im.n_img * S), 512, 0, s>>>(x, n, S, part, imap));
  GLR_LAUNCH("k_image_mean_final", s,
             k_image_mean_final<<<(unsigned)ceil_div(im.n_img, 128), 128, 0, s>>>(part, im.n_img, S, n, mean));
  return GLR_OK;
}

glr_status launch_key_vectors(const float* x, const float* mean, const int32_t* keys, const int32_t* n_found,
                              const glr_images& im, int N, int Npad, float* keyv, StatusBlock* st, ImgMap imap,
                              cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  const long long total = (long long)im.n_img * Npad * d;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
  GLR_LAUNCH("k_key_vectors", s, k_key_vectors<<<blocks, 256, 0, s>>>(x, mean, keys, n_found, im.n_img, im.C, im.H,
                                                                       im.W, im.P, N, Npad, keyv, st, imap));
  return GLR_OK;
}

glr_status launch_rerank_streams(const float* x, const int32_t* keys, const int32_t* n_found, const glr_images& im,
                                 int N, int Npad, int K, int streams_per_key, int cap, int Kp, int finish,
                                 const uint2* bufs, const int* bufcnt, int32_t* idx, float* dist, ImgMap imap,
                                 cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  int pow2 = 32;
  while (pow2 < streams_per_key * (finish ? Kp : cap + 32)) pow2 <<= 1;
  const int dpad = (d + 31) & ~31;
  const size_t smem = (size_t)RR_WARPS * pow2 * 8 + (size_t)RR_WARPS * (dpad + 256) * 4;
  if (smem > 227 * 1024 || d > 640) return GLR_ENOTSUP;
  if (cudaFuncSetAttribute(k_rerank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GLR_ECUDA;
  const long long nkeys = (long long)im.n_img * N;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, RR_WARPS), (long long)num_sms() * 16));
  GLR_LAUNCH("k_rerank", s, k_rerank<<<blocks, RR_WARPS * 32, smem, s>>>(x, keys, n_found, im.n_img, im.C, im.H, im.W,
                                                                          im.P, N, Npad, K, streams_per_key, cap + 32,
                                                                          Kp, pow2, bufs, bufcnt, 0, 1.f, 0, idx, dist,
                                                                          imap));
  return GLR_OK;
}

// Learned proposal after the embedding scan (bound_pass 2): the bound and candidate chunks of
// every key, then their FP32 embedding scores, the exact distances of the K' best and the K
// best written.
glr_status launch_emb_topk(const float* x, const glr_images& im, const int32_t* keys, const int32_t* n_found, int N,
                           const MatchPlan& pl, char* ws, int32_t* idx, float* dist, cudaStream_t s) {
  const long long nkeys = (long long)im.n_img * N;
  const int nchunks = 8 * pl.pos_tiles;
  const uint16_t* mins16 = reinterpret_cast<const uint16_t*>(ws + pl.mins_off);
  uint32_t* tau16s = reinterpret_cast<uint32_t*>(ws + pl.taugl_off);
  int32_t* ccount = reinterpret_cast<int32_t*>(ws + pl.ccnt_off);
  uint32_t* clist_g = reinterpret_cast<uint32_t*>(ws + pl.clist_off);
  {
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, 8), (long long)num_sms() * 16));
    GLR_LAUNCH("k_tau_chunk", s, k_tau_chunk<24><<<blocks, 256, 0, s>>>(mins16, n_found, im.n_img, N, pl.Npad,
                                                                         nchunks, pl.Kp, CT_CL_EMB, tau16s, ccount,
                                                                         clist_g, reinterpret_cast<StatusBlock*>(ws)));
  }
  const size_t smem = (size_t)ET_WARPS * ET_WARP_BYTES;
  auto kern = pl.emb_fmt == 1 ? k_emb_topk<true> : k_emb_topk<false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GLR_ECUDA;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, ET_WARPS), (long long)num_sms() * 8));
  GLR_LAUNCH("k_emb_topk", s,
             kern<<<blocks, ET_WARPS * 32, smem, s>>>(x, keys, n_found, reinterpret_cast<const uint8_t*>(ws + pl.embq_off),
                                                      reinterpret_cast<const uint8_t*>(ws + pl.embk_off), mins16, tau16s,
                                                      ccount, clist_g, CT_CL_EMB, im.n_img, im.C, im.H, im.W, im.P, N,
                                                      pl.Npad, pl.npos_pad, nchunks, pl.K, pl.Kp, idx, dist));
  return GLR_OK;
}

// Exact evaluation of the candidate chunks (bound_pass 2).
glr_status launch_chunk_topk(const float* x, const glr_images& im, const int32_t* keys, const int32_t* n_found,
                             int N, const MatchPlan& pl, const float* mean, const float* qn, const float* keyv,
                             const uint16_t* mins16, char* ws, int32_t* idx, float* dist, cudaStream_t s) {
  const long long nkeys = (long long)im.n_img * N;
  const int nchunks = 8 * pl.pos_tiles;
  uint32_t* tau16s = reinterpret_cast<uint32_t*>(ws + pl.taugl_off);
  int32_t* ccount = reinterpret_cast<int32_t*>(ws + pl.ccnt_off);
  uint32_t* clist_g = reinterpret_cast<uint32_t*>(ws + pl.clist_off);
  int* ticket = reinterpret_cast<int*>(ws + pl.ticket_off);
  {
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, 8), (long long)num_sms() * 16));
    GLR_LAUNCH("k_tau_chunk", s, k_tau_chunk<8><<<blocks, 256, 0, s>>>(mins16, n_found, im.n_img, N, pl.Npad,
                                                                        nchunks, pl.Kp, CT_CL, tau16s, ccount, clist_g,
                                                                        reinterpret_cast<StatusBlock*>(ws), ticket));
  }
#define GLR_CHUNK_CASE(PP, CM)                                                                                  \
  {                                                                                                             \
    const size_t smem = (size_t)CT_WARPS * chunk_topk_warp_bytes<PP, CM>();                                     \
    if (cudaFuncSetAttribute(k_chunk_topk<PP, CM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=    \
        cudaSuccess)                                                                                            \
      return GLR_ECUDA;                                                                                         \
    int per_sm = 0; /* resident CTAs: every warp of the grid is on an SM at once */                            \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chunk_topk<PP, CM>, CT_WARPS * 32, smem) !=    \
        cudaSuccess)                                                                                            \
      return GLR_ECUDA;                                                                                         \
    const int blocks =                                                                                          \
        (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, CT_WARPS), (long long)num_sms() * std::max(per_sm, 1))); \
    GLR_LAUNCH("k_chunk_topk", s,                                                                               \
               (k_chunk_topk<PP, CM><<<blocks, CT_WARPS * 32, smem, s>>>(x, mean, qn, keyv, keys, n_found, mins16, \
                                                                        tau16s, ccount, clist_g, im.n_img, im.C, \
                                                                        im.H, im.W, N, pl.Npad, nchunks, pl.K,   \
                                                                        pl.Kp, idx, dist, ticket)));             \
  }
  if (im.P == 8 && im.C == 1) GLR_CHUNK_CASE(8, 1)
  else if (im.P == 6 && im.C <= 2) GLR_CHUNK_CASE(6, 2)
  else if (im.P == 4 && im.C <= 4) GLR_CHUNK_CASE(4, 4)
  else return GLR_ENOTSUP;
#undef GLR_CHUNK_CASE
  return GLR_OK;
}

MatchPlan match_plan(const glr_images& im, int N, int K, const glr_match_opts* o) {
  MatchPlan pl{};
  pl.mode = o ? o->mode : GLR_MATCH_FP32;
  pl.K = K;
  const bool edge = pl.mode == GLR_MATCH_EDGE;
  const bool tc = pl.mode == GLR_MATCH_BF16 || pl.mode == GLR_MATCH_LEARNED || edge;
  pl.edge_th = (o && edge) ? o->edge_th : 0.f;
  pl.window = (o && pl.mode == GLR_MATCH_WINDOW) ? o->window : 0;
  pl.Kp = (o && o->k_over > 0) ? o->k_over : (pl.mode == GLR_MATCH_LEARNED ? std::max(256, K + 16) : K + 16);
  pl.Kp = std::max(pl.Kp, K);
  // a small compaction trigger publishes a first threshold early; each compaction keeps ~Kp + (cap - Kp) / 4
  pl.cap = (o && o->cap > 0) ? o->cap : std::min(std::max(2 * pl.Kp + 64, 256), kStreamMaxEntries - 32);
  pl.cap = (int)(pl.cap / 32) * 32;
  pl.subs = 2;
  pl.epi_batch = (o && o->epi_batch == 4) ? 4 : 2;  // 2 chunks per visit: no register spills
  pl.key_tile = FT;
  pl.Npad = (int)(ceil_div(N, FT) * FT);
  const int Hq = im.H - im.P + 1, Wq = im.W - im.P + 1;
  const int ktiles = pl.Npad / FT;
  if (tc) {
    pl.pos_tile = 256;
    pl.pos_tiles = (int)ceil_div((long long)Hq * Wq, pl.pos_tile);
  } else {
    pl.pos_tile = FT;
    pl.pos_tiles = Hq * (int)ceil_div(Wq, FT);
  }
  // fewer splits mean fewer streams per key (less re-rank work and threshold learning):
  // split the positions only when key tiles alone would leave SMs idle
  int splits = (o && o->splits > 0) ? o->splits : (int)ceil_div((long long)num_sms(), (long long)ktiles * im.n_img);
  // the exact re-rank holds every stream's candidates of one key in shared memory
  const int max_splits = std::max(1, kRerankMaxList / (pl.subs * pl.Kp));
  splits = std::max(1, std::min({splits, pl.pos_tiles, max_splits}));
  pl.tiles_per_split = (int)ceil_div(pl.pos_tiles, splits);
  pl.splits = (int)ceil_div(pl.pos_tiles, pl.tiles_per_split);
  pl.streams_per_key = pl.splits * pl.subs;
  // the re-rank keeps the K' best stream entries of a key itself; when every buffer
  // fits its list unreduced, the streams skip their own final exact selection
  pl.finish = (long long)pl.streams_per_key * (pl.cap + 32) <= kRerankMaxList ? 0 : 1;
  // the heat map of Eq. 4 contracts the 4 C binary edge planes instead of the image
  const int d = (edge ? 4 : 1) * im.C * im.P * im.P;
  const long long npos = (long long)Hq * Wq;
  WsLayout L;
  pl.mean_off = L.take((size_t)im.n_img * 4);
  pl.meanp_off = L.take((size_t)im.n_img * kMeanMaxSlices * 8);
  pl.qn_off = L.take((size_t)im.n_img * npos * 4);
  pl.keyv_off = L.take((size_t)im.n_img * pl.Npad * d * 4);
  // chunk-minima scan + exact evaluation of the candidate chunks (bound_pass 2): BF16 mode,
  // one 64-column chunk per operand row, a patch side the evaluation kernel is compiled for
  const int bp = o ? o->bound_pass : 0;
  const bool chunk_ok = pl.mode == GLR_MATCH_BF16 && d <= 74 && (im.P == 4 || im.P == 6 || im.P == 8) &&
                        im.C * im.P <= 16 && npos < (1LL << 24) - 64;  // position ids exact in FP32
  // the learned proposal's embedding scan takes the same chunk-minima form (bound_pass 2)
  const bool emb_chunk = pl.mode == GLR_MATCH_LEARNED && (bp == 2 || bp == 0) && npos < (1LL << 24) - 64;
  const bool chunk = (chunk_ok && (bp == 2 || bp == 0)) || emb_chunk;
  const long long nstreams = chunk ? 0 : (long long)im.n_img * pl.Npad * pl.streams_per_key;
  pl.buf_off = L.take((size_t)nstreams * (pl.cap + 32) * 8);
  pl.bufcnt_off = L.take((size_t)nstreams * 4);
  pl.taugl_off = L.take((size_t)im.n_img * pl.Npad * 4);
  if (tc) {
    // BF16 operands: positions [img][npos_pad][dk] and keys [img][Npad][dk]: 80 columns
    // (patch values and norm terms) for d <= 74; for wider patches nkc chunks of 64
    // patch columns, then 16 norm columns
    const int dmat = pl.mode == GLR_MATCH_LEARNED ? 16 : d;
    pl.nkc = dmat > 74 ? (int)ceil_div(dmat, 64) : 1;
    const int dk = 64 * pl.nkc + 16;
    pl.dk = dk;
    pl.npos_pad = (long long)pl.pos_tiles * pl.pos_tile;
    if (!emb_chunk) {
      pl.qpack_off = L.take((size_t)im.n_img * pl.npos_pad * dk * 2);
      pl.kpack_off = L.take((size_t)im.n_img * pl.Npad * dk * 2);
    }
    // the bound of the minima scan needs Kp half tiles.  Automatic: on for one-chunk
    // rows, where the candidate appends cost more than a second contraction; off for
    // chunked rows (d > 74), where the contraction itself dominates
    if (chunk) {
      pl.bound_pass = 2;  // 16-bit minima of every 32-position chunk
      pl.mins_off = L.take((size_t)im.n_img * pl.Npad * 8 * pl.pos_tiles * 2);
      pl.ccnt_off = L.take((size_t)im.n_img * pl.Npad * 4);
      pl.ticket_off = L.take(4);
      pl.clist_off = L.take((size_t)im.n_img * pl.Npad * (emb_chunk ? CT_CL_EMB : CT_CL) * 4);
    } else {
      pl.bound_pass = ((bp == 1 || ((bp == 0 || bp == 2) && pl.nkc == 1)) && 2LL * pl.pos_tiles >= pl.Kp) ? 1 : 0;
      if (pl.bound_pass) pl.mins_off = L.take((size_t)im.n_img * pl.Npad * 2 * pl.pos_tiles * 4);
    }
  }
  if (edge) pl.edge_off = L.take((size_t)im.n_img * 4 * im.C * im.H * im.W * 4);
  if (pl.mode == GLR_MATCH_LEARNED) {
    pl.embp_off = L.take((size_t)im.n_img * npos * 16 * 4);  // FP32 embeddings of every position
    if (emb_chunk) {
      pl.emb_fmt = (o && o->emb_format == 1) ? 1 : 0;
      const size_t rb = pl.emb_fmt == 1 ? 32 : 64;  // operand row bytes
      pl.n2_off = L.take(4);
      pl.embq_off = L.take((size_t)im.n_img * pl.npos_pad * rb);
      pl.embk_off = L.take((size_t)im.n_img * pl.Npad * rb);
    } else {
      pl.embk_off = L.take((size_t)im.n_img * pl.Npad * 16 * 4);
    }
  }
  pl.total = L.off;
  return pl;
}

glr_status launch_match(const float* x, const glr_images& im, const int32_t* keys, const int32_t* n_found, int N,
                        const MatchPlan& pl, const float* encoder, int32_t* idx, float* dist, char* ws,
                        cudaStream_t s) {
  const int Hq = im.H - im.P + 1, Wq = im.W - im.P + 1;
  const long long npos = (long long)Hq * Wq;
  const bool edge = pl.mode == GLR_MATCH_EDGE;
  const bool tc = pl.mode == GLR_MATCH_BF16 || pl.mode == GLR_MATCH_LEARNED || edge;
  if (pl.window > 0) {
    // block matching in a local window: every candidate is scored exactly by the re-rank kernel
    const int d0 = im.C * im.P * im.P;
    const int dpad = (d0 + 31) & ~31;
    int pow2 = 32;
    const int nwin = (2 * pl.window + 1) * (2 * pl.window + 1);
    while (pow2 < nwin) pow2 <<= 1;
    const size_t smem = (size_t)RR_WARPS * pow2 * 8 + (size_t)RR_WARPS * (dpad + 256) * 4;
    if (smem > 227 * 1024 || pow2 > kRerankMaxList) return GLR_ENOTSUP;
    if (cudaFuncSetAttribute(k_rerank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GLR_ECUDA;
    const long long nkeys = (long long)im.n_img * N;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, RR_WARPS), (long long)num_sms() * 16));
    GLR_LAUNCH("k_rerank", s, k_rerank<<<blocks, RR_WARPS * 32, smem, s>>>(x, keys, n_found, im.n_img, im.C, im.H, im.W, im.P, N, pl.Npad,
                                                 pl.K, 0, 0, 0, pow2, nullptr, nullptr, 0, 1.f, pl.window, idx, dist,
                                                 ImgMap{}));
    return GLR_OK;
  }
  // GLR_MATCH_EDGE: every later step sees the 4 C binary edge planes as the image
  glr_images ime = im;
  if (edge) ime.C = 4 * im.C;
  const int d = ime.C * im.P * im.P;
  float* mean = reinterpret_cast<float*>(ws + pl.mean_off);
  float* qn = reinterpret_cast<float*>(ws + pl.qn_off);
  float* keyv = reinterpret_cast<float*>(ws + pl.keyv_off);
  uint2* bufs = reinterpret_cast<uint2*>(ws + pl.buf_off);
  int* bufcnt = reinterpret_cast<int*>(ws + pl.bufcnt_off);
  const long long HW = (long long)im.H * im.W;
  uint32_t* taugl = reinterpret_cast<uint32_t*>(ws + pl.taugl_off);
  if (cudaMemsetAsync(taugl, 0xff, (size_t)im.n_img * pl.Npad * 4, s) != cudaSuccess) return GLR_ECUDA;
  (void)HW;
  const float* xs = x;
  if (edge) {
    // binary edge planes, no mean shift (the correlation is not shift-invariant)
    float* planes = reinterpret_cast<float*>(ws + pl.edge_off);
    glr_status st = launch_edge_planes(x, im, pl.edge_th, planes, s);
    if (st != GLR_OK) return st;
    xs = planes;
    if (cudaMemsetAsync(mean, 0, (size_t)im.n_img * 4, s) != cudaSuccess) return GLR_ECUDA;
  } else {
    const glr_status st = launch_image_mean(x, im, mean, reinterpret_cast<double*>(ws + pl.meanp_off), s);
    if (st != GLR_OK) return st;
  }
  // the FP32 scorers add ||q||^2 themselves; the tensor-core operands carry theirs
  if (!tc || (pl.bound_pass == 2 && pl.mode != GLR_MATCH_LEARNED)) {
    const long long total = (long long)im.n_img * npos;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
    GLR_LAUNCH("k_patch_norms", s, k_patch_norms<<<blocks, 256, 0, s>>>(x, mean, im.n_img, im.C, im.H, im.W, im.P, qn));
  }
  {
    const long long total = (long long)im.n_img * pl.Npad * d;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
    GLR_LAUNCH("k_key_vectors", s, k_key_vectors<<<blocks, 256, 0, s>>>(xs, mean, keys, n_found, im.n_img, ime.C, im.H, im.W, im.P, N, pl.Npad,
                                        keyv, reinterpret_cast<StatusBlock*>(ws), ImgMap{}));
  }
  StreamCfg cfg{pl.cap, pl.Kp, pl.finish};
  if (pl.mode == GLR_MATCH_LEARNED) {
    float* emb_p = reinterpret_cast<float*>(ws + pl.embp_off);
    const bool emb_chunk = pl.bound_pass == 2;
    glr_status st = launch_encode_positions(x, im, mean, encoder, emb_p,
                                            emb_chunk ? reinterpret_cast<unsigned*>(ws + pl.n2_off) : nullptr,
                                            reinterpret_cast<StatusBlock*>(ws), s);
    if (st != GLR_OK) return st;
    if (emb_chunk) {
      st = launch_match_emb(im, keys, n_found, N, pl, ws, g_tc_dump, s);
      if (st != GLR_OK) return st;
      return launch_emb_topk(x, im, keys, n_found, N, pl, ws, idx, dist, s);
    }
    float* emb_k = reinterpret_cast<float*>(ws + pl.embk_off);
    st = launch_encode_vectors(keyv, (long long)im.n_img * pl.Npad, d, encoder, emb_k, s);
    if (st != GLR_OK) return st;
  }
  if (tc) {
    const glr_status st = launch_match_tc(xs, ime, keys, n_found, N, pl, ws, s);
    if (st != GLR_OK) return st;
    if (pl.bound_pass == 2)
      return launch_chunk_topk(x, im, keys, n_found, N, pl, mean, qn, keyv,
                               reinterpret_cast<const uint16_t*>(ws + pl.mins_off), ws, idx, dist, s);
  } else {
    // channels per chunk: all of them if the transposed key tile fits, else as many as fit
    auto fp32_smem = [&](int cc) {
      return (size_t)(cc * im.P * im.P * FT + cc * im.P * (FT + 8) + FT * SC_LD + FT) * 4 + 8 * 256 * 4 + FT * 4;
    };
    int cc = im.C;
    while (cc > 1 && fp32_smem(cc) > 227 * 1024) --cc;
    const size_t smem = fp32_smem(cc);
    if (smem > 227 * 1024) return GLR_ENOTSUP;
    dim3 grid((unsigned)(pl.Npad / FT), (unsigned)im.n_img, (unsigned)pl.splits);
#define GLR_FP32_CASE(PP)                                                                                    \
  case PP: {                                                                                                 \
    if (cudaFuncSetAttribute(k_match_fp32<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=     \
        cudaSuccess)                                                                                         \
      return GLR_ECUDA;                                                                                      \
    GLR_LAUNCH("k_match_fp32", s,                                                                           \
               k_match_fp32<PP><<<grid, 256, smem, s>>>(x, mean, qn, keyv, n_found, im.C, im.H, im.W, pl.Npad,  \
                                                        pl.splits, pl.tiles_per_split, cc, cfg, bufs, bufcnt, taugl, \
                                                        reinterpret_cast<StatusBlock*>(ws)));                      \
  } break;
    switch (im.P) {
      GLR_FP32_CASE(2)
      GLR_FP32_CASE(3)
      GLR_FP32_CASE(4)
      GLR_FP32_CASE(5)
      GLR_FP32_CASE(6)
      GLR_FP32_CASE(7)
      GLR_FP32_CASE(8)
      default:
        return GLR_ENOTSUP;
    }
#undef GLR_FP32_CASE
  }
  {
    int pow2 = 32;
    while (pow2 < pl.streams_per_key * (pl.finish ? pl.Kp : pl.cap + 32)) pow2 <<= 1;
    const int dpad = (d + 31) & ~31;
    const size_t smem = (size_t)RR_WARPS * pow2 * 8 + (size_t)RR_WARPS * (dpad + 256) * 4;
    if (smem > 227 * 1024 || d > 640) return GLR_ENOTSUP;
    if (cudaFuncSetAttribute(k_rerank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GLR_ECUDA;
    const long long nkeys = (long long)im.n_img * N;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, RR_WARPS), (long long)num_sms() * 16));
    GLR_LAUNCH("k_rerank", s, k_rerank<<<blocks, RR_WARPS * 32, smem, s>>>(x, keys, n_found, im.n_img, im.C, im.H, im.W, im.P, N, pl.Npad,
                                                 pl.K, pl.streams_per_key, pl.cap + 32, pl.Kp, pow2, bufs, bufcnt,
                                                 edge ? 1 : 0, edge ? -0.5f : 1.f, 0, idx, dist, ImgMap{}));
  }
  return GLR_OK;
}

}  // namespace glr
