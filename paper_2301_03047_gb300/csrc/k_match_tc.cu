// BF16 tensor-core scorer for glr_match_topk: the heat map of Eq. 4 evaluated
// as a dense contraction on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory), operands staged by TMA, fused with the
// running per-key top-K' of topk_stream.cuh so no score reaches HBM.
//
// Operands (packed once per call by k_pack_keys / k_pack_positions), 80 BF16
// columns per row, the first 64 in a 128-byte swizzled tile, the last 16 in a
// 32-byte swizzled tile:
//   A (keys)      row = [-2 p~ (d values) | 1 1 1 pn_hi pn_mid pn_lo | 0..]
//   B (positions) row = [   q~ (d values) | qn_hi qn_mid qn_lo 1 1 1 | 0..]
// with the six norm columns starting at column max(d, 64), so d <= 74.
// where p~, q~ are the mean-shifted patches rounded to BF16 and pn, qn their
// squared norms computed in FP32 from the rounded values, split into three
// BF16 terms.  One 128 x 256 x 80 product therefore gives, per key/position,
// ||p~||^2 + ||q~||^2 - 2<p~,q~> = ||p~ - q~||^2 up to FP32 accumulation:
// the exact distance of the BF16-rounded patches.  Candidates are re-ranked
// with the exact FP32 distance afterwards (k_rerank).
//
// CTA = 128 keys x one split of the positions, 320 threads:
//   warp 0      TMA producer (one thread): key tile once, then position tiles
//               into a 4-stage ring (SW128 for the 64 patch columns, SW32 for
//               the 16 norm columns)
//   warp 1      TMEM allocator (512 columns = two 128x256 FP32 accumulators)
//               and MMA issuer (one thread): 4 x K16 + 1 x K16 per tile
//   warps 2-9   epilogue: tcgen05.ld 32 lanes x 32 columns, push into the
//               per-row top-K' stream; warps w and w+4 share a TMEM lane
//               quadrant and take one column half each
// Two scans of the same contraction (bound_pass): k_match_tc<4, W, true> keeps no
// candidate and writes the minimum score of every (key, 128-position half tile);
// k_tau_bound turns the K'-th smallest of a key's minima into its starting bound;
// k_match_tc<EB, W, false> then pushes only scores below that bound into the
// streams.  Chunked rows (d > 74, W = true) stream key and position chunks
// through a 4-stage ring and append from registers (no shared tile).
// Every mbarrier wait is bounded (1 s of %globaltimer): on expiry the CTA sets
// GLR_DEV_TIMEOUT and an abort flag, every role leaves its loop, in-flight TMA
// loads and MMAs are waited for (bounded) and TMEM is freed before exit.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "glr_kernels.cuh"
#include "tc_ptx.cuh"
#include "topk_stream.cuh"

namespace glr {

namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 256;
constexpr int TC_STAGES = 4;
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 64 + TC_EPI_WARPS * 32;
constexpr int DK_MAIN = 64;  // patch columns (bf16), one 128-byte swizzle row
constexpr int DK_AUX = 16;   // norm columns (bf16), one 32-byte swizzle row
constexpr uint32_t A_MAIN_BYTES = TC_M * DK_MAIN * 2;  // 16384
constexpr uint32_t A_AUX_BYTES = TC_M * DK_AUX * 2;    // 4096
constexpr uint32_t B_MAIN_BYTES = TC_N * DK_MAIN * 2;  // 32768
constexpr uint32_t B_AUX_BYTES = TC_N * DK_AUX * 2;    // 8192
constexpr uint32_t OFF_A_MAIN = 0;
constexpr uint32_t OFF_A_AUX = OFF_A_MAIN + A_MAIN_BYTES;
constexpr uint32_t OFF_B_MAIN = OFF_A_AUX + A_AUX_BYTES;
constexpr uint32_t OFF_B_AUX = OFF_B_MAIN + TC_STAGES * B_MAIN_BYTES;
constexpr uint32_t OFF_BAR = OFF_B_AUX + TC_STAGES * B_AUX_BYTES;  // 8-byte barriers
constexpr int NBAR = 2 * TC_STAGES + 4 + 2;                        // full, empty, tmem_full x2, tmem_empty x2, a_full, mma_done
constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;                  // tmem base, abort flag
constexpr uint32_t OFF_HIST = (OFF_MISC + 64 + 15) / 16 * 16;
// per-warp 32 x 32 score tile for the row-wise append: rows written as eight 16-byte
// stores (a stride of 36 words keeps each quarter-warp phase on distinct banks), read
// one row per instruction
constexpr int TILE_LD = 36;
constexpr uint32_t OFF_TILE = OFF_HIST + TC_EPI_WARPS * 256 * 4;
constexpr uint32_t OFF_TAU = OFF_TILE + TC_EPI_WARPS * 32 * TILE_LD * 4;  // published thresholds of the 128 rows
constexpr uint32_t TC_SMEM = OFF_TAU + TC_M * 4 + 1024;                   // + alignment slack
static_assert(TC_SMEM <= 232448, "shared memory budget");
static_assert(OFF_TILE % 16 == 0 && (TILE_LD * 4) % 16 == 0, "16-byte aligned tile rows");
// Wide operands (d > 74): the key tile no longer fits next to a position ring, so
// every 64-column chunk of keys and positions streams through a 4-stage ring of
// (A chunk, B chunk) pairs; the 16 norm columns come last as a 16-column chunk.
// The fourth stage takes the room of the append tile (appends go through
// shuffles here: the contraction of a tile is long enough to hide them).
constexpr int W_STAGES = 4;
static_assert(W_STAGES <= TC_STAGES, "barrier slots");
constexpr uint32_t W_STAGE_BYTES = A_MAIN_BYTES + B_MAIN_BYTES;  // 48 KB
constexpr uint32_t W_OFF_BAR = W_STAGES * W_STAGE_BYTES;
constexpr uint32_t W_OFF_MISC = W_OFF_BAR + NBAR * 8;
constexpr uint32_t W_OFF_HIST = (W_OFF_MISC + 64 + 15) / 16 * 16;
constexpr uint32_t W_OFF_TAU = W_OFF_HIST + TC_EPI_WARPS * 256 * 4;  // no append tile: rows go through shuffles
constexpr uint32_t W_SMEM = W_OFF_TAU + TC_M * 4 + 1024;
static_assert(W_SMEM <= 232448, "shared memory budget (wide)");
// (PTX helpers: tc_ptx.cuh)

// ------------------------------------------------------------------- kernels
__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// First norm column of the 80-column operand rows for d patch values.
__host__ __device__ constexpr int norm_col(int d) { return d > DK_MAIN ? d : DK_MAIN; }

// Positions: thread per position builds its 64 + 16 bf16; a warp stores its 32 rows as
// contiguous blocks through shared memory.
// emb != nullptr: pack the 16-value embeddings emb[img][q][16] instead of the patches.
// PT: the patch side when it is known at compile time (cheap index arithmetic), 0 = P
template <int PT>
__global__ void __launch_bounds__(256) k_pack_positions(const float* __restrict__ x, const float* __restrict__ mean,
                                                        int n_img, int C, int H, int W, int P_, long long npos_pad,
                                                        const float* __restrict__ emb, int raw,
                                                        __nv_bfloat16* __restrict__ qmain,
                                                        __nv_bfloat16* __restrict__ qaux) {
  const int P = PT ? PT : P_;
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const int d = emb != nullptr ? 16 : C * P * P;
  const int nb = norm_col(d) - DK_MAIN;  // first norm column inside the aux tile
  const long long total = (long long)n_img * npos_pad;  // a multiple of 32: whole warps per pass
  __shared__ __align__(16) __nv_bfloat16 stage[8][32][DK_MAIN + DK_AUX];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / npos_pad;
    const long long q = i - f * npos_pad;
    __align__(16) __nv_bfloat16 row[DK_MAIN + DK_AUX];
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);
#pragma unroll
    for (int e = 0; e < DK_MAIN + DK_AUX; ++e) row[e] = z;
    if (q < npos) {
      const int r = (int)(q / Wq), c = (int)(q - (q / Wq) * Wq);
      const float mu = mean[f];
      float nrm = 0.f;
#pragma unroll
      for (int e = 0; e < DK_MAIN + DK_AUX; ++e) {
        if (e < d) {
          float v;
          if (emb != nullptr) {
            v = __ldg(emb + (f * npos + q) * 16 + e);
          } else {
            const int ch = e / (P * P), dr = (e / P) % P, dc = e % P;
            v = __ldg(x + (((long long)f * C + ch) * H + r + dr) * W + c + dc) - mu;
          }
          row[e] = __float2bfloat16_rn(v);
          const float rv = __bfloat162float(row[e]);
          nrm = fmaf(rv, rv, nrm);
        }
      }
      __nv_bfloat16 h, m, l;
      split3(nrm, h, m, l);
#pragma unroll
      for (int e = 0; e < DK_AUX; ++e) {  // static register indices: select by offset
        const int t = raw ? -1 : e - nb;  // raw operands (heat map): no norm columns
        if (t == 0) row[DK_MAIN + e] = h;
        else if (t == 1) row[DK_MAIN + e] = m;
        else if (t == 2) row[DK_MAIN + e] = l;
        else if (t >= 3 && t < 6) row[DK_MAIN + e] = one;
      }
    }
    // the warp's 32 rows (consecutive positions) go through shared memory and leave as
    // two contiguous blocks (4 KB of patch columns, 1 KB of norm columns)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint4* srow = reinterpret_cast<uint4*>(stage[wid][lane]);
    const uint4* src = reinterpret_cast<const uint4*>(row);
#pragma unroll
    for (int k = 0; k < (DK_MAIN + DK_AUX) / 8; ++k) srow[k] = src[k];
    __syncwarp();
    const long long i0 = i - lane;
    uint4* dmain = reinterpret_cast<uint4*>(qmain + i0 * DK_MAIN);
#pragma unroll
    for (int t = lane; t < 32 * DK_MAIN / 8; t += 32)
      dmain[t] = reinterpret_cast<const uint4*>(stage[wid][t / (DK_MAIN / 8)])[t % (DK_MAIN / 8)];
    uint4* daux = reinterpret_cast<uint4*>(qaux + i0 * DK_AUX);
#pragma unroll
    for (int t = lane; t < 32 * DK_AUX / 8; t += 32)
      daux[t] = reinterpret_cast<const uint4*>(stage[wid][t / (DK_AUX / 8)])[DK_MAIN / 8 + t % (DK_AUX / 8)];
    __syncwarp();
  }
}

// Keys: thread per key slot of the padded key array.
__global__ void __launch_bounds__(256) k_pack_keys(const float* __restrict__ keyv, int n_keys_total, int d, int raw,
                                                   __nv_bfloat16* __restrict__ kmain,
                                                   __nv_bfloat16* __restrict__ kaux) {
  const int nb = norm_col(d) - DK_MAIN;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_keys_total; i += gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 row[DK_MAIN + DK_AUX];
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);
    float nrm = 0.f;
#pragma unroll
    for (int e = 0; e < DK_MAIN + DK_AUX; ++e) {
      row[e] = z;
      if (e < d) {
        const __nv_bfloat16 b = __float2bfloat16_rn(keyv[(long long)i * d + e]);
        const float rv = __bfloat162float(b);
        nrm = fmaf(rv, rv, nrm);
        row[e] = __float2bfloat16_rn(-2.f * rv);  // exact: scaling by -2
      }
    }
    __nv_bfloat16 h, m, l;
    split3(nrm, h, m, l);
#pragma unroll
    for (int e = 0; e < DK_AUX; ++e) {
      const int t = raw ? -1 : e - nb;
      if (t >= 0 && t < 3) row[DK_MAIN + e] = one;
      else if (t == 3) row[DK_MAIN + e] = h;
      else if (t == 4) row[DK_MAIN + e] = m;
      else if (t == 5) row[DK_MAIN + e] = l;
    }
    uint4* dst = reinterpret_cast<uint4*>(kmain + (long long)i * DK_MAIN);
    const uint4* src = reinterpret_cast<const uint4*>(row);
#pragma unroll
    for (int k = 0; k < DK_MAIN / 8; ++k) dst[k] = src[k];
    uint4* dsta = reinterpret_cast<uint4*>(kaux + (long long)i * DK_AUX);
    dsta[0] = src[DK_MAIN / 8];
    dsta[1] = src[DK_MAIN / 8 + 1];
  }
}

// Wide operands (d > 74): rows of nkc 64-column chunks of patch values, then a
// separate 16-column row of norm terms ([qn_hi qn_mid qn_lo 1 1 1] for positions,
// [1 1 1 pn_hi pn_mid pn_lo] for keys).
// 32 consecutive positions per CTA: each warp packs whole channels (lane = position,
// coalesced image reads) into rows staged in shared memory; the channel partial
// norms are added in channel order (deterministic) and the rows leave as one
// contiguous block of 16-byte stores.
constexpr int PW_POS = 32;
template <int PT>  // P at compile time (0: runtime): unrolled patch loops
__global__ void __launch_bounds__(256) k_pack_positions_w(const float* __restrict__ x, const float* __restrict__ mean,
                                                          int n_img, int C, int H, int W, int P_, long long npos_pad,
                                                          int nkc, int raw, __nv_bfloat16* __restrict__ qmain,
                                                          __nv_bfloat16* __restrict__ qaux, ImgMap imap) {
  const int P = PT ? PT : P_;
  extern __shared__ __align__(16) uint8_t pw_smem[];
  const int rowlen = nkc * DK_MAIN;  // bf16 per row
  const int ld = rowlen + 2;         // shared-memory row stride: an odd number of words (no bank conflicts)
  __nv_bfloat16* rows = reinterpret_cast<__nv_bfloat16*>(pw_smem);        // [PW_POS][ld]
  float* pnorm = reinterpret_cast<float*>(pw_smem + (size_t)PW_POS * ld * 2);  // [C][PW_POS]
  const int Hq = H - P + 1, Wq = W - P + 1;
  const long long npos = (long long)Hq * Wq;
  const int PP = P * P, d = C * PP;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long blocks_per_img = npos_pad / PW_POS;
  for (long long blk = blockIdx.x; blk < (long long)n_img * blocks_per_img; blk += gridDim.x) {
    const long long f = blk / blocks_per_img;
    const long long q0 = (blk - f * blocks_per_img) * PW_POS;
    const float mu = mean[f];
    // padding columns (e >= d) of every row
    for (int i = threadIdx.x; i < PW_POS * (rowlen - d); i += blockDim.x) {
      const int j = i / (rowlen - d), e = d + i - (i / (rowlen - d)) * (rowlen - d);
      rows[j * ld + e] = __float2bfloat16_rn(0.f);
    }
    const long long q = q0 + lane;
    const bool valid = q < npos;
    const int r = valid ? (int)(q / Wq) : 0, c = valid ? (int)(q - (q / Wq) * Wq) : 0;
    for (int ch = wid; ch < C; ch += nw) {
      const float* xc = x + imap.pix((int)f, (long long)C * H * W) + (long long)ch * H * W;
      float nrm = 0.f;
      const float* xp = xc + (long long)r * W + c;
#pragma unroll
      for (int dr = 0; dr < (PT ? PT : 1) * 0 + P; ++dr)
#pragma unroll
        for (int dc = 0; dc < P; ++dc) {
          const float v = valid ? __ldg(xp + (long long)dr * W + dc) - mu : 0.f;
          const __nv_bfloat16 b = __float2bfloat16_rn(v);
          const float rv = __bfloat162float(b);
          nrm = fmaf(rv, rv, nrm);
          rows[lane * ld + ch * PP + dr * P + dc] = b;
        }
      pnorm[ch * PW_POS + lane] = nrm;
    }
    __syncthreads();
    if (wid == 0) {
      float nrm = 0.f;
      for (int ch = 0; ch < C; ++ch) nrm += pnorm[ch * PW_POS + lane];
      __align__(16) __nv_bfloat16 aux[DK_AUX];
      const __nv_bfloat16 z = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);
#pragma unroll
      for (int e = 0; e < DK_AUX; ++e) aux[e] = z;
      if (valid && !raw) {
        split3(nrm, aux[0], aux[1], aux[2]);
        aux[3] = aux[4] = aux[5] = one;
      }
      uint4* dsta = reinterpret_cast<uint4*>(qaux + (f * npos_pad + q) * DK_AUX);
      dsta[0] = reinterpret_cast<const uint4*>(aux)[0];
      dsta[1] = reinterpret_cast<const uint4*>(aux)[1];
    }
    // the 32 rows are contiguous in the packed array (4-byte words: the staged rows are
    // padded by one word)
    const uint32_t* src = reinterpret_cast<const uint32_t*>(rows);
    uint32_t* dst = reinterpret_cast<uint32_t*>(qmain + (f * npos_pad + q0) * (long long)rowlen);
    const int wpr = rowlen / 2;
    for (int i = threadIdx.x; i < PW_POS * wpr; i += blockDim.x) {
      const int j = i / wpr;
      dst[i] = src[j * (wpr + 1) + (i - j * wpr)];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_pack_keys_w(const float* __restrict__ keyv, int n_keys_total, int d, int nkc,
                                                     int raw, __nv_bfloat16* __restrict__ kmain,
                                                     __nv_bfloat16* __restrict__ kaux) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_keys_total; i += gridDim.x * blockDim.x) {
    float nrm = 0.f;
    uint4* dst = reinterpret_cast<uint4*>(kmain + (long long)i * nkc * DK_MAIN);
    for (int kc = 0; kc < nkc; ++kc) {
      __align__(16) __nv_bfloat16 row[DK_MAIN];
#pragma unroll
      for (int j = 0; j < DK_MAIN; ++j) {
        const int e = kc * DK_MAIN + j;
        const __nv_bfloat16 b = __float2bfloat16_rn(e < d ? keyv[(long long)i * d + e] : 0.f);
        const float rv = __bfloat162float(b);
        nrm = fmaf(rv, rv, nrm);
        row[j] = __float2bfloat16_rn(-2.f * rv);  // exact: scaling by -2
      }
      const uint4* src = reinterpret_cast<const uint4*>(row);
#pragma unroll
      for (int k = 0; k < DK_MAIN / 8; ++k) dst[kc * (DK_MAIN / 8) + k] = src[k];
    }
    __align__(16) __nv_bfloat16 aux[DK_AUX];
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);
#pragma unroll
    for (int e = 0; e < DK_AUX; ++e) aux[e] = z;
    if (!raw) {
      aux[0] = aux[1] = aux[2] = one;
      split3(nrm, aux[3], aux[4], aux[5]);
    }
    uint4* dsta = reinterpret_cast<uint4*>(kaux + (long long)i * DK_AUX);
    dsta[0] = reinterpret_cast<const uint4*>(aux)[0];
    dsta[1] = reinterpret_cast<const uint4*>(aux)[1];
  }
}

// Bound from the half-tile minima: the kp-th smallest of the 2 ntiles minima of a
// key's row.  kp half tiles each hold a score no larger than it, so at least kp
// scores of the key are <= it: published (+1 in the order key, the filter is
// strict) it is a valid bound for the scan that keeps candidates.  One warp per
// key, 4-pass radix select over the order-preserving keys, stopping after the third
// pass when the kp-th minimum closes its bin (the bin's upper end is then as valid a
// bound, at most 256 ulps looser).
__global__ void __launch_bounds__(256) k_tau_bound(const float* __restrict__ mins, const int32_t* __restrict__ n_found,
                                                   int n_img, int N, int Npad, int L, int kp,
                                                   uint32_t* __restrict__ tau_gl) {
  __shared__ unsigned hist_s[8][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* hist = hist_s[wid];
  const long long nkeys = (long long)n_img * N;
  for (long long gk = blockIdx.x * 8LL + wid; gk < nkeys; gk += gridDim.x * 8LL) {
    const int f = (int)(gk / N), k = (int)(gk - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    const float* m = mins + ((long long)f * Npad + k) * L;
    uint32_t prefix = 0, pmask = 0;
    int rank = kp;
#pragma unroll 1
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
#pragma unroll
      for (int t = 0; t < 8; ++t) hist[lane * 8 + t] = 0;
      __syncwarp();
      for (int i = lane; i < L; i += 32) {
        const uint32_t kk = float_order_key(m[i]);
        if ((kk & pmask) == prefix) atomicAdd(&hist[(kk >> shift) & 255u], 1u);
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
      prefix |= (uint32_t)sel << shift;
      pmask |= 255u << shift;
      __syncwarp();
      // the kp-th minimum is the largest of its bin: at least kp minima lie at or below
      // the bin's upper end, which bounds the scan as well; stop refining once a bin
      // spans at most 2^8 order keys (the bound stays within 256 ulps)
      if (rank == in_bin && shift <= 8) {
        prefix |= (1u << shift) - 1u;
        break;
      }
    }
    // a finite kp-th minimum bounds the scan (an infinite one says nothing)
    if (lane == 0 && prefix < float_order_key(INFINITY)) atomicMin(tau_gl + (long long)f * Npad + k, prefix + 1u);
  }
}

// Seed bounds: for each key, the K'-th smallest tensor-core score over 16 x 16
// positions sampled at stride 2 around it.  That sample is a subset of the
// positions, so at least K' positions score below this value: it is a valid
// initial published bound.  The scores are recomputed here from the same
// packed BF16 operands in FP32; a margin covers the different summation order.
// One warp per key; 8 positions per lane; exact warp radix select.
constexpr int SEED_WIN = 16;    // samples per side
constexpr int SEED_STRIDE = 2;  // spacing of the samples
__global__ void __launch_bounds__(256) k_seed_bounds(const __nv_bfloat16* __restrict__ qmain,
                                                     const __nv_bfloat16* __restrict__ qaux,
                                                     const __nv_bfloat16* __restrict__ kmain,
                                                     const __nv_bfloat16* __restrict__ kaux,
                                                     const int32_t* __restrict__ keys,
                                                     const int32_t* __restrict__ n_found, int n_img, int N, int Npad,
                                                     int Hq, int Wq, long long npos_pad, int kp, int d,
                                                     uint32_t* __restrict__ tau_gl) {
  const int nb = norm_col(d) - DK_MAIN;  // patch values in the aux tile: columns 0 .. nb-1
  __shared__ unsigned hist_s[8][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned* hist = hist_s[wid];
  const long long nkeys = (long long)n_img * N;
  for (long long gk = blockIdx.x * 8LL + wid; gk < nkeys; gk += gridDim.x * 8LL) {
    const int f = (int)(gk / N), k = (int)(gk - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    const int kq = keys[gk];
    if ((unsigned)kq >= (unsigned)(Hq * Wq)) continue;
    constexpr int SPAN = SEED_WIN * SEED_STRIDE;
    if (Hq < SPAN || Wq < SPAN) continue;  // small images: no seed
    const int kr = kq / Wq, kc = kq - (kq / Wq) * Wq;
    const int r0 = min(max(kr - SPAN / 2, 0), Hq - SPAN);
    const int c0 = min(max(kc - SPAN / 2, 0), Wq - SPAN);
    const int rows = SEED_WIN, cols = SEED_WIN;
    // key operand: -2 p~ (64) and the three pn terms
    const __nv_bfloat16* ka = kmain + ((long long)f * Npad + k) * DK_MAIN;
    const __nv_bfloat16* kx = kaux + ((long long)f * Npad + k) * DK_AUX;
    const float pn = __bfloat162float(kx[nb + 3]) + __bfloat162float(kx[nb + 4]) + __bfloat162float(kx[nb + 5]);
    float kv[DK_MAIN], kxv[DK_AUX];
#pragma unroll
    for (int e = 0; e < DK_MAIN; ++e) kv[e] = __bfloat162float(ka[e]);
#pragma unroll
    for (int e = 0; e < DK_AUX; ++e) kxv[e] = e < nb ? __bfloat162float(kx[e]) : 0.f;
    constexpr int PER_LANE = SEED_WIN * SEED_WIN / 32;
    uint32_t key_s[PER_LANE];
    float qmax = 0.f;
#pragma unroll
    for (int i = 0; i < PER_LANE; ++i) {
      // sample j = 32 i + lane: row j / 16, column j % 16 of the strided grid
      uint32_t kk = 0xffffffffu;
      {
        const int j = 32 * i + lane;
        const long long q = (long long)(r0 + SEED_STRIDE * (j / SEED_WIN)) * Wq + c0 + SEED_STRIDE * (j % SEED_WIN);
        const uint4* qa = reinterpret_cast<const uint4*>(qmain + ((long long)f * npos_pad + q) * DK_MAIN);
        float acc = 0.f;
#pragma unroll
        for (int v = 0; v < DK_MAIN / 8; ++v) {
          const uint4 w = __ldg(qa + v);
          const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&w);
#pragma unroll
          for (int t = 0; t < 8; ++t) acc = fmaf(kv[v * 8 + t], __bfloat162float(hb[t]), acc);
        }
        const __nv_bfloat16* qx = qaux + ((long long)f * npos_pad + q) * DK_AUX;
        if (nb > 0) {
#pragma unroll
          for (int e = 0; e < DK_AUX; ++e)
            if (e < nb) acc = fmaf(kxv[e], __bfloat162float(qx[e]), acc);
        }
        const float qn = __bfloat162float(qx[nb]) + __bfloat162float(qx[nb + 1]) + __bfloat162float(qx[nb + 2]);
        qmax = fmaxf(qmax, qn);
        kk = float_order_key((acc + qn) + pn);
      }
      key_s[i] = kk;
    }
    const int n = rows * cols;
    if (n < kp) continue;
    // exact kp-th smallest of the 32 x 32 keys (4-pass radix select over the registers)
    uint32_t prefix = 0, pmask = 0;
    int rank = kp;
#pragma unroll 1
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
#pragma unroll
      for (int t = 0; t < 8; ++t) hist[lane * 8 + t] = 0;
      __syncwarp();
#pragma unroll
      for (int i = 0; i < PER_LANE; ++i)
        if (key_s[i] != 0xffffffffu && (key_s[i] & pmask) == prefix) atomicAdd(&hist[(key_s[i] >> shift) & 255u], 1u);
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
      int sel = 0, before = 0;
      if (lane == owner) {
        int c = excl;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (c + loc[t] >= rank) {
            sel = lane * 8 + t;
            before = c;
            break;
          }
          c += loc[t];
        }
      }
      sel = __shfl_sync(0xffffffffu, sel, owner);
      before = __shfl_sync(0xffffffffu, before, owner);
      rank -= before;
      prefix |= (uint32_t)sel << shift;
      pmask |= 255u << shift;
      __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
    if (lane == 0) {
      // margin: FP32 summation-order difference of ~80 products (far above its actual size)
      const float s_k = float_from_order_key(prefix);
      const float margin = 1e-5f * (pn + qmax + 2.f * sqrtf(pn * qmax)) + 1e-7f;
      tau_gl[(long long)f * Npad + k] = float_order_key(s_k + margin) + 1u;
    }
  }
}

template <int EB, bool WIDE, int MINS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_match_tc(const __grid_constant__ CUtensorMap tm_qmain, const __grid_constant__ CUtensorMap tm_qaux,
               const __grid_constant__ CUtensorMap tm_kmain, const __grid_constant__ CUtensorMap tm_kaux,
               const int32_t* __restrict__ n_found, int Npad, long long npos, long long npos_pad, int splits,
               int tiles_per_split, int ntiles, int nkc, StreamCfg cfg, uint2* __restrict__ bufs,
               int* __restrict__ buf_cnt, uint32_t* __restrict__ tau_gl, StatusBlock* st, float* __restrict__ dump,
               float* __restrict__ mins) {
  // MINS = 1: bound pass.  No candidate is kept; each epilogue lane writes the minimum
  // score of its row over every half tile (128 positions) to mins[key][2 tile + half]
  // instead (all four 32-column chunks read from TMEM in one visit).
  // (the chunk-minima scan of bound_pass 2 is k_match_chunk)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t kBar = WIDE ? W_OFF_BAR : OFF_BAR, kMisc = WIDE ? W_OFF_MISC : OFF_MISC;
  constexpr uint32_t kHist = WIDE ? W_OFF_HIST : OFF_HIST, kTile = WIDE ? W_OFF_TAU : OFF_TILE;
  constexpr uint32_t kTau = WIDE ? W_OFF_TAU : OFF_TAU;
  constexpr int NST = WIDE ? W_STAGES : TC_STAGES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kBar);
  uint64_t* full = bars;
  uint64_t* empty = bars + TC_STAGES;
  uint64_t* tfull = bars + 2 * TC_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* a_full = tempty + 2;
  uint64_t* mma_done = a_full + 1;
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(smem + kMisc);
  volatile int* abort_s = reinterpret_cast<volatile int*>(smem + kMisc + 4);
  unsigned* hist = reinterpret_cast<unsigned*>(smem + kHist);
  float* tiles = reinterpret_cast<float*>(smem + kTile);
  uint32_t* tau_sh = reinterpret_cast<uint32_t*>(smem + kTau);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kt = blockIdx.x, f = blockIdx.y, split = blockIdx.z;
  const int t_begin = split * tiles_per_split;
  const int t_end = min(ntiles, t_begin + tiles_per_split);
  const int nt = max(0, t_end - t_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, TC_EPI_WARPS);
    }
    mbar_init(a_full, 1);
    mbar_init(mma_done, 1);
    *abort_s = 0;
    for (int i = 0; i < TC_M; ++i) tau_sh[i] = 0xffffffffu;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_base_s;

  if (WIDE && warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ producer (wide operands)
      const int arow = f * Npad + kt * TC_M;
      int it = 0;
      bool ok = true;
      for (int i = 0; ok && i < nt; ++i) {
        const int brow = (int)(f * npos_pad + (long long)(t_begin + i) * TC_N);
        for (int kc = 0; kc <= nkc; ++kc) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          if (!mbar_wait(empty + s, ph ^ 1u, abort_s, st, true, cfg.wait_ns)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * W_STAGE_BYTES;
          uint8_t* sb = sa + A_MAIN_BYTES;
          if (kc < nkc) {
            mbar_arrive_expect_tx(full + s, A_MAIN_BYTES + B_MAIN_BYTES);
            tma_load_2d(&tm_kmain, full + s, sa, DK_MAIN * kc, arow);
            tma_load_2d(&tm_qmain, full + s, sb, DK_MAIN * kc, brow);
          } else {
            mbar_arrive_expect_tx(full + s, A_AUX_BYTES + B_AUX_BYTES);
            tma_load_2d(&tm_kaux, full + s, sa, 0, arow);
            tma_load_2d(&tm_qaux, full + s, sb, 0, brow);
          }
          ++it;
        }
      }
      // teardown: every issued copy has landed before the CTA may exit
      for (int j = max(0, it - NST); j < it; ++j)
        mbar_wait(full + (j % NST), (uint32_t)(j / NST) & 1u, abort_s, st, false);
    }
  } else if (WIDE && warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------- MMA issuer (wide operands)
      constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
      int it = 0;
      bool ok = true;
      for (int i = 0; ok && i < nt; ++i) {
        const int b = i & 1;
        const uint32_t bph = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait(tempty + b, bph ^ 1u, abort_s, st, true, cfg.wait_ns)) break;
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * TC_N);
        for (int kc = 0; kc <= nkc; ++kc) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          if (!mbar_wait(full + s, ph, abort_s, st, true, cfg.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * W_STAGE_BYTES);
          const uint32_t sb = sa + A_MAIN_BYTES;
          if (kc < nkc) {
#pragma unroll
            for (int k = 0; k < DK_MAIN / 16; ++k)
              mma_f16(d_tmem, smem_desc(sa + 32 * k, 1024, LAYOUT_SW128), smem_desc(sb + 32 * k, 1024, LAYOUT_SW128),
                       idesc, (kc > 0 || k > 0) ? 1u : 0u);
          } else {
            mma_f16(d_tmem, smem_desc(sa, 256, LAYOUT_SW32), smem_desc(sb, 256, LAYOUT_SW32), idesc, 1u);
          }
          mma_commit(empty + s);
          ++it;
        }
        if (ok) mma_commit(tfull + b);
      }
      // teardown: all issued MMAs have completed
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, abort_s, st, false);
    }
  } else if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      mbar_arrive_expect_tx(a_full, A_MAIN_BYTES + A_AUX_BYTES);
      const int arow = f * Npad + kt * TC_M;
      tma_load_2d(&tm_kmain, a_full, smem + OFF_A_MAIN, 0, arow);
      tma_load_2d(&tm_kaux, a_full, smem + OFF_A_AUX, 0, arow);
      int issued = 0;
      for (int i = 0; i < nt; ++i) {
        const int s = i % TC_STAGES;
        const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, abort_s, st, true, cfg.wait_ns)) break;
        mbar_arrive_expect_tx(full + s, B_MAIN_BYTES + B_AUX_BYTES);
        const int brow = (int)(f * npos_pad + (long long)(t_begin + i) * TC_N);
        tma_load_2d(&tm_qmain, full + s, smem + OFF_B_MAIN + s * B_MAIN_BYTES, 0, brow);
        tma_load_2d(&tm_qaux, full + s, smem + OFF_B_AUX + s * B_AUX_BYTES, 0, brow);
        issued = i + 1;
      }
      // teardown: every issued copy has landed before the CTA may exit
      mbar_wait(a_full, 0, abort_s, st, false);
      for (int i = max(0, issued - TC_STAGES); i < issued; ++i)
        mbar_wait(full + (i % TC_STAGES), (uint32_t)(i / TC_STAGES) & 1u, abort_s, st, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
      const uint32_t a_main = smem_u32(smem + OFF_A_MAIN), a_aux = smem_u32(smem + OFF_A_AUX);
      bool ok = mbar_wait(a_full, 0, abort_s, st, true, cfg.wait_ns);
      tc_fence_after();
      for (int i = 0; ok && i < nt; ++i) {
        const int s = i % TC_STAGES;
        const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
        const int b = i & 1;
        const uint32_t bph = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait(full + s, ph, abort_s, st, true, cfg.wait_ns)) break;
        if (!mbar_wait(tempty + b, bph ^ 1u, abort_s, st, true, cfg.wait_ns)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * TC_N);
        const uint32_t b_main = smem_u32(smem + OFF_B_MAIN + s * B_MAIN_BYTES);
        const uint32_t b_aux = smem_u32(smem + OFF_B_AUX + s * B_AUX_BYTES);
#pragma unroll
        for (int k = 0; k < DK_MAIN / 16; ++k)
          mma_f16(d_tmem, smem_desc(a_main + 32 * k, 1024, LAYOUT_SW128), smem_desc(b_main + 32 * k, 1024, LAYOUT_SW128),
                   idesc, k > 0 ? 1u : 0u);
        mma_f16(d_tmem, smem_desc(a_aux, 256, LAYOUT_SW32), smem_desc(b_aux, 256, LAYOUT_SW32), idesc, 1u);
        mma_commit(empty + s);
        mma_commit(tfull + b);
      }
      // teardown: all issued MMAs have completed
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, abort_s, st, false);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int e = warp - 2;
    const int quad = warp & 3;
    const int h = e >> 2;
    const int row = 32 * quad + lane;
    const int key = kt * TC_M + row;
    const int nf = min(n_found[f], Npad);
    const long long stream = (((long long)f * Npad + key) * splits + split) * 2 + h;
    uint2* mybuf = bufs + stream * (cfg.cap + 32);
    float tau = (key < nf) ? INFINITY : -INFINITY;
    int cnt = 0;
    uint32_t gl_next;  // seeded / published bound of the row, loaded one tile ahead
    uint2 stats = make_uint2(0u, 0u);
    unsigned* whist = hist + e * 256;
    float* wtile = tiles + e * 32 * TILE_LD;
    uint32_t* pub_sh = tau_sh + 32 * quad;
    uint32_t* pub_gl = tau_gl + (long long)f * Npad + (long long)kt * TC_M + 32 * quad;
    gl_next = *reinterpret_cast<volatile uint32_t*>(pub_gl + lane);
    for (int i = 0; i < nt; ++i) {
      const int b = i & 1;
      const uint32_t bph = (uint32_t)(i >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull + b, bph, abort_s, st, true, cfg.wait_ns));
      if (!ok) break;
      tc_fence_after();
      const long long tile_q0 = (long long)(t_begin + i) * TC_N;
      if constexpr (MINS == 1) {
        float w[4][32], v[128];
        const uint32_t taddr = tmem_base + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * TC_N + h * 128);
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld_32x32_nowait(taddr + 32 * c, w[c]);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 128; ++j) v[j] = w[j >> 5][j & 31];
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty + b);
        const int nvalid = (int)max(0LL, min(128LL, npos - (tile_q0 + h * 128)));
        if (nvalid < 128) {
#pragma unroll
          for (int j = 0; j < 128; ++j) v[j] = j < nvalid ? v[j] : INFINITY;
        }
        mins[(((long long)f * Npad + key) * ntiles + t_begin + i) * 2 + h] = min_tree3(v);
        continue;
      }
      const uint32_t gl = gl_next;
      gl_next = *reinterpret_cast<volatile uint32_t*>(pub_gl + lane);
      // EB chunks of 32 columns are read from TMEM per visit; the buffer goes back to
      // the MMA warp after the last visit (EB = 4: one visit, earliest release)
#pragma unroll 1
      for (int c0 = 0; c0 < 4; c0 += EB) {
        float v[EB][32];
        {
          const uint32_t taddr =
              tmem_base + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * TC_N + h * 128 + 32 * c0);
#pragma unroll
          for (int c = 0; c < EB; ++c) tmem_ld_32x32_nowait(taddr + 32 * c, v[c]);
          tmem_ld_wait();
        }
        if (c0 + EB >= 4) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty + b);
        }
#pragma unroll
        for (int c = 0; c < EB; ++c) {
          const int col = h * 128 + (c0 + c) * 32;
          const long long q0 = tile_q0 + col;
          const int nvalid = (int)max(0LL, min(32LL, npos - q0));
          if (dump != nullptr && i == 0 && t_begin == 0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) dump[((long long)f * Npad + key) * TC_N + col + j] = v[c][j];
          }
          const float te = stream_tau_eff(tau, *reinterpret_cast<volatile uint32_t*>(pub_sh + lane), gl);
          const unsigned rows = stream_filter(v[c], nvalid, te);
          if (rows) {
            if constexpr (WIDE) {
              stream_append_regs(rows, v[c], (int)q0, nvalid, te, tau, cnt, mybuf, cfg, whist, pub_sh, pub_gl, stats);
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                reinterpret_cast<float4*>(wtile + lane * TILE_LD)[j] =
                    make_float4(v[c][4 * j], v[c][4 * j + 1], v[c][4 * j + 2], v[c][4 * j + 3]);
              __syncwarp();
              stream_append(rows, wtile, TILE_LD, (int)q0, nvalid, te, tau, cnt, mybuf, cfg, whist, pub_sh, pub_gl,
                            stats);
            }
          }
        }
      }
    }
    if constexpr (MINS == 0) {
      if (cfg.finish) stream_finish(tau, cnt, mybuf, cfg, whist);
      stream_stats_flush(stats, st);
      buf_cnt[stream] = (key < nf) ? cnt : 0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// One size class of an uneven batch in the persistent scorer.  Its images are contiguous in
// the flat packed operands (key rows from krow0, position rows from qrow0) and in the image map.
constexpr int kMaxClasses = 8;
struct QClass {
  int n_img;       // images of the class
  int Npad;        // key rows per image (keys padded to 128)
  int N;           // keys per image
  int ntiles;      // position tiles per image
  int tps;         // position tiles per split
  int img0;        // first entry of the class in the image map
  long long npos;  // valid positions per image
  long long npos_pad;
  long long krow0, qrow0;
  long long item0;  // first work item of the class
};
struct QBatch {
  int n_classes;
  int splits;
  long long n_items;
  QClass c[kMaxClasses];
};

// Persistent candidate scan over an uneven batch (chunked operand rows).  One CTA per SM claims
// work items -- (class, image, key tile, position split) -- from a counter until the queue is
// empty; an item is the scan of one CTA of the uniform kernel (k_match_tc<EB, true, 0>): the same
// producer / MMA / epilogue roles, the operand ring and TMEM buffers continuing from item to item
// (their phases run on), the streams of the item's keys initialised at its start and closed at
// its end.  Between items the CTA synchronises: by then every copy and MMA of the item has been
// consumed.  The waits are bounded as in the uniform kernel.
template <int EB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_match_tc_queue(const __grid_constant__ CUtensorMap tm_qmain, const __grid_constant__ CUtensorMap tm_qaux,
                     const __grid_constant__ CUtensorMap tm_kmain, const __grid_constant__ CUtensorMap tm_kaux,
                     const __grid_constant__ QBatch qb, const int32_t* __restrict__ img_map,
                     const int32_t* __restrict__ n_found, int nkc, StreamCfg cfg, uint2* __restrict__ bufs,
                     int* __restrict__ buf_cnt, uint32_t* __restrict__ tau_gl, unsigned* __restrict__ queue,
                     StatusBlock* st) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int NST = W_STAGES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + W_OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + TC_STAGES;
  uint64_t* tfull = bars + 2 * TC_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* mma_done = tempty + 3;
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(smem + W_OFF_MISC);
  volatile int* abort_s = reinterpret_cast<volatile int*>(smem + W_OFF_MISC + 4);
  volatile long long* item_s = reinterpret_cast<volatile long long*>(smem + W_OFF_MISC + 8);
  unsigned* hist = reinterpret_cast<unsigned*>(smem + W_OFF_HIST);
  uint32_t* tau_sh = reinterpret_cast<uint32_t*>(smem + W_OFF_TAU);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int splits = qb.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, TC_EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_base_s;
  int it_ring = 0;  // operand ring slots used so far (producer and MMA count alike)
  int it_tile = 0;  // position tiles scored so far (TMEM buffer and phase)
  for (;;) {
    if (threadIdx.x == 0) *item_s = (long long)atomicAdd(queue, 1u);
    if (threadIdx.x < TC_M) tau_sh[threadIdx.x] = 0xffffffffu;
    __syncthreads();
    const long long item = *item_s;
    const bool stop = item >= qb.n_items || *abort_s;
    __syncthreads();  // every thread has read the item before thread 0 claims the next one
    if (stop) break;
    // decode: class, image, key tile, split
    int c = 0;
    while (c + 1 < qb.n_classes && item >= qb.c[c + 1].item0) ++c;
    const QClass& qc = qb.c[c];
    const long long local = item - qc.item0;
    const int ktiles = qc.Npad / TC_M;
    const int f = (int)(local / ((long long)ktiles * splits));
    const int rem = (int)(local - (long long)f * ktiles * splits);
    const int kt = rem / splits, split = rem - (rem / splits) * splits;
    const int t_begin = split * qc.tps;
    const int t_end = min(qc.ntiles, t_begin + qc.tps);
    const int nt = max(0, t_end - t_begin);
    const long long krow = qc.krow0 + (long long)f * qc.Npad;  // first key row of the image
    const long long qrow = qc.qrow0 + (long long)f * qc.npos_pad;
    if (warp == 0) {
      if (lane == 0) {
        // ---------------------------------------------------------- producer
        const int arow = (int)(krow + (long long)kt * TC_M);
        bool ok = true;
        for (int i = 0; ok && i < nt; ++i) {
          const int brow = (int)(qrow + (long long)(t_begin + i) * TC_N);
          for (int kc = 0; kc <= nkc; ++kc) {
            const int s = it_ring % NST;
            const uint32_t ph = (uint32_t)(it_ring / NST) & 1u;
            if (!mbar_wait(empty + s, ph ^ 1u, abort_s, st, true, cfg.wait_ns)) {
              ok = false;
              break;
            }
            uint8_t* sa = smem + s * W_STAGE_BYTES;
            uint8_t* sb = sa + A_MAIN_BYTES;
            if (kc < nkc) {
              mbar_arrive_expect_tx(full + s, A_MAIN_BYTES + B_MAIN_BYTES);
              tma_load_2d(&tm_kmain, full + s, sa, DK_MAIN * kc, arow);
              tma_load_2d(&tm_qmain, full + s, sb, DK_MAIN * kc, brow);
            } else {
              mbar_arrive_expect_tx(full + s, A_AUX_BYTES + B_AUX_BYTES);
              tma_load_2d(&tm_kaux, full + s, sa, 0, arow);
              tma_load_2d(&tm_qaux, full + s, sb, 0, brow);
            }
            ++it_ring;
          }
        }
        if (!ok) {
          // teardown after an expired wait: every issued copy lands before the CTA may exit
          for (int j = max(0, it_ring - NST); j < it_ring; ++j)
            mbar_wait(full + (j % NST), (uint32_t)(j / NST) & 1u, abort_s, st, false);
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        // --------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
        bool ok = true;
        for (int i = 0; ok && i < nt; ++i) {
          const int b = it_tile & 1;
          const uint32_t bph = (uint32_t)(it_tile >> 1) & 1u;
          if (!mbar_wait(tempty + b, bph ^ 1u, abort_s, st, true, cfg.wait_ns)) break;
          const uint32_t d_tmem = tmem_base + (uint32_t)(b * TC_N);
          for (int kc = 0; kc <= nkc; ++kc) {
            const int s = it_ring % NST;
            const uint32_t ph = (uint32_t)(it_ring / NST) & 1u;
            if (!mbar_wait(full + s, ph, abort_s, st, true, cfg.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * W_STAGE_BYTES);
            const uint32_t sb = sa + A_MAIN_BYTES;
            if (kc < nkc) {
#pragma unroll
              for (int k = 0; k < DK_MAIN / 16; ++k)
                mma_f16(d_tmem, smem_desc(sa + 32 * k, 1024, LAYOUT_SW128), smem_desc(sb + 32 * k, 1024, LAYOUT_SW128),
                         idesc, (kc > 0 || k > 0) ? 1u : 0u);
            } else {
              mma_f16(d_tmem, smem_desc(sa, 256, LAYOUT_SW32), smem_desc(sb, 256, LAYOUT_SW32), idesc, 1u);
            }
            mma_commit(empty + s);
            ++it_ring;
          }
          if (ok) mma_commit(tfull + b);
          ++it_tile;
        }
      }
      // (it_tile is tracked by the epilogue warps and lane 0 of this warp alike)
    } else {
      // ------------------------------------------------------------- epilogue
      const int e = warp - 2;
      const int quad = warp & 3;
      const int h = e >> 2;
      const int row = 32 * quad + lane;
      const int key = kt * TC_M + row;  // key of the image
      const int nf = min(n_found[img_map[qc.img0 + f]], qc.Npad);
      const long long stream = ((krow + key) * splits + split) * 2 + h;
      uint2* mybuf = bufs + stream * (cfg.cap + 32);
      float tau = (key < nf) ? INFINITY : -INFINITY;
      int cnt = 0;
      uint2 stats = make_uint2(0u, 0u);
      unsigned* whist = hist + e * 256;
      uint32_t* pub_sh = tau_sh + 32 * quad;
      uint32_t* pub_gl = tau_gl + krow + (long long)kt * TC_M + 32 * quad;
      uint32_t gl_next = *reinterpret_cast<volatile uint32_t*>(pub_gl + lane);
      for (int i = 0; i < nt; ++i) {
        const int b = it_tile & 1;
        const uint32_t bph = (uint32_t)(it_tile >> 1) & 1u;
        ++it_tile;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull + b, bph, abort_s, st, true, cfg.wait_ns));
        if (!ok) break;
        tc_fence_after();
        const long long tile_q0 = (long long)(t_begin + i) * TC_N;
        const uint32_t gl = gl_next;
        gl_next = *reinterpret_cast<volatile uint32_t*>(pub_gl + lane);
#pragma unroll 1
        for (int c0 = 0; c0 < 4; c0 += EB) {
          float v[EB][32];
          {
            const uint32_t taddr =
                tmem_base + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * TC_N + h * 128 + 32 * c0);
#pragma unroll
            for (int cc = 0; cc < EB; ++cc) tmem_ld_32x32_nowait(taddr + 32 * cc, v[cc]);
            tmem_ld_wait();
          }
          if (c0 + EB >= 4) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + b);
          }
#pragma unroll
          for (int cc = 0; cc < EB; ++cc) {
            const int col = h * 128 + (c0 + cc) * 32;
            const long long q0 = tile_q0 + col;
            const int nvalid = (int)max(0LL, min(32LL, qc.npos - q0));
            const float te = stream_tau_eff(tau, *reinterpret_cast<volatile uint32_t*>(pub_sh + lane), gl);
            const unsigned rows = stream_filter(v[cc], nvalid, te);
            if (rows)
              stream_append_regs(rows, v[cc], (int)q0, nvalid, te, tau, cnt, mybuf, cfg, whist, pub_sh, pub_gl, stats);
          }
        }
      }
      if (cfg.finish) stream_finish(tau, cnt, mybuf, cfg, whist);
      stream_stats_flush(stats, st);
      buf_cnt[stream] = (key < nf) ? cnt : 0;
    }
    // the MMA warp's lanes other than 0 and the producer warp's keep the tile count in step
    if ((warp == 0) || (warp == 1 && lane != 0)) it_tile += nt;
    __syncthreads();
  }
  // teardown: all issued MMAs have completed before TMEM is freed
  if (warp == 1 && lane == 0) {
    mma_commit(mma_done);
    mbar_wait(mma_done, 0, abort_s, st, false);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// ------------------------------------------------------ learned proposal scan
// The proposal contracts 16-value embeddings instead of patches.  Operand rows of 32
// elements, one per position / key:
//   BF16 (64-byte rows, two 32-byte swizzled chunks of 16 columns):
//     positions [ a = e~ (16)            | qn_hi qn_mid qn_lo 1 1 1 0 .. ]
//     keys      [ b = -2 e~ (16)         | 1 1 1 pn_hi pn_mid pn_lo 0 .. ]
//   E4M3 (32-byte rows, one 32-byte swizzled chunk, kind::f8f6f4, K = 32 per MMA):
//     positions [ a = e4m3(s e) (16)     | qn_hi qn_mid qn_lo 1 1 1 0 .. ]
//     keys      [ b = e4m3(-2 a) (16)    | 1 1 1 pn_hi pn_mid pn_lo 0 .. ]
// with e the FP32 embedding, e~ its BF16 rounding, qn = sum a^2 (FP32) of the position and
// pn the same of the key's own position, each split into three terms of the operand type,
// and s the per-tensor scale: the largest power of two with s^2 max ||e||^2 <= 384 (squared
// norms stay below E4M3's largest finite 448; doubling is exact).  A tile product gives per
// key p and position q the score
//   ||a_q||^2 - 2 <a_p, a_q> + ||a_p||^2 = ||a_p - a_q||^2,
// the squared distance of the rounded embeddings (scaled by s^2 for E4M3), so the 16-bit
// chunk minima resolve it relative to the distance itself.
constexpr int EMB_COLS = 32;

__device__ __forceinline__ float emb_scale(const unsigned* n2max) {
  const float m = __uint_as_float(*n2max);
  if (!(m > 0.f) || !(m < INFINITY)) return 1.f;
  int ex;
  frexpf(sqrtf(384.f / m), &ex);  // sqrt(384 / m) in [2^(ex-1), 2^ex)
  return ldexpf(1.f, ex - 1);
}
__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(uint8_t b) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
  return __half2float(__half(h));
}

// Position rows from the FP32 embeddings emb[img][npos][16]; rows past npos are zero.
template <bool FP8>
__global__ void __launch_bounds__(256) k_pack_emb_pos(const float* __restrict__ emb, int n_img, long long npos,
                                                      long long npos_pad, const unsigned* __restrict__ n2max,
                                                      uint8_t* __restrict__ out) {
  constexpr int RB = FP8 ? 32 : 64;  // row bytes
  const float s = FP8 ? emb_scale(n2max) : 1.f;
  const long long total = (long long)n_img * npos_pad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / npos_pad, q = i - f * npos_pad;
    __align__(16) uint8_t row[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) row[k] = 0;
    if (q < npos) {
      const float4* src = reinterpret_cast<const float4*>(emb + (f * npos + q) * 16);
      float e[16];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 v = __ldg(src + k);
        e[4 * k] = v.x;
        e[4 * k + 1] = v.y;
        e[4 * k + 2] = v.z;
        e[4 * k + 3] = v.w;
      }
      float n = 0.f;
      if constexpr (FP8) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          row[j] = to_e4m3(s * e[j]);
          const float a = from_e4m3(row[j]);
          n = fmaf(a, a, n);
        }
        row[16] = to_e4m3(n);
        const float r1 = n - from_e4m3(row[16]);
        row[17] = to_e4m3(r1);
        row[18] = to_e4m3(r1 - from_e4m3(row[17]));
        row[19] = row[20] = row[21] = to_e4m3(1.f);
      } else {
        __nv_bfloat16* rb = reinterpret_cast<__nv_bfloat16*>(row);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          rb[j] = __float2bfloat16_rn(e[j]);
          const float a = __bfloat162float(rb[j]);
          n = fmaf(a, a, n);
        }
        split3(n, rb[16], rb[17], rb[18]);
        rb[19] = rb[20] = rb[21] = __float2bfloat16_rn(1.f);
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(out + i * RB);
#pragma unroll
    for (int k = 0; k < RB / 16; ++k) dst[k] = reinterpret_cast<const uint4*>(row)[k];
  }
}

// Key rows: the embedding of each key's own position (so a key scores its own position
// like any other); rows of keys >= n_found and of the padding are zero.
template <bool FP8>
__global__ void __launch_bounds__(256) k_pack_emb_keys(const float* __restrict__ emb, const int32_t* __restrict__ keys,
                                                       const int32_t* __restrict__ n_found, int n_img, int N, int Npad,
                                                       long long npos, const unsigned* __restrict__ n2max,
                                                       uint8_t* __restrict__ out) {
  constexpr int RB = FP8 ? 32 : 64;
  const float s = FP8 ? emb_scale(n2max) : 1.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n_img * Npad;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / Npad), k = (int)(i - (long long)f * Npad);
    __align__(16) uint8_t row[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) row[j] = 0;
    const int kq = k < min(n_found[f], N) ? keys[(long long)f * N + k] : -1;
    if (kq >= 0 && kq < npos) {
      const float* src = emb + ((long long)f * npos + kq) * 16;
      float n = 0.f;  // the key position's own squared norm, formed as for the position rows
      if constexpr (FP8) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float a = from_e4m3(to_e4m3(s * __ldg(src + j)));
          n = fmaf(a, a, n);
          row[j] = to_e4m3(-2.f * a);
        }
        row[16] = row[17] = row[18] = to_e4m3(1.f);
        row[19] = to_e4m3(n);
        const float r1 = n - from_e4m3(row[19]);
        row[20] = to_e4m3(r1);
        row[21] = to_e4m3(r1 - from_e4m3(row[20]));
      } else {
        __nv_bfloat16* rb = reinterpret_cast<__nv_bfloat16*>(row);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float a = __bfloat162float(__float2bfloat16_rn(__ldg(src + j)));
          n = fmaf(a, a, n);
          rb[j] = __float2bfloat16_rn(-2.f * a);
        }
        rb[16] = rb[17] = rb[18] = __float2bfloat16_rn(1.f);
        split3(n, rb[19], rb[20], rb[21]);
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(out + i * RB);
#pragma unroll
    for (int j = 0; j < RB / 16; ++j) dst[j] = reinterpret_cast<const uint4*>(row)[j];
  }
}

// Chunk-minima scans (bound_pass 2) of both the exact BF16 matcher and the learned proposal:
// CTA = 128 keys x one split of the positions, 320 threads: warp 0 = TMA producer (one
// thread), warp 1 = TMEM allocator and MMA issuer (one thread), warps 2-9 = epilogue (warps
// w and w + 4 share a TMEM lane quadrant and take one column half each).  Position tiles are
// NT wide and tensor memory holds 512 / NT accumulators: each tile's handshake (MMA commit ->
// epilogue reads -> buffer released -> next MMA into it) is a chain of barrier wake-ups, and
// more buffers in flight overlap more of those chains.  Operand forms:
//   CF_PATCH      BF16 rows of 64 patch columns (128-byte swizzle) + 16 norm columns
//                 (32-byte swizzle): 4 + 1 kind::f16 MMAs per tile
//   CF_EMB_BF16   BF16 embedding rows of 32 columns as two 32-byte swizzled chunks:
//                 2 kind::f16 MMAs per tile
//   CF_EMB_E4M3   E4M3 embedding rows of 32 bytes: 1 kind::f8f6f4 MMA per tile
// Minima: the upper 16 bits of the order key of each 32-position chunk minimum (the key
// truncated), mins viewed as uint16 [key][chunk] (chunk = position / 32).
constexpr int CF_PATCH = 0, CF_EMB_BF16 = 1, CF_EMB_E4M3 = 2;
constexpr int kChunkNT = 256;  // position tile of the chunk-minima scans (128 measured slower)
constexpr int CH_EPI_WARPS = 8;
constexpr int CH_THREADS = 64 + CH_EPI_WARPS * 32;
template <int FORM, int NT>
struct ChunkForm {
  static constexpr int nbuf = 512 / NT;  // accumulators in tensor memory
  static constexpr uint32_t a_main = FORM == CF_PATCH ? A_MAIN_BYTES : (FORM == CF_EMB_BF16 ? 4096 : 4096);
  static constexpr uint32_t a_bytes = FORM == CF_PATCH ? A_MAIN_BYTES + A_AUX_BYTES : (FORM == CF_EMB_BF16 ? 8192 : 4096);
  static constexpr uint32_t b_main = FORM == CF_PATCH ? NT * 128 : NT * 32;  // first column chunk of a tile
  static constexpr uint32_t b_bytes = FORM == CF_PATCH ? NT * 160 : (FORM == CF_EMB_BF16 ? NT * 64 : NT * 32);
  static constexpr int stages = (FORM == CF_PATCH ? 160 * 1024 : 128 * 1024) / (int)b_bytes < 16
                                    ? (FORM == CF_PATCH ? 160 * 1024 : 128 * 1024) / (int)b_bytes
                                    : 16;
  static constexpr uint32_t off_b = (a_bytes + 1023) / 1024 * 1024;
  static constexpr uint32_t off_bar = off_b + stages * b_bytes;
  static constexpr uint32_t off_misc = off_bar + (2 * stages + 2 * nbuf + 2) * 8;
  static constexpr uint32_t smem = off_misc + 64 + 1024;
};
static_assert(ChunkForm<CF_PATCH, 128>::smem <= 232448 && ChunkForm<CF_PATCH, 256>::smem <= 232448, "smem budget");
static_assert(ChunkForm<CF_EMB_BF16, 128>::smem <= 232448, "smem budget");

template <int FORM, int NT>
__global__ void __launch_bounds__(CH_THREADS, 1)
    k_match_chunk(const __grid_constant__ CUtensorMap tm_qmain, const __grid_constant__ CUtensorMap tm_qaux,
                  const __grid_constant__ CUtensorMap tm_kmain, const __grid_constant__ CUtensorMap tm_kaux,
                  int Npad, long long npos, long long npos_pad, int tiles_per_split, int ntiles,
                  unsigned long long wait_ns, StatusBlock* st, float* __restrict__ dump,
                  uint16_t* __restrict__ mins) {
  using CF = ChunkForm<FORM, NT>;
  constexpr int NST = CF::stages, NB = CF::nbuf, CPW = NT / 64;  // chunks per epilogue thread and tile
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + CF::off_bar);
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* tfull = bars + 2 * NST;
  uint64_t* tempty = tfull + NB;
  uint64_t* a_full = tempty + NB;
  uint64_t* mma_done = a_full + 1;
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(smem + CF::off_misc);
  volatile int* abort_s = reinterpret_cast<volatile int*>(smem + CF::off_misc + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kt = blockIdx.x, f = blockIdx.y, split = blockIdx.z;
  // tiles_per_split and ntiles count 256-position tiles; this kernel walks NT-position tiles
  constexpr int R = 256 / NT;
  const int t_begin = split * tiles_per_split * R;
  const int nt = max(0, min(ntiles * R, t_begin + tiles_per_split * R) - t_begin);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, CH_EPI_WARPS);
    }
    mbar_init(a_full, 1);
    mbar_init(mma_done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_base_s, 512);
    tmem_relinquish();
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_base_s;
  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      const int arow = f * Npad + kt * TC_M;
      mbar_arrive_expect_tx(a_full, CF::a_bytes);
      tma_load_2d(&tm_kmain, a_full, smem, 0, arow);
      if constexpr (FORM == CF_PATCH) tma_load_2d(&tm_kaux, a_full, smem + CF::a_main, 0, arow);
      if constexpr (FORM == CF_EMB_BF16) tma_load_2d(&tm_kmain, a_full, smem + CF::a_main, 16, arow);
      int issued = 0;
      for (int i = 0; i < nt; ++i) {
        const int s = i % NST;
        const uint32_t ph = (uint32_t)(i / NST) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, abort_s, st, true, wait_ns)) break;
        mbar_arrive_expect_tx(full + s, CF::b_bytes);
        const int brow = (int)(f * npos_pad + (long long)(t_begin + i) * NT);
        uint8_t* sb = smem + CF::off_b + s * CF::b_bytes;
        tma_load_2d(&tm_qmain, full + s, sb, 0, brow);
        if constexpr (FORM == CF_PATCH) tma_load_2d(&tm_qaux, full + s, sb + CF::b_main, 0, brow);
        if constexpr (FORM == CF_EMB_BF16) tma_load_2d(&tm_qmain, full + s, sb + CF::b_main, 16, brow);
        issued = i + 1;
      }
      // teardown: every issued copy has landed before the CTA may exit
      mbar_wait(a_full, 0, abort_s, st, false);
      for (int i = max(0, issued - NST); i < issued; ++i)
        mbar_wait(full + (i % NST), (uint32_t)(i / NST) & 1u, abort_s, st, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // --------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = FORM == CF_EMB_E4M3 ? idesc_e4m3(TC_M, NT) : idesc_bf16(TC_M, NT);
      const uint32_t sa = smem_u32(smem);
      bool ok = mbar_wait(a_full, 0, abort_s, st, true, wait_ns);
      tc_fence_after();
      for (int i = 0; ok && i < nt; ++i) {
        const int s = i % NST;
        const uint32_t ph = (uint32_t)(i / NST) & 1u;
        const int b = i % NB;
        const uint32_t bph = (uint32_t)(i / NB) & 1u;
        if (!mbar_wait(full + s, ph, abort_s, st, true, wait_ns)) break;
        if (!mbar_wait(tempty + b, bph ^ 1u, abort_s, st, true, wait_ns)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * NT);
        const uint32_t sb = smem_u32(smem + CF::off_b + s * CF::b_bytes);
        if constexpr (FORM == CF_PATCH) {
#pragma unroll
          for (int k = 0; k < DK_MAIN / 16; ++k)
            mma_f16(d_tmem, smem_desc(sa + 32 * k, 1024, LAYOUT_SW128), smem_desc(sb + 32 * k, 1024, LAYOUT_SW128),
                    idesc, k > 0 ? 1u : 0u);
          mma_f16(d_tmem, smem_desc(sa + CF::a_main, 256, LAYOUT_SW32), smem_desc(sb + CF::b_main, 256, LAYOUT_SW32),
                  idesc, 1u);
        } else if constexpr (FORM == CF_EMB_E4M3) {
          mma_e4m3(d_tmem, smem_desc(sa, 256, LAYOUT_SW32), smem_desc(sb, 256, LAYOUT_SW32), idesc, 0u);
        } else {
          mma_f16(d_tmem, smem_desc(sa, 256, LAYOUT_SW32), smem_desc(sb, 256, LAYOUT_SW32), idesc, 0u);
          mma_f16(d_tmem, smem_desc(sa + CF::a_main, 256, LAYOUT_SW32), smem_desc(sb + CF::b_main, 256, LAYOUT_SW32),
                  idesc, 1u);
        }
        mma_commit(empty + s);
        mma_commit(tfull + b);
      }
      // teardown: all issued MMAs have completed
      mma_commit(mma_done);
      mbar_wait(mma_done, 0, abort_s, st, false);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int quad = warp & 3;        // TMEM lane quadrant this warp may read
    const int h = (warp - 2) >> 2;    // column half of the tile: NT / 2 positions, CPW chunks
    const int key = kt * TC_M + 32 * quad + lane;
    const uint32_t taddr0 = tmem_base + ((uint32_t)(32 * quad) << 16) + (uint32_t)(h * (NT / 2));
    uint16_t* mrow = mins + ((long long)f * Npad + key) * ntiles * 8 + h * CPW;
    for (int i = 0; i < nt; ++i) {
      const int b = i % NB;
      const uint32_t bph = (uint32_t)(i / NB) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(tfull + b, bph, abort_s, st, true, wait_ns))) break;
      tc_fence_after();
      float w[CPW][32];
#pragma unroll
      for (int c = 0; c < CPW; ++c) tmem_ld_32x32_nowait(taddr0 + (uint32_t)(b * NT + 32 * c), w[c]);
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);
      const long long q0 = (long long)(t_begin + i) * NT + h * (NT / 2);
      if (dump != nullptr && q0 < TC_N) {  // raw scores of the first 256 positions
        float* dr = dump + ((long long)f * Npad + key) * TC_N + q0;
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
          for (int j = 0; j < 32; ++j) dr[32 * c + j] = w[c][j];
      }
      // the upper 16 bits of each chunk minimum's order key (truncation: monotone, so a key's
      // K'-th smallest truncated minimum still bounds its candidate chunks); positions past the
      // grid only occur in the last tile
      uint32_t k16[CPW];
      if (q0 + NT / 2 <= npos) {
#pragma unroll
        for (int c = 0; c < CPW; ++c) k16[c] = float_order_key(min_tree3(w[c])) >> 16;
      } else {
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const int nvalid = (int)max(0LL, min(32LL, npos - (q0 + 32 * c)));
          k16[c] = float_order_key(stream_min(w[c], nvalid)) >> 16;
        }
      }
      uint16_t* dst = mrow + (long long)(t_begin + i) * (NT / 32);
      if constexpr (CPW == 4) {
        *reinterpret_cast<uint2*>(dst) = make_uint2(k16[0] | (k16[1] << 16), k16[2] | (k16[3] << 16));
      } else {
        *reinterpret_cast<uint32_t*>(dst) = k16[0] | (k16[1] << 16);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, void* base, uint64_t rows, uint32_t cols, uint32_t box_rows, CUtensorMapSwizzle sw,
              uint32_t box_cols = 0, CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, uint32_t esz = 2) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
  const cuuint32_t box[2] = {box_cols ? box_cols : cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern float* g_tc_dump;

glr_status launch_tau_bound(const float* mins, const int32_t* n_found, int n_img, int N, const MatchPlan& pl,
                            uint32_t* taugl, cudaStream_t s) {
  const long long nkeys = (long long)n_img * N;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, 8), (long long)num_sms() * 16));
  GLR_LAUNCH("k_tau_bound", s,
             k_tau_bound<<<blocks, 256, 0, s>>>(mins, n_found, n_img, N, pl.Npad, 2 * pl.pos_tiles, pl.Kp, taugl));
  return GLR_OK;
}

glr_status launch_match_tc_impl(const float* x, const glr_images& im, const int32_t* n_found, const MatchPlan& pl,
                                char* ws, float* dump, const int32_t* seed_keys, int seed_N, const float* emb_pos,
                                const float* emb_keys, cudaStream_t s) {
  const int d = emb_keys ? 16 : im.C * im.P * im.P;
  const bool wide = pl.nkc > 1;
  const int raw = pl.mode == GLR_MATCH_EDGE ? 1 : 0;  // heat-map operands: no norm columns
  if (!wide && norm_col(d) + 6 > DK_MAIN + DK_AUX) return GLR_ENOTSUP;
  if (wide && (emb_keys != nullptr || dump != nullptr || pl.nkc * DK_MAIN < d)) return GLR_ENOTSUP;
  const float* mean = reinterpret_cast<const float*>(ws + pl.mean_off);
  const float* keyv = emb_keys ? emb_keys : reinterpret_cast<const float*>(ws + pl.keyv_off);
  uint2* bufs = reinterpret_cast<uint2*>(ws + pl.buf_off);
  int* bufcnt = reinterpret_cast<int*>(ws + pl.bufcnt_off);
  uint32_t* taugl = reinterpret_cast<uint32_t*>(ws + pl.taugl_off);
  float* mins = pl.bound_pass ? reinterpret_cast<float*>(ws + pl.mins_off) : nullptr;
  StatusBlock* st = reinterpret_cast<StatusBlock*>(ws);
  __nv_bfloat16* qmain = reinterpret_cast<__nv_bfloat16*>(ws + pl.qpack_off);
  __nv_bfloat16* qaux = qmain + (size_t)im.n_img * pl.npos_pad * DK_MAIN * pl.nkc;
  __nv_bfloat16* kmain = reinterpret_cast<__nv_bfloat16*>(ws + pl.kpack_off);
  __nv_bfloat16* kaux = kmain + (size_t)im.n_img * pl.Npad * DK_MAIN * pl.nkc;
  if (wide) {
    {
      const size_t psmem = (size_t)PW_POS * (pl.nkc * DK_MAIN + 2) * 2 + (size_t)im.C * PW_POS * 4;
      if (psmem > 227 * 1024) return GLR_ENOTSUP;
      const long long nblk = (long long)im.n_img * (pl.npos_pad / PW_POS);
      const int pblocks = (int)std::max<long long>(1, std::min<long long>(nblk, (long long)num_sms() * 16));
#define GLR_PACKW_CASE(PP)                                                                                     \
  {                                                                                                            \
    if (cudaFuncSetAttribute(k_pack_positions_w<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem) != \
        cudaSuccess)                                                                                           \
      return GLR_ECUDA;                                                                                        \
    GLR_LAUNCH("k_pack_positions", s,                                                                          \
               k_pack_positions_w<PP><<<pblocks, 256, psmem, s>>>(x, mean, im.n_img, im.C, im.H, im.W, im.P,     \
                                                                  pl.npos_pad, pl.nkc, raw, qmain, qaux,       \
                                                                  ImgMap{}));                                  \
  }
      switch (im.P) {
        case 6: GLR_PACKW_CASE(6); break;
        case 8: GLR_PACKW_CASE(8); break;
        default: GLR_PACKW_CASE(0); break;
      }
#undef GLR_PACKW_CASE
    }
    {
      const int nk = im.n_img * pl.Npad;
      const int blocks = (int)std::max<long long>(1, ceil_div(nk, 256));
      GLR_LAUNCH("k_pack_keys", s, k_pack_keys_w<<<blocks, 256, 0, s>>>(keyv, nk, d, pl.nkc, raw, kmain, kaux));
    }
    CUtensorMap tq, tqa, tk, tka;
    const uint64_t qrows = (uint64_t)im.n_img * pl.npos_pad, krows = (uint64_t)im.n_img * pl.Npad;
    const uint32_t wcols = (uint32_t)(pl.nkc * DK_MAIN);
    if (!make_map(&tq, qmain, qrows, wcols, TC_N, CU_TENSOR_MAP_SWIZZLE_128B, DK_MAIN) ||
        !make_map(&tqa, qaux, qrows, DK_AUX, TC_N, CU_TENSOR_MAP_SWIZZLE_32B) ||
        !make_map(&tk, kmain, krows, wcols, TC_M, CU_TENSOR_MAP_SWIZZLE_128B, DK_MAIN) ||
        !make_map(&tka, kaux, krows, DK_AUX, TC_M, CU_TENSOR_MAP_SWIZZLE_32B))
      return GLR_ECUDA;
    auto kern = pl.epi_batch == 2 ? k_match_tc<2, true, 0> : k_match_tc<4, true, 0>;
    auto kmin = k_match_tc<4, true, 1>;
    if (pl.bound_pass &&
        cudaFuncSetAttribute(kmin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W_SMEM) != cudaSuccess)
      return GLR_ECUDA;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W_SMEM) != cudaSuccess)
      return GLR_ECUDA;
    int blocks_per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, TC_THREADS, W_SMEM) != cudaSuccess ||
        blocks_per_sm != 1)  // all of TMEM: exactly one resident CTA per SM
      return GLR_ENOTSUP;
    const long long npos = (long long)(im.H - im.P + 1) * (im.W - im.P + 1);
    const StreamCfg cfg{pl.cap, pl.Kp, pl.finish, g_match_wait_ns > 0 ? g_match_wait_ns : kWaitNs};
    dim3 grid((unsigned)(pl.Npad / TC_M), (unsigned)im.n_img, (unsigned)pl.splits);
    if (pl.bound_pass) {
      GLR_LAUNCH("k_match_tc_min", s,
                 kmin<<<grid, TC_THREADS, W_SMEM, s>>>(tq, tqa, tk, tka, n_found, pl.Npad, npos, pl.npos_pad,
                                                       pl.splits, pl.tiles_per_split, pl.pos_tiles, pl.nkc, cfg, bufs,
                                                       bufcnt, taugl, st, nullptr, mins));
      const glr_status bs = launch_tau_bound(mins, n_found, im.n_img, seed_N, pl, taugl, s);
      if (bs != GLR_OK) return bs;
    }
    GLR_LAUNCH("k_match_tc", s,
               kern<<<grid, TC_THREADS, W_SMEM, s>>>(tq, tqa, tk, tka, n_found, pl.Npad, npos, pl.npos_pad, pl.splits,
                                                     pl.tiles_per_split, pl.pos_tiles, pl.nkc, cfg, bufs, bufcnt,
                                                     taugl, st, nullptr, nullptr));
    return GLR_OK;
  }
  {
    const long long total = (long long)im.n_img * pl.npos_pad;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
#define GLR_PACK_CASE(PP)                                                                                  \
  GLR_LAUNCH("k_pack_positions", s,                                                                          \
             k_pack_positions<PP><<<blocks, 256, 0, s>>>(x, mean, im.n_img, im.C, im.H, im.W, im.P, pl.npos_pad, \
                                                         emb_pos, raw, qmain, qaux))
    switch (im.P) {
      case 4: GLR_PACK_CASE(4); break;
      case 5: GLR_PACK_CASE(5); break;
      case 6: GLR_PACK_CASE(6); break;
      case 8: GLR_PACK_CASE(8); break;
      default: GLR_PACK_CASE(0); break;
    }
#undef GLR_PACK_CASE
  }
  {
    const int nk = im.n_img * pl.Npad;
    const int blocks = (int)std::max<long long>(1, ceil_div(nk, 256));
    GLR_LAUNCH("k_pack_keys", s, k_pack_keys<<<blocks, 256, 0, s>>>(keyv, nk, d, raw, kmain, kaux));
  }
  if (seed_keys != nullptr) {
    const long long nkeys = (long long)im.n_img * seed_N;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(nkeys, 8), (long long)num_sms() * 16));
    GLR_LAUNCH("k_seed_bounds", s,
               k_seed_bounds<<<blocks, 256, 0, s>>>(qmain, qaux, kmain, kaux, seed_keys, n_found, im.n_img, seed_N,
                                                    pl.Npad, im.H - im.P + 1, im.W - im.P + 1, pl.npos_pad, pl.Kp,
                                                    d, taugl));
  }
  CUtensorMap tq, tqa, tk, tka;
  const uint64_t qrows = (uint64_t)im.n_img * pl.npos_pad, krows = (uint64_t)im.n_img * pl.Npad;
  if (!make_map(&tq, qmain, qrows, DK_MAIN, TC_N, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map(&tqa, qaux, qrows, DK_AUX, TC_N, CU_TENSOR_MAP_SWIZZLE_32B) ||
      !make_map(&tk, kmain, krows, DK_MAIN, TC_M, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map(&tka, kaux, krows, DK_AUX, TC_M, CU_TENSOR_MAP_SWIZZLE_32B))
    return GLR_ECUDA;
  auto kern = pl.epi_batch == 2 ? k_match_tc<2, false, 0> : k_match_tc<4, false, 0>;
  auto kmin = k_match_tc<4, false, 1>;
  if (pl.bound_pass == 2) {
    // chunk-minima scan only; the exact evaluation of the candidate chunks follows (k_match.cu)
    auto kch = k_match_chunk<CF_PATCH, kChunkNT>;
    constexpr uint32_t smem = ChunkForm<CF_PATCH, kChunkNT>::smem;
    CUtensorMap cq, cqa;  // position tiles of kChunkNT rows
    if (!make_map(&cq, qmain, qrows, DK_MAIN, kChunkNT, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&cqa, qaux, qrows, DK_AUX, kChunkNT, CU_TENSOR_MAP_SWIZZLE_32B))
      return GLR_ECUDA;
    if (cudaFuncSetAttribute(kch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GLR_ECUDA;
    int blocks_per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kch, CH_THREADS, smem) != cudaSuccess ||
        blocks_per_sm != 1)  // all of TMEM: exactly one resident CTA per SM
      return GLR_ENOTSUP;
    const long long npos = (long long)(im.H - im.P + 1) * (im.W - im.P + 1);
    dim3 grid((unsigned)(pl.Npad / TC_M), (unsigned)im.n_img, (unsigned)pl.splits);
    GLR_LAUNCH("k_match_tc_chunk", s,
               kch<<<grid, CH_THREADS, smem, s>>>(cq, cqa, tk, tka, pl.Npad, npos, pl.npos_pad, pl.tiles_per_split,
                                                 pl.pos_tiles, g_match_wait_ns > 0 ? g_match_wait_ns : kWaitNs, st,
                                                 dump, reinterpret_cast<uint16_t*>(mins)));
    return GLR_OK;
  }
  if (pl.bound_pass &&
      cudaFuncSetAttribute(kmin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess)
    return GLR_ECUDA;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess)
    return GLR_ECUDA;
  {
    int blocks_per_sm = 0;  // the kernel needs exactly one resident CTA per SM (all of TMEM)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, TC_THREADS, TC_SMEM) != cudaSuccess ||
        blocks_per_sm < 1)
      return GLR_ENOTSUP;
  }
  const long long npos = (long long)(im.H - im.P + 1) * (im.W - im.P + 1);
  const StreamCfg cfg{pl.cap, pl.Kp, pl.finish, g_match_wait_ns > 0 ? g_match_wait_ns : kWaitNs};
  dim3 grid((unsigned)(pl.Npad / TC_M), (unsigned)im.n_img, (unsigned)pl.splits);
  if (pl.bound_pass && dump == nullptr) {
    GLR_LAUNCH("k_match_tc_min", s,
               kmin<<<grid, TC_THREADS, TC_SMEM, s>>>(tq, tqa, tk, tka, n_found, pl.Npad, npos, pl.npos_pad,
                                                      pl.splits, pl.tiles_per_split, pl.pos_tiles, 1, cfg, bufs,
                                                      bufcnt, taugl, st, nullptr, mins));
    const glr_status bs = launch_tau_bound(mins, n_found, im.n_img, seed_N, pl, taugl, s);
    if (bs != GLR_OK) return bs;
  }
  GLR_LAUNCH("k_match_tc", s,
             kern<<<grid, TC_THREADS, TC_SMEM, s>>>(tq, tqa, tk, tka, n_found, pl.Npad, npos, pl.npos_pad,
                                                          pl.splits, pl.tiles_per_split, pl.pos_tiles, 1, cfg, bufs,
                                                          bufcnt, taugl, st, dump, nullptr));
  return GLR_OK;
}

// ---- uneven batches (glr_batch.cu): packing of one size class into the flat operands, and the
//      persistent scan over all classes
glr_status launch_pack_class_w(const float* x, const float* mean, const glr_images& im, long long npos_pad, int nkc,
                               const float* keyv, int Npad, __nv_bfloat16* qmain, __nv_bfloat16* qaux,
                               __nv_bfloat16* kmain, __nv_bfloat16* kaux, ImgMap imap, cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  {
    const size_t psmem = (size_t)PW_POS * (nkc * DK_MAIN + 2) * 2 + (size_t)im.C * PW_POS * 4;
    if (psmem > 227 * 1024) return GLR_ENOTSUP;
    const long long nblk = (long long)im.n_img * (npos_pad / PW_POS);
    const int pblocks = (int)std::max<long long>(1, std::min<long long>(nblk, (long long)num_sms() * 16));
#define GLR_PACKB_CASE(PP)                                                                                     \
  {                                                                                                            \
    if (cudaFuncSetAttribute(k_pack_positions_w<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem) != \
        cudaSuccess)                                                                                           \
      return GLR_ECUDA;                                                                                        \
    GLR_LAUNCH("k_pack_positions", s,                                                                          \
               k_pack_positions_w<PP><<<pblocks, 256, psmem, s>>>(x, mean, im.n_img, im.C, im.H, im.W, im.P,     \
                                                                  npos_pad, nkc, 0, qmain, qaux, imap));       \
  }
    switch (im.P) {
      case 6: GLR_PACKB_CASE(6); break;
      case 8: GLR_PACKB_CASE(8); break;
      default: GLR_PACKB_CASE(0); break;
    }
#undef GLR_PACKB_CASE
  }
  const int nk = im.n_img * Npad;
  const int blocks = (int)std::max<long long>(1, ceil_div(nk, 256));
  GLR_LAUNCH("k_pack_keys", s, k_pack_keys_w<<<blocks, 256, 0, s>>>(keyv, nk, d, nkc, 0, kmain, kaux));
  return GLR_OK;
}

glr_status launch_match_tc_queue(const QBatchHost& hb, const int32_t* img_map, const int32_t* n_found, int nkc,
                                 int cap, int Kp, int finish, int epi_batch, __nv_bfloat16* qmain,
                                 __nv_bfloat16* qaux, __nv_bfloat16* kmain, __nv_bfloat16* kaux, long long qrows,
                                 long long krows, uint2* bufs, int* bufcnt, uint32_t* taugl, unsigned* queue,
                                 StatusBlock* st, cudaStream_t s) {
  if (hb.n_classes < 1 || hb.n_classes > kMaxClasses) return GLR_ENOTSUP;
  QBatch qb{};
  qb.n_classes = hb.n_classes;
  qb.splits = hb.splits;
  qb.n_items = hb.n_items;
  for (int c = 0; c < hb.n_classes; ++c) {
    const QClassHost& h = hb.c[c];
    qb.c[c] = QClass{h.n_img, h.Npad, h.N, h.ntiles, h.tps, h.img0, h.npos, h.npos_pad, h.krow0, h.qrow0, h.item0};
  }
  CUtensorMap tq, tqa, tk, tka;
  const uint32_t wcols = (uint32_t)(nkc * DK_MAIN);
  if (!make_map(&tq, qmain, (uint64_t)qrows, wcols, TC_N, CU_TENSOR_MAP_SWIZZLE_128B, DK_MAIN) ||
      !make_map(&tqa, qaux, (uint64_t)qrows, DK_AUX, TC_N, CU_TENSOR_MAP_SWIZZLE_32B) ||
      !make_map(&tk, kmain, (uint64_t)krows, wcols, TC_M, CU_TENSOR_MAP_SWIZZLE_128B, DK_MAIN) ||
      !make_map(&tka, kaux, (uint64_t)krows, DK_AUX, TC_M, CU_TENSOR_MAP_SWIZZLE_32B))
    return GLR_ECUDA;
  auto kern = epi_batch == 4 ? k_match_tc_queue<4> : k_match_tc_queue<2>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W_SMEM) != cudaSuccess)
    return GLR_ECUDA;
  int blocks_per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, TC_THREADS, W_SMEM) != cudaSuccess ||
      blocks_per_sm != 1)  // all of TMEM: exactly one resident CTA per SM
    return GLR_ENOTSUP;
  if (cudaMemsetAsync(queue, 0, sizeof(unsigned), s) != cudaSuccess) return GLR_ECUDA;
  const StreamCfg cfg{cap, Kp, finish, g_match_wait_ns > 0 ? g_match_wait_ns : kWaitNs};
  const int grid = (int)std::max<long long>(1, std::min<long long>(hb.n_items, (long long)num_sms()));
  GLR_LAUNCH("k_match_tc_queue", s,
             kern<<<grid, TC_THREADS, W_SMEM, s>>>(tq, tqa, tk, tka, qb, img_map, n_found, nkc, cfg, bufs, bufcnt,
                                                    taugl, queue, st));
  return GLR_OK;
}

glr_status launch_match_tc(const float* x, const glr_images& im, const int32_t* keys, const int32_t* n_found, int N,
                           const MatchPlan& pl, char* ws, cudaStream_t s) {
  const float* ep = pl.mode == GLR_MATCH_LEARNED ? reinterpret_cast<const float*>(ws + pl.embp_off) : nullptr;
  const float* ek = pl.mode == GLR_MATCH_LEARNED ? reinterpret_cast<const float*>(ws + pl.embk_off) : nullptr;
  // seed bounds read the narrow operand layout only; the minima scan gives a tighter bound
  const int32_t* seed = (g_tc_dump || pl.nkc > 1 || pl.bound_pass) ? nullptr : keys;
  return launch_match_tc_impl(x, im, n_found, pl, ws, g_tc_dump, seed, N, ep, ek, s);
}

// Learned proposal (GLR_MATCH_LEARNED, bound_pass 2): pack the embedding operands (BF16 or
// E4M3 with its per-tensor scale) and run the chunk-minima scan over them.  The FP32
// embeddings and the largest squared norm are in the workspace (k_encode_tc).
glr_status launch_match_emb(const glr_images& im, const int32_t* keys, const int32_t* n_found, int N,
                            const MatchPlan& pl, char* ws, float* dump, cudaStream_t s) {
  const long long npos = (long long)(im.H - im.P + 1) * (im.W - im.P + 1);
  const float* emb = reinterpret_cast<const float*>(ws + pl.embp_off);
  const unsigned* n2 = reinterpret_cast<const unsigned*>(ws + pl.n2_off);
  uint8_t* qop = reinterpret_cast<uint8_t*>(ws + pl.embq_off);
  uint8_t* kop = reinterpret_cast<uint8_t*>(ws + pl.embk_off);
  const bool fp8 = pl.emb_fmt == 1;
  {
    const long long total = (long long)im.n_img * pl.npos_pad;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(total, 256), (long long)num_sms() * 32));
    if (fp8)
      GLR_LAUNCH("k_pack_emb_pos", s,
                 k_pack_emb_pos<true><<<blocks, 256, 0, s>>>(emb, im.n_img, npos, pl.npos_pad, n2, qop));
    else
      GLR_LAUNCH("k_pack_emb_pos", s,
                 k_pack_emb_pos<false><<<blocks, 256, 0, s>>>(emb, im.n_img, npos, pl.npos_pad, n2, qop));
    const int kb = (int)std::max<long long>(1, ceil_div((long long)im.n_img * pl.Npad, 256));
    if (fp8)
      GLR_LAUNCH("k_pack_emb_keys", s,
                 k_pack_emb_keys<true><<<kb, 256, 0, s>>>(emb, keys, n_found, im.n_img, N, pl.Npad, npos, n2, kop));
    else
      GLR_LAUNCH("k_pack_emb_keys", s,
                 k_pack_emb_keys<false><<<kb, 256, 0, s>>>(emb, keys, n_found, im.n_img, N, pl.Npad, npos, n2, kop));
  }
  CUtensorMap tq, tk;
  const uint64_t qrows = (uint64_t)im.n_img * pl.npos_pad, krows = (uint64_t)im.n_img * pl.Npad;
  const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint32_t esz = fp8 ? 1 : 2, box_cols = fp8 ? 32 : 16;
  if (!make_map(&tq, qop, qrows, EMB_COLS, kChunkNT, CU_TENSOR_MAP_SWIZZLE_32B, box_cols, dt, esz) ||
      !make_map(&tk, kop, krows, EMB_COLS, TC_M, CU_TENSOR_MAP_SWIZZLE_32B, box_cols, dt, esz))
    return GLR_ECUDA;
  auto kern = fp8 ? k_match_chunk<CF_EMB_E4M3, kChunkNT> : k_match_chunk<CF_EMB_BF16, kChunkNT>;
  const uint32_t smem = fp8 ? ChunkForm<CF_EMB_E4M3, kChunkNT>::smem : ChunkForm<CF_EMB_BF16, kChunkNT>::smem;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GLR_ECUDA;
  int blocks_per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, CH_THREADS, smem) != cudaSuccess ||
      blocks_per_sm != 1)  // all of TMEM: exactly one resident CTA per SM
    return GLR_ENOTSUP;
  dim3 grid((unsigned)(pl.Npad / TC_M), (unsigned)im.n_img, (unsigned)pl.splits);
  GLR_LAUNCH("k_match_emb", s,
             kern<<<grid, CH_THREADS, smem, s>>>(tq, tq, tk, tk, pl.Npad, npos, pl.npos_pad, pl.tiles_per_split,
                                                 pl.pos_tiles, g_match_wait_ns > 0 ? g_match_wait_ns : kWaitNs,
                                                 reinterpret_cast<StatusBlock*>(ws), dump,
                                                 reinterpret_cast<uint16_t*>(ws + pl.mins_off)));
  return GLR_OK;
}

float* g_tc_dump = nullptr;
unsigned long long g_match_wait_ns = 0;

}  // namespace glr
