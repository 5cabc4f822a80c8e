// Running per-key top-K' over a stream of scores, shared by the FP32 and the
// tensor-core scorers.  A warp serves 32 key rows; lane r holds the state of
// row r: a threshold tau and a candidate buffer (global memory, cap + 32
// entries of {order-preserving score bits, position id}).
//
// One 32-column chunk is pushed in two steps:
//   1. filter   each lane takes the minimum of its row's 32 scores (in
//               registers, a tree of three-input minima: about half an
//               instruction per score) and compares it with its tau; a warp
//               vote gives the rows that have a candidate.
//   2. append   for each such row the warp reads the row from a shared-memory
//               tile (or, without one, through 32 shuffles; lane = column),
//               votes on s < tau and appends the candidates in position order
//               with one coalesced store.
// When a buffer holds more than cap entries the warp compacts it: the new
// threshold is a pivot drawn from 32 sorted samples such that at least K'
// entries lie below it (entries >= pivot are dropped), or, if the sample
// misses, the exact K'-th smallest found by a 4-pass radix select.  The
// buffer therefore always holds every entry that can still be among the K'
// smallest (score, id) pairs of the stream.  At the end of the stream an
// exact compaction leaves exactly the K' smallest, ties by smaller id
// (entries are appended in increasing id order), unless the re-rank takes the
// unreduced buffers and selects the K' best itself (StreamCfg::finish = 0).
//
// Several streams serve one key (column halves of a tile, position splits).
// A compaction that leaves at least K' entries strictly below a value v
// publishes v (atomic min, in shared memory for the streams of one CTA and in
// global memory across CTAs): at least K' scores of the key lie below v, so
// no score >= v can be among its K' smallest, and every stream of the key
// filters against min(own threshold, published value).  The union of the
// streams of a key therefore still contains its K' smallest scores.
#pragma once

#include "glr_common.cuh"

namespace glr {

struct StreamCfg {
  int cap;     // compaction trigger (entries)
  int kp;      // entries kept per stream
  int finish;  // 0: leave the buffers as they are (the re-rank selects the K' best itself)
  unsigned long long wait_ns;  // limit of the pipeline's mbarrier waits (teardown waits keep 1 s)
};

constexpr int kStreamSlots = 17;                      // buffer entries per lane of the compacting warp
constexpr int kStreamMaxEntries = 32 * kStreamSlots;  // cap + 32 <= 544

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exact: keep the kp smallest (key, buffer order) entries of b[0..n).  Returns the new count;
// *tau_key receives the kp-th smallest key.  Warp-collective (uniform arguments).
static __device__ __noinline__ int compact_exact(uint2* b, int n, int kp, unsigned* hist, uint32_t* tau_key) {
  const int lane = threadIdx.x & 31;
  uint2 e[kStreamSlots];
#pragma unroll
  for (int i = 0; i < kStreamSlots; ++i) {
    const int j = lane + 32 * i;
    e[i] = (j < n) ? b[j] : make_uint2(0xffffffffu, 0u);
  }
  uint32_t prefix = 0, pmask = 0;
  int k = kp;  // 1-based rank of the wanted element among those matching the prefix
#pragma unroll 1
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kStreamSlots; ++i) {
      const int j = lane + 32 * i;
      if (j < n && (e[i].x & pmask) == prefix) atomicAdd(&hist[(e[i].x >> shift) & 255u], 1u);
    }
    __syncwarp();
    int loc[8];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      loc[i] = (int)hist[lane * 8 + i];
      sum += loc[i];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - sum;
    const unsigned bal = __ballot_sync(0xffffffffu, excl < k && k <= incl);
    const int owner = __ffs(bal) - 1;
    int sel = 0, before = 0;
    if (lane == owner) {
      int c = excl;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (c + loc[i] >= k) {
          sel = lane * 8 + i;
          before = c;
          break;
        }
        c += loc[i];
      }
    }
    sel = __shfl_sync(0xffffffffu, sel, owner);
    before = __shfl_sync(0xffffffffu, before, owner);
    k -= before;
    prefix |= (uint32_t)sel << shift;
    pmask |= 255u << shift;
    __syncwarp();
  }
  const uint32_t T = prefix;
  int out = 0, ties = 0;
  const unsigned lt_mask = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kStreamSlots; ++i) {
    const int j = lane + 32 * i;
    const bool lt = (j < n) && e[i].x < T;
    const bool eq = (j < n) && e[i].x == T;
    const unsigned eqm = __ballot_sync(0xffffffffu, eq);
    const int tie_rank = ties + __popc(eqm & lt_mask);
    const bool keep = lt || (eq && tie_rank < k);
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    if (keep) b[out + __popc(km & lt_mask)] = e[i];
    out += __popc(km);
    ties += __popc(eqm);
  }
  __syncwarp();
  *tau_key = T;
  return out;
}

// Mid-stream compaction of b[0..n) (warp-collective).  Entries >= te_key (the
// effective threshold) are dropped first; if that is not enough, a pivot from
// 32 sorted samples that leaves between kp and cap - 32 entries strictly
// below it becomes the new threshold, else the exact kp-th smallest.
// Returns the new count; *tau_own gets the stream's new threshold and
// *pub the value to publish (0xffffffff = nothing).
static __device__ __noinline__ int compact_mid(uint2* b, int n, int kp, int cap, uint32_t te_key, unsigned* hist,
                                               float* tau_own, uint32_t* pub) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = lanemask_lt();
  uint2 e[kStreamSlots];
  int below_te = 0;
#pragma unroll
  for (int i = 0; i < kStreamSlots; ++i) {
    const int j = lane + 32 * i;
    e[i] = (j < n) ? b[j] : make_uint2(0xffffffffu, 0u);
    below_te += (j < n && e[i].x < te_key) ? 1 : 0;
  }
  below_te = __reduce_add_sync(0xffffffffu, below_te);
  uint32_t cut = te_key;
  *pub = 0xffffffffu;
  if (below_te > (cap + kp) / 2) {
    // 32 samples (a block of 32 consecutive entries from the middle of the buffer,
    // already in registers), sorted across the warp (bitonic, ascending)
    uint32_t smp = e[0].x;
    {
      const int mid = min(kStreamSlots - 1, max(0, (n / 32) / 2));
#pragma unroll
      for (int i = 0; i < kStreamSlots; ++i)
        if (i == mid) smp = e[i].x;
    }
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const uint32_t o = __shfl_xor_sync(0xffffffffu, smp, j);
        const bool up = ((lane & k) == 0);
        const bool lower = ((lane & j) == 0);
        smp = (lower == up) ? min(smp, o) : max(smp, o);
      }
    }
    const int target = kp + (cap - kp) / 4;
    const int pidx = min(31, max(0, (int)(((long long)target * 32) / n)));
    const uint32_t pivot = min(__shfl_sync(0xffffffffu, smp, pidx), te_key);
    int below = 0;
#pragma unroll
    for (int i = 0; i < kStreamSlots; ++i) below += (lane + 32 * i < n && e[i].x < pivot) ? 1 : 0;
    below = __reduce_add_sync(0xffffffffu, below);
    if (below < kp || below > cap - 32) {
      uint32_t T;
      const int out = compact_exact(b, n, kp, hist, &T);
      *tau_own = float_from_order_key(T);
      *pub = T + 1u;  // the kp kept entries are <= T: at least kp scores lie strictly below T + 1
      return out;
    }
    cut = pivot;
    *pub = pivot;
    *tau_own = float_from_order_key(pivot);
  }
  int out = 0;
#pragma unroll
  for (int i = 0; i < kStreamSlots; ++i) {
    const int j = lane + 32 * i;
    const bool keep = (j < n) && e[i].x < cut;
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    if (keep) b[out + __popc(km & lt_mask)] = e[i];
    out += __popc(km);
  }
  __syncwarp();
  return out;
}

// Per-warp counters (appends, compactions) go to the status block once per stream.
__device__ __forceinline__ void stream_stats_flush(const uint2& stats, StatusBlock* st) {
  if ((threadIdx.x & 31) == 0 && st != nullptr) {
    atomicAdd(&st->cand_appends, (unsigned long long)stats.x);
    atomicAdd(&st->compactions, (unsigned long long)stats.y);
  }
}

// Effective threshold of this lane's row: own threshold and the published bounds.
__device__ __forceinline__ float stream_tau_eff(float tau_own, uint32_t pub_shared, uint32_t pub_global) {
  return fminf(tau_own, float_from_order_key(min(pub_shared, pub_global)));  // 0xffffffff decodes to NaN: ignored
}

// Three-input minimum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Minimum of N register values as a tree of three-input minima: about N / 2
// instructions, depth log3(N).
template <int N>
__device__ __forceinline__ float min_tree3(const float (&a)[N]) {
  if constexpr (N == 1) {
    return a[0];
  } else if constexpr (N == 2) {
    return fminf(a[0], a[1]);
  } else {
    constexpr int M = (N + 2) / 3;
    float b[M];
#pragma unroll
    for (int j = 0; j < N / 3; ++j) b[j] = fmin3(a[3 * j], a[3 * j + 1], a[3 * j + 2]);
    if constexpr (N % 3 == 1) b[N / 3] = a[N - 1];
    if constexpr (N % 3 == 2) b[N / 3] = fminf(a[N - 2], a[N - 1]);
    return min_tree3<M>(b);
  }
}

// Step 1 of a chunk push: rows (bit r = lane r) whose 32 scores contain one
// below their tau.  s = this lane's row scores, column j = position q0 + j;
// columns j >= nvalid do not exist.
__device__ __forceinline__ float stream_min(const float (&s)[32], int nvalid) {
  if (nvalid < 32) {
    float m[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) m[j] = j < nvalid ? s[j] : INFINITY;
    return min_tree3(m);
  }
  return min_tree3(s);
}

__device__ __forceinline__ unsigned stream_filter(const float (&s)[32], int nvalid, float tau) {
  return __ballot_sync(0xffffffffu, stream_min(s, nvalid) < tau);
}

// Step 2: append the candidates of the selected rows.  tile holds the same
// 32 x 32 scores in shared memory, row r at tile + r * ld (lane = column).
// te = effective threshold of this lane's row; tau / cnt / row_buf are its
// own state; pub_sh / pub_gl point at the published bounds of the warp's
// row 0 (row r at + r).
// row_value(r): this lane's column of row r (lane = column).
template <class RowValue>
__device__ __forceinline__ void stream_append_rows(unsigned rows, RowValue row_value, int q0, int nvalid, float te,
                                                   float& tau, int& cnt, uint2* row_buf, const StreamCfg& cfg,
                                                   unsigned* hist, uint32_t* pub_sh, uint32_t* pub_gl, uint2& stats) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = lanemask_lt();
  while (rows) {
    const int r = __ffs(rows) - 1;
    rows &= rows - 1;
    const float t_r = __shfl_sync(0xffffffffu, te, r);
    int c_r = __shfl_sync(0xffffffffu, cnt, r);
    uint2* b_r = reinterpret_cast<uint2*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(row_buf), r));
    const float v = row_value(r);
    const bool c = (lane < nvalid) && v < t_r;
    const unsigned bal = __ballot_sync(0xffffffffu, c);
    if (c) b_r[c_r + __popc(bal & lt_mask)] = make_uint2(float_order_key(v), (unsigned)(q0 + lane));
    c_r += __popc(bal);
    stats.x += __popc(bal);
    if (c_r > cfg.cap) {
      __syncwarp();
      float own = __shfl_sync(0xffffffffu, tau, r);
      stats.y += 1;
      uint32_t pub;
      c_r = compact_mid(b_r, c_r, cfg.kp, cfg.cap, float_order_key(t_r), hist, &own, &pub);
      if (lane == r) {
        tau = own;
        if (pub != 0xffffffffu) {
          atomicMin(pub_sh + r, pub);
          atomicMin(pub_gl + r, pub);
        }
      }
    }
    if (lane == r) cnt = c_r;
  }
  __syncwarp();
}

// The rows from a 32 x 32 shared-memory tile (row r at tile + r * ld).
__device__ __forceinline__ void stream_append(unsigned rows, const float* tile, int ld, int q0, int nvalid, float te,
                                              float& tau, int& cnt, uint2* row_buf, const StreamCfg& cfg,
                                              unsigned* hist, uint32_t* pub_sh, uint32_t* pub_gl, uint2& stats) {
  const int lane = threadIdx.x & 31;
  stream_append_rows(rows, [&](int r) { return tile[r * ld + lane]; }, q0, nvalid, te, tau, cnt, row_buf, cfg, hist,
                     pub_sh, pub_gl, stats);
}

// The rows straight from registers (lane r holds row r's 32 values): a row reaches
// the warp through 32 shuffles.  For kernels without room for the tile.
__device__ __forceinline__ void stream_append_regs(unsigned rows, const float (&s)[32], int q0, int nvalid, float te,
                                                   float& tau, int& cnt, uint2* row_buf, const StreamCfg& cfg,
                                                   unsigned* hist, uint32_t* pub_sh, uint32_t* pub_gl,
                                                   uint2& stats) {
  const int lane = threadIdx.x & 31;
  auto row_value = [&](int r) {
    float mine = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float t = __shfl_sync(0xffffffffu, s[j], r);
      mine = lane == j ? t : mine;
    }
    return mine;
  };
  stream_append_rows(rows, row_value, q0, nvalid, te, tau, cnt, row_buf, cfg, hist, pub_sh, pub_gl, stats);
}

// End of a stream: every buffer keeps exactly its min(cnt, kp) smallest entries.
__device__ __forceinline__ void stream_finish(float& tau, int& cnt, uint2* row_buf, const StreamCfg& cfg,
                                              unsigned* hist) {
  __syncwarp();
  unsigned need = __ballot_sync(0xffffffffu, cnt > cfg.kp);
  while (need) {
    const int r = __ffs(need) - 1;
    need &= need - 1;
    const int c_r = __shfl_sync(0xffffffffu, cnt, r);
    uint2* b_r = reinterpret_cast<uint2*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(row_buf), r));
    uint32_t T;
    const int out = compact_exact(b_r, c_r, cfg.kp, hist, &T);
    if ((threadIdx.x & 31) == r) {
      cnt = out;
      tau = float_from_order_key(T);
    }
  }
}

}  // namespace glr
