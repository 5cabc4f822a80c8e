// Running per-key top-K' over a stream of scores, shared by the FP32 and the
// tensor-core scorers.  Each lane of a warp owns one key row; the 32 lanes
// push 32-column chunks of their rows in lock step.
//
//   * A lane keeps a threshold tau and a candidate buffer (global memory,
//     cap + 32 entries of {order-preserving score bits, position id}).
//     A score s < tau is appended; a chunk whose minimum is >= tau for every
//     lane costs one min-reduction and a warp vote.
//   * When a lane's buffer holds more than cap entries the whole warp
//     compacts it: a 4-pass 8-bit radix select finds the K'-th smallest
//     score, entries below it are kept, and among entries equal to it the
//     earliest (= smallest position ids, since a stream is scanned in
//     increasing id order) fill the remaining slots.  tau becomes the K'-th
//     smallest score; later equal scores have larger ids and lose the tie.
//   * The buffer therefore always contains the K' smallest (score, id) pairs
//     seen so far, plus at most cap + 32 - K' others.
#pragma once

#include "glr_common.cuh"

namespace glr {

struct StreamCfg {
  int cap;  // compaction trigger (entries)
  int kp;   // entries kept by a compaction
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Compact the buffer of lane L to its kp smallest (key, id) entries.  All 32 lanes call.
static __device__ __noinline__ void stream_compact(int L, float& tau, int& cnt, uint2* buf, int kp, unsigned* hist) {
  const int lane = threadIdx.x & 31;
  const int n = __shfl_sync(0xffffffffu, cnt, L);
  uint2* b = reinterpret_cast<uint2*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(buf), L));
  __syncwarp();
  if (n <= kp) return;
  uint32_t prefix = 0, pmask = 0;
  int k = kp;  // 1-based rank of the wanted element among those matching the prefix
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint32_t key = b[i].x;
      if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
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
  const uint32_t T = prefix;  // kp-th smallest key; keep k entries equal to T
  int out = 0, ties = 0;
  const unsigned lt_mask = lanemask_lt();
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    uint2 e = make_uint2(0xffffffffu, 0u);
    if (i < n) e = b[i];
    const bool lt = (i < n) && e.x < T;
    const bool eq = (i < n) && e.x == T;
    const unsigned eqm = __ballot_sync(0xffffffffu, eq);
    const int tie_rank = ties + __popc(eqm & lt_mask);
    const bool keep = lt || (eq && tie_rank < k);
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) b[out + __popc(km & lt_mask)] = e;
    out += __popc(km);
    ties += __popc(eqm);
    __syncwarp();
  }
  if (lane == L) {
    cnt = out;
    tau = float_from_order_key(T);
  }
  __syncwarp();
}

// Push one 32-column chunk of this lane's row: s[j] is the score of position q0 + j,
// columns j >= nvalid do not exist.  All 32 lanes call with the same q0 / nvalid.
template <int NC>
__device__ __forceinline__ void stream_push(const float (&s)[NC], int q0, int nvalid, float& tau, int& cnt,
                                            uint2* buf, const StreamCfg& cfg, unsigned* hist) {
  float m = INFINITY;
#pragma unroll
  for (int j = 0; j < NC; ++j) m = fminf(m, j < nvalid ? s[j] : INFINITY);
  const bool any = m < tau;
  if (__any_sync(0xffffffffu, any)) {
    if (any) {
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        if (j < nvalid && s[j] < tau) {
          buf[cnt] = make_uint2(float_order_key(s[j]), (unsigned)(q0 + j));
          ++cnt;
        }
      }
    }
    __syncwarp();
    unsigned need = __ballot_sync(0xffffffffu, cnt > cfg.cap);
    while (need) {
      const int L = __ffs(need) - 1;
      need &= need - 1;
      stream_compact(L, tau, cnt, buf, cfg.kp, hist);
    }
  }
}

// End of a stream: bring every buffer down to kp entries.
__device__ __forceinline__ void stream_finish(float& tau, int& cnt, uint2* buf, const StreamCfg& cfg,
                                              unsigned* hist) {
  __syncwarp();
  unsigned need = __ballot_sync(0xffffffffu, cnt > cfg.kp);
  while (need) {
    const int L = __ffs(need) - 1;
    need &= need - 1;
    stream_compact(L, tau, cnt, buf, cfg.kp, hist);
  }
}

}  // namespace glr
