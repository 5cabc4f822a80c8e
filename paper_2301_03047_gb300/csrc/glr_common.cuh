// Shared definitions of the GLR CUDA library (device and host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/glr.h"

namespace glr {

// ---------------------------------------------------------------------------
// status block: the first 256 bytes of every workspace
// ---------------------------------------------------------------------------
struct StatusBlock {
  uint32_t bits;           // GLR_DEV_* flags
  uint32_t cand_overflow;  // streams whose candidate buffer overflowed
  uint32_t svd_noconv;     // groups that reached the sweep cap
  uint32_t sweeps;         // total Jacobi sweeps
  uint32_t groups;         // groups processed
  uint32_t fb_count;       // groups queued for the FP64 low-rank fallback
  unsigned long long cand_appends;  // candidates appended by the top-K streams
  unsigned long long compactions;   // stream compactions
  uint32_t fb_noconv;      // groups the FP64 fallback did not converge within its sweep cap
  uint32_t rank1;          // groups settled by the rank-1 certificate (no Jacobi sweep)
  uint32_t power_steps;    // power steps of the rank-1 certificate (all groups that tried it)
  uint32_t rank1_gram;     // of rank1: settled by the Gram bound (the energy bound did not hold)
  uint32_t gram_evals;     // Gram bounds evaluated
  uint32_t pad[49];
};
static_assert(sizeof(StatusBlock) == 256, "status block is 256 bytes");

constexpr size_t kAlign = 256;
__host__ __device__ inline size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Bump allocator over a caller workspace (host side only computes offsets).
struct WsLayout {
  size_t off = sizeof(StatusBlock);
  size_t take(size_t bytes) {
    size_t o = align_up(off);
    off = o + align_up(bytes);
    return o;
  }
};

// Monotone map float -> uint32 (larger float -> larger uint).
__host__ __device__ inline uint32_t float_order_key(float f) {
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float float_from_order_key(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

#ifdef __CUDACC__
__device__ inline void status_set(StatusBlock* st, uint32_t bit) { atomicOr(&st->bits, bit); }
#endif

// Images of an uneven batch seen by a kernel written for a uniform batch: the kernel's image f
// is image map[f] of the caller's batch, whose pixels start pix_off[] floats into x and whose
// keys (and rows of idx / dist) start key_off[] keys into keys.  map == nullptr: the uniform
// layout (image f at f C H W, keys at f N).
struct ImgMap {
  const int32_t* map = nullptr;
  const int64_t* pix_off = nullptr;
  const int64_t* key_off = nullptr;
#ifdef __CUDACC__
  __device__ __forceinline__ int id(int f) const { return map ? map[f] : f; }
  __device__ __forceinline__ long long pix(int f, long long per_img) const {
    return map ? (long long)pix_off[map[f]] : (long long)f * per_img;
  }
  __device__ __forceinline__ long long key(int f, long long N) const {
    return map ? (long long)key_off[map[f]] : (long long)f * N;
  }
#endif
};

// host: launch counting and optional per-kernel event timing (glr_api.cu)
void note_launch(int n = 1);
// host: streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, cached)
int num_sms();
// host: device address of glr_aggregate_noalloc's scratch array on the current device
// (its first 256 bytes are that entry point's status block; glr_noalloc.cu)
glr_status noalloc_scratch_address(void** out);
void prof_begin(cudaStream_t s);
void prof_end(const char* name, cudaStream_t s);

}  // namespace glr

// Launch a kernel (the variadic part is the <<<...>>> expression) on stream S:
// optional timing events, launch-error check, launch count.
#define GLR_LAUNCH(NAME, S, ...)                 \
  do {                                           \
    ::glr::prof_begin(S);                        \
    __VA_ARGS__;                                 \
    cudaError_t e_ = cudaGetLastError();         \
    if (e_ != cudaSuccess) return GLR_ECUDA;     \
    ::glr::prof_end(NAME, S);                    \
    ::glr::note_launch();                        \
  } while (0)
