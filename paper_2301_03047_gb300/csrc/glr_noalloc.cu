// glr_aggregate_noalloc: aggregation without a caller workspace.
//
// Some callers cannot allocate device memory at the point where they need the
// aggregation step: a plug-in running inside a host framework or inference
// server that owns every device allocation and forbids cudaMalloc on its
// request path, or a real-time capture loop that runs under a fixed memory
// budget and has no workspace to hand in.  For them this entry point takes its
// scratch (the numerator planes, the coverage counts and a status block) from
// a fixed array in device memory that the library reserves when it is loaded.
//
// Properties a caller must know:
//   * The array holds kNoAllocScratchBytes (16 MiB) and is reserved on every
//     GPU that loads the library, until the process exits.
//   * Problems whose scratch does not fit are rejected with GLR_ETOOBIG before
//     anything is launched (scratch = 256 + n_img*C*H*W*8 + n_img*Hq*Wq*4 bytes,
//     each part rounded up to 256 bytes).
//   * Every call shares the same array and leaves its contents behind; each call
//     clears what must start at zero.  Calls whose work overlaps on the GPU
//     (different streams, or several host threads) race on the array and give
//     wrong results: serialise them.
//   * The first call on a device looks up the array's device address (with that
//     device current) and caches it; make that first call before any stream
//     capture on the device.
//   * Device-side conditions (a match id outside the position grid, whose entry is
//     skipped) are recorded in a status block at the start of the array; read it
//     with glr_poll_status(NULL, ...) on the same device after the stream is done.
//   * No cudaMalloc, cudaFree or other allocating routine is called.
#include <mutex>

#include "glr_kernels.cuh"

namespace glr {

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

// Device address of the scratch array on the current device (looked up once per device).
glr_status noalloc_scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GLR_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return GLR_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GLR_OK;
}

}  // namespace glr

using namespace glr;

extern "C" glr_status glr_aggregate_noalloc(const float* groups, const int32_t* idx, const int32_t* n_found,
                                            const glr_images* im, int32_t N, int32_t K, const float* x_in,
                                            float* v_out, void* stream) {
  if (!im || !groups || !idx || !n_found || !x_in || !v_out) return GLR_EINVAL;
  if (im->n_img < 1 || im->C < 1 || im->H < 1 || im->W < 1 || im->P < 1 || im->P > im->H || im->P > im->W ||
      im->P > 16)
    return GLR_EINVAL;
  const long long npos = (long long)(im->H - im->P + 1) * (im->W - im->P + 1);
  if (N < 1 || K < 1 || K > npos) return GLR_EINVAL;
  if ((const void*)v_out == (const void*)groups) return GLR_EINVAL;
  const AggWs L = agg_ws_layout(*im);
  if (L.total > kNoAllocScratchBytes) return GLR_ETOOBIG;
  void* ws = nullptr;
  const glr_status st = noalloc_scratch_address(&ws);
  if (st != GLR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, sizeof(StatusBlock), s) != cudaSuccess) return GLR_ECUDA;
  return launch_aggregate(groups, idx, n_found, *im, N, K, x_in, v_out, static_cast<char*>(ws), L, s);
}
