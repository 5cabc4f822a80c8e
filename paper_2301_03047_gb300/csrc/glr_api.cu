// C ABI of the GLR library: argument validation, workspace layout and launch
// sequencing.  Every entry point validates on the host before launching
// anything and never allocates device memory.
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "glr_kernels.cuh"

namespace glr {

static std::atomic<unsigned long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// Streaming multiprocessors of the current device, read once per device (grid sizing).
static std::atomic<int> g_sm_count[64];
int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = g_sm_count[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 152;
  g_sm_count[dev].store(n, std::memory_order_relaxed);
  return n;
}

// ---- optional per-kernel event timing (host side, single-threaded use)
namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
constexpr int kProfPool = 8192;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;  // pool, first g_prof_used entries recorded
int g_prof_used = 0;
bool g_prof_pending = false;  // prof_begin recorded `a` of entry g_prof_used
}  // namespace

void prof_begin(cudaStream_t s) {
  g_prof_pending = false;
  if (!g_prof_on || g_prof_used >= (int)g_prof.size()) return;
  if (cudaEventRecord(g_prof[g_prof_used].a, s) == cudaSuccess) g_prof_pending = true;
}
void prof_end(const char* name, cudaStream_t s) {
  if (!g_prof_pending) return;
  g_prof_pending = false;
  ProfRec& r = g_prof[g_prof_used];
  if (cudaEventRecord(r.b, s) != cudaSuccess) return;
  r.name = name;
  ++g_prof_used;
}

static bool images_ok(const glr_images* im) {
  if (!im) return false;
  if (im->n_img < 1 || im->C < 1 || im->H < 1 || im->W < 1 || im->P < 1) return false;
  if (im->P > im->H || im->P > im->W || im->P > 16) return false;
  if ((long long)im->H * im->W > (1LL << 30)) return false;
  if ((long long)im->n_img * im->C * im->H * im->W > (1LL << 36)) return false;
  return true;
}
static long long npos_of(const glr_images* im) { return (long long)(im->H - im->P + 1) * (im->W - im->P + 1); }
static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

static glr_status begin_ws(void* ws, size_t ws_bytes, size_t need, cudaStream_t s) {
  if (!ws) return GLR_EINVAL;
  if (!aligned(ws, kAlign)) return GLR_EINVAL;
  if (ws_bytes < need) return GLR_ENOMEM;
  if (cudaMemsetAsync(ws, 0, sizeof(StatusBlock), s) != cudaSuccess) return GLR_ECUDA;
  return GLR_OK;
}

}  // namespace glr

using namespace glr;

extern "C" {

const char* glr_status_string(glr_status s) {
  switch (s) {
    case GLR_OK: return "GLR_OK";
    case GLR_EINVAL: return "GLR_EINVAL: invalid argument";
    case GLR_ECUDA: return "GLR_ECUDA: CUDA runtime error";
    case GLR_ENOMEM: return "GLR_ENOMEM: workspace too small";
    case GLR_ETIMEDOUT: return "GLR_ETIMEDOUT: bounded device wait expired";
    case GLR_ENOTSUP: return "GLR_ENOTSUP: shape or mode not supported by this build";
    case GLR_EDEVICE: return "GLR_EDEVICE: device-side error flag set";
    case GLR_ETOOBIG: return "GLR_ETOOBIG: problem exceeds the 16 MiB scratch of the no-allocation entry point";
    default: return "GLR_?: unknown status";
  }
}

uint64_t glr_launch_count(void) { return (uint64_t)g_launches.load(); }

const char* glr_version(void) { return "glr-gb300 0.1 (sm_103a)"; }

glr_status glr_profile_enable(int32_t on) {
  if (on && g_prof.empty()) {
    g_prof.resize(kProfPool);
    for (auto& r : g_prof) {
      if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
        g_prof.clear();
        return GLR_ECUDA;
      }
    }
  }
  g_prof_on = on != 0;
  g_prof_used = 0;
  return GLR_OK;
}

int32_t glr_profile_collect(char* names, float* total_ms, int32_t* launches, int32_t cap) {
  std::map<std::string, std::pair<double, int>> agg;
  std::vector<std::string> order;
  for (int i = 0; i < g_prof_used; ++i) {
    ProfRec& r = g_prof[i];
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return -1;
    auto it = agg.find(r.name);
    if (it == agg.end()) {
      order.push_back(r.name);
      agg[r.name] = {ms, 1};
    } else {
      it->second.first += ms;
      it->second.second += 1;
    }
  }
  g_prof_used = 0;
  int n = 0;
  for (const auto& nm : order) {
    if (n >= cap) break;
    if (names) {
      strncpy(names + 48 * n, nm.c_str(), 47);
      names[48 * n + 47] = 0;
    }
    if (total_ms) total_ms[n] = (float)agg[nm].first;
    if (launches) launches[n] = agg[nm].second;
    ++n;
  }
  return n;
}

size_t glr_workspace_size(int32_t op, const glr_images* im, int32_t N, int32_t K, const glr_match_opts* opts) {
  if (!images_ok(im)) return 0;
  const long long npos = npos_of(im);
  switch (op) {
    case GLR_OP_SELECT:
      if (N < 1 || N > npos || N > 16384) return 0;
      return select_ws_layout(*im, N).total;
    case GLR_OP_MATCH:
      if (N < 1 || K < 1 || K > 128 || K > npos) return 0;
      return match_plan(*im, N, K, opts).total;
    case GLR_OP_LOWRANK: {
      if (N < 1) return 0;
      WsLayout L;
      L.take((size_t)im->n_img * N * 4);  // queue of the FP64 fallback
      return L.off;
    }
    case GLR_OP_ADMM: {
      WsLayout L;
      L.take((size_t)im->n_img * sizeof(double));  // residual accumulators
      return L.off;
    }
    case GLR_OP_AGGREGATE:
      return agg_ws_layout(*im).total;
    case GLR_OP_ENCODER: {
      WsLayout L;
      L.take((size_t)im->n_img * 4);             // image means
      L.take((size_t)GLR_ENCODER_PARAMS * 4);    // gradient
      L.take((size_t)im->n_img * kMeanMaxSlices * 8);  // partial sums of the means
      return L.off;
    }
    default:
      return 0;
  }
}

glr_status glr_select_keys(const float* x, const glr_images* im, float edge_th, int32_t N, int32_t* keys,
                           int32_t* n_found, int32_t* n_corner, void* ws, size_t ws_bytes, void* stream) {
  return glr_select_keys_mixed(x, im, edge_th, N, 0, keys, n_found, n_corner, ws, ws_bytes, stream);
}

glr_status glr_select_keys_mixed(const float* x, const glr_images* im, float edge_th, int32_t N, int32_t n_uniform,
                                 int32_t* keys, int32_t* n_found, int32_t* n_corner, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (n_uniform < 0 || n_uniform > N) return GLR_EINVAL;
  if (!images_ok(im) || !x || !keys || !n_found) return GLR_EINVAL;
  if (!(edge_th >= 0.f) || !aligned(x, 4) || !aligned(keys, 4)) return GLR_EINVAL;
  const long long npos = npos_of(im);
  if (N < 1 || N > npos) return GLR_EINVAL;
  if (N > 16384) return GLR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const SelectWs L = select_ws_layout(*im, N);
  glr_status st = begin_ws(ws, ws_bytes, L.total, s);
  if (st != GLR_OK) return st;
  return launch_select(x, *im, edge_th, N, n_uniform, keys, n_found, n_corner, (char*)ws, L, s);
}

glr_status glr_match_topk(const float* x, const glr_images* im, const int32_t* keys, const int32_t* n_found,
                          int32_t N, int32_t K, const glr_match_opts* opts, int32_t* idx, float* dist, void* ws,
                          size_t ws_bytes, void* stream) {
  if (!images_ok(im) || !x || !keys || !n_found || (!idx && !g_tc_dump)) return GLR_EINVAL;
  const long long npos = npos_of(im);
  if (N < 1 || K < 1 || K > npos) return GLR_EINVAL;
  if (K > 128) return GLR_ENOTSUP;
  if (opts && opts->mode != GLR_MATCH_FP32 && opts->mode != GLR_MATCH_BF16 && opts->mode != GLR_MATCH_LEARNED &&
      opts->mode != GLR_MATCH_EDGE && opts->mode != GLR_MATCH_WINDOW)
    return GLR_EINVAL;
  if (opts && opts->mode == GLR_MATCH_WINDOW) {
    if (opts->window < 1 || opts->window > 22) return GLR_EINVAL;
    const int wl = 2 * opts->window + 1;
    if (K > wl * wl || im->H - im->P + 1 < wl || im->W - im->P + 1 < wl) return GLR_EINVAL;
    if (im->C * im->P * im->P > 640) return GLR_ENOTSUP;
  }
  if (opts && opts->mode == GLR_MATCH_EDGE) {
    if (!(opts->edge_th >= 0.f)) return GLR_EINVAL;
    if (4 * im->C * im->P * im->P > 640) return GLR_ENOTSUP;
  }
  if (opts && opts->mode == GLR_MATCH_LEARNED && (!opts->encoder || im->C * im->P * im->P > 64)) return GLR_EINVAL;
  if (opts && (opts->k_over < 0 || opts->splits < 0 || opts->cap < 0 || (opts->k_over > 0 && opts->k_over < K)))
    return GLR_EINVAL;
  if (opts && opts->cap > 512) return GLR_ENOTSUP;
  if (opts && opts->epi_batch != 0 && opts->epi_batch != 2 && opts->epi_batch != 4) return GLR_EINVAL;
  const MatchPlan pl = match_plan(*im, N, K, opts);
  if (pl.Kp > 256 || pl.Kp >= pl.cap) return GLR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  glr_status st = begin_ws(ws, ws_bytes, pl.total, s);
  if (st != GLR_OK) return st;
  return launch_match(x, *im, keys, n_found, N, pl, opts ? opts->encoder : nullptr, idx, dist, (char*)ws, s);
}

uint64_t glr_debug_match_wait_ns(uint64_t ns) {
  const uint64_t old = g_match_wait_ns;
  g_match_wait_ns = ns;
  return old;
}

int32_t glr_debug_wnnm_sweep_cap(int32_t cap) {
  const int32_t old = g_wnnm_sweep_cap;
  g_wnnm_sweep_cap = cap > 0 ? cap : 0;
  return old;
}

glr_status glr_debug_match_scores(const float* x, const glr_images* im, const int32_t* keys,
                                  const int32_t* n_found, int32_t N, int32_t K, float* scores, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!scores) return GLR_EINVAL;
  glr_match_opts o{};
  o.mode = GLR_MATCH_BF16;
  o.bound_pass = -1;  // the raw scores come from the candidate scan
  g_tc_dump = scores;
  glr_status st = glr_match_topk(x, im, keys, n_found, N, K, &o, nullptr, nullptr, ws, ws_bytes, stream);
  g_tc_dump = nullptr;
  return st;
}

glr_status glr_debug_proposal_scores(const float* x, const glr_images* im, const int32_t* keys,
                                     const int32_t* n_found, int32_t N, int32_t K, const float* encoder,
                                     int32_t emb_format, float* scores, void* ws, size_t ws_bytes, void* stream) {
  if (!scores || !encoder || (emb_format != 0 && emb_format != 1)) return GLR_EINVAL;
  glr_match_opts o{};
  o.mode = GLR_MATCH_LEARNED;
  o.encoder = encoder;
  o.bound_pass = 2;
  o.emb_format = emb_format;
  g_tc_dump = scores;
  glr_status st = glr_match_topk(x, im, keys, n_found, N, K, &o, nullptr, nullptr, ws, ws_bytes, stream);
  g_tc_dump = nullptr;
  return st;
}

glr_status glr_encoder_embed(const float* x, const glr_images* im, const float* params, float* emb, void* ws,
                             size_t ws_bytes, void* stream) {
  if (!images_ok(im) || !x || !params || !emb) return GLR_EINVAL;
  if (im->C * im->P * im->P > 64) return GLR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t need = glr_workspace_size(GLR_OP_ENCODER, im, 1, 1, nullptr);
  glr_status st = begin_ws(ws, ws_bytes, need, s);
  if (st != GLR_OK) return st;
  WsLayout L;
  float* mean = reinterpret_cast<float*>((char*)ws + L.take((size_t)im->n_img * 4));
  L.take((size_t)GLR_ENCODER_PARAMS * 4);
  double* part = reinterpret_cast<double*>((char*)ws + L.take((size_t)im->n_img * kMeanMaxSlices * 8));
  st = launch_image_mean(x, *im, mean, part, s);
  if (st != GLR_OK) return st;
  return launch_encode_positions(x, *im, mean, params, emb, nullptr, reinterpret_cast<StatusBlock*>(ws), s);
}

glr_status glr_encoder_train_step(const float* x, const glr_images* im, const int32_t* pairs, int32_t n_pairs,
                                  float* params, float* adam_m, float* adam_v, int32_t step, float lr,
                                  float weight_decay, float* loss, void* ws, size_t ws_bytes, void* stream) {
  if (!images_ok(im) || !x || !pairs || !params || !adam_m || !adam_v || !loss) return GLR_EINVAL;
  if (n_pairs < 1 || step < 1 || !(lr > 0.f) || !(weight_decay >= 0.f)) return GLR_EINVAL;
  if (im->C * im->P * im->P > 64) return GLR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t need = glr_workspace_size(GLR_OP_ENCODER, im, 1, 1, nullptr);
  glr_status st = begin_ws(ws, ws_bytes, need, s);
  if (st != GLR_OK) return st;
  WsLayout L;
  float* mean = reinterpret_cast<float*>((char*)ws + L.take((size_t)im->n_img * 4));
  float* grad = reinterpret_cast<float*>((char*)ws + L.take((size_t)GLR_ENCODER_PARAMS * 4));
  double* part = reinterpret_cast<double*>((char*)ws + L.take((size_t)im->n_img * kMeanMaxSlices * 8));
  st = launch_image_mean(x, *im, mean, part, s);
  if (st != GLR_OK) return st;
  return launch_encoder_train(x, *im, mean, pairs, n_pairs, params, adam_m, adam_v, step, lr, weight_decay, grad,
                              loss, s);
}

glr_status glr_lowrank_groups(const float* x, const glr_images* im, const int32_t* idx, const int32_t* n_found,
                              int32_t N, int32_t K, float sigma_w, float c_wnnm, float* groups, int32_t* rank,
                              void* ws, size_t ws_bytes, void* stream) {
  if (!images_ok(im) || !x || !idx || !n_found || !groups) return GLR_EINVAL;
  if (N < 1 || K < 1 || K > npos_of(im)) return GLR_EINVAL;
  if (!(sigma_w >= 0.f) || !(c_wnnm >= 0.f)) return GLR_EINVAL;
  if (!aligned(groups, 16)) return GLR_EINVAL;
  const int d = im->C * im->P * im->P;
  if (d > 640 || K > 128 || d % 4 != 0) return GLR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  glr_status st = begin_ws(ws, ws_bytes, glr_workspace_size(GLR_OP_LOWRANK, im, N, K, nullptr), s);
  if (st != GLR_OK) return st;
  st = launch_gather(x, *im, idx, n_found, N, K, groups, (StatusBlock*)ws, s);
  if (st != GLR_OK) return st;
  WsLayout L;
  int32_t* fb_queue = reinterpret_cast<int32_t*>((char*)ws + L.take((size_t)im->n_img * N * 4));
  if (d <= 64 && K <= 64)
    return launch_wnnm(*im, n_found, N, K, sigma_w, c_wnnm, groups, rank, (StatusBlock*)ws, fb_queue, s);
  // tall groups: Gram matrix + two-sided Jacobi (work O(d K^2) once instead of per sweep)
  if (K <= 32 && d >= 2 * K)
    return launch_gram_wnnm(*im, n_found, N, K, sigma_w, c_wnnm, groups, rank, (StatusBlock*)ws, fb_queue, s);
  return launch_wnnm_smem(*im, false, n_found, N, K, sigma_w, c_wnnm, groups, rank, (StatusBlock*)ws, fb_queue, s);
}

glr_status glr_lowrank_aggregate(const float* x, const glr_images* im, const int32_t* idx, const int32_t* n_found,
                                 int32_t N, int32_t K, float sigma_w, float c_wnnm, float* v_out, int32_t* rank,
                                 void* ws, size_t ws_bytes, void* stream) {
  if (!images_ok(im) || !x || !idx || !n_found || !v_out) return GLR_EINVAL;
  if (N < 1 || K < 1 || K > npos_of(im)) return GLR_EINVAL;
  if (!(sigma_w >= 0.f) || !(c_wnnm >= 0.f)) return GLR_EINVAL;
  if ((const void*)v_out == (const void*)x) return GLR_EINVAL;
  if (im->C * im->P * im->P > 64 || K > 64) return GLR_ENOTSUP;
  const AggWs L = agg_ws_layout(*im);
  cudaStream_t s = (cudaStream_t)stream;
  glr_status st = begin_ws(ws, ws_bytes, L.total, s);
  if (st != GLR_OK) return st;
  return launch_fused_lowrank_aggregate(x, *im, idx, n_found, N, K, sigma_w, c_wnnm, v_out, rank, (char*)ws, L, s);
}

glr_status glr_lowrank_groups_complex(const float* x, const glr_images* im, const int32_t* idx,
                                      const int32_t* n_found, int32_t N, int32_t K, float sigma_w, float c_wnnm,
                                      float* groups, int32_t* rank, void* ws, size_t ws_bytes, void* stream) {
  if (!images_ok(im) || !x || !idx || !n_found || !groups) return GLR_EINVAL;
  if (im->C != 2) return GLR_EINVAL;
  if (N < 1 || K < 1 || K > npos_of(im)) return GLR_EINVAL;
  if (!(sigma_w >= 0.f) || !(c_wnnm >= 0.f)) return GLR_EINVAL;
  if (!aligned(groups, 16)) return GLR_EINVAL;
  const int d = im->C * im->P * im->P;
  if (d > 640 || K > 128 || d % 4 != 0) return GLR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  glr_status st = begin_ws(ws, ws_bytes, glr_workspace_size(GLR_OP_LOWRANK, im, N, K, nullptr), s);
  if (st != GLR_OK) return st;
  st = launch_gather(x, *im, idx, n_found, N, K, groups, (StatusBlock*)ws, s);
  if (st != GLR_OK) return st;
  WsLayout L;
  int32_t* fb_queue = reinterpret_cast<int32_t*>((char*)ws + L.take((size_t)im->n_img * N * 4));
  if (d <= 72 && K <= 64)
    return launch_wnnm_complex_regs(*im, n_found, N, K, sigma_w, c_wnnm, groups, rank, (StatusBlock*)ws, fb_queue, s);
  return launch_wnnm_smem(*im, true, n_found, N, K, sigma_w, c_wnnm, groups, rank, (StatusBlock*)ws, fb_queue, s);
}

glr_status glr_admm_sci_step(const float* y, const float* masks, int64_t mask_group_stride, const float* z,
                             const float* x, float* u, int32_t G, int32_t T, int32_t H, int32_t W, float rho,
                             float* x_out, float* w_out, void* stream) {
  if (!y || !masks || !z || !x || !u || !x_out || !w_out || G < 1 || T < 1 || H < 1 || W < 1) return GLR_EINVAL;
  if (!(rho > 0.f) || !std::isfinite(rho) || mask_group_stride < 0) return GLR_EINVAL;
  if ((long long)G * T * H * W > (1LL << 36)) return GLR_EINVAL;
  if ((const void*)x_out == (const void*)w_out || (const void*)x_out == (const void*)u ||
      (const void*)w_out == (const void*)u || (const void*)x_out == (const void*)z ||
      (const void*)w_out == (const void*)x)
    return GLR_EINVAL;
  return launch_admm_sci(y, masks, mask_group_stride, z, x, u, G, T, (long long)H * W, rho, x_out, w_out,
                         (cudaStream_t)stream);
}

glr_status glr_mosaic_init(const float* y, const float* masks, int64_t mask_group_stride, int32_t G, int32_t T,
                           int32_t H, int32_t W, int32_t s, float* x_out, void* stream) {
  if (!y || !masks || !x_out || G < 1 || T < 1 || H < 1 || W < 1 || s < 1 || s > 16) return GLR_EINVAL;
  if (mask_group_stride < 0 || (long long)G * T * H * W > (1LL << 36)) return GLR_EINVAL;
  if ((const void*)x_out == (const void*)y || (const void*)x_out == (const void*)masks) return GLR_EINVAL;
  return launch_mosaic_init(y, masks, mask_group_stride, G, T, H, W, s, x_out, (cudaStream_t)stream);
}

static bool pow2_side(int32_t n) { return n >= 2 && n <= 4096 && (n & (n - 1)) == 0; }

glr_status glr_fft2(const float* in, float* out, int32_t n_img, int32_t H, int32_t W, int32_t inverse,
                    void* stream) {
  if (!in || !out || n_img < 1) return GLR_EINVAL;
  if (!pow2_side(H) || !pow2_side(W)) return GLR_ENOTSUP;
  if ((long long)n_img * 2 * H * W > (1LL << 34)) return GLR_EINVAL;
  return launch_fft2(in, out, n_img, H, W, inverse != 0, (cudaStream_t)stream);
}

glr_status glr_admm_step(const float* y, const float* mask, const float* z, const float* x, float* u,
                         int32_t n_img, int32_t H, int32_t W, float rho, float* x_out, float* w_out,
                         double* residual, void* ws, size_t ws_bytes, void* stream) {
  if (!y || !mask || !z || !x || !u || !x_out || !w_out || n_img < 1) return GLR_EINVAL;
  if (!(rho > 0.f) || !std::isfinite(rho)) return GLR_EINVAL;
  if (!pow2_side(H) || !pow2_side(W)) return GLR_ENOTSUP;
  if ((long long)n_img * 2 * H * W > (1LL << 34)) return GLR_EINVAL;
  const void* outs[2] = {x_out, w_out};
  for (const void* o : outs)
    if (o == (const void*)y || o == (const void*)mask || o == (const void*)u) return GLR_EINVAL;
  if ((const void*)x_out == (const void*)z || (const void*)w_out == (const void*)x || x_out == w_out)
    return GLR_EINVAL;
  glr_images im{n_img, 2, H, W, 1};
  const size_t need = glr_workspace_size(GLR_OP_ADMM, &im, 1, 1, nullptr);
  cudaStream_t s = (cudaStream_t)stream;
  glr_status st = begin_ws(ws, ws_bytes, need, s);
  if (st != GLR_OK) return st;
  WsLayout L;
  double* acc = reinterpret_cast<double*>((char*)ws + L.take((size_t)n_img * sizeof(double)));
  if (cudaMemsetAsync(acc, 0, (size_t)n_img * sizeof(double), s) != cudaSuccess) return GLR_ECUDA;
  return launch_admm_step(y, mask, z, x, u, n_img, H, W, rho, x_out, w_out, residual, acc, s);
}

glr_status glr_aggregate(const float* groups, const int32_t* idx, const int32_t* n_found, const glr_images* im,
                         int32_t N, int32_t K, const float* x_in, float* v_out, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!images_ok(im) || !groups || !idx || !n_found || !x_in || !v_out) return GLR_EINVAL;
  if (N < 1 || K < 1 || K > npos_of(im)) return GLR_EINVAL;
  if ((const void*)v_out == (const void*)groups) return GLR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const AggWs L = agg_ws_layout(*im);
  glr_status st = begin_ws(ws, ws_bytes, L.total, s);
  if (st != GLR_OK) return st;
  return launch_aggregate(groups, idx, n_found, *im, N, K, x_in, v_out, (char*)ws, L, s);
}

glr_status glr_gap_step(const float* y, const float* masks, int64_t mask_group_stride, const float* v, int32_t G,
                        int32_t T, int32_t H, int32_t W, int32_t accelerate, float* y_acc, float* x_out,
                        void* stream) {
  if (!y || !masks || !x_out) return GLR_EINVAL;
  if (G < 1 || T < 1 || H < 1 || W < 1 || mask_group_stride < 0) return GLR_EINVAL;
  if (accelerate && !y_acc) return GLR_EINVAL;
  if ((long long)G * T * H * W > (1LL << 36)) return GLR_EINVAL;
  return launch_gap_step(y, masks, (long long)mask_group_stride, v, G, T, (long long)H * W, accelerate ? 1 : 0,
                         accelerate ? y_acc : nullptr, x_out, (cudaStream_t)stream);
}

glr_status glr_poll_status(const void* ws, uint32_t* bits, uint32_t* counters, int32_t reset, void* stream) {
  if (!bits) return GLR_EINVAL;
  if (!ws) {
    // the status block of glr_aggregate_noalloc's scratch array on the current device
    void* p = nullptr;
    const glr_status r = noalloc_scratch_address(&p);
    if (r != GLR_OK) return r;
    ws = p;
  }
  cudaStream_t s = (cudaStream_t)stream;
  StatusBlock h;
  if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GLR_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GLR_ECUDA;
  *bits = h.bits;
  if (counters) {
    counters[0] = h.cand_overflow;
    counters[1] = h.svd_noconv;
    counters[2] = h.sweeps;
    counters[3] = h.groups;
    counters[4] = (uint32_t)std::min<unsigned long long>(h.cand_appends, 0xffffffffull);
    counters[5] = (uint32_t)std::min<unsigned long long>(h.compactions, 0xffffffffull);
    counters[6] = h.fb_noconv;
    counters[7] = h.rank1;
    counters[8] = h.power_steps;
    counters[9] = h.rank1_gram;
    counters[10] = h.gram_evals;
  }
  if (reset) {
    if (cudaMemsetAsync(const_cast<void*>(ws), 0, sizeof(StatusBlock), s) != cudaSuccess) return GLR_ECUDA;
  }
  if (h.bits & GLR_DEV_TIMEOUT) return GLR_ETIMEDOUT;
  return (h.bits & (GLR_DEV_NONFINITE | GLR_DEV_BAD_INDEX)) ? GLR_EDEVICE : GLR_OK;
}

}  // extern "C"
