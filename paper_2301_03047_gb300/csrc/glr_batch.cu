// Uneven batches: glr_match_topk_batch.
//
// The images of a glr_batch are grouped into size classes on the host (at most 8 classes; images
// of one size must have the same number of keys).  A set-up kernel lists each class's images
// (their position in the caller's back-to-back layout) from the device mirrors of the sizes, so
// the call can be captured into a CUDA graph.  Per class, the uniform-batch kernels compute the
// image means, the shifted key patches and the BF16 operands, reading the caller's images through
// that list and writing each class into its slice of one flat operand array.  Then ONE launch of
// the persistent tensor-core scorer walks the work queue of every class's (image, key tile,
// position split) items, and per class the exact re-rank writes the K best matches of every key
// to its rows of idx and dist.
#include <algorithm>
#include <vector>

#include "glr_kernels.cuh"

namespace glr {

namespace {

constexpr int kMaxBatchClasses = 8;

struct ClassSizes {
  int n;
  int H[kMaxBatchClasses], W[kMaxBatchClasses];
};

// img_map[img0[c] + j] = index of the j-th image of class c in the caller's batch (caller order)
__global__ void k_batch_classes(const int32_t* __restrict__ d_H, const int32_t* __restrict__ d_W, int n_img,
                                ClassSizes cls, int32_t* __restrict__ img_map) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int pos = 0;
  for (int c = 0; c < cls.n; ++c)
    for (int i = 0; i < n_img; ++i)
      if (d_H[i] == cls.H[c] && d_W[i] == cls.W[c]) img_map[pos++] = i;
}

struct BatchPlan {
  int n_classes = 0, d = 0, nkc = 1, K = 0, Kp = 0, cap = 0, finish = 0, splits = 1, epi_batch = 2;
  int H[kMaxBatchClasses], W[kMaxBatchClasses], N[kMaxBatchClasses], n[kMaxBatchClasses];
  int Npad[kMaxBatchClasses], ntiles[kMaxBatchClasses], img0[kMaxBatchClasses];
  long long npos[kMaxBatchClasses], npos_pad[kMaxBatchClasses], krow0[kMaxBatchClasses], qrow0[kMaxBatchClasses];
  long long keyv0[kMaxBatchClasses], item0[kMaxBatchClasses];
  long long krows = 0, qrows = 0, keyv_total = 0, n_items = 0;
  size_t map_off, queue_off, mean_off, meanp_off, keyv_off, qmain_off, qaux_off, kmain_off, kaux_off, buf_off,
      bufcnt_off, taugl_off, total;
};

// Host validation and layout; returns GLR_OK and fills pl.
glr_status batch_plan(const glr_batch* b, int K, const glr_match_opts* o, BatchPlan& pl) {
  if (!b || b->n_img < 1 || b->C < 1 || b->P < 1 || b->P > 16 || !b->H || !b->W || !b->N || !b->d_H || !b->d_W ||
      !b->d_pix_off || !b->d_key_off)
    return GLR_EINVAL;
  if (K < 1) return GLR_EINVAL;
  if (o && o->mode != GLR_MATCH_BF16) return GLR_ENOTSUP;  // the batch path is the tensor-core form
  if (o && (o->k_over < 0 || o->splits < 0 || o->cap < 0 || (o->k_over > 0 && o->k_over < K))) return GLR_EINVAL;
  if (o && o->cap > 512) return GLR_ENOTSUP;
  const int d = b->C * b->P * b->P;
  if (d > 640 || K > 128) return GLR_ENOTSUP;
  pl.d = d;
  pl.K = K;
  pl.nkc = (d + 63) / 64;
  // size classes, largest images first (their items lead the work queue)
  std::vector<int> order(b->n_img);
  for (int i = 0; i < b->n_img; ++i) {
    if (b->H[i] < b->P || b->W[i] < b->P) return GLR_EINVAL;
    const long long np = (long long)(b->H[i] - b->P + 1) * (b->W[i] - b->P + 1);
    if (b->N[i] < 1 || b->N[i] > np || K > np) return GLR_EINVAL;
    if ((long long)b->H[i] * b->W[i] > (1LL << 30)) return GLR_EINVAL;
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return (long long)b->H[a] * b->W[a] > (long long)b->H[c] * b->W[c];
  });
  for (int i : order) {
    int c = 0;
    while (c < pl.n_classes && !(pl.H[c] == b->H[i] && pl.W[c] == b->W[i])) ++c;
    if (c == pl.n_classes) {
      if (pl.n_classes == kMaxBatchClasses) return GLR_ENOTSUP;
      pl.H[c] = b->H[i];
      pl.W[c] = b->W[i];
      pl.N[c] = b->N[i];
      pl.n[c] = 0;
      ++pl.n_classes;
    }
    if (pl.N[c] != b->N[i]) return GLR_EINVAL;  // one key count per size
    ++pl.n[c];
  }
  pl.Kp = (o && o->k_over > 0) ? o->k_over : K + 16;
  pl.cap = (o && o->cap > 0) ? o->cap : std::min(std::max(2 * pl.Kp + 64, 256), 512 - 32);
  pl.cap = pl.cap / 32 * 32;
  if (pl.Kp > 256 || pl.Kp >= pl.cap) return GLR_ENOTSUP;
  pl.epi_batch = (o && o->epi_batch == 4) ? 4 : 2;
  long long ktiles = 0;
  int img0 = 0;
  for (int c = 0; c < pl.n_classes; ++c) {
    pl.Npad[c] = (pl.N[c] + 127) / 128 * 128;
    pl.npos[c] = (long long)(pl.H[c] - b->P + 1) * (pl.W[c] - b->P + 1);
    pl.ntiles[c] = (int)((pl.npos[c] + 255) / 256);
    pl.npos_pad[c] = (long long)pl.ntiles[c] * 256;
    pl.img0[c] = img0;
    img0 += pl.n[c];
    pl.krow0[c] = pl.krows;
    pl.qrow0[c] = pl.qrows;
    pl.keyv0[c] = pl.keyv_total;
    pl.krows += (long long)pl.n[c] * pl.Npad[c];
    pl.qrows += (long long)pl.n[c] * pl.npos_pad[c];
    pl.keyv_total += (long long)pl.n[c] * pl.Npad[c] * d;
    ktiles += (long long)pl.n[c] * (pl.Npad[c] / 128);
  }
  // position splits: enough items to fill the SMs; the re-rank holds every stream of a key
  const int max_splits = std::max(1, 2048 / (2 * pl.Kp));
  int sp = (o && o->splits > 0) ? o->splits : (int)std::max<long long>(1, (num_sms() + ktiles - 1) / ktiles);
  pl.splits = std::max(1, std::min(sp, max_splits));
  pl.finish = 2LL * pl.splits * (pl.cap + 32) <= 2048 ? 0 : 1;
  for (int c = 0; c < pl.n_classes; ++c) {
    pl.item0[c] = pl.n_items;
    pl.n_items += (long long)pl.n[c] * (pl.Npad[c] / 128) * pl.splits;
  }
  WsLayout L;
  pl.map_off = L.take((size_t)b->n_img * 4);
  pl.queue_off = L.take(256);
  pl.mean_off = L.take((size_t)b->n_img * 4);
  pl.meanp_off = L.take((size_t)b->n_img * kMeanMaxSlices * 8);
  pl.keyv_off = L.take((size_t)pl.keyv_total * 4);
  const int rowlen = pl.nkc * 64;
  pl.qmain_off = L.take((size_t)pl.qrows * rowlen * 2);
  pl.qaux_off = L.take((size_t)pl.qrows * 16 * 2);
  pl.kmain_off = L.take((size_t)pl.krows * rowlen * 2);
  pl.kaux_off = L.take((size_t)pl.krows * 16 * 2);
  const long long nstreams = pl.krows * pl.splits * 2;
  pl.buf_off = L.take((size_t)nstreams * (pl.cap + 32) * 8);
  pl.bufcnt_off = L.take((size_t)nstreams * 4);
  pl.taugl_off = L.take((size_t)pl.krows * 4);
  pl.total = L.off;
  return GLR_OK;
}

}  // namespace

}  // namespace glr

using namespace glr;

extern "C" {

size_t glr_workspace_size_batch(const glr_batch* b, int32_t K, const glr_match_opts* opts) {
  BatchPlan pl;
  return batch_plan(b, K, opts, pl) == GLR_OK ? pl.total : 0;
}

glr_status glr_match_topk_batch(const float* x, const glr_batch* b, const int32_t* keys, const int32_t* n_found,
                                int32_t K, const glr_match_opts* opts, int32_t* idx, float* dist, void* ws,
                                size_t ws_bytes, void* stream) {
  if (!x || !keys || !n_found || !idx || !ws) return GLR_EINVAL;
  BatchPlan pl;
  glr_status st = batch_plan(b, K, opts, pl);
  if (st != GLR_OK) return st;
  if (((uintptr_t)ws % 256) != 0) return GLR_EINVAL;
  if (ws_bytes < pl.total) return GLR_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)ws;
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(w);
  if (cudaMemsetAsync(w, 0, sizeof(StatusBlock), s) != cudaSuccess) return GLR_ECUDA;
  int32_t* img_map = reinterpret_cast<int32_t*>(w + pl.map_off);
  {
    ClassSizes cls{};
    cls.n = pl.n_classes;
    for (int c = 0; c < pl.n_classes; ++c) {
      cls.H[c] = pl.H[c];
      cls.W[c] = pl.W[c];
    }
    GLR_LAUNCH("k_batch_classes", s, k_batch_classes<<<1, 32, 0, s>>>(b->d_H, b->d_W, b->n_img, cls, img_map));
  }
  float* mean = reinterpret_cast<float*>(w + pl.mean_off);
  double* meanp = reinterpret_cast<double*>(w + pl.meanp_off);
  float* keyv = reinterpret_cast<float*>(w + pl.keyv_off);
  __nv_bfloat16* qmain = reinterpret_cast<__nv_bfloat16*>(w + pl.qmain_off);
  __nv_bfloat16* qaux = reinterpret_cast<__nv_bfloat16*>(w + pl.qaux_off);
  __nv_bfloat16* kmain = reinterpret_cast<__nv_bfloat16*>(w + pl.kmain_off);
  __nv_bfloat16* kaux = reinterpret_cast<__nv_bfloat16*>(w + pl.kaux_off);
  uint2* bufs = reinterpret_cast<uint2*>(w + pl.buf_off);
  int* bufcnt = reinterpret_cast<int*>(w + pl.bufcnt_off);
  uint32_t* taugl = reinterpret_cast<uint32_t*>(w + pl.taugl_off);
  if (cudaMemsetAsync(taugl, 0xff, (size_t)pl.krows * 4, s) != cudaSuccess) return GLR_ECUDA;
  const int rowlen = pl.nkc * 64;
  for (int c = 0; c < pl.n_classes; ++c) {
    const glr_images im{pl.n[c], b->C, pl.H[c], pl.W[c], b->P};
    const ImgMap imap{img_map + pl.img0[c], b->d_pix_off, b->d_key_off};
    st = launch_image_mean(x, im, mean + pl.img0[c], meanp + (size_t)pl.img0[c] * kMeanMaxSlices, s, imap);
    if (st != GLR_OK) return st;
    float* kv = keyv + pl.keyv0[c];
    st = launch_key_vectors(x, mean + pl.img0[c], keys, n_found, im, pl.N[c], pl.Npad[c], kv, sb, imap, s);
    if (st != GLR_OK) return st;
    st = launch_pack_class_w(x, mean + pl.img0[c], im, pl.npos_pad[c], pl.nkc, kv, pl.Npad[c],
                             qmain + (size_t)pl.qrow0[c] * rowlen, qaux + (size_t)pl.qrow0[c] * 16,
                             kmain + (size_t)pl.krow0[c] * rowlen, kaux + (size_t)pl.krow0[c] * 16, imap, s);
    if (st != GLR_OK) return st;
  }
  QBatchHost hb{};
  hb.n_classes = pl.n_classes;
  hb.splits = pl.splits;
  hb.n_items = pl.n_items;
  for (int c = 0; c < pl.n_classes; ++c) {
    const int tps = (pl.ntiles[c] + pl.splits - 1) / pl.splits;
    hb.c[c] = QClassHost{pl.n[c], pl.Npad[c], pl.N[c], pl.ntiles[c], tps, pl.img0[c],
                         pl.npos[c], pl.npos_pad[c], pl.krow0[c], pl.qrow0[c], pl.item0[c]};
  }
  st = launch_match_tc_queue(hb, img_map, n_found, pl.nkc, pl.cap, pl.Kp, pl.finish, pl.epi_batch, qmain, qaux,
                             kmain, kaux, pl.qrows, pl.krows, bufs, bufcnt, taugl,
                             reinterpret_cast<unsigned*>(w + pl.queue_off), sb, s);
  if (st != GLR_OK) return st;
  const int spk = 2 * pl.splits;
  for (int c = 0; c < pl.n_classes; ++c) {
    const glr_images im{pl.n[c], b->C, pl.H[c], pl.W[c], b->P};
    const ImgMap imap{img_map + pl.img0[c], b->d_pix_off, b->d_key_off};
    st = launch_rerank_streams(x, keys, n_found, im, pl.N[c], pl.Npad[c], K, spk, pl.cap, pl.Kp, pl.finish,
                               bufs + (size_t)pl.krow0[c] * spk * (pl.cap + 32), bufcnt + (size_t)pl.krow0[c] * spk,
                               idx, dist, imap, s);
    if (st != GLR_OK) return st;
  }
  return GLR_OK;
}

}  // extern "C"
