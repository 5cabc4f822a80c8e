// Launch functions of the GLR kernels (host side), one translation unit per step.
#pragma once

#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>

#include "glr_common.cuh"

namespace glr {

// ---- GAP projection (k_gap.cu)
glr_status launch_gap_step(const float* y, const float* masks, long long mstride, const float* v, int G, int T,
                           long long HW, int accelerate, float* y_acc, float* x_out, cudaStream_t s);

// ---- key selection (k_select.cu)
struct SelectWs {
  size_t S_off, R_off, cand_off, cnt_off, bitmap_off, total;
};
SelectWs select_ws_layout(const glr_images& im, int N);
glr_status launch_select(const float* x, const glr_images& im, float th, int N, int n_uniform, int32_t* keys, int32_t* n_found,
                         int32_t* n_corner, char* ws, const SelectWs& L, cudaStream_t s);

// ---- matching (k_match.cu, k_match_tc.cu)
struct MatchPlan {
  int mode;
  int K, Kp;            // matches, candidates kept per stream
  int cap;              // stream compaction trigger (entries; buffers hold cap + 32)
  int splits;           // position splits per key tile
  int subs;             // streams per key and split (column halves inside a tile)
  int streams_per_key;  // splits * subs
  int finish;           // streams end with their exact K' selection (else the re-rank makes it)
  int key_tile;         // keys per CTA
  int Npad;             // N rounded up to key_tile
  int pos_tile;         // positions per scorer tile
  int pos_tiles;        // position tiles per image
  int tiles_per_split;
  int dk;               // BF16 operand row length (elements)
  int nkc;              // 64-column chunks of patch values in a BF16 operand row (1 unless d > 74)
  float edge_th;        // GLR_MATCH_EDGE: threshold of the edge maps
  int window;           // GLR_MATCH_WINDOW: half-width of the search window
  size_t edge_off;      // GLR_MATCH_EDGE: edge planes [n_img][4 C][H][W]
  int epi_batch;        // tensor-core epilogue: 32-column chunks read from TMEM per visit (2 or 4)
  long long npos_pad;   // BF16 position rows per image (pos_tiles * pos_tile)
  int bound_pass;       // tensor-core scorer: minima scan first (bound from half-tile minima)
  size_t mins_off;      // bound_pass 1: half-tile minima [n_img][Npad][2 pos_tiles] float32;
                        // bound_pass 2: 16-bit chunk minima [n_img][Npad][8 pos_tiles]
  size_t ccnt_off, clist_off;  // bound_pass 2: candidate chunks per key (count, the first ids)
  size_t ticket_off;           // bound_pass 2: next key of the exact evaluation (int)
  int emb_fmt;                 // GLR_MATCH_LEARNED, bound_pass 2: proposal operand 0 = BF16, 1 = E4M3
  size_t embq_off, n2_off;     // its position operand rows, the largest squared embedding norm
  size_t mean_off, meanp_off, qn_off, keyv_off, buf_off, bufcnt_off, taugl_off, qpack_off, kpack_off, embp_off, embk_off, total;
};
MatchPlan match_plan(const glr_images& im, int N, int K, const glr_match_opts* o);
glr_status launch_match(const float* x, const glr_images& im, const int32_t* keys, const int32_t* n_found, int N,
                        const MatchPlan& plan, const float* encoder, int32_t* idx, float* dist, char* ws,
                        cudaStream_t s);
// tensor-core scorer (k_match_tc.cu); returns GLR_ENOTSUP when the shape is not covered
glr_status launch_match_tc(const float* x, const glr_images& im, const int32_t* keys, const int32_t* n_found,
                           int N, const MatchPlan& plan, char* ws, cudaStream_t s);
// learned proposal scan over the packed embedding operands (k_match_tc.cu)
glr_status launch_match_emb(const glr_images& im, const int32_t* keys, const int32_t* n_found, int N,
                            const MatchPlan& pl, char* ws, float* dump, cudaStream_t s);
glr_status launch_match_tc_impl(const float* x, const glr_images& im, const int32_t* n_found, const MatchPlan& pl,
                                char* ws, float* dump, const int32_t* seed_keys, int seed_N, const float* emb_pos,
                                const float* emb_keys, cudaStream_t s);

// ---- learned proposal (k_encoder.cu)
glr_status launch_encode_positions(const float* x, const glr_images& im, const float* mean, const float* params,
                                   float* emb, unsigned* n2max, StatusBlock* st, cudaStream_t s);
glr_status launch_encode_vectors(const float* vecs, long long n, int d, const float* params, float* emb,
                                 cudaStream_t s);
// image means: part = scratch of n_img x kMeanMaxSlices doubles
constexpr int kMeanMaxSlices = 256;
glr_status launch_image_mean(const float* x, const glr_images& im, float* mean, double* part, cudaStream_t s,
                             ImgMap imap = ImgMap{});
glr_status launch_encoder_train(const float* x, const glr_images& im, const float* mean, const int32_t* pairs,
                                int n_pairs, float* params, float* m, float* v, int step, float lr, float wd,
                                float* grad, float* loss, cudaStream_t s);

// ---- uneven batches (glr_batch.cu)
struct QClassHost {  // one size class of the persistent scorer's work queue
  int n_img, Npad, N, ntiles, tps, img0;
  long long npos, npos_pad, krow0, qrow0, item0;
};
struct QBatchHost {
  int n_classes, splits;
  long long n_items;
  QClassHost c[8];
};
glr_status launch_pack_class_w(const float* x, const float* mean, const glr_images& im, long long npos_pad, int nkc,
                               const float* keyv, int Npad, __nv_bfloat16* qmain, __nv_bfloat16* qaux,
                               __nv_bfloat16* kmain, __nv_bfloat16* kaux, ImgMap imap, cudaStream_t s);
glr_status launch_match_tc_queue(const QBatchHost& hb, const int32_t* img_map, const int32_t* n_found, int nkc,
                                 int cap, int Kp, int finish, int epi_batch, __nv_bfloat16* qmain,
                                 __nv_bfloat16* qaux, __nv_bfloat16* kmain, __nv_bfloat16* kaux, long long qrows,
                                 long long krows, uint2* bufs, int* bufcnt, uint32_t* taugl, unsigned* queue,
                                 StatusBlock* st, cudaStream_t s);
glr_status launch_key_vectors(const float* x, const float* mean, const int32_t* keys, const int32_t* n_found,
                              const glr_images& im, int N, int Npad, float* keyv, StatusBlock* st, ImgMap imap,
                              cudaStream_t s);
glr_status launch_rerank_streams(const float* x, const int32_t* keys, const int32_t* n_found, const glr_images& im,
                                 int N, int Npad, int K, int streams_per_key, int cap, int Kp, int finish,
                                 const uint2* bufs, const int* bufcnt, int32_t* idx, float* dist, ImgMap imap,
                                 cudaStream_t s);

// testing aid: when set, the tensor-core scorer also writes the raw scores of the
// first position tile, [n_img][Npad][256] float32, to this device buffer
extern float* g_tc_dump;
// testing aid: limit of the tensor-core scorer's pipeline waits in ns (0: 1 s)
extern unsigned long long g_match_wait_ns;

// ---- low-rank step (k_lowrank.cu)
glr_status launch_gather(const float* x, const glr_images& im, const int32_t* idx, const int32_t* n_found, int N,
                         int K, float* groups, StatusBlock* st, cudaStream_t s);
// fb_queue (may be nullptr): groups at the sweep cap are queued for the FP64 fallback instead of
// keeping their FP32 result (the caller then runs launch_wnnm_fp64)
glr_status launch_gram_wnnm(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                            float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue, cudaStream_t s);
glr_status launch_wnnm_smem(const glr_images& im, bool cplx, const int32_t* n_found, int N, int K, float sigma_w,
                            float c_wnnm, float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue,
                            cudaStream_t s);
glr_status launch_edge_planes(const float* x, const glr_images& im, float th, float* planes, cudaStream_t s);
glr_status launch_admm_sci(const float* y, const float* masks, long long mstride, const float* z, const float* x,
                           float* u, int G, int T, long long HW, float rho, float* x_out, float* w_out, cudaStream_t s);
glr_status launch_mosaic_init(const float* y, const float* masks, long long mstride, int G, int T, int H, int W, int s,
                              float* x_out, cudaStream_t st);
glr_status launch_fft2(const float* in, float* out, int n_img, int H, int W, int inverse, cudaStream_t s);
glr_status launch_admm_step(const float* y, const float* mask, const float* z, const float* x, float* u, int n_img,
                            int H, int W, float rho, float* x_out, float* w_out, double* residual, double* res_acc,
                            cudaStream_t s);
glr_status launch_wnnm_fused(const float* x, const glr_images& im, const int32_t* idx, const int32_t* n_found, int N,
                             int K, float sigma_w, float c_wnnm, unsigned long long* num, int* cnt, int32_t* rank,
                             StatusBlock* st, cudaStream_t s);
glr_status launch_wnnm_complex_regs(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w,
                                   float c_wnnm, float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue,
                                   cudaStream_t s);
// fb_queue: n_img * N int32 of scratch for the FP64 fallback (nullptr: no fallback)
glr_status launch_wnnm(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                       float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue, cudaStream_t s);
// FP64 Gram + two-sided Jacobi for the groups queued by the FP32 kernels (k_lowrank_fp64.cu);
// complex groups (cplx) through their real 2m x 2K form; supported while K (2K complex) <= 96
bool wnnm_fp64_supported(int K, bool cplx);
glr_status launch_wnnm_fp64(int d, int K, float sigma_w, float c_wnnm, float* groups, int32_t* rank,
                            const int32_t* queue, StatusBlock* st, cudaStream_t s, bool cplx = false);
// testing aid: sweep cap of the register Jacobi (0: 30)
extern int g_wnnm_sweep_cap;

// ---- aggregation (k_aggregate.cu)
struct AggWs {
  size_t num_off, cnt_off, total;
};
AggWs agg_ws_layout(const glr_images& im);
glr_status launch_fused_lowrank_aggregate(const float* x, const glr_images& im, const int32_t* idx,
                                         const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                                         float* v_out, int32_t* rank, char* ws, const AggWs& L, cudaStream_t s);
glr_status launch_aggregate(const float* groups, const int32_t* idx, const int32_t* n_found, const glr_images& im,
                            int N, int K, const float* x_in, float* v_out, char* ws, const AggWs& L,
                            cudaStream_t s);

}  // namespace glr
