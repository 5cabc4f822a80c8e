/*
 * glr.h -- C ABI of the GB300 global low-rank (GLR) denoising library.
 *
 * The library implements the hot path of "Large-scale Global Low-rank
 * Optimization for Computational Compressed Imaging" (Li et al., 2023):
 * key-patch selection from corners of the edge map (Section 2, Eq. 2-3),
 * global patch matching with a running top-K (Section 2, Eq. 1 made global,
 * Eq. 4 computed as a dense contraction), grouping R~_i x and the WNNM
 * low-rank step (Eq. 5), aggregation, and the GAP projection for the coded
 * aperture model y = sum_t A_t x_t (Eq. 6, Eq. 8).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers owned by the caller, except
 *    where an argument is documented as a host pointer.  The library never
 *    allocates or frees device memory; scratch space is the caller's
 *    workspace `ws` of `ws_bytes` bytes (query the size with
 *    glr_workspace_size; the base must be 256-byte aligned).
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream).  Arguments are validated on the host
 *    before anything is launched; on an error nothing is launched and the
 *    status code says why.  Nothing aborts, exits or traps.
 *  - Device-side conditions (a bounded wait that expired, a group whose SVD
 *    did not converge, a key whose candidate list had to be rebuilt) are
 *    recorded as bits and counters in a status block at the start of the
 *    workspace; read it with glr_poll_status after the stream is done.
 *  - Images: x is float32 [n_img][C][H][W], row-major.  A patch is P x P x C;
 *    its vector index is ch*P*P + dr*P + dc.  Patch positions are the
 *    Hq x Wq = (H-P+1) x (W-P+1) top-left corners (the valid positions of the
 *    Conv2d heat map in Section 2); a position id is q = r*Wq + c.
 *  - Keys, groups and matches are per image: keys int32 [n_img][N],
 *    idx int32 [n_img][N][K], dist float32 [n_img][N][K],
 *    groups float32 [n_img][N][K][C*P*P].
 */
#ifndef GLR_H_
#define GLR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t glr_status;
enum {
  GLR_OK = 0,
  GLR_EINVAL = 1,    /* an argument is out of range or a pointer is NULL/misaligned */
  GLR_ECUDA = 2,     /* a CUDA runtime call failed (launch error, bad stream, ...) */
  GLR_ENOMEM = 3,    /* the workspace is smaller than glr_workspace_size() */
  GLR_ETIMEDOUT = 4, /* a bounded device-side wait expired (status bit set) */
  GLR_ENOTSUP = 5,   /* the shape / mode is valid but not supported by this build */
  GLR_EDEVICE = 6,   /* a device-side error bit is set in the status block */
  GLR_ETOOBIG = 7    /* the problem needs more scratch than glr_aggregate_noalloc reserves */
};

/* Status-block bits (glr_poll_status, `bits`). */
enum {
  GLR_DEV_TIMEOUT = 1u << 0,       /* an mbarrier / flag wait hit its iteration cap */
  GLR_DEV_NONFINITE = 1u << 1,     /* NaN or Inf met in an input */
  GLR_DEV_SVD_NOCONV = 1u << 2,    /* a Jacobi SVD reached its sweep cap */
  GLR_DEV_CAND_OVERFLOW = 1u << 3, /* a candidate buffer overflowed (result still exact, slower) */
  GLR_DEV_BAD_INDEX = 1u << 4      /* a key / match position id was outside 0..Hq*Wq-1 (entry skipped) */
};

/* A batch of equally sized images searched independently. */
typedef struct glr_images {
  int32_t n_img; /* number of images (video frames, MSFA images, ...) */
  int32_t C;     /* channels per image (1 for SCI frames) */
  int32_t H, W;  /* image size */
  int32_t P;     /* patch side; 1 <= P <= min(H, W) */
} glr_images;

/*
 * A batch of images of different sizes (an uneven batch, e.g. multispectral
 * images of several sides, Section 3 MSFA), stored back to back: image i holds
 * C * H[i] * W[i] values of x from d_pix_off[i], its N[i] keys (and the N[i]
 * rows of idx / dist) from d_key_off[i].  C and P are common to all images;
 * images of the same size must have the same N.  The host arrays plan the call;
 * the device arrays (which must hold the same values) are what the kernels read,
 * so a call can be captured into a CUDA graph.
 */
typedef struct glr_batch {
  int32_t n_img;            /* number of images */
  int32_t C;                /* channels per image */
  int32_t P;                /* patch side */
  const int32_t* H;         /* host [n_img]: image heights */
  const int32_t* W;         /* host [n_img]: image widths */
  const int32_t* N;         /* host [n_img]: keys per image */
  const int32_t* d_H;       /* device mirror of H */
  const int32_t* d_W;       /* device mirror of W */
  const int64_t* d_pix_off; /* device [n_img]: first value of image i in x */
  const int64_t* d_key_off; /* device [n_img]: first key of image i in keys (first row of idx / dist) */
} glr_batch;

/* Contraction used by glr_match_topk. */
enum {
  GLR_MATCH_FP32 = 0,   /* plain form: FP32 FMA on the CUDA cores */
  GLR_MATCH_BF16 = 1,   /* chosen form: BF16 tcgen05.mma into TMEM, FP32 accumulate, FP32 re-rank */
  GLR_MATCH_LEARNED = 2, /* learned proposal: k_over candidates by the 16-dim encoder embedding
                           (BF16 tcgen05 contraction), then the exact FP32 re-rank on patches */
  GLR_MATCH_EDGE = 3,    /* the paper's heat map (Eq. 4): binary edge patches (Eq. 2, threshold
                           edge_th) correlated over the four maps and all channels on the tensor
                           cores (0/1 operands: exact); the K largest values, ties by smaller id */
  GLR_MATCH_WINDOW = 4   /* block matching in a local window (Eq. 1 restricted to positions within
                           `window` rows and columns of the key, the baseline the paper's global
                           matching replaces): exact FP32 distances, the K smallest */
};

/* Number of floats of an encoder parameter buffer: W1[64][64], b1[64], W2[16][64], b2[16]. */
#define GLR_ENCODER_PARAMS 5200

typedef struct glr_match_opts {
  int32_t mode;   /* GLR_MATCH_* */
  int32_t k_over; /* candidates kept per key and position split before the exact
                     FP32 re-rank; 0 = default (K+16) */
  int32_t splits; /* position splits per key tile; 0 = automatic */
  int32_t cap;    /* candidates a top-K stream may hold before it compacts
                     (> k_over, <= 512); 0 = automatic */
  const float* encoder; /* GLR_MATCH_LEARNED: device encoder parameters (GLR_ENCODER_PARAMS
                           floats); k_over = candidates per key (0 = 256) */
  int32_t epi_batch;    /* tensor-core epilogue: 32-column chunks read from tensor memory per
                           visit, 2 or 4 (0 = 2) */
  float edge_th;        /* GLR_MATCH_EDGE: the threshold th of Eq. 3 on Sobel output (>= 0) */
  int32_t window;       /* GLR_MATCH_WINDOW: half-width w of the search window, 1 <= w <= 22:
                           the (2w+1)^2 positions centred on the key, shifted inside the
                           position grid at its borders; K <= (2w+1)^2 */
  int32_t bound_pass;   /* tensor-core scorer:
                           2 = one scan that records the minimum BF16 score of every
                             32-position chunk per key, then every chunk whose minimum is
                             at or below the key's K'-th smallest chunk minimum is scored
                             exactly in FP32 (a superset of the K' best BF16 scores), and
                             the K' best of those are re-ranked (GLR_MATCH_BF16 with d <= 74
                             and P in {4, 6, 8}, C P <= 16);
                           1 = a first scan that only records the minimum of every
                             128-position half tile, and a candidate scan started from the
                             bound they give (same matches as -1);
                           -1 = one candidate scan;
                           0 = automatic (2 where it applies, else 1 when d <= 74, else -1).
                           GLR_MATCH_LEARNED: 2 or 0 = one scan over the embedding operands
                             that records the minimum score of every 32-position chunk per
                             key; the chunks at or below the key's K'-th smallest minimum are
                             scored again in FP32 from the same operand values, and the K'
                             best of those re-ranked exactly (positions < 2^24 - 64);
                             1 or -1 = the candidate-stream scan over BF16 embeddings */
  int32_t emb_format;   /* GLR_MATCH_LEARNED with bound_pass 2: the embedding operand of the
                           proposal scan, 0 = BF16 (kind::f16), 1 = FP8 E4M3 with one
                           power-of-two scale per call (kind::f8f6f4) */
} glr_match_opts;

/* Operation codes for glr_workspace_size. */
enum { GLR_OP_SELECT = 1, GLR_OP_MATCH = 2, GLR_OP_LOWRANK = 3, GLR_OP_AGGREGATE = 4, GLR_OP_ENCODER = 5,
       GLR_OP_ADMM = 6 };

/*
 * Workspace bytes needed by one operation.  `opts` is used by GLR_OP_MATCH
 * only and may be NULL (defaults).  Returns 0 for invalid arguments.
 */
size_t glr_workspace_size(int32_t op, const glr_images* im, int32_t N, int32_t K,
                          const glr_match_opts* opts);

/*
 * Key (exemplar) patch selection -- Section 2: the exemplars sit at corners of
 * the averaged binary edge map (edge maps of Eq. 2, threshold function of
 * Eq. 3).
 *
 *   x        [n_img][C][H][W] float32, the current estimate.
 *   edge_th  the threshold th of Eq. 3 (applied to Sobel output).
 *   N        keys per image, 1 <= N <= Hq*Wq.
 *   keys     out, int32 [n_img][N]: position ids in rank order -- corners by
 *            descending integer Harris response (k = 1/25) of the summed
 *            signed edge maps, ties by pixel id, mapped to the patch whose
 *            top-left is (r - P/2, c - P/2) clamped, duplicates dropped;
 *            then a row-major uniform grid of stride max(1, isqrt(Hq*Wq/N))
 *            fills the remaining slots.
 *   n_found  out, int32 [n_img]: number of valid keys (= N).
 *   n_corner out (may be NULL), int32 [n_img]: keys that came from corners.
 * Result is bit-exact given the edge maps (integer arithmetic after Eq. 3).
 */
glr_status glr_select_keys(const float* x, const glr_images* im, float edge_th, int32_t N,
                           int32_t* keys, int32_t* n_found, int32_t* n_corner, void* ws,
                           size_t ws_bytes, void* stream);

/*
 * Corner + uniform exemplar mixes (Section 3: the CACTI experiments add uniformly
 * selected exemplars to the corner-based ones; the matching-strategy comparison
 * uses as many uniform as corner exemplars).  At most N - n_uniform corners (in
 * the rank order above), then the row-major grid of the smallest stride s with
 * ceil(Hq/s) ceil(Wq/s) <= n_uniform (a grid over the whole image), skipping
 * chosen positions, then the stride-isqrt(Hq*Wq/N) grid up to N keys.  0 <= n_uniform <= N;
 * n_uniform = 0 is glr_select_keys.  Same workspace as glr_select_keys.
 */
glr_status glr_select_keys_mixed(const float* x, const glr_images* im, float edge_th, int32_t N,
                                 int32_t n_uniform, int32_t* keys, int32_t* n_found, int32_t* n_corner,
                                 void* ws, size_t ws_bytes, void* stream);

/*
 * Global matching -- Section 2 (Eq. 1 over the entire image; the heat map of
 * Eq. 4 computed as ||p||^2 - 2<p,q> + ||q||^2 for every key p and every
 * position q of the same image, fused with a running per-key top-K so the
 * heat map never reaches memory).
 *
 *   keys     int32 [n_img][N] position ids (from glr_select_keys or the caller).
 *   n_found  int32 [n_img] valid keys per image (<= N); rows beyond are not written.
 *   K        matches per key, 1 <= K <= 128, K <= Hq*Wq.
 *   modes    GLR_MATCH_FP32: d = C*P*P <= 256 and P <= 8; GLR_MATCH_BF16: d <= 640;
 *            GLR_MATCH_LEARNED: d <= 64; GLR_MATCH_EDGE: 4 C P^2 <= 640
 *            (GLR_ENOTSUP / GLR_EINVAL otherwise).
 *            FP32, BF16 and LEARNED select K' = k_over candidates per key by
 *            the scorer's value (FP32 or BF16 expanded-form distance, embedding
 *            distance; ties to smaller ids) and re-rank exactly those K'.
 *            With GLR_MATCH_EDGE, idx is ordered by descending heat-map value H
 *            (ties by smaller id) and dist receives H (an integer count).
 *   idx      out, int32 [n_img][N][K]: the K positions with the smallest
 *            squared L2 distance, ordered by (distance, position id); the key
 *            itself is included (distance 0).
 *   dist     out (may be NULL), float32 [n_img][N][K]: those distances,
 *            recomputed directly as sum((p - q)^2) in FP32.
 */
glr_status glr_match_topk(const float* x, const glr_images* im, const int32_t* keys,
                          const int32_t* n_found, int32_t N, int32_t K,
                          const glr_match_opts* opts, int32_t* idx, float* dist, void* ws,
                          size_t ws_bytes, void* stream);

/*
 * glr_match_topk for an uneven batch (the batching pattern of the project):
 * the same matches per image as glr_match_topk in GLR_MATCH_BF16 mode (K'
 * candidates by the BF16 tensor-core score, exact FP32 re-rank), computed by
 * ONE launch of a persistent tensor-core kernel that claims work items --
 * (image, key tile of 128 keys, position split) over every image of the
 * batch, largest images first -- from a counter until the queue is empty, so
 * the SMs stay busy across image sizes.  The preparation (image means, BF16
 * operands) and the exact re-rank run per size class.
 *   x       float32, the images back to back (see glr_batch).
 *   keys    int32, image i's N[i] position ids from d_key_off[i].
 *   n_found int32 [n_img]: valid keys per image (<= N[i]).
 *   idx, dist: out, rows d_key_off[i] .. + N[i] - 1 of [sum N][K].
 *   opts    NULL or mode GLR_MATCH_BF16 (GLR_ENOTSUP otherwise); k_over,
 *           splits (the same for every image), cap and epi_batch as for
 *           glr_match_topk.
 * Limits: at most 8 different image sizes, d = C P^2 <= 640, K <= 128.
 * Workspace: glr_workspace_size_batch(b, K, opts) bytes (0: invalid).
 */
size_t glr_workspace_size_batch(const glr_batch* b, int32_t K, const glr_match_opts* opts);
glr_status glr_match_topk_batch(const float* x, const glr_batch* b, const int32_t* keys, const int32_t* n_found,
                                int32_t K, const glr_match_opts* opts, int32_t* idx, float* dist, void* ws,
                                size_t ws_bytes, void* stream);

/*
 * Learned matching proposal (the project's learned-proposal pattern; the
 * paper's Outlook only mentions low-rank networks).  The encoder
 * f(p) = W2 relu(W1 p + b1) + b2 maps a mean-shifted patch (d <= 64, zero
 * padded) to 16 values; GLR_MATCH_LEARNED retrieves candidates by
 * ||f(p) - f(q)||^2 and re-ranks them with the exact patch distance.
 * Inference rounds the weights to FP16 and computes in FP32.
 *
 * glr_encoder_embed: emb float32 [n_img][Hq*Wq][16] for every position.
 *
 * glr_encoder_train_step: one AdamW step (lr, weight decay on W1 and W2;
 * betas 0.9 / 0.999, eps 1e-8; `step` >= 1 is the step number for the bias
 * correction) on the loss mean_i w_i (||f(p_i) - f(q_i)||^2 - d_i)^2 with
 * d_i the exact squared distance of the two patches and
 * w_i = 1 / (d_i + 0.05)^2.  pairs int32 [n_pairs][3] = (image, position of
 * p, position of q).  params, adam_m, adam_v: GLR_ENCODER_PARAMS floats each,
 * updated in place (FP32 master).  loss: device float, receives the batch
 * loss before the update.  Workspace: glr_workspace_size(GLR_OP_ENCODER, ...).
 */
glr_status glr_encoder_embed(const float* x, const glr_images* im, const float* params, float* emb, void* ws,
                             size_t ws_bytes, void* stream);
glr_status glr_encoder_train_step(const float* x, const glr_images* im, const int32_t* pairs, int32_t n_pairs,
                                  float* params, float* adam_m, float* adam_v, int32_t step, float lr,
                                  float weight_decay, float* loss, void* ws, size_t ws_bytes, void* stream);

/*
 * Testing aid for the BF16 tensor-core scorer: runs glr_match_topk in
 * GLR_MATCH_BF16 mode (no idx / dist output) and also writes the raw scores
 * ||p~ - q~||^2 of every key against the first 256 positions of its image,
 * float32 [n_img][ceil(N/128)*128][256], to `scores` (device).  p~, q~ are the
 * mean-shifted patches rounded to BF16.  The paper has no counterpart; this
 * exists to check the tensor-core operand layout against a host computation.
 */
glr_status glr_debug_match_scores(const float* x, const glr_images* im, const int32_t* keys,
                                  const int32_t* n_found, int32_t N, int32_t K, float* scores, void* ws,
                                  size_t ws_bytes, void* stream);

/*
 * Testing aid for the learned proposal's scan: runs glr_match_topk in
 * GLR_MATCH_LEARNED mode with bound_pass 2 (no idx / dist output) and also writes
 * the raw scan scores of every key against the first 256 positions of its image,
 * float32 [n_img][ceil(N/128)*128][256], to `scores` (device): the
 * contraction over the 32 operand columns, ||a_q||^2 - 2 <a_p, a_q> + ||a_p||^2
 * with both squared norms carried as three terms of the operand type, for the
 * embedding operands a (BF16 roundings of the embeddings, or E4M3 roundings of
 * s times them, s the per-call power-of-two scale; emb_format 0 or 1).  Exists to check the operand packing and the
 * kind::f16 / kind::f8f6f4 contraction against a host computation.
 */
glr_status glr_debug_proposal_scores(const float* x, const glr_images* im, const int32_t* keys,
                                     const int32_t* n_found, int32_t N, int32_t K, const float* encoder,
                                     int32_t emb_format, float* scores, void* ws, size_t ws_bytes, void* stream);

/*
 * Testing aid for the bounded waits of the tensor-core scorer (BF16, LEARNED and
 * EDGE modes): sets the limit, in nanoseconds of %globaltimer, of the waits
 * between its producer, MMA and epilogue warps for later calls of this process
 * (0: the default of 1 s) and returns the previous setting.  A wait that runs
 * out sets GLR_DEV_TIMEOUT (glr_poll_status then returns GLR_ETIMEDOUT) and the
 * CTA stops its work; the copies and MMAs it already issued are still waited
 * for with the full second, so nothing is in flight when it exits.  The
 * matches of such a call are incomplete.  The paper has no counterpart.  Not
 * thread-safe.
 */
uint64_t glr_debug_match_wait_ns(uint64_t ns);

/*
 * Testing aid for the FP64 fallback of the low-rank step: sets the sweep cap of
 * the FP32 register Jacobi used by glr_lowrank_groups (cap <= 0: the default 30)
 * for later calls of this process and returns the previous setting (0 =
 * default).  Groups that reach the cap are recomputed in FP64 (Gram matrix and a
 * two-sided Jacobi); a small cap sends most groups there.  Not thread-safe.
 */
int32_t glr_debug_wnnm_sweep_cap(int32_t cap);

/*
 * Grouping and low-rank step -- Eq. 5 (R~_i x) solved by WNNM (Section 2).
 * For every key the K matched patches form Y (d x K, d = C*P*P); with
 * Y = U S V^T, sigma_hat_i = sqrt(max(s_i^2 - K sigma_w^2, 0)),
 * tau_i = c_wnnm sigma_w^2 / (sigma_hat_i + 1e-8), s'_i = max(s_i - tau_i, 0),
 * the output is X^ = U diag(s') V^T.  The SVD is a one-sided Jacobi in FP32
 * (columns in registers for d <= 64 and K <= 64, in shared memory otherwise;
 * tall groups with K <= 32 through the Gram matrix).  Groups that reach the
 * 30-sweep cap of any of these paths are recomputed in FP64 (Gram matrix,
 * two-sided Jacobi) by a second kernel in the same call (K <= 96; above that a
 * capped group keeps its FP32 result); the status block counts them
 * (svd_noconv, and fb_noconv for groups the FP64 sweeps cannot finish either).
 *
 *   idx      int32 [n_img][N][K] matches (from glr_match_topk).
 *   groups   out, float32 [n_img][N][K][d]: row j = column j of X^.
 *   rank     out (may be NULL), int32 [n_img][N]: number of s'_i > 0.
 *   ws       glr_workspace_size(GLR_OP_LOWRANK, im, N, K, NULL) bytes (status block
 *            and the FP64 fallback's queue).
 * Limits of this build: d <= 640, K <= 128, d % 4 == 0 (GLR_ENOTSUP otherwise).
 */
glr_status glr_lowrank_groups(const float* x, const glr_images* im, const int32_t* idx,
                              const int32_t* n_found, int32_t N, int32_t K, float sigma_w,
                              float c_wnnm, float* groups, int32_t* rank, void* ws,
                              size_t ws_bytes, void* stream);

/*
 * Grouping, low-rank step and aggregation in one pass (the fused form of
 * glr_lowrank_groups followed by glr_aggregate with x_in = x): each group's K
 * patches are read from x, shrunk exactly as glr_lowrank_groups does, and the
 * estimates are added straight into the aggregation sums, so no group buffer is
 * written.  v_out [n_img][C][H][W] receives what glr_aggregate would, bit for bit
 * (the sums are fixed point; the per-group arithmetic is the same code).
 * rank (may be NULL) as in glr_lowrank_groups.  v_out must not alias x.
 * Limits: d = C P^2 <= 64 and K <= 64 (GLR_ENOTSUP otherwise).
 * Workspace: glr_workspace_size(GLR_OP_AGGREGATE, ...).
 */
glr_status glr_lowrank_aggregate(const float* x, const glr_images* im, const int32_t* idx,
                                 const int32_t* n_found, int32_t N, int32_t K, float sigma_w, float c_wnnm,
                                 float* v_out, int32_t* rank, void* ws, size_t ws_bytes, void* stream);

/*
 * The same step for a complex image (Section 3, MRI): x holds C == 2 planes
 * per image (real, imaginary), so a gathered column is the real half followed
 * by the imaginary half of a complex patch (m = P*P entries).  Y is the complex
 * m x K matrix of the K patches; its SVD Y = U S V^H (one-sided Jacobi with
 * Hermitian rotations, FP32) is shrunk with the same formula, sigma_w being
 * the noise standard deviation per complex entry, and X^ = U diag(s') V^H is
 * written back in the same two-half layout.  Groups at the sweep cap are
 * recomputed in FP64 as the real 2 P^2 x 2K matrix [[Re, -Im], [Im, Re]] (same
 * singular values, each twice) when K <= 48.  Limits: 2 P^2 <= 640, K <= 128.
 * Workspace: glr_workspace_size(GLR_OP_LOWRANK, ...).
 */
glr_status glr_lowrank_groups_complex(const float* x, const glr_images* im, const int32_t* idx,
                                      const int32_t* n_found, int32_t N, int32_t K, float sigma_w,
                                      float c_wnnm, float* groups, int32_t* rank, void* ws,
                                      size_t ws_bytes, void* stream);

/*
 * Aggregation: every group column is added back at its patch position with
 * weight 1 and overlapping estimates are averaged; pixels no patch covers
 * keep x_in.  The sums are accumulated in 64-bit fixed point (2^-32 units), so
 * the result does not depend on the order of the additions (run to run and
 * eager vs graph replay give identical bits).  v_out must not alias groups; it
 * may alias x_in.
 *   groups float32 [n_img][N][K][d], idx int32 [n_img][N][K],
 *   x_in, v_out float32 [n_img][C][H][W].
 */
glr_status glr_aggregate(const float* groups, const int32_t* idx, const int32_t* n_found,
                         const glr_images* im, int32_t N, int32_t K, const float* x_in,
                         float* v_out, void* ws, size_t ws_bytes, void* stream);

/*
 * glr_aggregate without a workspace argument: the same computation and
 * arguments as glr_aggregate, for callers that cannot allocate device memory
 * (a plug-in inside a framework or server that owns all device allocations
 * and forbids cudaMalloc on its request path, or a real-time loop with a fixed
 * memory budget and no workspace to hand in).  The paper has no counterpart;
 * this is a deployment convenience.
 *
 * Scratch comes from a 16 MiB array in device memory that the library
 * reserves on every GPU that loads it, until the process exits.  Problems whose
 * scratch (256 + n_img*C*H*W*8 + n_img*Hq*Wq*4 bytes, each part rounded up to
 * 256) exceeds it return GLR_ETOOBIG without launching.  All calls share the
 * array and leave their contents in it (each call clears what must start at
 * zero); calls that overlap on the GPU race on it, so serialise them.  The
 * first call on a device looks the array's address up with that device
 * current and caches it: make that call before any stream capture.  Device-side
 * conditions (a match id outside the position grid: that entry is skipped) go
 * to a status block in the array; read it with glr_poll_status(NULL, ...) on
 * the same device once the stream is done.  Nothing is allocated or freed.
 */
glr_status glr_aggregate_noalloc(const float* groups, const int32_t* idx, const int32_t* n_found,
                                 const glr_images* im, int32_t N, int32_t K, const float* x_in,
                                 float* v_out, void* stream);

/*
 * GAP projection for y = sum_t A_t x_t (Eq. 6 for video SCI; Eq. 8 for an
 * MSFA with orthogonal masks, Eq. 9, where R == 1):
 *   R = sum_t A_t^2 (0 -> 1),  x_t = v_t + A_t (y - sum_s A_s v_s) / R.
 * With accelerate != 0 (accelerated GAP): y_acc += y - sum_s A_s v_s and y_acc
 * replaces y in the update.  v == NULL means v = 0, which gives the usual
 * start x0 = Phi^T (y / R).
 *
 *   y      float32 [G][H][W]          measurements
 *   masks  float32 [T][H][W] per group, at element stride mask_group_stride
 *          between groups (0 = one mask set shared by all groups)
 *   v, x_out float32 [G][T][H][W]; x_out may alias v.
 *   y_acc  float32 [G][H][W], in/out, required iff accelerate != 0.
 */
glr_status glr_gap_step(const float* y, const float* masks, int64_t mask_group_stride,
                        const float* v, int32_t G, int32_t T, int32_t H, int32_t W,
                        int32_t accelerate, float* y_acc, float* x_out, void* stream);

/*
 * ADMM for y = sum_t A_t x_t (the paper's SCI reconstruction uses GAP or ADMM,
 * Section 2 after Eq. 5), scaled form, after the denoiser z = D(x + u):
 *   u  <- u + x - z                                  (in place)
 *   x'  = w + Phi^T ((y - Phi w) / (R + rho)),  w = z - u,  R = sum_t A_t^2
 *         (the minimiser of ||y - Phi x||^2 + rho ||x - w||^2)      -> x_out
 *   x' + u                                           -> w_out (next denoiser input)
 * y [G][H][W]; masks [T][H][W] per group at element stride mask_group_stride
 * (0 = shared); z, x, u, x_out, w_out [G][T][H][W]; rho > 0.  x_out may alias x,
 * w_out may alias z; no other aliasing.
 */
glr_status glr_admm_sci_step(const float* y, const float* masks, int64_t mask_group_stride, const float* z,
                             const float* x, float* u, int32_t G, int32_t T, int32_t H, int32_t W, float rho,
                             float* x_out, float* w_out, void* stream);

/*
 * Start of multispectral-filter-array demosaicing (Section 3, MSFA; the GAP
 * iterations then refine it): per band t, the normalised convolution of the
 * sampled values with a separable tent of half-width s,
 *   x_t(p) = sum_q w(q - p) A_t(q) y(q) / sum_q w(q - p) A_t(q),
 *   w(dr, dc) = (1 - |dr|/s)(1 - |dc|/s) for |dr|, |dc| < s, q inside the image,
 * which is bilinear interpolation for a periodic mosaic of period s; 0 where
 * no sample of band t is in the window.  The paper gives no initialisation; a
 * zero-filled start leaves the mosaic pattern in every patch and the low-rank
 * step cannot remove it.
 *   y [G][H][W], masks [T][H][W] per group at element stride mask_group_stride
 *   (0 = shared), x_out [G][T][H][W]; 1 <= s <= 16.
 */
glr_status glr_mosaic_init(const float* y, const float* masks, int64_t mask_group_stride, int32_t G, int32_t T,
                           int32_t H, int32_t W, int32_t s, float* x_out, void* stream);

/*
 * Orthonormal 2-D DFT of complex images (the F of the MRI model y = M F(x),
 * Section 3): X[k][l] = sum_{r,c} x[r][c] exp(-+2 pi i (k r / H + l c / W)) / sqrt(H W)
 * (minus sign forward, plus sign when inverse != 0), unshifted (index 0 is
 * frequency 0).  in, out: float32 [n_img][2][H][W] (real plane, imaginary
 * plane); out may alias in.  H and W are powers of two in [2, 4096].  FP32
 * radix-2 transforms of the rows and then of the columns; no workspace.
 */
glr_status glr_fft2(const float* in, float* out, int32_t n_img, int32_t H, int32_t W, int32_t inverse,
                    void* stream);

/*
 * One ADMM step after the denoiser for y = M F(x) (Section 3, MRI; ADMM
 * ref. [26]), scaled form, given x (previous data-consistent image), z (the
 * denoiser output D(x + u)) and u:
 *   u   <- u + x - z                                  (in place)
 *   x'   = F^-1((M y + rho F(z - u)) / (M + rho))      -> x_out
 *   w    = x' + u                                      -> w_out (next denoiser input)
 *   residual[i] = ||M F(x') - y||_2 of image i, accumulated in FP64 (F(x') is
 *   the k-space array the step inverts, so no extra transform is needed).
 * y (k-space, zero where M = 0), z, x, u, x_out, w_out: float32
 * [n_img][2][H][W]; mask float32 [n_img][H][W] (>= 0, normally 0/1); rho > 0;
 * residual: device double [n_img] (may be NULL).  x_out may alias x, w_out may
 * alias z; no other aliasing.  H, W powers of two in [2, 4096].
 * Workspace: glr_workspace_size(GLR_OP_ADMM, im with n_img, H, W, ...).
 */
glr_status glr_admm_step(const float* y, const float* mask, const float* z, const float* x, float* u,
                         int32_t n_img, int32_t H, int32_t W, float rho, float* x_out, float* w_out,
                         double* residual, void* ws, size_t ws_bytes, void* stream);

/*
 * Reads the status block of a workspace used by an earlier call (blocks on
 * `stream`).  ws == NULL reads the status block of glr_aggregate_noalloc's
 * scratch array on the current device instead.  bits = OR of GLR_DEV_*;
 * counters (may be NULL) receives 11 uint32 values: [0] keys whose candidate
 * buffer overflowed, [1] groups whose SVD hit the FP32 sweep cap, [2] total
 * Jacobi sweeps, [3] groups processed, [4] candidates appended by the matching
 * top-K streams or candidate chunks of the chunk form (saturating), [5] top-K
 * stream compactions (saturating), [6] groups whose FP64 fallback also reached
 * its sweep cap, [7] groups settled by the rank-1 certificate without sweeps,
 * [8] power steps the certificate took (over every group that tried it), [9]
 * groups of [7] settled by its Gram bound (the energy bound did not hold),
 * [10] Gram bounds evaluated.
 * Returns GLR_ETIMEDOUT if a bounded device wait expired (GLR_DEV_TIMEOUT),
 * else GLR_EDEVICE if another error bit (non-finite, bad index) is set.
 * Pass reset != 0 to clear the block afterwards.
 */
glr_status glr_poll_status(const void* ws, uint32_t* bits, uint32_t* counters, int32_t reset,
                           void* stream);

/* Human-readable name of a status code (static string). */
const char* glr_status_string(glr_status s);

/* Number of kernels this library has launched in this process (all devices). */
uint64_t glr_launch_count(void);

/*
 * Per-kernel timing: when enabled, the library records a CUDA event pair on
 * the launch stream around every kernel it launches (do not enable while a
 * stream is being captured into a CUDA graph).  glr_profile_collect waits for
 * the recorded events, sums the durations per kernel name since the previous
 * collect and clears the record.  names receives `cap` NUL-terminated strings
 * of 48 bytes each; total_ms and launches receive `cap` values.  Returns the
 * number of distinct kernels written (<= cap), or -1 on a CUDA error.
 */
glr_status glr_profile_enable(int32_t on);
int32_t glr_profile_collect(char* names, float* total_ms, int32_t* launches, int32_t cap);

/* Version string of the library build. */
const char* glr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GLR_H_ */
