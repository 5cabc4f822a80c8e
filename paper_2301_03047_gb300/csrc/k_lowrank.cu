// Grouping R~_i x and the WNNM low-rank step of Eq. 5.
//
//  k_gather      groups[f][k][j][:] = patch at idx[f][k][j] (vector order
//                ch, dr, dc).  One CTA per group, one thread per 4 output
//                floats: coalesced 16-byte stores; loads hit the L2-resident
//                image.  HBM-write bound.
//  k_jacobi_wnnm one warp per group Y (d x K).  One-sided Jacobi (Hestenes)
//                SVD in FP32 with the columns held in registers: lane L owns two
//                column slots (zero beyond K); the 32 lanes rotate their pairs in
//                parallel and re-pair by a recursive-halving ordering (cyclic
//                shifts within lane groups, one shuffle per element), so every
//                pair meets once per sweep.  Rotation angles use the stable
//                formulas of Rutishauser (t = sign(z)/(|z| + sqrt(1 + z^2))).
//                Sweeps stop when no pair has |a.b| > tol sqrt(|a|^2 |b|^2).
//                With W = Y V (columns w_i = s_i u_i) the WNNM estimate is
//                X^ = U diag(s') V^T = sum_i (s'_i / s_i^3) w_i (w_i^T Y),
//                formed from the active w_i staged in shared memory and the
//                original Y re-read from the group buffer.
#include "glr_kernels.cuh"

namespace glr {

namespace {

// PT = P (compile-time patch side; 0: the runtime value).  One CTA per group:
// thread t writes float4 number e4 = t mod q4 of members j = t / q4, t / q4 + 256 / q4,
// ... (q4 = d / 4), so the index arithmetic per value is a few constant divisions.
template <int PT>
__global__ void __launch_bounds__(256) k_gather(const float* __restrict__ x, int n_img, int C, int H, int W, int Prt,
                                                const int32_t* __restrict__ idx, const int32_t* __restrict__ n_found,
                                                int N, int K, float* __restrict__ groups, StatusBlock* st) {
  const int P = PT ? PT : Prt;
  const int PP = P * P;
  const int d = C * PP;
  const int q4 = d / 4;  // d % 4 == 0 on this path
  const int Wq = W - P + 1, npos = Wq * (H - P + 1);
  const int jstep = 256 / q4;  // members per pass (q4 <= 160 for d <= 640)
  const int t = threadIdx.x;
  const int j0 = t / q4, e0 = (t - j0 * q4) * 4;
  if (j0 >= jstep) return;
  // vector index -> (channel, row, column) offsets of the four values, fixed per thread
  int off[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u;
    const int ch = e / PP, rem = e - ch * PP, rr = rem / P, cc = rem - rr * P;
    off[u] = (ch * H + rr) * W + cc;
  }
  const long long ngroups = (long long)n_img * N;
  for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int f = (int)(g / N), k = (int)(g - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    const float* xf = x + (long long)f * C * H * W;
    float4* out = reinterpret_cast<float4*>(groups + g * (long long)K * d);
    for (int j = j0; j < K; j += jstep) {
      const int q = idx[g * K + j];
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((unsigned)q >= (unsigned)npos) {
        if (e0 == 0) status_set(st, GLR_DEV_BAD_INDEX);
      } else {
        const int r = q / Wq, c = q - (q / Wq) * Wq;
        const float* base = xf + (long long)r * W + c;
        v = make_float4(__ldg(base + off[0]), __ldg(base + off[1]), __ldg(base + off[2]), __ldg(base + off[3]));
      }
      out[(long long)j * q4 + e0 / 4] = v;
    }
  }
}

// One Jacobi rotation of the column pair held by this lane.  The columns are kept
// scaled: the true columns are da a and db b.  A rotation by (c, s) = c (1, t) of
// the true columns is then a shear of the stored ones plus the factor c on both
// scales (a' = a - t (db / da) b, b' = b + t (da / db) a, da' = c da, db' = c db):
// two FMAs per row instead of four operations.  alpha / beta are the tracked
// squared norms of the true columns (updated exactly as the rotation changes
// them: alpha - t gamma, beta + t gamma); only gamma = da db (a.b) is summed.
template <int DMAX>
__device__ __forceinline__ void jacobi_pair(float (&a)[DMAX], float (&b)[DMAX], float& da, float& db, float& alpha,
                                            float& beta, float tol, float lam_skip, float lam, float& acc_a,
                                            float& acc_b, bool active, bool& rotated) {
  float ga[4] = {0.f, 0.f, 0.f, 0.f};  // four partial sums shorten the dependency chain
#pragma unroll
  for (int r = 0; r < DMAX; ++r) ga[r & 3] = fmaf(a[r], b[r], ga[r & 3]);
  const float gamma = ((ga[0] + ga[1]) + (ga[2] + ga[3])) * (da * db);
  // Gershgorin sums of the block of columns below lam (see the sweep loop)
  if (beta < lam) acc_a += fabsf(gamma);
  if (alpha < lam) acc_b += fabsf(gamma);
  // pairs of columns that are both below lam_skip are left alone (see the sweep loop)
  if (active && fabsf(gamma) > tol * sqrtf(alpha * beta) && gamma != 0.f && (alpha >= lam_skip || beta >= lam_skip)) {
    const float zeta = __fdividef(beta - alpha, 2.f * gamma);
    const float az = fabsf(zeta);
    float t = (az < 1e18f) ? __frcp_rn(az + sqrtf(fmaf(zeta, zeta, 1.f))) : __fdividef(0.5f, az);
    t = copysignf(t, zeta);
    const float cs = rsqrtf(fmaf(t, t, 1.f));
    const float ta = t * __fdividef(db, da), tb = t * __fdividef(da, db);
#pragma unroll
    for (int r = 0; r < DMAX; ++r) {
      const float ar = a[r], br = b[r];
      a[r] = fmaf(-ta, br, ar);
      b[r] = fmaf(tb, ar, br);
    }
    da *= cs;
    db *= cs;
    alpha = fmaf(-t, gamma, alpha);
    beta = fmaf(t, gamma, beta);
    rotated = true;
  }
}

// Complex columns (real halves in [0, DMAX/2), imaginary halves in [DMAX/2, DMAX)):
// with g = a^H b = |g| e, rotate (a, conj(e) b) as a real pair:
// a' = c a - s conj(e) b, b' = s e a + c b, which zeroes a'^H b'.
// Scaled as the real pair: a' = a - t (db / da) conj(e) b, b' = b + t (da / db) e a,
// both scales times c (four FMAs per complex row and column instead of eight).
template <int DMAX>
__device__ __forceinline__ void jacobi_pair_c(float (&a)[DMAX], float (&b)[DMAX], float& da, float& db, float& alpha,
                                              float& beta, float tol, float lam_skip, float lam, float& acc_a,
                                              float& acc_b, bool& rotated) {
  constexpr int H2 = DMAX / 2;
  float pr[2] = {0.f, 0.f}, pi[2] = {0.f, 0.f};
#pragma unroll
  for (int r = 0; r < H2; ++r) {
    pr[r & 1] = fmaf(a[r], b[r], pr[r & 1]);
    pr[r & 1] = fmaf(a[H2 + r], b[H2 + r], pr[r & 1]);
    pi[r & 1] = fmaf(a[r], b[H2 + r], pi[r & 1]);
    pi[r & 1] = fmaf(-a[H2 + r], b[r], pi[r & 1]);
  }
  const float sab = da * db;
  const float gr = (pr[0] + pr[1]) * sab, gi = (pi[0] + pi[1]) * sab;
  const float gm = sqrtf(fmaf(gr, gr, gi * gi));
  if (beta < lam) acc_a += gm;
  if (alpha < lam) acc_b += gm;
  if (gm > tol * sqrtf(alpha * beta) && gm != 0.f && (alpha >= lam_skip || beta >= lam_skip)) {
    const float zeta = __fdividef(beta - alpha, 2.f * gm);
    const float az = fabsf(zeta);
    float t = (az < 1e18f) ? __frcp_rn(az + sqrtf(fmaf(zeta, zeta, 1.f))) : __fdividef(0.5f, az);
    t = copysignf(t, zeta);
    const float cs = rsqrtf(fmaf(t, t, 1.f));
    const float inv = __frcp_rn(gm);
    const float er = gr * inv, ei = gi * inv;
    const float p = t * __fdividef(db, da), q = t * __fdividef(da, db);
    const float per = p * er, pei = p * ei, qer = q * er, qei = q * ei;
#pragma unroll
    for (int r = 0; r < H2; ++r) {
      const float ar = a[r], ai = a[H2 + r], br = b[r], bi = b[H2 + r];
      a[r] = fmaf(-per, br, fmaf(-pei, bi, ar));      // a - p conj(e) b
      a[H2 + r] = fmaf(-per, bi, fmaf(pei, br, ai));
      b[r] = fmaf(qer, ar, fmaf(-qei, ai, br));       // b + q e a
      b[H2 + r] = fmaf(qer, ai, fmaf(qei, ar, bi));
    }
    da *= cs;
    db *= cs;
    alpha = fmaf(-t, gm, alpha);
    beta = fmaf(t, gm, beta);
    rotated = true;
  }
}

// Column j of a group in global memory <-> registers.  Real: d values.  Complex:
// m = d / 2 real parts then m imaginary parts, placed at [0, m) and [DMAX/2, DMAX/2 + m).
template <int DMAX, bool CPLX>
__device__ __forceinline__ void load_col(float (&a)[DMAX], const float* __restrict__ y, int d, bool own) {
  if (CPLX) {
    constexpr int H2 = DMAX / 2;
    const int m = d / 2;
#pragma unroll
    for (int r = 0; r < H2; ++r) {
      a[r] = (own && r < m) ? y[r] : 0.f;
      a[H2 + r] = (own && r < m) ? y[m + r] : 0.f;
    }
  } else {
#pragma unroll
    for (int r = 0; r < DMAX; ++r) a[r] = (own && r < d) ? y[r] : 0.f;
  }
}
template <int DMAX, bool CPLX>
__device__ __forceinline__ void store_col(const float (&a)[DMAX], float* __restrict__ y, int d) {
  if (CPLX) {
    constexpr int H2 = DMAX / 2;
    const int m = d / 2;
#pragma unroll
    for (int r = 0; r < H2; ++r)
      if (r < m) {
        y[r] = a[r];
        y[m + r] = a[H2 + r];
      }
  } else {
#pragma unroll
    for (int r = 0; r < DMAX; ++r)
      if (r < d) y[r] = a[r];
  }
}

// Fused path: the group's columns are gathered from the image (R~_i x of Eq. 5)
// and the estimates are added straight into the aggregation planes (64-bit fixed
// point, as k_scatter does), so the group never goes to memory.
struct FusedIO {
  const float* x;
  int C, H, W, P;
  const int32_t* idx;        // [n_img][N][K]
  unsigned long long* num;   // [n_img][C][H][W] fixed-point numerators
  int* cnt;                  // [n_img][Hq][Wq] patch counts
};

template <int DMAX>
__device__ __forceinline__ void gather_col(float (&a)[DMAX], const FusedIO& io, int f, int q, int d, bool own) {
  const int Wq = io.W - io.P + 1, PP = io.P * io.P;
  const int r0 = own ? q / Wq : 0, c0 = own ? q - (q / Wq) * Wq : 0;
  const float* xf = io.x + (long long)f * io.C * io.H * io.W;
#pragma unroll
  for (int r = 0; r < DMAX; ++r) {
    float v = 0.f;
    if (own && r < d) {
      const int ch = r / PP, rem = r - ch * PP, dr = rem / io.P, dc = rem - dr * io.P;
      v = __ldg(xf + ((long long)ch * io.H + r0 + dr) * io.W + c0 + dc);
    }
    a[r] = v;
  }
}

template <int DMAX>
__device__ __forceinline__ void scatter_col(const float (&a)[DMAX], const FusedIO& io, int f, int q, int d) {
  const int Wq = io.W - io.P + 1, Hq = io.H - io.P + 1, PP = io.P * io.P;
  const int r0 = q / Wq, c0 = q - (q / Wq) * Wq;
  unsigned long long* nf = io.num + (long long)f * io.C * io.H * io.W;
#pragma unroll
  for (int r = 0; r < DMAX; ++r)
    if (r < d) {
      const int ch = r / PP, rem = r - ch * PP, dr = rem / io.P, dc = rem - dr * io.P;
      const float v = fminf(fmaxf(a[r], -1073741824.f), 1073741824.f);
      atomicAdd(nf + ((long long)ch * io.H + r0 + dr) * io.W + c0 + dc,
                (unsigned long long)__float2ll_rn(v * 4294967296.f));
    }
  atomicAdd(io.cnt + (long long)f * Hq * Wq + q, 1);
}

template <int DMAX>
__device__ __forceinline__ float sq_norm(const float (&a)[DMAX]) {
  float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < DMAX; ++r) p[r & 3] = fmaf(a[r], a[r], p[r & 3]);
  return (p[0] + p[1]) + (p[2] + p[3]);
}

// The rank-1 certificate of k_jacobi_wnnm (real groups of up to 64 rows).  WNNM removes
// every component with s <= s_crit, s_crit^2 = sw^2 (K + sqrt(K^2 + 4 C^2)) / 2 (where
// s = C sw^2 / sqrt(s^2 - K sw^2)).  Power steps on Y^T Y from the all-ones vector give a unit
// vector v near the dominant right singular vector and mu = ||Y v||^2 <= s_1^2.  Two upper
// bounds on s_2^2 settle the group as rank <= 1:
//  1. energy: ||Y||_F^2 - mu >= sum_{i >= 2} s_i^2 >= s_2^2;
//  2. Gram: with R = Y (I - v v^T), R^T R is Y^T Y compressed to the complement of v, so by
//     Cauchy interlacing s_2^2 <= lambda_max(R^T R) <= ||R^T R||_F.  Where the residual energy
//     is spread over many small components (noise at the start of the schedule) this is up to
//     sqrt(K - 1) times tighter than the energy bound.
// Either bound at most s_crit^2 (less margins for the FP32 sums) means WNNM keeps at most the
// first component; once the eigen-residual ||Y^T Y v - mu v|| is below 2e-6 (mu - bound) (v
// within 2e-6 of the dominant vector) X^ = s_1' u u^T Y with u = Y v / ||Y v||.
// y = Y v is summed through the warp's shared-memory slice buf (32 partial rows of 68 floats,
// then y at 32 x 68): every lane adds two rows of the 32 lane partials in lane order.  The
// Gram bound stores the columns of R in buf (slot l: lane l's first column, slot 32 + l: its
// second; float4 r4 of slot s at 4 (r4 ^ (s & 15)), so that both the column stores and the
// broadcast reads avoid bank conflicts) and the eigen-residual components in res[64].
// Returns 0 (not certified), 1 (energy bound) or 2 (Gram bound), with ylo, yhi = rows
// 2 lane, 2 lane + 1 of y, mu, and zA, zB = y . y_j of the lane's two columns (so that
// x^_j = s_1' / (s_1 mu) (y . y_j) y); gram tells whether the Gram bound was evaluated.
constexpr int kPowerSteps = 12;
constexpr int kPartLd = 68;  // partial-row stride (floats): 16-byte stores without bank conflicts
__device__ __forceinline__ int rank1_certificate(const float (&a)[64], const float (&b)[64], bool has_a,
                                                 bool has_b, int K, float sigma_w, float c_wnnm, int lane,
                                                 float* buf, float* res, float& ylo, float& yhi, float& mu,
                                                 float& zA, float& zB, int& steps, bool& gram) {
  const float sw2 = sigma_w * sigma_w;
  const float scrit2 = 0.5f * sw2 * ((float)K + sqrtf((float)K * (float)K + 4.f * c_wnnm * c_wnnm));
  const float lim = 0.9999f * scrit2;
  const float sqrt_m = sqrtf((float)max(K - 1, 1));  // R has rank <= K - 1
  float fro = sq_norm<64>(a) + sq_norm<64>(b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  float va = has_a ? rsqrtf((float)K) : 0.f, vb = has_b ? rsqrtf((float)K) : 0.f;
  float* yv = buf + 32 * kPartLd;
  mu = 0.f;
  gram = false;
  float ra = 0.f, rb = 0.f, res_n = 0.f, lim_g = 0.f;
  bool try_gram = false;
  for (int it = 0; it < kPowerSteps; ++it) {
    steps = it + 1;
    // y = Y v: this lane's share (its two columns), then the 32 shares added
    float4* pw = reinterpret_cast<float4*>(buf + lane * kPartLd);
#pragma unroll
    for (int r4 = 0; r4 < 16; ++r4)
      pw[r4] = make_float4(fmaf(va, a[4 * r4], vb * b[4 * r4]), fmaf(va, a[4 * r4 + 1], vb * b[4 * r4 + 1]),
                           fmaf(va, a[4 * r4 + 2], vb * b[4 * r4 + 2]), fmaf(va, a[4 * r4 + 3], vb * b[4 * r4 + 3]));
    __syncwarp();
    float sx = 0.f, sy = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float2 v = *reinterpret_cast<const float2*>(buf + k * kPartLd + 2 * lane);
      sx += v.x;
      sy += v.y;
    }
    ylo = sx;
    yhi = sy;
    *reinterpret_cast<float2*>(yv + 2 * lane) = make_float2(sx, sy);
    __syncwarp();
    float p[4] = {0.f, 0.f, 0.f, 0.f}, za[4] = {0.f, 0.f, 0.f, 0.f}, zb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r4 = 0; r4 < 16; ++r4) {
      const float4 t = reinterpret_cast<const float4*>(yv)[r4];
      const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        p[u] = fmaf(tv[u], tv[u], p[u]);
        za[u] = fmaf(a[4 * r4 + u], tv[u], za[u]);
        zb[u] = fmaf(b[4 * r4 + u], tv[u], zb[u]);
      }
    }
    __syncwarp();  // y and the partials are read before the next step rewrites them
    const float mu_new = (p[0] + p[1]) + (p[2] + p[3]);  // ||Y v||^2, v of unit length
    zA = (za[0] + za[1]) + (za[2] + za[3]);
    zB = (zb[0] + zb[1]) + (zb[2] + zb[3]);
    const bool done = it > 0 && mu_new - mu <= 1e-7f * mu_new;
    mu = mu_new;
    if (!(mu > 0.f)) return fro <= lim ? 1 : 0;  // Y = 0 (or below s_crit altogether)
    // residual of the eigen-equation: r = Y^T Y v - mu v; v is within |r| / gap of the
    // dominant vector, gap >= mu - (upper bound on s_2^2)
    ra = zA - mu * va;
    rb = zB - mu * vb;
    float r2 = ra * ra + rb * rb, n2 = zA * zA + zB * zB;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    res_n = sqrtf(r2);
    const float rest = fro - mu;  // = ||R||_F^2 >= sum_{i >= 2} s_i^2 (mu only grows)
    const bool energy_ok = rest <= lim - 4e-6f * fro;
    if (energy_ok && res_n <= 2e-6f * (mu - rest)) return 1;
    // the Gram bound's level, less its FP32 error (the products a.r_c and the residual terms
    // below: about 4e-6 sqrt(||Y||_F^2 ||R||_F^2) and 4e-6 ||Y||_F^2 at worst, taken 10 and 2
    // times); it can only hold when ||R||_F^2 / sqrt(K - 1) <= ||R^T R||_F is below it
    lim_g = lim - 8e-6f * fro - 4e-5f * sqrtf(fro * fmaxf(rest, 0.f));
    const bool gram_ok = lim_g > 0.f && rest <= lim_g * sqrt_m;
    if (!energy_ok && gram_ok && res_n <= 2e-6f * (mu - lim_g)) {
      try_gram = true;
      break;
    }
    if (done && !energy_ok && !gram_ok) return 0;  // converged above both levels: not rank 1
    const float inv = rsqrtf(n2);
    va = zA * inv;
    vb = zB * inv;
  }
  if (!try_gram) return 0;
  // Gram bound: R columns r_j = y_j - v_j y into buf (y rows from the lanes that hold them),
  // res_j = y . r_j = (Y^T y)_j - v_j ||y||^2 (the eigen-residual), then per lane the entries
  // (R^T R)_{j s} = r_j . r_s = y_j . r_s - v_j res_s of its two rows j
  gram = true;
  res[lane] = ra;
  res[32 + lane] = rb;
  {
    const int sw = lane & 15;
    float4* ca = reinterpret_cast<float4*>(buf + lane * 64);
    float4* cb = reinterpret_cast<float4*>(buf + (32 + lane) * 64);
#pragma unroll
    for (int r4 = 0; r4 < 16; ++r4) {
      float yr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 4 * r4 + u;
        yr[u] = __shfl_sync(0xffffffffu, (r & 1) ? yhi : ylo, r >> 1);
      }
      ca[r4 ^ sw] = make_float4(fmaf(-va, yr[0], a[4 * r4]), fmaf(-va, yr[1], a[4 * r4 + 1]),
                                fmaf(-va, yr[2], a[4 * r4 + 2]), fmaf(-va, yr[3], a[4 * r4 + 3]));
      cb[r4 ^ sw] = make_float4(fmaf(-vb, yr[0], b[4 * r4]), fmaf(-vb, yr[1], b[4 * r4 + 1]),
                                fmaf(-vb, yr[2], b[4 * r4 + 2]), fmaf(-vb, yr[3], b[4 * r4 + 3]));
    }
  }
  __syncwarp();
  float gs = 0.f;
#pragma unroll 1
  for (int s = 0; s < 64; ++s) {
    const float4* cs = reinterpret_cast<const float4*>(buf + s * 64);
    const int sw = s & 15;
    float da[4] = {0.f, 0.f, 0.f, 0.f}, db[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r4 = 0; r4 < 16; ++r4) {
      const float4 t = cs[r4 ^ sw];
      da[0] = fmaf(a[4 * r4], t.x, da[0]);
      da[1] = fmaf(a[4 * r4 + 1], t.y, da[1]);
      da[2] = fmaf(a[4 * r4 + 2], t.z, da[2]);
      da[3] = fmaf(a[4 * r4 + 3], t.w, da[3]);
      db[0] = fmaf(b[4 * r4], t.x, db[0]);
      db[1] = fmaf(b[4 * r4 + 1], t.y, db[1]);
      db[2] = fmaf(b[4 * r4 + 2], t.z, db[2]);
      db[3] = fmaf(b[4 * r4 + 3], t.w, db[3]);
    }
    const float rs = res[s];
    const float ga = fmaf(-va, rs, (da[0] + da[1]) + (da[2] + da[3]));
    const float gb = fmaf(-vb, rs, (db[0] + db[1]) + (db[2] + db[3]));
    gs = fmaf(ga, ga, fmaf(gb, gb, gs));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
  __syncwarp();  // the R columns and res are read before the caller reuses buf
  const float rho = sqrtf(gs);  // ||R^T R||_F >= s_2^2
  return (rho <= lim_g && res_n <= 2e-6f * (mu - rho)) ? 2 : 0;
}

// Staging slice of a 64 x 64 group: float4 r4 (rows 4 r4 .. 4 r4 + 3) of column j at
// 16 j + (r4 ^ ((j >> 1) & 15)).  Coalesced copies (8 consecutive float4 of one column per
// quarter warp) and the lanes' reads of their own columns 2 lane, 2 lane + 1 both fall on 8
// distinct 16-byte bank groups.
__device__ __forceinline__ int stage_at(int j, int r4) { return 16 * j + (r4 ^ ((j >> 1) & 15)); }

// Columns at or above the skip level up to which a sweep is replaced by a direct test of
// their pairs (each costs one broadcast column: DMAX shuffles and 2 DMAX FMAs per lane).
constexpr int kDirectCheckCols = 4;

// DMAX rows per column, KMAX <= 64 columns, one warp per group, WARPS groups per CTA.
template <int DMAX, int WARPS, bool CPLX, bool FUSED>
__global__ void __launch_bounds__(WARPS * 32, CPLX ? 2 : 3) k_jacobi_wnnm(int n_img, int d, int N, int K,
                                                            const int32_t* __restrict__ n_found, float sigma_w,
                                                            float c_wnnm, float tol, int max_sweeps,
                                                            float* __restrict__ groups, int32_t* __restrict__ rank,
                                                            StatusBlock* st, FusedIO io,
                                                            int32_t* __restrict__ fb_queue) {
  extern __shared__ float wsm[];  // [WARPS][64][DMAX]: active columns of W
  __shared__ float coef_s[WARPS][64];  // shrinkage coefficients (the certificate's scratch before)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* Ws = wsm + (size_t)wid * 64 * DMAX;
  const long long ngroups = (long long)n_img * N;
  const int m = (K + 1) / 2;  // lanes holding at least one real column; the other slots are zero
  const bool live = true;     // zero columns never rotate (their inner products vanish)
  for (long long g = blockIdx.x * (long long)WARPS + wid; g < ngroups; g += (long long)gridDim.x * WARPS) {
    const int f = (int)(g / N), k = (int)(g - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    float* Y = FUSED ? nullptr : groups + g * (long long)K * d;
    // real 64-row groups in memory move through the staging slice with 16-byte accesses
    const bool stage_ok = !FUSED && !CPLX && DMAX == 64 && d == 64;
    float a[DMAX], b[DMAX];
    const int ja = 2 * lane, jb = 2 * lane + 1;
    int qa = -1, qb = -1;  // FUSED: patch positions of the two columns (-1: none / invalid)
    if (FUSED) {
      const int npos = (io.H - io.P + 1) * (io.W - io.P + 1);
      if (ja < K) qa = io.idx[g * K + ja];
      if (jb < K) qb = io.idx[g * K + jb];
      if ((ja < K && (unsigned)qa >= (unsigned)npos) || (jb < K && (unsigned)qb >= (unsigned)npos))
        status_set(st, GLR_DEV_BAD_INDEX);
      if ((unsigned)qa >= (unsigned)npos) qa = -1;
      if ((unsigned)qb >= (unsigned)npos) qb = -1;
      gather_col<DMAX>(a, io, f, qa, d, qa >= 0);
      gather_col<DMAX>(b, io, f, qb, d, qb >= 0);
    } else if (stage_ok) {
      // the group's K rows of 64 floats, coalesced through the warp's staging slice
      const float4* src = reinterpret_cast<const float4*>(Y);
      float4* W4 = reinterpret_cast<float4*>(Ws);
      for (int t = lane; t < K * 16; t += 32) W4[stage_at(t >> 4, t & 15)] = src[t];
      __syncwarp();
#pragma unroll
      for (int r4 = 0; r4 < 16; ++r4) {
        const float4 ta = ja < K ? W4[stage_at(ja, r4)] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 tb = jb < K ? W4[stage_at(jb, r4)] : make_float4(0.f, 0.f, 0.f, 0.f);
        a[4 * r4] = ta.x;
        a[4 * r4 + 1] = ta.y;
        a[4 * r4 + 2] = ta.z;
        a[4 * r4 + 3] = ta.w;
        b[4 * r4] = tb.x;
        b[4 * r4 + 1] = tb.y;
        b[4 * r4 + 2] = tb.z;
        b[4 * r4 + 3] = tb.w;
      }
      __syncwarp();  // the slice is read before the certificate reuses it
    } else {
      load_col<DMAX, CPLX>(a, Y + (long long)ja * d, d, ja < K);
      load_col<DMAX, CPLX>(b, Y + (long long)jb * d, d, live && jb < K);
    }
    // non-finite input: leave the group unchanged and flag it
    float s0 = 0.f;
#pragma unroll
    for (int r = 0; r < DMAX; ++r) s0 += a[r] + b[r];
    if (__any_sync(0xffffffffu, !isfinite(s0))) {
      if (lane == 0) status_set(st, GLR_DEV_NONFINITE);
      if (rank && lane == 0) rank[g] = -1;
      continue;
    }
    int sweep = 0;
    bool converged = (m < 1);
    // real groups of up to 64 rows: settle rank <= 1 without sweeps where the certificate holds
    bool rank1 = false;
    float ylo = 0.f, yhi = 0.f, mu1 = 0.f, zA = 0.f, zB = 0.f;
    if constexpr (!CPLX && DMAX == 64) {
      if (sigma_w > 0.f && !converged) {
        int steps = 0;
        bool gram = false;
        const int how = rank1_certificate(a, b, ja < K, jb < K, K, sigma_w, c_wnnm, lane, Ws, coef_s[wid], ylo,
                                          yhi, mu1, zA, zB, steps, gram);
        rank1 = how != 0;
        converged = converged || rank1;
        if (lane == 0) {
          atomicAdd(&st->power_steps, (unsigned)steps);
          if (gram) atomicAdd(&st->gram_evals, 1u);
          if (how == 2) atomicAdd(&st->rank1_gram, 1u);
        }
      }
    }
    // Components with s^2 < K sw^2 are always removed by the shrinkage.  When the
    // columns below that level carry less than K sw^2 in total, no combination of
    // them can reach it, so rotations among them cannot change X^ and are skipped
    // (decided per sweep; a sweep without rotations ends the iteration).
    const float lam = (float)K * sigma_w * sigma_w;
    bool gersh_ok = false;
    // Parallel ordering by recursive halving (32 lanes, 64 column slots): at a
    // level with lane groups of size g, the B columns shift cyclically inside
    // each group for g rounds, so every A meets every B of its group; then each
    // group of 2g lanes regroups into A-A pairs (first half) and B-B pairs
    // (second half) for the next level.  Levels g = 32, 16, ..., 1 give
    // 63 rounds covering all 2016 pairs; a shift costs one shuffle per element.
    float da = 1.f, db = 1.f;  // column scales (see jacobi_pair)
    while (!converged && sweep < max_sweeps) {
      bool rotated = false;
      // fold the scales into the columns, then exact norms once per sweep (tracked
      // through the rotations within it; a sweep shrinks a scale by at most 2^-32)
#pragma unroll
      for (int r = 0; r < DMAX; ++r) {
        a[r] *= da;
        b[r] *= db;
      }
      da = db = 1.f;
      float alpha = sq_norm<DMAX>(a), beta = sq_norm<DMAX>(b);
      float small = (alpha < lam ? alpha : 0.f) + (beta < lam ? beta : 0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) small += __shfl_xor_sync(0xffffffffu, small, o);
      // skip pairs inside the below-lam block when no combination of its columns can
      // reach lam: its total is below lam, or the previous sweep's Gershgorin bound
      // (norm^2 + sum of |a.b| over block partners, largest over the block) was
      // below lam / 2
      const float lam_skip = (lam > 0.f && (small < lam || gersh_ok)) ? lam : 0.f;
      // With the skip rule on, only pairs with a column at or above lam_skip can rotate.
      // When there are few such columns, test those pairs directly (each such column
      // broadcast once, the same inner products and test as the sweep's): if none
      // passes, the sweep would rotate nothing, so it is not run.
      if (!CPLX && lam_skip > 0.f) {
        unsigned ma = __ballot_sync(0xffffffffu, alpha >= lam_skip);
        unsigned mb = __ballot_sync(0xffffffffu, beta >= lam_skip);
        if (__popc(ma) + __popc(mb) <= kDirectCheckCols) {
          bool need = false;
          while (ma | mb) {
            const bool from_a = ma != 0;
            const int src = __ffs(from_a ? ma : mb) - 1;
            if (from_a) ma &= ma - 1;
            else mb &= mb - 1;
            const float nb = __shfl_sync(0xffffffffu, from_a ? alpha : beta, src);
            float ga[4] = {0.f, 0.f, 0.f, 0.f}, gb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < DMAX; ++r) {
              const float bv = __shfl_sync(0xffffffffu, from_a ? a[r] : b[r], src);
              ga[r & 3] = fmaf(a[r], bv, ga[r & 3]);
              gb[r & 3] = fmaf(b[r], bv, gb[r & 3]);
            }
            const float g_a = (ga[0] + ga[1]) + (ga[2] + ga[3]), g_b = (gb[0] + gb[1]) + (gb[2] + gb[3]);
            const bool self_a = from_a && lane == src, self_b = !from_a && lane == src;
            need |= !self_a && fabsf(g_a) > tol * sqrtf(alpha * nb) && g_a != 0.f;
            need |= !self_b && fabsf(g_b) > tol * sqrtf(beta * nb) && g_b != 0.f;
          }
          if (!__any_sync(0xffffffffu, need)) {
            converged = true;
            break;
          }
        }
      }
      float acc_a = 0.f, acc_b = 0.f;
#pragma unroll 1
      for (int g = 32; g >= 1; g >>= 1) {
        if (g < 32) {
          const bool first = (lane & g) == 0;
#pragma unroll
          for (int r = 0; r < DMAX; ++r) {
            const float recv = __shfl_xor_sync(0xffffffffu, first ? b[r] : a[r], g);
            if (first)
              b[r] = recv;
            else
              a[r] = recv;
          }
          const float rn = __shfl_xor_sync(0xffffffffu, first ? beta : alpha, g);
          const float ra = __shfl_xor_sync(0xffffffffu, first ? acc_b : acc_a, g);
          const float rs = __shfl_xor_sync(0xffffffffu, first ? db : da, g);
          if (first) {
            beta = rn;
            acc_b = ra;
            db = rs;
          } else {
            alpha = rn;
            acc_a = ra;
            da = rs;
          }
        }
        const int src = (lane & ~(g - 1)) | ((lane + 1) & (g - 1));
#pragma unroll 1
        for (int rd = 0; rd < g; ++rd) {
          if (CPLX)
            jacobi_pair_c<DMAX>(a, b, da, db, alpha, beta, tol, lam_skip, lam, acc_a, acc_b, rotated);
          else
            jacobi_pair<DMAX>(a, b, da, db, alpha, beta, tol, lam_skip, lam, acc_a, acc_b, live, rotated);
          if (rd + 1 < g) {
#pragma unroll
            for (int r = 0; r < DMAX; ++r) b[r] = __shfl_sync(0xffffffffu, b[r], src);
            beta = __shfl_sync(0xffffffffu, beta, src);
            acc_b = __shfl_sync(0xffffffffu, acc_b, src);
            db = __shfl_sync(0xffffffffu, db, src);
          }
        }
      }
      ++sweep;
      converged = !__any_sync(0xffffffffu, rotated);
      float gb = fmaxf(alpha < lam ? alpha + acc_a : 0.f, beta < lam ? beta + acc_b : 0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) gb = fmaxf(gb, __shfl_xor_sync(0xffffffffu, gb, o));
      gersh_ok = gb < 0.5f * lam;
    }
#pragma unroll
    for (int r = 0; r < DMAX; ++r) {
      a[r] *= da;
      b[r] *= db;
    }
    if (!converged && lane == 0) {
      atomicAdd(&st->svd_noconv, 1u);
      status_set(st, GLR_DEV_SVD_NOCONV);
    }
    if (!FUSED && !converged && fb_queue != nullptr) {
      // the sweep cap was reached: leave the group as gathered and queue it for the
      // FP64 fallback, which writes X^ and the rank
      if (lane == 0) {
        fb_queue[atomicAdd(&st->fb_count, 1u)] = (int32_t)g;
        atomicAdd(&st->sweeps, (unsigned)sweep);
        atomicAdd(&st->groups, 1u);
      }
      continue;
    }
    if (lane == 0) {
      atomicAdd(&st->sweeps, (unsigned)sweep);
      atomicAdd(&st->groups, 1u);
      if (rank1) atomicAdd(&st->rank1, 1u);
    }
    int rnk;
    if (rank1) {
      // X^ = coef w (w^T Y) with w = Y v: coef = s' / (s ||w||^2), s = ||w|| (as below)
      const float sw2 = sigma_w * sigma_w;
      const float s1 = sqrtf(mu1);
      const float h1 = sqrtf(fmaxf(mu1 - (float)K * sw2, 0.f));
      const float p1 = fmaxf(s1 - c_wnnm * sw2 / (h1 + 1e-8f), 0.f);
      const float coef = (p1 > 0.f && mu1 > 0.f) ? p1 / (s1 * mu1) : 0.f;
      rnk = coef != 0.f ? 1 : 0;
      if (rank && lane == 0) rank[g] = rnk;
      __syncwarp();  // the certificate's last reads of Ws are done
      if (stage_ok) {
        // x^_j = coef (y . y_j) y from the certificate's own products: y to every lane through
        // coef_s, the columns staged as they were loaded, stored with 16-byte accesses
        float* yv = coef_s[wid];
        yv[2 * lane] = ylo;
        yv[2 * lane + 1] = yhi;
        __syncwarp();
        float4* W4 = reinterpret_cast<float4*>(Ws);
        const float ka = zA * coef, kb = zB * coef;
#pragma unroll
        for (int r4 = 0; r4 < 16; ++r4) {
          const float4 t = reinterpret_cast<const float4*>(yv)[r4];
          W4[stage_at(ja, r4)] = make_float4(ka * t.x, ka * t.y, ka * t.z, ka * t.w);
          W4[stage_at(jb, r4)] = make_float4(kb * t.x, kb * t.y, kb * t.z, kb * t.w);
        }
        __syncwarp();
        float4* dst = reinterpret_cast<float4*>(Y);
        for (int t = lane; t < K * 16; t += 32) dst[t] = W4[stage_at(t >> 4, t & 15)];
        __syncwarp();
        continue;
      }
      Ws[2 * lane] = ylo;
      Ws[2 * lane + 1] = yhi;
      if (lane == 0) coef_s[wid][0] = coef;
    } else {
    // singular values and WNNM shrinkage (reading: tau_i = C sw^2 / (sigma_hat_i + eps))
    float na2 = 0.f, nb2 = 0.f;
#pragma unroll
    for (int r = 0; r < DMAX; ++r) {
      na2 = fmaf(a[r], a[r], na2);
      nb2 = fmaf(b[r], b[r], nb2);
    }
    const float sw2 = sigma_w * sigma_w;
    float coef_a = 0.f, coef_b = 0.f;
    // numerical rank: singular values at or below max(d, K) 2^-24 s_max are FP32
    // rounding residue (the null space of a group with K > d), not components
    float smax = fmaxf(na2, nb2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    const float rtol = (float)max(CPLX ? d / 2 : d, K) * 5.9604645e-8f;
    const float floor2 = rtol * rtol * smax;
    {
      const float sa = sqrtf(na2), sb = sqrtf(nb2);
      const float ha = sqrtf(fmaxf(na2 - (float)K * sw2, 0.f)), hb = sqrtf(fmaxf(nb2 - (float)K * sw2, 0.f));
      const float pa = fmaxf(sa - c_wnnm * sw2 / (ha + 1e-8f), 0.f);
      const float pb = fmaxf(sb - c_wnnm * sw2 / (hb + 1e-8f), 0.f);
      if (live && pa > 0.f && na2 > floor2) coef_a = pa / (sa * na2);
      if (live && pb > 0.f && nb2 > floor2) coef_b = pb / (sb * nb2);
    }
    const unsigned act_a = __ballot_sync(0xffffffffu, coef_a != 0.f);
    const unsigned act_b = __ballot_sync(0xffffffffu, coef_b != 0.f);
    const int ra = __popc(act_a), rb = __popc(act_b);
    rnk = ra + rb;
    if (rank && lane == 0) rank[g] = rnk;
    // stage the active columns w_i into shared memory (compacted) with coefficients
    {
      const int pa = __popc(act_a & ((1u << lane) - 1u));
      const int pb = ra + __popc(act_b & ((1u << lane) - 1u));
      if (coef_a != 0.f) {
#pragma unroll
        for (int r = 0; r < DMAX; ++r) Ws[pa * DMAX + r] = a[r];
        coef_s[wid][pa] = coef_a;
      }
      if (coef_b != 0.f) {
#pragma unroll
        for (int r = 0; r < DMAX; ++r) Ws[pb * DMAX + r] = b[r];
        coef_s[wid][pb] = coef_b;
      }
    }
    }  // rank1
    __syncwarp();
    // X^ columns j = 2 lane, 2 lane + 1: x^_j = sum_i coef_i w_i (w_i . y_j)
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * lane + h;
      const bool own = live && j < K;
      // a / b are free once W is staged: reuse them as y_j and x^_j
      const int qj = h == 0 ? qa : qb;
      if (FUSED)
        gather_col<DMAX>(a, io, f, qj, d, own && qj >= 0);
      else
        load_col<DMAX, CPLX>(a, Y + (long long)j * d, d, own);
#pragma unroll
      for (int r = 0; r < DMAX; ++r) b[r] = 0.f;
      for (int i = 0; i < rnk; ++i) {
        const float* w = Ws + i * DMAX;
        if (CPLX) {
          // z = coef w^H y (complex); x^ += w z
          constexpr int H2 = DMAX / 2;
          float zr = 0.f, zi = 0.f;
#pragma unroll
          for (int r = 0; r < H2; ++r) {
            zr = fmaf(w[r], a[r], zr);
            zr = fmaf(w[H2 + r], a[H2 + r], zr);
            zi = fmaf(w[r], a[H2 + r], zi);
            zi = fmaf(-w[H2 + r], a[r], zi);
          }
          zr *= coef_s[wid][i];
          zi *= coef_s[wid][i];
#pragma unroll
          for (int r = 0; r < H2; ++r) {
            b[r] = fmaf(w[r], zr, fmaf(-w[H2 + r], zi, b[r]));
            b[H2 + r] = fmaf(w[r], zi, fmaf(w[H2 + r], zr, b[H2 + r]));
          }
        } else {
          float zp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int r = 0; r < DMAX; ++r) zp[r & 3] = fmaf(w[r], a[r], zp[r & 3]);
          const float z = ((zp[0] + zp[1]) + (zp[2] + zp[3])) * coef_s[wid][i];
#pragma unroll
          for (int r = 0; r < DMAX; ++r) b[r] = fmaf(z, w[r], b[r]);
        }
      }
      __syncwarp();
      if (FUSED && rnk <= 32 && DMAX == 64) {
        // coalesced scatter: the 32 columns of this half go through the free half of
        // the staging area (active columns use rows < rnk <= 32), XOR-swizzled so
        // that both the column writes and the element reads avoid bank conflicts;
        // then the warp adds one column at a time, lane = element
        float* T = Ws + 32 * DMAX;
#pragma unroll
        for (int r = 0; r < DMAX; ++r) T[r * 32 + (lane ^ (r & 31))] = b[r];
        __syncwarp();
        const int Wq = io.W - io.P + 1, Hq = io.H - io.P + 1, PP = io.P * io.P;
        unsigned long long* nf = io.num + (long long)f * io.C * io.H * io.W;
        const int ok = own && qj >= 0;
        for (int c = 0; c < 32; ++c) {
          const int qc = __shfl_sync(0xffffffffu, ok ? qj : -1, c);
          if (qc < 0) continue;  // uniform over the warp
          const int r0 = qc / Wq, c0 = qc - (qc / Wq) * Wq;
          for (int e = lane; e < d; e += 32) {
            const float v = fminf(fmaxf(T[e * 32 + (c ^ (e & 31))], -1073741824.f), 1073741824.f);
            const int ch = e / PP, rem = e - ch * PP, dr = rem / io.P, dc = rem - dr * io.P;
            atomicAdd(nf + ((long long)ch * io.H + r0 + dr) * io.W + c0 + dc,
                      (unsigned long long)__float2ll_rn(v * 4294967296.f));
          }
          if (lane == 0) atomicAdd(io.cnt + (long long)f * Hq * Wq + qc, 1);
        }
        __syncwarp();
      } else if (FUSED) {
        if (own && qj >= 0) scatter_col<DMAX>(b, io, f, qj, d);
      } else if (own) {
        store_col<DMAX, CPLX>(b, Y + (long long)j * d, d);
      }
    }
    __syncwarp();
  }
}

}  // namespace

glr_status launch_gather(const float* x, const glr_images& im, const int32_t* idx, const int32_t* n_found, int N,
                         int K, float* groups, StatusBlock* st, cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  if (d % 4 != 0) return GLR_ENOTSUP;
  if (d / 4 > 256) return GLR_ENOTSUP;
  const long long ngroups = (long long)im.n_img * N;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ngroups, (long long)num_sms() * 16));
#define GLR_GATHER_CASE(PP) \
  GLR_LAUNCH("k_gather", s, k_gather<PP><<<blocks, 256, 0, s>>>(x, im.n_img, im.C, im.H, im.W, im.P, idx, n_found, N, K, groups, st))
  switch (im.P) {
    case 4: GLR_GATHER_CASE(4); break;
    case 6: GLR_GATHER_CASE(6); break;
    case 8: GLR_GATHER_CASE(8); break;
    default: GLR_GATHER_CASE(0); break;
  }
#undef GLR_GATHER_CASE
  return GLR_OK;
}

// testing aid: sweep cap of the register Jacobi (0: 30)
int g_wnnm_sweep_cap = 0;

template <int DMAX, bool CPLX, bool FUSED = false>
glr_status launch_wnnm_regs(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                            float* groups, int32_t* rank, StatusBlock* st, cudaStream_t s, const char* name,
                            FusedIO io = FusedIO{}, int32_t* fb_queue = nullptr) {
  constexpr int WARPS = 4;
  const int d = im.C * im.P * im.P;
  const size_t smem = (size_t)WARPS * 64 * DMAX * sizeof(float);
  if (cudaFuncSetAttribute(k_jacobi_wnnm<DMAX, WARPS, CPLX, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return GLR_ECUDA;
  const long long ngroups = (long long)im.n_img * N;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(ngroups, WARPS), (long long)num_sms() * 64));
  const float tol = 1e-5f;
  const int cap = g_wnnm_sweep_cap > 0 ? g_wnnm_sweep_cap : 30;
  GLR_LAUNCH(name, s, (k_jacobi_wnnm<DMAX, WARPS, CPLX, FUSED><<<blocks, WARPS * 32, smem, s>>>(im.n_img, d, N, K, n_found, sigma_w, c_wnnm, tol, cap, groups, rank, st, io, fb_queue)));
  return GLR_OK;
}

glr_status launch_wnnm(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                       float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue, cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  if (d > 64 || K > 64 || K < 1) return GLR_ENOTSUP;
  glr_status r = launch_wnnm_regs<64, false>(im, n_found, N, K, sigma_w, c_wnnm, groups, rank, st, s,
                                             "k_jacobi_wnnm", FusedIO{}, fb_queue);
  if (r != GLR_OK || fb_queue == nullptr) return r;
  return launch_wnnm_fp64(d, K, sigma_w, c_wnnm, groups, rank, fb_queue, st, s);
}

glr_status launch_wnnm_fused(const float* x, const glr_images& im, const int32_t* idx, const int32_t* n_found, int N,
                             int K, float sigma_w, float c_wnnm, unsigned long long* num, int* cnt, int32_t* rank,
                             StatusBlock* st, cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  if (d > 64 || K > 64 || K < 1) return GLR_ENOTSUP;
  FusedIO io{x, im.C, im.H, im.W, im.P, idx, num, cnt};
  return launch_wnnm_regs<64, false, true>(im, n_found, N, K, sigma_w, c_wnnm, nullptr, rank, st, s,
                                           "k_jacobi_wnnm_fused", io);
}

glr_status launch_wnnm_complex_regs(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w,
                                   float c_wnnm, float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue,
                                   cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  if (d > 72 || (d % 2) != 0 || K > 64 || K < 1) return GLR_ENOTSUP;
  if (!wnnm_fp64_supported(K, true)) fb_queue = nullptr;  // capped groups keep their FP32 result (flagged)
  glr_status r = launch_wnnm_regs<72, true>(im, n_found, N, K, sigma_w, c_wnnm, groups, rank, st, s,
                                            "k_jacobi_wnnm_c", FusedIO{}, fb_queue);
  if (r != GLR_OK || fb_queue == nullptr) return r;
  return launch_wnnm_fp64(d, K, sigma_w, c_wnnm, groups, rank, fb_queue, st, s, true);
}

}  // namespace glr
