// WNNM low-rank step (Eq. 5) for groups whose columns do not fit in registers:
// long real patches (d up to 640, e.g. multi-channel 6 x 6 x 16) and complex
// patches (complex images stored as two planes; a column is the real half
// followed by the imaginary half).
//
//  k_jacobi_smem  one CTA (8 warps) per group, the K columns in shared memory.
//                 One-sided Jacobi (Hestenes) SVD in FP32; the K(K-1)/2 pairs of
//                 a sweep are scheduled by the round-robin (circle) ordering: in
//                 each of the K-1 rounds K/2 disjoint pairs rotate in parallel,
//                 one warp per pair, lanes striding over the entries.
//                 Complex columns use the Hermitian rotation: with
//                 g = a^H b = |g| e, the pair (a, e^-1 b) is real-orthogonalised
//                 (a' = c a - s conj(e) b, b' = s e a + c b), which zeroes a'^H b'.
//                 Stable angle as in the register kernel
//                 (t = sign(z) / (|z| + sqrt(1 + z^2)), z = (|b|^2 - |a|^2) / 2|g|).
//                 Rotations between two columns that cannot reach the WNNM
//                 threshold lam = K sw^2 are skipped by the same rule as the
//                 register kernel (block total below lam, or the previous
//                 sweep's Gershgorin bound of the block below lam / 2).
//                 Output X^ = sum_i (s'_i / s_i^3) w_i (w_i^H y_j) for every
//                 column y_j, re-read from the group buffer.
#include "glr_kernels.cuh"

namespace glr {

namespace {

constexpr int WJ_WARPS = 8;
constexpr int WJ_THREADS = WJ_WARPS * 32;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Columns: Wc[j * dr + e], dr real values per column (complex: m = dr / 2
// entries, real parts at e < m, imaginary parts at m + e).
template <bool CPLX>
__global__ void __launch_bounds__(WJ_THREADS) k_jacobi_smem(int n_img, int dr, int N, int K,
                                                            const int32_t* __restrict__ n_found, float sigma_w,
                                                            float c_wnnm, float tol, int max_sweeps,
                                                            float* __restrict__ groups, int32_t* __restrict__ rank,
                                                            StatusBlock* st, int32_t* __restrict__ fb_queue) {
  extern __shared__ float sm[];
  const int Kp = K + (K & 1);  // an odd K gets one zero column (it never rotates)
  float* Wc = sm;              // [Kp][dr]
  float* nrm = Wc + (size_t)Kp * dr;
  float* acc = nrm + Kp;
  float* coef = acc + Kp;
  int* act = reinterpret_cast<int*>(coef + Kp);  // then per warp 2 Kp floats of z_i
  __shared__ float skip_s, negl_s;
  __shared__ int nact_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int m = CPLX ? dr / 2 : dr;
  const long long ngroups = (long long)n_img * N;
  const float lam = (float)K * sigma_w * sigma_w;
  for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int f = (int)(g / N), k = (int)(g - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;  // uniform over the CTA
    float* Y = groups + g * (long long)K * dr;
    bool bad = false;
    for (int i = tid; i < K * dr; i += WJ_THREADS) {
      const float v = Y[i];
      bad |= !isfinite(v);
      Wc[i] = v;
    }
    for (int i = tid; i < (Kp - K) * dr; i += WJ_THREADS) Wc[(size_t)K * dr + i] = 0.f;
    for (int j = tid; j < Kp; j += WJ_THREADS) acc[j] = 0.f;
    if (__syncthreads_or(bad)) {
      if (tid == 0) {
        status_set(st, GLR_DEV_NONFINITE);
        if (rank) rank[g] = -1;
      }
      continue;
    }
    int sweep = 0;
    bool converged = (K < 2);
    while (!converged && sweep < max_sweeps) {
      // exact squared norms at the start of the sweep
      for (int j = wid; j < Kp; j += WJ_WARPS) {
        const float* w = Wc + (size_t)j * dr;
        float s = 0.f;
        for (int e = lane; e < dr; e += 32) s = fmaf(w[e], w[e], s);
        s = warp_sum(s);
        if (lane == 0) nrm[j] = s;
      }
      __syncthreads();
      if (wid == 0) {
        float small = 0.f, gb = 0.f, nmax = 0.f;
        for (int j = lane; j < Kp; j += 32) {
          if (nrm[j] < lam) {
            small += nrm[j];
            gb = fmaxf(gb, nrm[j] + acc[j]);
          }
          nmax = fmaxf(nmax, nrm[j]);
          acc[j] = 0.f;
        }
        small = warp_sum(small);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          gb = fmaxf(gb, __shfl_xor_sync(0xffffffffu, gb, o));
          nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        }
        if (lane == 0) {
          // the previous sweep's bound only (acc is empty before the first sweep)
          const bool gersh = sweep > 0 && gb < 0.5f * lam;
          skip_s = (lam > 0.f && (small < lam || gersh)) ? lam : 0.f;
          // pairs of columns at the rounding level of the largest one (the null space
          // when K exceeds the rank) are not rotated
          negl_s = 1e-12f * nmax;
        }
      }
      __syncthreads();
      const float lam_skip = skip_s, negl = negl_s;
      bool rotated = false;
      for (int r = 0; r < Kp - 1; ++r) {
        for (int i = wid; i < Kp / 2; i += WJ_WARPS) {
          const int p = (i == 0) ? r : (r + i) % (Kp - 1);
          const int q = (i == 0) ? Kp - 1 : (r - i + Kp - 1) % (Kp - 1);
          float* a = Wc + (size_t)p * dr;
          float* b = Wc + (size_t)q * dr;
          float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
          for (int e = lane; e < m; e += 32) {
            const float ar = a[e], br = b[e];
            al = fmaf(ar, ar, al);
            be = fmaf(br, br, be);
            gr = fmaf(ar, br, gr);
            if (CPLX) {
              const float ai = a[m + e], bi = b[m + e];
              al = fmaf(ai, ai, al);
              be = fmaf(bi, bi, be);
              gr = fmaf(ai, bi, gr);  // Re(a^H b) = ar br + ai bi
              gi = fmaf(ar, bi, gi);  // Im(a^H b) = ar bi - ai br
              gi = fmaf(-ai, br, gi);
            }
          }
          al = warp_sum(al);
          be = warp_sum(be);
          gr = warp_sum(gr);
          if (CPLX) gi = warp_sum(gi);
          const float gmag = CPLX ? sqrtf(fmaf(gr, gr, gi * gi)) : fabsf(gr);
          if (lane == 0) {
            if (be < lam) acc[p] += gmag;
            if (al < lam) acc[q] += gmag;
          }
          if (gmag > tol * sqrtf(al * be) && gmag != 0.f && (al >= lam_skip || be >= lam_skip) &&
              fmaxf(al, be) > negl) {
            const float zeta = (be - al) / (2.f * gmag);
            const float az = fabsf(zeta);
            float t = (az < 1e18f) ? 1.f / (az + sqrtf(fmaf(zeta, zeta, 1.f))) : 0.5f / az;
            t = copysignf(t, zeta);
            const float cs = rsqrtf(fmaf(t, t, 1.f));
            const float sn = cs * t;
            if (CPLX) {
              const float er = gr / gmag, ei = gi / gmag;  // e = g / |g|
              for (int e = lane; e < m; e += 32) {
                const float ar = a[e], ai = a[m + e], br = b[e], bi = b[m + e];
                // conj(e) b = (er br + ei bi) + i (er bi - ei br); e a = (er ar - ei ai) + i (er ai + ei ar)
                const float cbr = fmaf(er, br, ei * bi), cbi = fmaf(er, bi, -ei * br);
                const float ear = fmaf(er, ar, -ei * ai), eai = fmaf(er, ai, ei * ar);
                a[e] = fmaf(cs, ar, -sn * cbr);
                a[m + e] = fmaf(cs, ai, -sn * cbi);
                b[e] = fmaf(sn, ear, cs * br);
                b[m + e] = fmaf(sn, eai, cs * bi);
              }
            } else {
              const float se = gr < 0.f ? -sn : sn;  // s * e with e = sign(a.b) for real columns
              for (int e = lane; e < m; e += 32) {
                const float ar = a[e], br = b[e];
                a[e] = fmaf(cs, ar, -se * br);
                b[e] = fmaf(se, ar, cs * br);
              }
            }
            rotated = true;
          }
        }
        __syncthreads();
      }
      ++sweep;
      converged = !__syncthreads_or(rotated);
    }
    if (tid == 0) {
      if (!converged) {
        atomicAdd(&st->svd_noconv, 1u);
        status_set(st, GLR_DEV_SVD_NOCONV);
        // the group stays as gathered and goes to the FP64 fallback, which writes X^ and the rank
        if (fb_queue != nullptr) fb_queue[atomicAdd(&st->fb_count, 1u)] = (int32_t)g;
      }
      atomicAdd(&st->sweeps, (unsigned)sweep);
      atomicAdd(&st->groups, 1u);
    }
    if (!converged && fb_queue != nullptr) continue;  // uniform over the CTA
    // singular values s_i = |w_i| and the WNNM coefficients s'_i / s_i^3
    for (int j = wid; j < Kp; j += WJ_WARPS) {
      const float* w = Wc + (size_t)j * dr;
      float s = 0.f;
      for (int e = lane; e < dr; e += 32) s = fmaf(w[e], w[e], s);
      s = warp_sum(s);
      if (lane == 0) nrm[j] = s;
    }
    __syncthreads();
    if (wid == 0) {
      float smax = 0.f;
      for (int j = lane; j < Kp; j += 32) smax = fmaxf(smax, nrm[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      for (int j = lane; j < Kp; j += 32) {
        const float s = nrm[j];
        const float sg = sqrtf(s);
        const float sh = sqrtf(fmaxf(s - lam, 0.f));
        const float sp = fmaxf(sg - c_wnnm * sigma_w * sigma_w / (sh + 1e-8f), 0.f);
        // numerical rank: singular values at or below max(rows, K) 2^-24 s_max are
        // FP32 rounding residue (the null space of a group with K > rows)
        const float rtol = (float)max(m, K) * 5.9604645e-8f;
        coef[j] = (sp > 0.f && s > rtol * rtol * smax) ? sp / (sg * s) : 0.f;
      }
      __syncwarp();
      int base = 0;
      for (int j0 = 0; j0 < Kp; j0 += 32) {
        const int j = j0 + lane;
        const bool on = j < Kp && coef[j] != 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) act[base + __popc(bal & ((1u << lane) - 1u))] = j;
        base += __popc(bal);
      }
      if (lane == 0) {
        nact_s = base;
        if (rank) rank[g] = base;
      }
    }
    __syncthreads();
    const int nact = nact_s;
    // X^ column by column, a warp per column: first every z_i = coef_i w_i^H y_j
    // (kept in the warp's slice of shared memory), then y_j is overwritten
    float* zs = reinterpret_cast<float*>(act + Kp) + (size_t)wid * 2 * Kp;
    for (int j = wid; j < K; j += WJ_WARPS) {
      float* y = Y + (size_t)j * dr;
      for (int u = 0; u < nact; ++u) {
        const float* w = Wc + (size_t)act[u] * dr;
        float pr = 0.f, pi = 0.f;
        for (int e = lane; e < m; e += 32) {
          const float wr = w[e], yr = y[e];
          pr = fmaf(wr, yr, pr);
          if (CPLX) {
            const float wi = w[m + e], yi = y[m + e];
            pr = fmaf(wi, yi, pr);  // Re(w^H y)
            pi = fmaf(wr, yi, pi);  // Im(w^H y)
            pi = fmaf(-wi, yr, pi);
          }
        }
        pr = warp_sum(pr);
        if (CPLX) pi = warp_sum(pi);
        if (lane == 0) {
          const float cf = coef[act[u]];
          zs[2 * u] = cf * pr;
          zs[2 * u + 1] = cf * pi;
        }
      }
      __syncwarp();
      for (int e = lane; e < m; e += 32) {
        float xr = 0.f, xi = 0.f;
        for (int u = 0; u < nact; ++u) {
          const float* w = Wc + (size_t)act[u] * dr;
          const float wr = w[e], zr = zs[2 * u];
          xr = fmaf(wr, zr, xr);
          if (CPLX) {
            const float wi = w[m + e], zi = zs[2 * u + 1];
            xr = fmaf(-wi, zi, xr);  // Re(w z)
            xi = fmaf(wr, zi, xi);   // Im(w z)
            xi = fmaf(wi, zr, xi);
          }
        }
        y[e] = xr;
        if (CPLX) y[m + e] = xi;
      }
      __syncwarp();
    }
    __syncthreads();  // the shared columns are reused by the next group
  }
}

// ---------------------------------------------------------------------------
// k_gram_wnnm: tall real groups (d >= 2K, K <= 32), one warp per group.
// The K x K Gram matrix G = Y^T Y is formed in FP32 (Y streamed through a
// 32 x 32 shared-memory tile), diagonalised by the cyclic two-sided Jacobi
// method (G <- J^T G J, V <- V J, 16 disjoint pairs per round, circle
// ordering), and X^ = Y V diag(c) V^T with c_i = s'_i / s_i, s_i = sqrt(l_i):
// since Y v_i = s_i u_i, this is U diag(s') V^T.  Work per group is
// O(d K^2) once instead of per sweep, and the weights c_i <= 1 never amplify
// rounding.  Eigenvalues carry an absolute error of order 2^-24 l_max, which
// moves components near the WNNM threshold only (the shrinkage removes them).
// The WNNM skip rule of the one-sided kernels applies to the diagonal, and
// off-diagonal entries below the Gram matrix's rounding level (4 ulps of its
// largest diagonal entry) are not rotated: they carry no information, and the
// relative test alone would never be met among components at that level.
// ---------------------------------------------------------------------------
constexpr int GW_WARPS = 4;
constexpr int GW_LD = 33;

__device__ __forceinline__ void circle_pair(int k, int r, int& p, int& q) {  // n = 32 slots
  if (k == 0) {
    p = r;
    q = 31;
  } else {
    p = (r + k) % 31;
    q = (r - k + 31) % 31;
  }
}

__global__ void __launch_bounds__(GW_WARPS * 32) k_gram_wnnm(int n_img, int d, int N, int K,
                                                             const int32_t* __restrict__ n_found, float sigma_w,
                                                             float c_wnnm, float tol, int max_sweeps,
                                                             float* __restrict__ groups, int32_t* __restrict__ rank,
                                                             StatusBlock* st, int32_t* __restrict__ fb_queue) {
  __shared__ float Gs[GW_WARPS][32][GW_LD];
  __shared__ float Vs[GW_WARPS][32][GW_LD];
  __shared__ float Ts[GW_WARPS][32][GW_LD];
  __shared__ float2 cs_s[GW_WARPS][16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float(*G)[GW_LD] = Gs[wid];
  float(*V)[GW_LD] = Vs[wid];
  float(*T)[GW_LD] = Ts[wid];
  float2* cs = cs_s[wid];
  const long long ngroups = (long long)n_img * N;
  const float lam = (float)K * sigma_w * sigma_w;
  for (long long g = blockIdx.x * (long long)GW_WARPS + wid; g < ngroups; g += (long long)gridDim.x * GW_WARPS) {
    const int f = (int)(g / N), k = (int)(g - (long long)f * N);
    if (k >= min(n_found[f], N)) continue;
    float* Y = groups + g * (long long)K * d;
    // ---- Gram matrix: lane j accumulates row j
    float gacc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) gacc[i] = 0.f;
    bool bad = false;
    for (int r0 = 0; r0 < d; r0 += 32) {
      const int rr = r0 + lane;
      for (int j = 0; j < 32; ++j) {
        const float v = (j < K && rr < d) ? Y[(long long)j * d + rr] : 0.f;
        bad |= !isfinite(v);
        T[lane][j] = v;
      }
      __syncwarp();
#pragma unroll 4
      for (int t = 0; t < 32; ++t) {
        const float yj = T[t][lane];
#pragma unroll
        for (int i = 0; i < 32; ++i) gacc[i] = fmaf(T[t][i], yj, gacc[i]);
      }
      __syncwarp();
    }
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) {
        status_set(st, GLR_DEV_NONFINITE);
        if (rank) rank[g] = -1;
      }
      continue;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      G[lane][i] = gacc[i];
      V[lane][i] = (i == lane) ? 1.f : 0.f;
    }
    __syncwarp();
    // ---- cyclic two-sided Jacobi on G
    int sweep = 0;
    bool converged = K < 2;
    bool gersh_ok = false;
    while (!converged && sweep < max_sweeps) {
      // WNNM skip rule (see the one-sided kernels): diagonal entries below lam form the block
      const float dii = G[lane][lane];
      float small = (lane < K && dii < lam) ? dii : 0.f;
      float dmax = dii;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        small += __shfl_xor_sync(0xffffffffu, small, o);
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      }
      // entries of G below its FP32 rounding level (a few ulps of the largest
      // diagonal entry) carry no information: they are not rotated away
      const float gfloor = 2.384e-7f * dmax;
      const float lam_skip = (lam > 0.f && (small < lam || gersh_ok)) ? lam : 0.f;
      bool rotated = false;
      for (int r = 0; r < 31; ++r) {
        if (lane < 16) {
          int p, q;
          circle_pair(lane, r, p, q);
          const float app = G[p][p], aqq = G[q][q], apq = G[p][q];
          float c = 1.f, s = 0.f;
          if (fabsf(apq) > tol * sqrtf(fabsf(app * aqq)) && fabsf(apq) > gfloor &&
              (app >= lam_skip || aqq >= lam_skip)) {
            const float tau = (aqq - app) / (2.f * apq);
            const float at = fabsf(tau);
            float t = (at < 1e18f) ? 1.f / (at + sqrtf(fmaf(tau, tau, 1.f))) : 0.5f / at;
            t = copysignf(t, tau);
            c = rsqrtf(fmaf(t, t, 1.f));
            s = t * c;
            rotated = true;
          }
          cs[lane] = make_float2(c, s);
        }
        __syncwarp();
        // columns of G and V: lane = row
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
          const float2 w = cs[kk];
          if (w.y == 0.f) continue;
          int p, q;
          circle_pair(kk, r, p, q);
          const float gp = G[lane][p], gq = G[lane][q];
          G[lane][p] = fmaf(w.x, gp, -w.y * gq);
          G[lane][q] = fmaf(w.y, gp, w.x * gq);
          const float vp = V[lane][p], vq = V[lane][q];
          V[lane][p] = fmaf(w.x, vp, -w.y * vq);
          V[lane][q] = fmaf(w.y, vp, w.x * vq);
        }
        __syncwarp();
        // rows of G: lane = column
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
          const float2 w = cs[kk];
          if (w.y == 0.f) continue;
          int p, q;
          circle_pair(kk, r, p, q);
          const float gp = G[p][lane], gq = G[q][lane];
          G[p][lane] = fmaf(w.x, gp, -w.y * gq);
          G[q][lane] = fmaf(w.y, gp, w.x * gq);
        }
        __syncwarp();
      }
      ++sweep;
      converged = !__any_sync(0xffffffffu, rotated);
      // Gershgorin bound of the block below lam on the current matrix, for the next sweep
      float gb = 0.f;
      if (lane < K && G[lane][lane] < lam) {
        float rs = G[lane][lane];
        for (int j = 0; j < K; ++j)
          if (j != lane && G[j][j] < lam) rs += fabsf(G[lane][j]);
        gb = rs;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) gb = fmaxf(gb, __shfl_xor_sync(0xffffffffu, gb, o));
      gersh_ok = gb < 0.5f * lam;
    }
    if (lane == 0) {
      if (!converged) {
        atomicAdd(&st->svd_noconv, 1u);
        status_set(st, GLR_DEV_SVD_NOCONV);
        // the group stays as gathered and goes to the FP64 fallback, which writes X^ and the rank
        if (fb_queue != nullptr) fb_queue[atomicAdd(&st->fb_count, 1u)] = (int32_t)g;
      }
      atomicAdd(&st->sweeps, (unsigned)sweep);
      atomicAdd(&st->groups, 1u);
    }
    if (!converged && fb_queue != nullptr) continue;  // uniform over the warp
    // ---- WNNM weights c_i = s'_i / s_i
    const float li = G[lane][lane];
    float ci = 0.f;
    if (lane < K && li > 0.f) {
      const float sg = sqrtf(li);
      const float sh = sqrtf(fmaxf(li - lam, 0.f));
      const float sp = fmaxf(sg - c_wnnm * sigma_w * sigma_w / (sh + 1e-8f), 0.f);
      ci = sp / sg;
    }
    const unsigned act = __ballot_sync(0xffffffffu, ci > 0.f);
    if (rank && lane == 0) rank[g] = __popc(act);
    __syncwarp();
    // M = V diag(c) V^T, lane j keeps column j
    float mcol[32];
    {
      float vj[32];
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) vj[kk] = V[lane][kk] * __shfl_sync(0xffffffffu, ci, kk);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float m = 0.f;
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) m = fmaf(V[i][kk], vj[kk], m);
        mcol[i] = m;
      }
    }
    // ---- X^ = Y M, 32 rows at a time, in place
    for (int r0 = 0; r0 < d; r0 += 32) {
      const int rr = r0 + lane;
      for (int j = 0; j < K; ++j) T[lane][j] = (rr < d) ? Y[(long long)j * d + rr] : 0.f;
      __syncwarp();
      float out[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) out[t] = 0.f;
      // columns i >= K of T and rows i >= K of M are zero
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float m = mcol[i];
#pragma unroll
        for (int t = 0; t < 32; ++t) out[t] = fmaf(T[t][i], m, out[t]);
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 32; ++t) T[t][lane] = out[t];
      __syncwarp();
      if (rr < d)
        for (int j = 0; j < K; ++j) Y[(long long)j * d + rr] = T[lane][j];
      __syncwarp();
    }
  }
}

}  // namespace

glr_status launch_gram_wnnm(const glr_images& im, const int32_t* n_found, int N, int K, float sigma_w, float c_wnnm,
                            float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue, cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  if (K < 1 || K > 32 || d < 2 * K) return GLR_ENOTSUP;
  const long long ngroups = (long long)im.n_img * N;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ceil_div(ngroups, GW_WARPS), (long long)num_sms() * 64));
  const int cap = g_wnnm_sweep_cap > 0 ? g_wnnm_sweep_cap : 30;
  GLR_LAUNCH("k_gram_wnnm", s, k_gram_wnnm<<<blocks, GW_WARPS * 32, 0, s>>>(im.n_img, d, N, K, n_found, sigma_w, c_wnnm, 1e-5f, cap, groups, rank, st, fb_queue));
  if (fb_queue == nullptr) return GLR_OK;
  return launch_wnnm_fp64(d, K, sigma_w, c_wnnm, groups, rank, fb_queue, st, s, false);
}

size_t wnnm_smem_bytes(int d, int K) {
  const int Kp = K + (K & 1);
  return (size_t)Kp * d * 4 + (size_t)Kp * 16 + (size_t)WJ_WARPS * 2 * Kp * 4;
}

glr_status launch_wnnm_smem(const glr_images& im, bool cplx, const int32_t* n_found, int N, int K, float sigma_w,
                            float c_wnnm, float* groups, int32_t* rank, StatusBlock* st, int32_t* fb_queue,
                            cudaStream_t s) {
  const int d = im.C * im.P * im.P;
  if (K < 1 || K > 128 || d > 640 || (cplx && (d % 2) != 0)) return GLR_ENOTSUP;
  const size_t smem = wnnm_smem_bytes(d, K);
  if (smem > 200 * 1024) return GLR_ENOTSUP;
  const long long ngroups = (long long)im.n_img * N;
  int per_sm = 1;
  if (cplx) {
    if (cudaFuncSetAttribute(k_jacobi_smem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GLR_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_smem<true>, WJ_THREADS, smem) != cudaSuccess)
      return GLR_ECUDA;
  } else {
    if (cudaFuncSetAttribute(k_jacobi_smem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GLR_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_smem<false>, WJ_THREADS, smem) !=
        cudaSuccess)
      return GLR_ECUDA;
  }
  if (per_sm < 1) return GLR_ENOTSUP;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(ngroups, (long long)num_sms() * per_sm * 4));
  const float tol = 1e-5f;
  const int cap = g_wnnm_sweep_cap > 0 ? g_wnnm_sweep_cap : 30;
  if (!wnnm_fp64_supported(K, cplx)) fb_queue = nullptr;  // capped groups keep their FP32 result (flagged)
  if (cplx)
    GLR_LAUNCH("k_jacobi_smem", s, k_jacobi_smem<true><<<blocks, WJ_THREADS, smem, s>>>(im.n_img, d, N, K, n_found, sigma_w, c_wnnm, tol, cap, groups, rank, st, fb_queue));
  else
    GLR_LAUNCH("k_jacobi_smem", s, k_jacobi_smem<false><<<blocks, WJ_THREADS, smem, s>>>(im.n_img, d, N, K, n_found, sigma_w, c_wnnm, tol, cap, groups, rank, st, fb_queue));
  if (fb_queue == nullptr) return GLR_OK;
  return launch_wnnm_fp64(d, K, sigma_w, c_wnnm, groups, rank, fb_queue, st, s, cplx);
}

}  // namespace glr
