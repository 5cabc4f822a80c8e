// FP64 fallback of the WNNM step (Eq. 5) for groups whose FP32 Jacobi reached its sweep
// cap.  The FP32 kernels (register, shared-memory, Gram and complex paths) leave such a group
// untouched in the group buffer and queue its index; this kernel then computes, in FP64,
//   G = Y_r^T Y_r,  G = V diag(lambda) V^T  (cyclic two-sided Jacobi),
//   s_i = sqrt(lambda_i),  coefficients c_i = s'_i / s_i  (the FP32 kernels' shrinkage,
//   reading: sigma_hat_i = sqrt(max(s_i^2 - K sw^2, 0)), tau_i = C sw^2 / (sigma_hat_i + eps),
//   s'_i = max(s_i - tau_i, 0)),
//   X^ = Y_r V diag(c) V^T,
// and writes X^ (FP32) and the rank over the same buffer.  Y_r is the group itself for real
// groups.  A complex group Y = A + iB (m x K, stored as real half then imaginary half per
// column) is taken as the real 2m x 2K matrix [[A, -B], [B, A]]: its singular values are
// those of Y, each twice, its Gram matrix is the real form of the Hermitian Y^H Y, and the
// first K columns of its shrunk matrix are [Re X^; Im X^], the stored layout; K in the
// shrinkage stays the complex K and the rank is half the real count.  The Gram matrix squares
// the condition number, which FP64 absorbs: components down to about 1e-7 s_1 are resolved,
// below the FP32 paths' 2^-24 max(d, K) s_1.
//
// One warp per queued group, one group per CTA at a time (G and V in shared memory, NM x NM
// doubles each with NM = 64 or 96, and a 32-row slab of the group for the Gram products); the
// queue length is read on the device, so the launch needs no host synchronisation.  A group
// whose FP64 sweeps also reach their cap is counted (fb_noconv) and flagged.
#include "glr_kernels.cuh"

namespace glr {

namespace {

// Circle ordering for NM slots: NM / 2 disjoint pairs per round, NM - 1 rounds per sweep.
template <int NM>
__device__ __forceinline__ void circle_pair(int k, int r, int& p, int& q) {
  if (k == 0) {
    p = r;
    q = NM - 1;
  } else {
    p = (r + k) % (NM - 1);
    q = (r - k + NM - 1) % (NM - 1);
  }
}

// Entry (row r, column c) of Y_r (see the header), d rows per stored column.
template <bool CPLX>
__device__ __forceinline__ double yr(const float* __restrict__ Y, int d, int K, int r, int c) {
  if (!CPLX || c < K) return (double)Y[(long long)c * d + r];
  const int m = d / 2, j = c - K;
  return r < m ? -(double)Y[(long long)j * d + m + r] : (double)Y[(long long)j * d + (r - m)];
}

template <int NM, bool CPLX>
__global__ void __launch_bounds__(32) k_wnnm_fp64(int d, int K, float sigma_w, float c_wnnm, int max_sweeps,
                                                  float* __restrict__ groups, int32_t* __restrict__ rank,
                                                  const int32_t* __restrict__ queue, StatusBlock* st) {
  constexpr int LD = NM + 1;  // odd stride: column accesses spread over the banks
  extern __shared__ double f64_smem[];
  double* G = f64_smem;                   // [NM][LD]
  double* V = f64_smem + NM * LD;         // [NM][LD]
  double* slab = f64_smem + 2 * NM * LD;  // [NM][33]: 32 rows of every real column
  __shared__ double2 cs[NM / 2];
  __shared__ double coef[NM];
  const int lane = threadIdx.x;
  const int KR = CPLX ? 2 * K : K;  // columns of Y_r
  const unsigned count = *reinterpret_cast<volatile unsigned*>(&st->fb_count);
  const double sw2 = (double)sigma_w * (double)sigma_w;
  const double lam = (double)K * sw2;
  for (unsigned qi = blockIdx.x; qi < count; qi += gridDim.x) {
    const long long g = queue[qi];
    float* Y = groups + g * (long long)K * d;  // column j at Y + j d
    // ---- G = Y_r^T Y_r, padded with zeros.  The group is read in slabs of 32 rows (lane = row
    //      inside the slab, coalesced); then lane = row i of G accumulates the slab's part.
    for (int i = lane; i < NM; i += 32)
      for (int j = 0; j < NM; ++j) {
        G[i * LD + j] = 0.0;
        V[i * LD + j] = (i == j) ? 1.0 : 0.0;
      }
    __syncwarp();
    for (int r0 = 0; r0 < d; r0 += 32) {
      const int r = r0 + lane;
      for (int c = 0; c < KR; ++c) slab[c * 33 + lane] = r < d ? yr<CPLX>(Y, d, K, r, c) : 0.0;
      __syncwarp();
      for (int i = lane; i < KR; i += 32)
        for (int j = 0; j < KR; ++j) {
          double acc = G[i * LD + j];
#pragma unroll 8
          for (int t = 0; t < 32; ++t) acc = fma(slab[i * 33 + t], slab[j * 33 + t], acc);
          G[i * LD + j] = acc;
        }
      __syncwarp();
    }
    // ---- cyclic two-sided Jacobi: G <- J^T G J, V <- V J per round
    double dmax = 0.0;
    for (int i = 0; i < KR; ++i) dmax = fmax(dmax, G[i * LD + i]);
    const double gfloor = 8.9e-16 * dmax;  // 4 ulps of the largest diagonal entry
    bool converged = KR < 2;
    for (int sweep = 0; !converged && sweep < max_sweeps; ++sweep) {
      bool rotated = false;
      for (int r = 0; r < NM - 1; ++r) {
        for (int kk = lane; kk < NM / 2; kk += 32) {
          int p, q;
          circle_pair<NM>(kk, r, p, q);
          const double app = G[p * LD + p], aqq = G[q * LD + q], apq = G[p * LD + q];
          double c = 1.0, s = 0.0;
          if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > gfloor) {
            const double theta = (aqq - app) / (2.0 * apq);
            double t = 1.0 / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
            t = theta < 0.0 ? -t : t;
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
            rotated = true;
          }
          cs[kk] = make_double2(c, s);
        }
        __syncwarp();
        // columns p, q of G and V (lane = row)
        for (int kk = 0; kk < NM / 2; ++kk) {
          const double2 w = cs[kk];
          if (w.y == 0.0) continue;
          int p, q;
          circle_pair<NM>(kk, r, p, q);
          for (int i = lane; i < NM; i += 32) {
            const double gp = G[i * LD + p], gq = G[i * LD + q];
            G[i * LD + p] = w.x * gp - w.y * gq;
            G[i * LD + q] = w.y * gp + w.x * gq;
            const double vp = V[i * LD + p], vq = V[i * LD + q];
            V[i * LD + p] = w.x * vp - w.y * vq;
            V[i * LD + q] = w.y * vp + w.x * vq;
          }
        }
        __syncwarp();
        // rows p, q of G (lane = column)
        for (int kk = 0; kk < NM / 2; ++kk) {
          const double2 w = cs[kk];
          if (w.y == 0.0) continue;
          int p, q;
          circle_pair<NM>(kk, r, p, q);
          for (int j = lane; j < NM; j += 32) {
            const double gp = G[p * LD + j], gq = G[q * LD + j];
            G[p * LD + j] = w.x * gp - w.y * gq;
            G[q * LD + j] = w.y * gp + w.x * gq;
          }
        }
        __syncwarp();
      }
      converged = !__any_sync(0xffffffffu, rotated);
    }
    if (!converged && lane == 0) {
      // the FP64 sweeps ran out too: X^ below is computed from the last rotation state
      atomicAdd(&st->fb_noconv, 1u);
      status_set(st, GLR_DEV_SVD_NOCONV);
    }
    // ---- shrinkage coefficients c_i = s'_i / s_i (components at the FP64 rounding level of
    //      the Gram matrix carry no information: treated as zero)
    const double lfloor = 2.0 * (double)max(d, KR) * 2.220446049250313e-16 * dmax;
    int nact = 0;
    for (int i = lane; i < NM; i += 32) {
      double ci = 0.0;
      const double li = (i < KR) ? G[i * LD + i] : 0.0;
      if (li > lfloor) {
        const double si = sqrt(li);
        const double sh = sqrt(fmax(li - lam, 0.0));
        const double sp = fmax(si - (double)c_wnnm * sw2 / (sh + 1e-8), 0.0);
        ci = sp / si;
      }
      coef[i] = ci;
      nact += ci > 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nact += __shfl_xor_sync(0xffffffffu, nact, o);
    __syncwarp();
    if (rank && lane == 0) rank[g] = CPLX ? nact / 2 : nact;
    // ---- M = V diag(c) V^T into G's storage (lane = row i of M; G is no longer read)
    for (int i = lane; i < NM; i += 32)
      for (int j = 0; j < KR; ++j) {
        double mm = 0.0;
        for (int kk = 0; kk < KR; ++kk) mm = fma(V[i * LD + kk] * coef[kk], V[j * LD + kk], mm);
        G[i * LD + j] = mm;
      }
    __syncwarp();
    // ---- X^ = Y_r M, columns j < K (the stored layout).  The values of Y_r a lane needs are
    //      copied into V's storage first (the eigenvectors are no longer needed), and every value
    //      is read before it is overwritten: a real lane owns row r; a complex lane owns rows r
    //      and r + m, the only two stored rows its two rows of Y_r read
    if (!CPLX) {
      double* yrow = V + lane * LD;
      for (int r = lane; r < d; r += 32) {
        for (int i = 0; i < KR; ++i) yrow[i] = (double)Y[(long long)i * d + r];
        for (int j = 0; j < K; ++j) {
          double xv = 0.0;
          for (int i = 0; i < KR; ++i) xv = fma(yrow[i], G[i * LD + j], xv);
          Y[(long long)j * d + r] = (float)xv;
        }
      }
    } else {
      const int m = d / 2;
      double* y0 = V + lane * LD;         // row r of Y_r
      double* y1 = V + (lane + 32) * LD;  // row r + m of Y_r
      for (int r = lane; r < m; r += 32) {
        for (int c = 0; c < K; ++c) {
          const double re = (double)Y[(long long)c * d + r], im = (double)Y[(long long)c * d + m + r];
          y0[c] = re;
          y0[K + c] = -im;
          y1[c] = im;
          y1[K + c] = re;
        }
        for (int j = 0; j < K; ++j) {
          double x0 = 0.0, x1 = 0.0;
          for (int i = 0; i < KR; ++i) {
            x0 = fma(y0[i], G[i * LD + j], x0);
            x1 = fma(y1[i], G[i * LD + j], x1);
          }
          Y[(long long)j * d + r] = (float)x0;
          Y[(long long)j * d + m + r] = (float)x1;
        }
      }
    }
    __syncwarp();
  }
}

template <int NM, bool CPLX>
glr_status launch_fp64(int d, int K, float sigma_w, float c_wnnm, float* groups, int32_t* rank,
                       const int32_t* queue, StatusBlock* st, int max_sweeps, cudaStream_t s) {
  const size_t smem = ((size_t)2 * NM * (NM + 1) + (size_t)NM * 33) * sizeof(double);
  if (cudaFuncSetAttribute(k_wnnm_fp64<NM, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return GLR_ECUDA;
  GLR_LAUNCH("k_wnnm_fp64", s,
             (k_wnnm_fp64<NM, CPLX><<<num_sms(), 32, smem, s>>>(d, K, sigma_w, c_wnnm, max_sweeps, groups, rank,
                                                                 queue, st)));
  return GLR_OK;
}

}  // namespace

bool wnnm_fp64_supported(int K, bool cplx) { return (cplx ? 2 * K : K) <= 96; }

glr_status launch_wnnm_fp64(int d, int K, float sigma_w, float c_wnnm, float* groups, int32_t* rank,
                            const int32_t* queue, StatusBlock* st, cudaStream_t s, bool cplx) {
  const int KR = cplx ? 2 * K : K;
  if (d < 1 || KR < 1 || (cplx && d % 2 != 0)) return GLR_ENOTSUP;
  if (KR <= 64)
    return cplx ? launch_fp64<64, true>(d, K, sigma_w, c_wnnm, groups, rank, queue, st, 30, s)
                : launch_fp64<64, false>(d, K, sigma_w, c_wnnm, groups, rank, queue, st, 30, s);
  if (KR <= 96)
    return cplx ? launch_fp64<96, true>(d, K, sigma_w, c_wnnm, groups, rank, queue, st, 30, s)
                : launch_fp64<96, false>(d, K, sigma_w, c_wnnm, groups, rank, queue, st, 30, s);
  return GLR_ENOTSUP;
}

}  // namespace glr
