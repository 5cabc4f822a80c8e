// FP64 fallback of the WNNM step (Eq. 5) for groups whose FP32 one-sided Jacobi
// reached its sweep cap.  The register kernel leaves such a group untouched in
// the group buffer and queues its index; this kernel then computes, in FP64,
//   G = Y^T Y,  G = V diag(lambda) V^T  (cyclic two-sided Jacobi),
//   s_i = sqrt(lambda_i),  coefficients c_i = s'_i / s_i  (the shrinkage of the
//   register kernel, reading: sigma_hat_i = sqrt(max(s_i^2 - K sw^2, 0)),
//   tau_i = C sw^2 / (sigma_hat_i + eps), s'_i = max(s_i - tau_i, 0)),
//   X^ = Y V diag(c) V^T,
// and writes X^ (FP32) and the rank over the same buffer.  The Gram matrix squares
// the condition number, which FP64 absorbs: components down to about 1e-7 s_1 are
// resolved, below the FP32 path's 2^-24 max(d, K) s_1.
//
// One warp per queued group, one group per CTA at a time (G and V in shared memory,
// 64 x 64 doubles each, and a 32-row slab of the group for the Gram products); the
// queue length is read on the device, so the launch needs no host synchronisation.
// A group whose FP64 sweeps also reach their cap is counted (fb_noconv) and flagged.
#include "glr_kernels.cuh"

namespace glr {

namespace {

constexpr int F64_N = 64;            // G is padded to 64 x 64 (zero rows / columns beyond K)
constexpr int F64_LD = F64_N + 1;    // odd stride: column accesses spread over the banks

// Circle ordering for 64 slots: 32 disjoint pairs per round, 63 rounds per sweep.
__device__ __forceinline__ void circle_pair64(int k, int r, int& p, int& q) {
  if (k == 0) {
    p = r;
    q = F64_N - 1;
  } else {
    p = (r + k) % (F64_N - 1);
    q = (r - k + F64_N - 1) % (F64_N - 1);
  }
}

__global__ void __launch_bounds__(32) k_wnnm_fp64(int d, int K, float sigma_w, float c_wnnm, int max_sweeps,
                                                  float* __restrict__ groups, int32_t* __restrict__ rank,
                                                  const int32_t* __restrict__ queue, StatusBlock* st) {
  extern __shared__ double f64_smem[];
  double* G = f64_smem;                      // [64][F64_LD]
  double* V = f64_smem + F64_N * F64_LD;     // [64][F64_LD]
  double* slab = f64_smem + 2 * F64_N * F64_LD;  // [64][33]: 32 rows of every column
  __shared__ double2 cs[F64_N / 2];
  const int lane = threadIdx.x;
  const unsigned count = *reinterpret_cast<volatile unsigned*>(&st->fb_count);
  const double sw2 = (double)sigma_w * (double)sigma_w;
  const double lam = (double)K * sw2;
  for (unsigned qi = blockIdx.x; qi < count; qi += gridDim.x) {
    const long long g = queue[qi];
    float* Y = groups + g * (long long)K * d;  // column j at Y + j d
    // ---- G = Y^T Y, padded with zeros.  The group is read in slabs of 32 rows, each staged
    //      in shared memory by coalesced loads (lane = row inside the slab); then lane = row i
    //      of G (two rows per lane) accumulates the slab's contribution to its 64 entries.
    for (int i = lane; i < F64_N; i += 32)
      for (int j = 0; j < F64_N; ++j) {
        G[i * F64_LD + j] = 0.0;
        V[i * F64_LD + j] = (i == j) ? 1.0 : 0.0;
      }
    __syncwarp();
    for (int r0 = 0; r0 < d; r0 += 32) {
      const int r = r0 + lane;
      for (int j = 0; j < K; ++j) slab[j * 33 + lane] = r < d ? (double)Y[(long long)j * d + r] : 0.0;
      __syncwarp();
      for (int i = lane; i < K; i += 32)
        for (int j = 0; j < K; ++j) {
          double acc = G[i * F64_LD + j];
#pragma unroll 8
          for (int t = 0; t < 32; ++t) acc = fma(slab[i * 33 + t], slab[j * 33 + t], acc);
          G[i * F64_LD + j] = acc;
        }
      __syncwarp();
    }
    // ---- cyclic two-sided Jacobi: G <- J^T G J, V <- V J per round
    double dmax = 0.0;
    for (int i = 0; i < K; ++i) dmax = fmax(dmax, G[i * F64_LD + i]);
    const double gfloor = 8.9e-16 * dmax;  // 4 ulps of the largest diagonal entry
    bool converged = K < 2;
    for (int sweep = 0; !converged && sweep < max_sweeps; ++sweep) {
      bool rotated = false;
      for (int r = 0; r < F64_N - 1; ++r) {
        {
          int p, q;
          circle_pair64(lane, r, p, q);
          const double app = G[p * F64_LD + p], aqq = G[q * F64_LD + q], apq = G[p * F64_LD + q];
          double c = 1.0, s = 0.0;
          if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > gfloor) {
            const double theta = (aqq - app) / (2.0 * apq);
            double t = 1.0 / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
            t = theta < 0.0 ? -t : t;
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
            rotated = true;
          }
          cs[lane] = make_double2(c, s);
        }
        __syncwarp();
        // columns p, q of G and V (lane = row, two rows per lane)
        for (int k = 0; k < F64_N / 2; ++k) {
          const double2 w = cs[k];
          if (w.y == 0.0) continue;
          int p, q;
          circle_pair64(k, r, p, q);
          for (int i = lane; i < F64_N; i += 32) {
            const double gp = G[i * F64_LD + p], gq = G[i * F64_LD + q];
            G[i * F64_LD + p] = w.x * gp - w.y * gq;
            G[i * F64_LD + q] = w.y * gp + w.x * gq;
            const double vp = V[i * F64_LD + p], vq = V[i * F64_LD + q];
            V[i * F64_LD + p] = w.x * vp - w.y * vq;
            V[i * F64_LD + q] = w.y * vp + w.x * vq;
          }
        }
        __syncwarp();
        // rows p, q of G (lane = column, two columns per lane)
        for (int k = 0; k < F64_N / 2; ++k) {
          const double2 w = cs[k];
          if (w.y == 0.0) continue;
          int p, q;
          circle_pair64(k, r, p, q);
          for (int j = lane; j < F64_N; j += 32) {
            const double gp = G[p * F64_LD + j], gq = G[q * F64_LD + j];
            G[p * F64_LD + j] = w.x * gp - w.y * gq;
            G[q * F64_LD + j] = w.y * gp + w.x * gq;
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
    __shared__ double coef[F64_N];
    const double lfloor = 2.0 * (double)max(d, K) * 2.220446049250313e-16 * dmax;
    for (int i = lane; i < F64_N; i += 32) {
      double ci = 0.0;
      const double li = (i < K) ? G[i * F64_LD + i] : 0.0;
      if (li > lfloor) {
        const double si = sqrt(li);
        const double sh = sqrt(fmax(li - lam, 0.0));
        const double sp = fmax(si - (double)c_wnnm * sw2 / (sh + 1e-8), 0.0);
        ci = sp / si;
      }
      coef[i] = ci;
    }
    __syncwarp();
    const unsigned act0 = __ballot_sync(0xffffffffu, coef[lane] > 0.0);
    const unsigned act1 = __ballot_sync(0xffffffffu, coef[lane + 32] > 0.0);
    if (rank && lane == 0) rank[g] = __popc(act0) + __popc(act1);
    // ---- M = V diag(c) V^T into G's storage (lane = row i of M; G is no longer read)
    for (int i = lane; i < F64_N; i += 32)
      for (int j = 0; j < F64_N; ++j) {
        double m = 0.0;
        for (int k = 0; k < F64_N; ++k) m = fma(V[i * F64_LD + k] * coef[k], V[j * F64_LD + k], m);
        G[i * F64_LD + j] = m;
      }
    __syncwarp();
    // ---- X^ = Y M in place: lane = row r of Y, its K values first copied into V's
    //      storage (the eigenvectors are no longer needed)
    double* yrow = V + lane * F64_LD;
    for (int r = lane; r < d; r += 32) {
      for (int i = 0; i < K; ++i) yrow[i] = (double)Y[(long long)i * d + r];
      for (int j = 0; j < K; ++j) {
        double x = 0.0;
        for (int i = 0; i < K; ++i) x = fma(yrow[i], G[i * F64_LD + j], x);
        Y[(long long)j * d + r] = (float)x;
      }
    }
    __syncwarp();
  }
}

}  // namespace

size_t wnnm_fp64_smem_bytes() { return ((size_t)2 * F64_N * F64_LD + (size_t)F64_N * 33) * sizeof(double); }

glr_status launch_wnnm_fp64(int d, int K, float sigma_w, float c_wnnm, float* groups, int32_t* rank,
                            const int32_t* queue, StatusBlock* st, cudaStream_t s) {
  if (K > F64_N || d < 1) return GLR_ENOTSUP;
  const size_t smem = wnnm_fp64_smem_bytes();
  if (cudaFuncSetAttribute(k_wnnm_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GLR_ECUDA;
  GLR_LAUNCH("k_wnnm_fp64", s,
             k_wnnm_fp64<<<num_sms(), 32, smem, s>>>(d, K, sigma_w, c_wnnm, 30, groups, rank, queue, st));
  return GLR_OK;
}

}  // namespace glr
