// Fourier transforms and the ADMM data-consistency step of the MRI model
// y = M F(x) (Section 3, MRI).
//
// Complex images are two planes ([n][2][H][W]: real plane, imaginary plane).
// F is the orthonormal, unshifted 2-D DFT: a pass over the rows (length W)
// and a pass over the columns (length H), each scaled by 1/sqrt(length).
//
//  k_fft_lines  one CTA transforms LPB lines held in shared memory: the line
//               is loaded in bit-reversed order, then log2(n) radix-2
//               decimation-in-time stages run with a __syncthreads between
//               them; twiddles exp(-+2 pi i k / n) come from sincospif once per
//               CTA.  Row lines are contiguous; column lines are loaded with
//               consecutive threads on consecutive columns (coalesced).
//               Optional fused load / store stages implement the ADMM step:
//                 load  LOAD_ADMM:  u' = u + x - z (stored), line value z - u'
//                 store STORE_DC:   X' = (M y + rho X) / (M + rho) and the FP64
//                                   sum of M |X' - y|^2 (F(x_new) = X' exactly)
//                 store STORE_ADMM: x_new, and w = x_new + u' (next denoiser input)
// The lines of one CTA are independent of every other CTA, so an output may
// overwrite the input it was read from.
#include "glr_kernels.cuh"

namespace glr {

namespace {

enum { LOAD_PLAIN = 0, LOAD_ADMM = 1 };
enum { STORE_PLAIN = 0, STORE_DC = 1, STORE_ADMM = 2 };

struct FftArgs {
  const float* in;
  float* out;
  int n_img, H, W;
  int cols;     // 0: rows (length W), 1: columns (length H)
  int inverse;  // sign of the exponent
  int log2n;
  int lpb;  // lines per CTA
  // LOAD_ADMM
  const float* x;
  const float* z;
  float* u;
  // STORE_DC
  const float* y;
  const float* mask;  // [n][H][W], 0/1
  float rho;
  double* res_acc;  // [n]
  // STORE_ADMM
  float* w_out;
  double* res_out;  // [n]: sqrt(res_acc), written by CTA 0
};

constexpr int FFT_THREADS = 256;

template <int LOAD, int STORE>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_lines(FftArgs a) {
  extern __shared__ float sm[];
  const int n = 1 << a.log2n;
  const int lpb = a.lpb;
  float* sre = sm;
  float* sim = sm + (size_t)lpb * n;
  float2* tw = reinterpret_cast<float2*>(sim + (size_t)lpb * n);
  __shared__ double red[FFT_THREADS / 32];
  const int tid = threadIdx.x;
  const float sgn = a.inverse ? 2.f : -2.f;
  for (int k = tid; k < n / 2; k += FFT_THREADS) {
    float sv, cv;
    sincospif(sgn * (float)k / (float)n, &sv, &cv);  // k / n is exact (n a power of two)
    tw[k] = make_float2(cv, sv);
  }
  const long long HW = (long long)a.H * a.W;
  const int lines_per_img = a.cols ? a.W : a.H;
  const long long total_lines = (long long)a.n_img * lines_per_img;
  const long long line0 = (long long)blockIdx.x * lpb;
  // global offset (real plane) of element e of local line l; -1 past the end
  auto offset = [&](int l, int e) -> long long {
    const long long gl = line0 + l;
    if (gl >= total_lines) return -1;
    const long long f = gl / lines_per_img;
    const int li = (int)(gl - f * lines_per_img);
    return f * 2 * HW + (a.cols ? (long long)e * a.W + li : (long long)li * a.W + e);
  };
  for (int i = tid; i < lpb * n; i += FFT_THREADS) {
    int l, e;
    if (a.cols) {
      l = i % lpb;
      e = i / lpb;
    } else {
      l = i / n;
      e = i - (i / n) * n;
    }
    const long long off = offset(l, e);
    float re = 0.f, im = 0.f;
    if (off >= 0) {
      if (LOAD == LOAD_ADMM) {
        const float xr = a.x[off], xi = a.x[off + HW];
        const float zr = a.z[off], zi = a.z[off + HW];
        const float ur = a.u[off] + xr - zr, ui = a.u[off + HW] + xi - zi;
        a.u[off] = ur;
        a.u[off + HW] = ui;
        re = zr - ur;
        im = zi - ui;
      } else {
        re = a.in[off];
        im = a.in[off + HW];
      }
    }
    const int br = (int)(__brev((unsigned)e) >> (32 - a.log2n));
    sre[l * n + br] = re;
    sim[l * n + br] = im;
  }
  __syncthreads();
  for (int s = 0; s < a.log2n; ++s) {
    const int h = 1 << s;
    const int tshift = a.log2n - 1 - s;
    for (int b = tid; b < lpb * (n / 2); b += FFT_THREADS) {
      const int l = b >> (a.log2n - 1);
      const int bb = b & (n / 2 - 1);
      const int pos = bb & (h - 1);
      const int i0 = l * n + ((bb >> s) << (s + 1)) + pos;
      const int i1 = i0 + h;
      const float2 w = tw[pos << tshift];
      const float xr = sre[i1], xi = sim[i1];
      const float vr = fmaf(w.x, xr, -w.y * xi), vi = fmaf(w.x, xi, w.y * xr);
      const float ur = sre[i0], ui = sim[i0];
      sre[i0] = ur + vr;
      sim[i0] = ui + vi;
      sre[i1] = ur - vr;
      sim[i1] = ui - vi;
    }
    __syncthreads();
  }
  const float scale = rsqrtf((float)n);
  double part = 0.0;
  long long part_img = -1;  // image of this CTA's lines (all lines of a CTA lie in one image)
  for (int i = tid; i < lpb * n; i += FFT_THREADS) {
    int l, e;
    if (a.cols) {
      l = i % lpb;
      e = i / lpb;
    } else {
      l = i / n;
      e = i - (i / n) * n;
    }
    const long long off = offset(l, e);
    if (off < 0) continue;
    float re = sre[l * n + e] * scale, im = sim[l * n + e] * scale;
    if (STORE == STORE_DC) {
      const long long f = off / (2 * HW);
      const long long pix = off - f * 2 * HW;
      const float mk = a.mask[f * HW + pix];
      const float yr = a.y[off], yi = a.y[off + HW];
      const float den = mk + a.rho;
      re = (mk * yr + a.rho * re) / den;
      im = (mk * yi + a.rho * im) / den;
      const double dr = (double)re - (double)yr, di = (double)im - (double)yi;
      part += (double)mk * (dr * dr + di * di);
      part_img = f;
    }
    a.out[off] = re;
    a.out[off + HW] = im;
    if (STORE == STORE_ADMM) {
      a.w_out[off] = re + a.u[off];
      a.w_out[off + HW] = im + a.u[off + HW];
    }
  }
  if (STORE == STORE_DC) {
    // lines of one CTA never straddle two images (lpb divides the lines per image)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    long long img = part_img;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) img = max(img, __shfl_xor_sync(0xffffffffu, img, o));
    __shared__ long long img_s[FFT_THREADS / 32];
    if ((tid & 31) == 0) img_s[tid >> 5] = img;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      long long fi = -1;
      for (int w = 0; w < FFT_THREADS / 32; ++w) {
        t += red[w];
        fi = max(fi, img_s[w]);
      }
      if (fi >= 0) atomicAdd(a.res_acc + fi, t);
    }
  }
  if (STORE == STORE_ADMM && a.res_out != nullptr && blockIdx.x == 0) {
    for (int f = tid; f < a.n_img; f += FFT_THREADS) a.res_out[f] = sqrt(a.res_acc[f]);
  }
}

int lines_per_block(int n, bool cols) {
  // rows: about 2048 elements per CTA; columns: 8 lines (32-byte segments) while it fits
  int lpb = cols ? 8 : std::max(1, 2048 / n);
  while (lpb > 1 && (size_t)lpb * n * 8 > 64 * 1024) lpb >>= 1;
  return lpb;
}

template <int LOAD, int STORE>
glr_status run_pass(FftArgs a, cudaStream_t s, const char* name) {
  const int n = a.cols ? a.H : a.W;
  a.log2n = 0;
  while ((1 << a.log2n) < n) ++a.log2n;
  a.lpb = lines_per_block(n, a.cols != 0);
  const int lines_per_img = a.cols ? a.W : a.H;
  while (a.lpb > 1 && lines_per_img % a.lpb != 0) a.lpb >>= 1;
  const size_t smem = (size_t)a.lpb * n * 8 + (size_t)(n / 2) * 8;
  if (cudaFuncSetAttribute(k_fft_lines<LOAD, STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return GLR_ECUDA;
  const long long blocks = (long long)a.n_img * lines_per_img / a.lpb;
  GLR_LAUNCH(name, s, k_fft_lines<LOAD, STORE><<<(unsigned)blocks, FFT_THREADS, smem, s>>>(a));
  return GLR_OK;
}

}  // namespace

glr_status launch_fft2(const float* in, float* out, int n_img, int H, int W, int inverse, cudaStream_t s) {
  FftArgs a{};
  a.in = in;
  a.out = out;
  a.n_img = n_img;
  a.H = H;
  a.W = W;
  a.inverse = inverse;
  a.cols = 0;
  glr_status st = run_pass<LOAD_PLAIN, STORE_PLAIN>(a, s, "k_fft_rows");
  if (st != GLR_OK) return st;
  a.in = out;
  a.cols = 1;
  return run_pass<LOAD_PLAIN, STORE_PLAIN>(a, s, "k_fft_cols");
}

glr_status launch_admm_step(const float* y, const float* mask, const float* z, const float* x, float* u, int n_img,
                            int H, int W, float rho, float* x_out, float* w_out, double* residual, double* res_acc,
                            cudaStream_t s) {
  FftArgs a{};
  a.n_img = n_img;
  a.H = H;
  a.W = W;
  a.rho = rho;
  // forward rows of z - (u + x - z), u updated in place
  a.x = x;
  a.z = z;
  a.u = u;
  a.out = x_out;
  a.cols = 0;
  a.inverse = 0;
  glr_status st = run_pass<LOAD_ADMM, STORE_PLAIN>(a, s, "k_fft_rows");
  if (st != GLR_OK) return st;
  // forward columns + data consistency in k-space
  a.in = x_out;
  a.cols = 1;
  a.y = y;
  a.mask = mask;
  a.res_acc = res_acc;
  st = run_pass<LOAD_PLAIN, STORE_DC>(a, s, "k_fft_cols");
  if (st != GLR_OK) return st;
  // inverse columns
  a.inverse = 1;
  st = run_pass<LOAD_PLAIN, STORE_PLAIN>(a, s, "k_fft_cols");
  if (st != GLR_OK) return st;
  // inverse rows: x_new and the next denoiser input
  a.cols = 0;
  a.w_out = w_out;
  a.res_out = residual;
  return run_pass<LOAD_PLAIN, STORE_ADMM>(a, s, "k_fft_rows");
}

}  // namespace glr
