// csl_precondition_static: P^{-1} v (the preconditioner application of
// csl_precondition) for callers that cannot allocate device memory -- for
// example code running inside a runtime whose memory pool owns all device
// memory, or a fixed-budget embedded service.  It allocates nothing: all
// scratch lives in the file-scope __device__ arrays below, sized for grids
// of at most kStaticMaxPoints points.
//
// Every call on a device shares these arrays (every GPU that loads the
// library holds them until the process exits), so calls that overlap on the
// GPU (different streams, or different host threads) race and must be
// serialised by the caller.  Each call rewrites every table and every
// intermediate it reads, so nothing needs clearing between calls.
//
// Set-up: the first call on a device looks up the device addresses of the
// arrays (cudaGetSymbolAddress) with that device current.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/csl.h"
#include "csl_passes.cuh"

using namespace csl;

void csl_internal_set_error(const char* msg);  // csl_api.cu

namespace {

constexpr long kStaticMaxPoints = 262144;  // e.g. 511^2 in 2D, 63^3 in 3D
constexpr int kMaxN = 1024;                 // transform length n + 1
constexpr int kMaxDevices = 64;

// per-axis table sizes (in doubles): twiddles (N/2 complex), half sines
// (N/2+1), extra twiddles (line_tp_size(N) complex), eigenvalues (n, FP64 and FP32)
constexpr int kTwD = kMaxN;                        // N/2 complex = N doubles
constexpr int kHsD = kMaxN / 2 + 2;
constexpr int kTpD = 2 * (8 * 8 + 8 * 8 * 16) + 2;  // largest line_tp_size (N = 1024), complex
constexpr int kAxisD = kTwD + kHsD + kTpD + 2 * kMaxN;

__device__ __align__(256) double g_static_T[2 * kStaticMaxPoints];     // intermediate (double2 / float2)
__device__ __align__(256) double g_static_scale[kStaticMaxPoints];     // per-mode scale (FP64 path)
__device__ __align__(256) double g_static_tables[3 * kAxisD];          // per-axis tables

struct StaticPtrs {
  double* T;
  double* scale;
  double* tables;
};
StaticPtrs g_ptrs[kMaxDevices];
std::once_flag g_once[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];

int ilog2_exact_s(long v) {
  if (v <= 0 || (v & (v - 1))) return -1;
  int l = 0;
  while ((1L << l) < v) ++l;
  return l;
}

// Tables of one axis, in the precision T, laid out in the axis slice:
//   tw[m] = exp(-2 pi i m/N) (m < N/2), hs[j] = sin(pi j/N)/2 (j <= N/2),
//   tp = extra twiddles (layout of LineDst<T,N>::TP), mu_d[k], mu_f[k]
//   (mu_k = (4/h^2) sin^2(k pi / (2N)), k = 1..n, h = 1/N).
template <typename T>
struct AxisTables {
  typename C2<T>::t* tw;
  T* hs;
  typename C2<T>::t* tp;
  double* mu_d;
  float* mu_f;
};

template <typename T>
__host__ __device__ AxisTables<T> axis_tables(double* base) {
  AxisTables<T> a;
  a.tw = (typename C2<T>::t*)base;
  a.hs = (T*)(base + kTwD);
  a.tp = (typename C2<T>::t*)(base + kTwD + kHsD);
  a.mu_d = base + kTwD + kHsD + kTpD;
  a.mu_f = (float*)(base + kTwD + kHsD + kTpD + kMaxN);
  return a;
}

// exp(-2 pi i num/den) with sincospi (exact argument reduction)
__device__ void root_of_unity(long num, long den, double& c, double& s) {
  double sn, cs;
  sincospi(2.0 * (double)(num % den) / (double)den, &sn, &cs);
  c = cs;
  s = -sn;
}

template <typename T>
__global__ void k_static_axis_tables(double* tables, int N) {
  AxisTables<T> a = axis_tables<T>(tables);
  const int H = N / 2, n = N - 1;
  const double h = 1.0 / (double)N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N + 8 * 8 * 16 + 8 * 8 + 2; i += gridDim.x * blockDim.x) {
    double c, s;
    if (i < H) {
      root_of_unity(i, N, c, s);
      a.tw[i] = mkc<T>((T)c, (T)s);
    }
    if (i <= H) a.hs[i] = (T)(i == H ? 0.5 : 0.5 * sinpi((double)i / (double)N));
    if (i >= 1 && i <= n) {
      const double sn = sinpi((double)i / (2.0 * N));
      a.mu_d[i - 1] = 4.0 / (h * h) * sn * sn;
      a.mu_f[i - 1] = (float)a.mu_d[i - 1];
    }
    // extra twiddles
    if (N >= 64 && N < 512) {
      int R1 = 0, R2 = 0;
      if (N == 64) { R1 = DstShape<64>::R1; R2 = DstShape<64>::R2; }
      if (N == 128) { R1 = DstShape<128>::R1; R2 = DstShape<128>::R2; }
      if (N == 256) { R1 = DstShape<256>::R1; R2 = DstShape<256>::R2; }
      if (i < R1 * R2) {
        const int k1 = i / R2, g = i - k1 * R2;
        root_of_unity((long)g * k1, N, c, s);
        a.tp[i] = mkc<T>((T)c, (T)s);
      }
    } else if (N >= 512) {
      const int R0 = 8, R1 = 8, R2 = N == 1024 ? 16 : 8;
      const int n2 = R0 * R1, n3 = R0 * R1 * R2;
      if (i < n2) {
        const int q = i / R0, k = i - q * R0;
        root_of_unity((long)q * k, (long)R0 * R1, c, s);
        a.tp[i] = mkc<T>((T)c, (T)s);
      } else if (i < n2 + n3) {
        const int r = i - n2, Ls = R0 * R1;
        const int q = r / Ls, k = r - q * Ls;
        root_of_unity((long)q * k, (long)Ls * R2, c, s);
        a.tp[i] = mkc<T>((T)c, (T)s);
      }
    }
  }
}

// per-mode scale cnorm / sqrt((gamma sum mu + alpha)^2 + beta^2) (FP64 path)
__global__ void k_static_scale(double* scale, const double* mux, const double* muy, const double* muz, int nx,
                               int ny, int nz, double gamma, double alpha, double beta, double cnorm) {
  const long M = (long)nx * ny * nz;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
    const long row = p / nx;
    const int ix = (int)(p - row * nx);
    const int iz = (int)(row / ny);
    const int iy = (int)(row - (long)iz * ny);
    double mu = mux[ix] + muy[iy];
    if (muz) mu += muz[iz];
    const double e = fma(gamma, mu, alpha);
    const double q = fma(e, e, beta * beta);
    scale[p] = q > 0.0 ? cnorm / sqrt(q) : 0.0;
  }
}

void setup_device(int dev) {
  StaticPtrs p;
  cudaError_t e = cudaGetSymbolAddress((void**)&p.T, g_static_T);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&p.scale, g_static_scale);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&p.tables, g_static_tables);
  g_ptrs[dev] = p;
  g_setup_err[dev] = e;
}

// CTA shape of one pass (same rules as the plan's default configuration)
template <typename T>
PassLaunch static_launch(int N, long nlines_or_tiles_per_cta_unit, bool strided, int ncols, int nouter) {
  const int wide = pass_has_wide(N) ? 1 : 0;
  const int tpl = pass_tpl(N, wide);
  int threads = 256;
  if (strided)
    while (threads > 32 && threads > tpl && (threads / tpl) / 2 >= ncols) threads >>= 1;
  while (threads > 32 && threads > tpl && pass_smem<T>(N, wide, threads / tpl) > 100 * 1024) threads >>= 1;
  const int lines = threads / tpl;
  PassLaunch L;
  L.threads = threads;
  L.smem = pass_smem<T>(N, wide, lines);
  long tiles = strided ? (long)((ncols + lines - 1) / lines) * nouter : (nlines_or_tiles_per_cta_unit + lines - 1) / lines;
  L.blocks = (int)(tiles < 4096 ? tiles : 4096);
  return L;
}

// Host-side check of the per-mode scales before anything is launched (the
// call is asynchronous, so the device cannot report a status): every mode's
// q = (gamma mu + alpha)^2 + beta^2 over the grid's modes, mu the sum of the
// per-axis eigenvalues mu_k = (4/h^2) sin^2(k pi / (2N)).  Returns
// CSL_SINGULAR_PRECOND when some q is zero to within rounding (only possible
// for beta = 0, as for csl_plan_create), and for FP32 the power of two sigma
// by which gamma, alpha, beta and cnorm are prescaled (as the plan does), or
// CSL_INVALID_ARG when the scales cnorm / sqrt(q) leave the FP32 range.
csl_status static_check_scales(int dim, const int n[3], double gamma, double alpha, double beta, double cnorm,
                               bool fp32, double* sigma) {
  std::vector<double> mu[3];
  for (int d = 0; d < dim; ++d) {
    const int N = n[d] + 1;
    const double h = 1.0 / (double)N;
    mu[d].resize(n[d]);
    for (int k = 1; k <= n[d]; ++k) {
      const double sn = sin(M_PI * (double)k / (2.0 * N));
      mu[d][k - 1] = 4.0 / (h * h) * sn * sn;
    }
  }
  double qmin = INFINITY, qmax = 0.0;
  bool zero = false;
  const int nz = dim == 3 ? n[2] : 1;
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < n[1]; ++iy)
      for (int ix = 0; ix < n[0]; ++ix) {
        const double m = mu[0][ix] + mu[1][iy] + (dim == 3 ? mu[2][iz] : 0.0);
        const double e = gamma * m + alpha;
        // |e| at the level of the rounding of gamma mu + alpha counts as zero
        if (beta == 0.0 && fabs(e) <= 16.0 * 2.2204460492503131e-16 * (fabs(gamma * m) + fabs(alpha))) zero = true;
        const double q = e * e + beta * beta;
        qmin = q < qmin ? q : qmin;
        qmax = q > qmax ? q : qmax;
      }
  if (zero || !(qmin > 0.0)) {
    csl_internal_set_error("csl_precondition_static: (gamma mu + alpha)^2 + beta^2 = 0 for some mode (singular P)");
    return CSL_SINGULAR_PRECOND;
  }
  *sigma = 1.0;
  if (fp32) {
    // the plan's FP32 rule: |e + i beta| is brought to at most 2^40 when it
    // leaves [2^-40, 2^60]; the scales themselves must be normal floats
    const double mmin = sqrt(qmin), mmax = sqrt(qmax);
    if (mmax > ldexp(1.0, 60) || mmin < ldexp(1.0, -40)) *sigma = ldexp(1.0, 40 - (int)ceil(log2(mmax)));
    const double smin = cnorm / mmax, smax = cnorm / mmin;
    if (!(smin >= ldexp(1.0, -120)) || !(smax <= ldexp(1.0, 120)) || !(mmin * *sigma >= ldexp(1.0, -60))) {
      csl_internal_set_error(
          "csl_precondition_static: the per-mode scales of P^-1 lie outside the FP32 range; use CSL_PREC_FP64");
      return CSL_INVALID_ARG;
    }
  }
  return CSL_OK;
}

template <typename T>
cudaError_t run_static(int dim, const int n[3], double gamma, double alpha, double beta, double sigma,
                       const double2* v, double2* out, cudaStream_t s, const StaticPtrs& P) {
  typedef typename C2<T>::t c_t;
  const long M = (long)n[0] * n[1] * n[2];
  double cnorm = 1.0;
  AxisTables<T> ax[3];
  for (int d = 0; d < dim; ++d) {
    const int N = n[d] + 1;
    cnorm *= 2.0 / (double)N;
    k_static_axis_tables<T><<<8, 256, 0, s>>>(P.tables + (long)d * kAxisD, N);
    ax[d] = axis_tables<T>(P.tables + (long)d * kAxisD);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (sizeof(T) == 8) {
    k_static_scale<<<256, 256, 0, s>>>(P.scale, ax[0].mu_d, ax[1].mu_d, dim == 3 ? ax[2].mu_d : nullptr, n[0], n[1],
                                       n[2], gamma, alpha, beta, cnorm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  c_t* Tbuf = (c_t*)P.T;
  const int nx = n[0], ny = n[1], nz = n[2];
  // x pass: v -> T
  RowArgs<T> r1;
  memset(&r1, 0, sizeof(r1));
  r1.n = nx;
  r1.nrows = (int)(M / nx);
  r1.tw = ax[0].tw;
  r1.hs = ax[0].hs;
  r1.tp = ax[0].tp;
  r1.vin = v;
  r1.tout = Tbuf;
  const PassLaunch Lr = static_launch<T>(nx + 1, M / nx, false, 0, 0);
  e = launch_row<T>(nx + 1, pass_has_wide(nx + 1) ? 1 : 0, LOAD_V, STORE_T, r1, Lr, s);
  if (e != cudaSuccess) return e;
  auto strided = [&](int axis, int nn, int nouter, long outer_stride, long line_stride, bool mid) {
    StridedArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.n = nn;
    a.ncols = nx;
    a.nouter = nouter;
    a.outer_stride = outer_stride;
    a.line_stride = line_stride;
    a.tw = ax[axis].tw;
    a.hs = ax[axis].hs;
    a.tp = ax[axis].tp;
    a.data = Tbuf;
    if (mid) {
      if (sizeof(T) == 8) {
        a.stab = P.scale;
      } else {
        a.mu_line = (const T*)ax[axis].mu_f;
        a.mu_col = (const T*)ax[0].mu_f;
        a.mu_outer = axis == 2 ? (const T*)ax[1].mu_f : nullptr;
      }
      // FP32: gamma, alpha, beta and cnorm times sigma (s_k unchanged, e^2 + beta^2 in range)
      a.gamma = (T)(gamma * sigma);
      a.alpha = (T)(alpha * sigma);
      a.beta2 = (T)((beta * sigma) * (beta * sigma));
      a.cnorm = (T)(cnorm * sigma);
    }
    const PassLaunch L = static_launch<T>(nn + 1, 0, true, nx, nouter);
    return launch_strided<T>(nn + 1, pass_has_wide(nn + 1) ? 1 : 0, mid, a, L, s);
  };
  if (dim == 2) {
    e = strided(1, ny, 1, 0, nx, true);
  } else {
    e = strided(1, ny, nz, (long)nx * ny, nx, false);
    if (e == cudaSuccess) e = strided(2, nz, ny, nx, (long)nx * ny, true);
    if (e == cudaSuccess) e = strided(1, ny, nz, (long)nx * ny, nx, false);
  }
  if (e != cudaSuccess) return e;
  RowArgs<T> r3 = r1;
  r3.vin = nullptr;
  r3.tout = nullptr;
  r3.tin = Tbuf;
  r3.dout = out;
  return launch_row<T>(nx + 1, pass_has_wide(nx + 1) ? 1 : 0, LOAD_T, STORE_D, r3, Lr, s);
}

}  // namespace

extern "C" csl_status csl_precondition_static(int dim, const int64_t n[3], double gamma, double alpha, double beta,
                                              int precision, const double* v, double* out, void* stream) {
  if (!n || !v || !out || (dim != 2 && dim != 3)) return CSL_INVALID_ARG;
  if (!(gamma > 0.0) || !isfinite(gamma) || !isfinite(alpha) || !isfinite(beta)) return CSL_INVALID_ARG;
  if (precision != CSL_PREC_FP64 && precision != CSL_PREC_FP32) return CSL_INVALID_ARG;
  int nn[3] = {1, 1, 1};
  long M = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 1) return CSL_INVALID_ARG;
    if (n[d] + 1 < 4 || n[d] + 1 > kMaxN || ilog2_exact_s(n[d] + 1) < 0) return CSL_UNSUPPORTED_SIZE;
    nn[d] = (int)n[d];
    M *= n[d];
  }
  if (M > kStaticMaxPoints) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "csl_precondition_static: %ld grid points exceed the static scratch capacity of %ld points", M,
             kStaticMaxPoints);
    csl_internal_set_error(msg);
    return CSL_UNSUPPORTED_SIZE;
  }
  double cnorm = 1.0, sigma = 1.0;
  for (int d = 0; d < dim; ++d) cnorm *= 2.0 / (double)(nn[d] + 1);
  const csl_status chk = static_check_scales(dim, nn, gamma, alpha, beta, cnorm, precision == CSL_PREC_FP32, &sigma);
  if (chk != CSL_OK) return chk;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    csl_internal_set_error("csl_precondition_static: no usable current device");
    return CSL_CUDA_ERROR;
  }
  std::call_once(g_once[dev], setup_device, dev);
  if (g_setup_err[dev] != cudaSuccess) {
    csl_internal_set_error("csl_precondition_static: cudaGetSymbolAddress failed during set-up");
    return CSL_CUDA_ERROR;
  }
  e = (precision == CSL_PREC_FP32)
          ? run_static<float>(dim, nn, gamma, alpha, beta, sigma, (const double2*)v, (double2*)out,
                              (cudaStream_t)stream, g_ptrs[dev])
          : run_static<double>(dim, nn, gamma, alpha, beta, 1.0, (const double2*)v, (double2*)out,
                               (cudaStream_t)stream, g_ptrs[dev]);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    csl_internal_set_error("csl_precondition_static: kernel launch failed");
    return CSL_CUDA_ERROR;
  }
  return CSL_OK;
}
