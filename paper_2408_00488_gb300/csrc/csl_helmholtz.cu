// The shifted system as a preconditioner (Section 1: the complex-shifted
// Laplacian was introduced as the "shifted Laplace" preconditioner of
// Helmholtz problems): restarted flexible GMRES for
//     (K + lambda_A I) u = f,      e.g. lambda_A = -k^2,
// right-preconditioned by z_j = M^{-1} v_j, M = K + lambda_M I (e.g.
// lambda_M = -k^2 (1 - 0.5 i)), each application one csl_solve of the
// library's preconditioned MINRES to a relative residual inner_tol.  The
// flexible variant keeps the z_j, so inexact inner solves are allowed.
//
// A z is (K + lambda_M I) z from csl_apply plus (lambda_A - lambda_M) z, so
// that one plan serves both operators (a plan for a real lambda_A could be
// refused as singular although only its operator is needed).  Arnoldi runs
// two passes of classical Gram-Schmidt with deterministic multi-dot and
// multi-axpy kernels; the (restart+1) x restart Hessenberg matrix and its
// complex Givens rotations live on the host.  Inner product <v, w> = sum
// conj(v) w over the M complex entries.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <complex>
#include <new>
#include <vector>

#include "../../include/csl.h"

void csl_internal_set_error(const char* msg);

namespace {

typedef std::complex<double> cplx;
constexpr int kHzThreads = 256;
constexpr int kHzChunks = 128;  // blocks per vector in the reductions

__device__ __forceinline__ double2 cmla(double2 acc, double2 c, double2 v) {  // acc + c v
  return make_double2(fma(c.x, v.x, fma(-c.y, v.y, acc.x)), fma(c.x, v.y, fma(c.y, v.x, acc.y)));
}

// part[(i * chunks + chunk)] = sum over the chunk of conj(V_i) w, i = blockIdx.y
__global__ void __launch_bounds__(kHzThreads) k_hz_multidot(const double2* V, const double2* w, long M,
                                                            double2* part) {
  const double2* v = V + (long)blockIdx.y * M;
  double re = 0.0, im = 0.0;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
    const double2 a = v[p], b = w[p];
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
  __shared__ double sh[2][kHzThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = re;
    sh[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kHzThreads / 32; ++i) {
      a += sh[0][i];
      b += sh[1][i];
    }
    part[(long)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(a, b);
  }
}

// w += sum_{i < nv} c_i V_i  (c on the device)
__global__ void __launch_bounds__(kHzThreads) k_hz_multiaxpy(const double2* V, int nv, const double2* c, double2* w,
                                                             long M) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
    double2 acc = w[p];
    for (int i = 0; i < nv; ++i) acc = cmla(acc, c[i], V[(long)i * M + p]);
    w[p] = acc;
  }
}

// out = s * in (real s)
__global__ void k_hz_scale(double2* out, const double2* in, double s, long M) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x)
    out[p] = make_double2(s * in[p].x, s * in[p].y);
}

// out = (K + lambda_M) z on entry; out += c z  ->  (K + lambda_A) z.  With f:
// out = f - out (a residual).
__global__ void k_hz_finish_apply(double2* out, const double2* z, double2 c, const double2* f, long M) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
    double2 a = cmla(out[p], c, z[p]);
    if (f) a = make_double2(f[p].x - a.x, f[p].y - a.y);
    out[p] = a;
  }
}

}  // namespace

struct csl_helmholtz {
  int restart = 0;
  long M = 0;
  cplx lamA, lamM;
  cudaStream_t s = nullptr;
  csl_plan* planM = nullptr;
  double2 *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *x = nullptr, *coef = nullptr, *part = nullptr;
  std::vector<void*> allocs;
  int blocks = 1;
};

namespace {
void* hz_alloc(csl_helmholtz* H, size_t bytes, cudaError_t* e) {
  if (*e != cudaSuccess) return nullptr;
  void* p = nullptr;
  *e = cudaMalloc(&p, bytes);
  if (*e == cudaSuccess) H->allocs.push_back(p);
  return p;
}
void hz_free(csl_helmholtz* H) {
  if (!H) return;
  if (H->planM) csl_plan_destroy(H->planM);
  for (void* p : H->allocs) cudaFree(p);
  delete H;
}

// conj(V_i) . w for i < nv, summed over the chunks in a fixed order
cudaError_t hz_dots(csl_helmholtz* H, const double2* V, int nv, const double2* w, std::vector<cplx>& out) {
  k_hz_multidot<<<dim3(kHzChunks, nv), kHzThreads, 0, H->s>>>(V, w, H->M, H->part);
  cudaError_t e = cudaGetLastError();
  std::vector<double2> part((size_t)nv * kHzChunks);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), H->part, sizeof(double2) * part.size(), cudaMemcpyDeviceToHost, H->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(H->s);
  out.assign(nv, cplx(0.0, 0.0));
  for (int i = 0; i < nv && e == cudaSuccess; ++i)
    for (int b = 0; b < kHzChunks; ++b) out[i] += cplx(part[(size_t)i * kHzChunks + b].x, part[(size_t)i * kHzChunks + b].y);
  return e;
}

// out = (K + lambda_A) z, or f - (K + lambda_A) z when f is given
csl_status hz_apply(csl_helmholtz* H, const double2* z, double2* out, const double2* f) {
  const csl_status st = csl_apply(H->planM, (const double*)z, (double*)out);
  if (st != CSL_OK) return st;
  const cplx c = H->lamA - H->lamM;
  k_hz_finish_apply<<<H->blocks, kHzThreads, 0, H->s>>>(out, z, make_double2(c.real(), c.imag()), f, H->M);
  return cudaGetLastError() == cudaSuccess ? CSL_OK : CSL_CUDA_ERROR;
}
}  // namespace

extern "C" {

csl_status csl_helmholtz_create(csl_helmholtz** out, int dim, const int64_t n[3], const double* const coef_faces[3],
                                double lam_re, double lam_im, double shift_re, double shift_im, int restart,
                                const csl_plan_options* opt, void* stream) {
  if (!out) return CSL_INVALID_ARG;
  *out = nullptr;
  if (!n || !coef_faces || restart < 1 || restart > 200) return CSL_INVALID_ARG;
  if (!isfinite(lam_re) || !isfinite(lam_im) || !isfinite(shift_re) || !isfinite(shift_im)) return CSL_INVALID_ARG;
  csl_helmholtz* H = new (std::nothrow) csl_helmholtz();
  if (!H) return CSL_OUT_OF_MEMORY;
  H->restart = restart;
  H->lamA = cplx(lam_re, lam_im);
  H->lamM = cplx(shift_re, shift_im);
  H->s = (cudaStream_t)stream;
  csl_status st = csl_plan_create(&H->planM, dim, n, coef_faces, shift_re, shift_im, opt, stream);
  if (st != CSL_OK) {
    hz_free(H);
    return st;
  }
  H->M = 1;
  for (int d = 0; d < dim; ++d) H->M *= n[d];
  const long M = H->M;
  const long b = (M + kHzThreads - 1) / kHzThreads;
  H->blocks = (int)(b < 4096 ? b : 4096);
  cudaError_t e = cudaSuccess;
  H->V = (double2*)hz_alloc(H, sizeof(double2) * (size_t)M * (restart + 1), &e);
  H->Z = (double2*)hz_alloc(H, sizeof(double2) * (size_t)M * restart, &e);
  H->w = (double2*)hz_alloc(H, sizeof(double2) * (size_t)M, &e);
  H->r = (double2*)hz_alloc(H, sizeof(double2) * (size_t)M, &e);
  H->x = (double2*)hz_alloc(H, sizeof(double2) * (size_t)M, &e);
  H->coef = (double2*)hz_alloc(H, sizeof(double2) * (restart + 1), &e);
  H->part = (double2*)hz_alloc(H, sizeof(double2) * (size_t)kHzChunks * (restart + 1), &e);
  if (e != cudaSuccess) {
    csl_internal_set_error(cudaGetErrorString(e));
    (void)cudaGetLastError();
    hz_free(H);
    return e == cudaErrorMemoryAllocation ? CSL_OUT_OF_MEMORY : CSL_CUDA_ERROR;
  }
  *out = H;
  return CSL_OK;
}

void csl_helmholtz_destroy(csl_helmholtz* H) { hz_free(H); }

csl_status csl_helmholtz_solve(csl_helmholtz* H, const double* f_, double* u, double tol, int maxit,
                               double inner_tol, int inner_maxit, csl_helmholtz_info* info) {
  if (!H || !f_ || !u || !(tol >= 0.0) || maxit < 0 || !(inner_tol > 0.0) || inner_maxit < 1)
    return CSL_INVALID_ARG;
  const long M = H->M;
  const int m = H->restart;
  const double2* f = (const double2*)f_;
  cudaStream_t s = H->s;
  csl_helmholtz_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.status = CSL_NOT_CONVERGED;
  csl_status result = CSL_OK;
  cudaError_t e = cudaMemsetAsync(H->x, 0, sizeof(double2) * M, s);
  std::vector<cplx> d;
  double fnorm = 0.0;
  if (e == cudaSuccess) e = hz_dots(H, f, 1, f, d);
  if (e == cudaSuccess) fnorm = sqrt(d[0].real());
  std::vector<cplx> Hm((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), hcol;
  auto Hat = [&](int i, int j) -> cplx& { return Hm[(size_t)i * m + j]; };
  while (e == cudaSuccess && result == CSL_OK) {
    // r = f - A x, beta = ||r||
    csl_status st = hz_apply(H, H->x, H->r, f);
    if (st != CSL_OK) {
      result = st;
      break;
    }
    e = hz_dots(H, H->r, 1, H->r, d);
    if (e != cudaSuccess) break;
    const double beta = sqrt(d[0].real());
    inf.relres = fnorm > 0.0 ? beta / fnorm : 0.0;
    if (!(inf.relres == inf.relres)) {
      result = CSL_BREAKDOWN;
      break;
    }
    if (inf.relres <= tol || fnorm == 0.0) {
      inf.status = CSL_OK;
      break;
    }
    if (inf.iters >= maxit) break;
    if (inf.iters > 0) inf.restarts += 1;
    k_hz_scale<<<H->blocks, kHzThreads, 0, s>>>(H->V, H->r, 1.0 / beta, M);
    std::fill(Hm.begin(), Hm.end(), cplx(0.0, 0.0));
    std::fill(g.begin(), g.end(), cplx(0.0, 0.0));
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m && e == cudaSuccess && result == CSL_OK; ++j) {
      double2* vj = H->V + (long)j * M;
      double2* zj = H->Z + (long)j * M;
      csl_solve_info si;
      st = csl_solve(H->planM, (const double*)vj, (double*)zj, inner_tol, inner_maxit, &si);
      if (st != CSL_OK && st != CSL_NOT_CONVERGED) {
        result = st;
        break;
      }
      inf.inner_iters_total += si.iters;
      st = hz_apply(H, zj, H->w, nullptr);
      if (st != CSL_OK) {
        result = st;
        break;
      }
      // two passes of classical Gram-Schmidt
      for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        e = hz_dots(H, H->V, j + 1, H->w, hcol);
        if (e != cudaSuccess) break;
        std::vector<double2> c(j + 1);
        for (int i = 0; i <= j; ++i) {
          Hat(i, j) += hcol[i];
          c[i] = make_double2(-hcol[i].real(), -hcol[i].imag());
        }
        e = cudaMemcpyAsync(H->coef, c.data(), sizeof(double2) * (j + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
          k_hz_multiaxpy<<<H->blocks, kHzThreads, 0, s>>>(H->V, j + 1, H->coef, H->w, M);
          e = cudaGetLastError();
        }
        // the coefficients' host buffer must outlive the copy
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      }
      if (e != cudaSuccess) break;
      e = hz_dots(H, H->w, 1, H->w, d);
      if (e != cudaSuccess) break;
      const double hn = sqrt(d[0].real());
      Hat(j + 1, j) = hn;
      k_hz_scale<<<H->blocks, kHzThreads, 0, s>>>(H->V + (long)(j + 1) * M, H->w, hn > 0.0 ? 1.0 / hn : 0.0, M);
      // rotations: with c = a/rho, s = b/rho,
      // (top, bottom) -> (conj(c) top + conj(s) bottom, -s top + c bottom)
      for (int i = 0; i < j; ++i) {
        const cplx t = std::conj(cs[i]) * Hat(i, j) + std::conj(sn[i]) * Hat(i + 1, j);
        Hat(i + 1, j) = -sn[i] * Hat(i, j) + cs[i] * Hat(i + 1, j);
        Hat(i, j) = t;
      }
      const cplx a = Hat(j, j), b = Hat(j + 1, j);
      const double rho = sqrt(std::norm(a) + std::norm(b));
      cs[j] = rho > 0.0 ? a / rho : cplx(1.0, 0.0);
      sn[j] = rho > 0.0 ? b / rho : cplx(0.0, 0.0);
      Hat(j, j) = rho;
      Hat(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = std::conj(cs[j]) * g[j];
      inf.iters += 1;
      jdone = j + 1;
      if (std::abs(g[j + 1]) <= tol * fnorm || inf.iters >= maxit || hn == 0.0) break;
    }
    if (e != cudaSuccess || result != CSL_OK || jdone == 0) break;
    // y = H^{-1} g (upper triangular), x += Z y
    std::vector<cplx> y(jdone);
    for (int i = jdone - 1; i >= 0; --i) {
      cplx acc = g[i];
      for (int k = i + 1; k < jdone; ++k) acc -= Hat(i, k) * y[k];
      y[i] = acc / Hat(i, i);
    }
    std::vector<double2> c(jdone);
    for (int i = 0; i < jdone; ++i) c[i] = make_double2(y[i].real(), y[i].imag());
    e = cudaMemcpyAsync(H->coef, c.data(), sizeof(double2) * jdone, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_hz_multiaxpy<<<H->blocks, kHzThreads, 0, s>>>(H->Z, jdone, H->coef, H->x, M);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, H->x, sizeof(double2) * M, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    csl_internal_set_error(cudaGetErrorString(e));
    (void)cudaGetLastError();
    result = CSL_CUDA_ERROR;
  }
  if (result != CSL_OK) inf.status = result;
  if (info) *info = inf;
  return result != CSL_OK ? result : (csl_status)inf.status;
}

}  // extern "C"
