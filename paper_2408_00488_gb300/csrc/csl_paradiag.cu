// All-at-once time solve built on the batched shifted solves (Section 1: the
// alpha-circulant approximation of a triangular time-discretisation matrix is
// block-diagonalised into complex-shifted Laplacian systems).
//
// Backward Euler for u' + K u = g on L steps of size tau is the block system
//     (B kron I + I kron K) U = F,   B = (I - S)/tau,   F_0 = g_0 + u0/tau,  F_n = g_n,
// solved by preconditioned Richardson U <- U + P_a^{-1} (F - A U) with
//     P_a = C_a kron I + I kron K,   C_a = (I - S_a)/tau   (S with a in its corner).
// With Gam = diag(a^{-j/L}) and the DFT matrix Fd, C_a = Gam Fd^{-1} diag(d_k) Fd Gam^{-1},
// d_k = (1 - a^{1/L} e^{-2 pi i k/L}) / tau, so P_a^{-1} R is
//     R_hat = Fd (a^{j/L} R_j)          k_pd_time_fft (forward)
//     (d_k I + K) Z_hat_k = R_hat_k     one csl_batch_solve over the L shifts
//     U += a^{-j/L} (Fd^{-1} Z_hat)_j   k_pd_time_fft (inverse, fused update)
// The residual uses the library's own stencil (csl_apply with lambda = 1/tau)
// and k_pd_residual; every sweep reads one norm back to the host.
//
// Time slices are stored slice-major: value of slice j at grid point p at
// index j*M + p (complex128).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/csl.h"

void csl_internal_set_error(const char* msg);

namespace {

constexpr int kPdThreads = 256;
constexpr int kPdRedBlocks = 512;
constexpr int kPdTile = 4096;  // complex values of one FFT tile: points per CTA x L

// Radix-2 decimation-in-time FFT over the time index of a tile of P grid
// points (values v[j*P + q] in shared memory, input written in bit-reversed
// order).  FWD: exp(-2 pi i m/L); inverse: conjugate twiddles.
template <bool FWD>
__device__ void tile_fft(double2* v, int P, int L, int logL, const double2* tw) {
  const int half_total = P * (L >> 1);
  for (int s = 1; s <= logL; ++s) {
    const int half = 1 << (s - 1), span = half << 1, tstride = L >> s;
    for (int b = threadIdx.x; b < half_total; b += blockDim.x) {
      const int q = b % P, bb = b / P;  // point, butterfly within the line
      const int grp = bb / half, pos = bb - grp * half;
      const int i0 = grp * span + pos, i1 = i0 + half;
      double2 w = tw[pos * tstride];
      if (!FWD) w.y = -w.y;
      const double2 x0 = v[i0 * P + q], x1 = v[i1 * P + q];
      const double2 t = make_double2(w.x * x1.x - w.y * x1.y, w.x * x1.y + w.y * x1.x);
      v[i0 * P + q] = make_double2(x0.x + t.x, x0.y + t.y);
      v[i1 * P + q] = make_double2(x0.x - t.x, x0.y - t.y);
    }
    __syncthreads();
  }
}

// forward: out_k = sum_j e^{-2 pi i jk/L} (scale_j in_j);
// inverse: acc_j += scale_j (1/L) sum_k e^{+2 pi i jk/L} in_k
template <bool FWD>
__global__ void __launch_bounds__(kPdThreads) k_pd_time_fft(const double2* in, double2* out, long M, int L,
                                                            int logL, const double* scale, const double2* tw) {
  extern __shared__ double2 pd_tile[];
  const int P = kPdTile / L;
  const long ntiles = (M + P - 1) / P;
  for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long p0 = t * P;
    for (int i = threadIdx.x; i < P * L; i += blockDim.x) {
      const int j = i / P, q = i - j * P;
      const long p = p0 + q;
      const int jr = (int)(__brev((unsigned)j) >> (32 - logL));
      double2 x = make_double2(0.0, 0.0);
      if (p < M) {
        x = in[(long)j * M + p];
        if (FWD) {
          x.x *= scale[j];
          x.y *= scale[j];
        }
      }
      pd_tile[jr * P + q] = x;
    }
    __syncthreads();
    tile_fft<FWD>(pd_tile, P, L, logL, tw);
    for (int i = threadIdx.x; i < P * L; i += blockDim.x) {
      const int k = i / P, q = i - k * P;
      const long p = p0 + q;
      if (p >= M) continue;
      const double2 y = pd_tile[k * P + q];
      if (FWD) {
        out[(long)k * M + p] = y;
      } else {
        const double s = scale[k] / (double)L;
        double2 u = out[(long)k * M + p];
        u.x = fma(s, y.x, u.x);
        u.y = fma(s, y.y, u.y);
        out[(long)k * M + p] = u;
      }
    }
    __syncthreads();
  }
}

// R_n = F_n - R_n + U_{n-1}/tau (R holds (K + I/tau) U_n on entry); partial
// sums of |R|^2 (and |F|^2 when fnorm) per block, in block order
__global__ void __launch_bounds__(kPdThreads) k_pd_residual(double2* R, const double2* F, const double2* U, long M,
                                                            int L, double inv_tau, double* part, int fnorm) {
  double acc = 0.0, accf = 0.0;
  const long tot = M * (long)L;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
    const long n = i / M;
    const double2 f = F[i];
    double2 r = R[i];
    r.x = f.x - r.x;
    r.y = f.y - r.y;
    if (n > 0) {
      const double2 up = U[i - M];
      r.x = fma(inv_tau, up.x, r.x);
      r.y = fma(inv_tau, up.y, r.y);
    }
    R[i] = r;
    acc = fma(r.x, r.x, fma(r.y, r.y, acc));
    if (fnorm) accf = fma(f.x, f.x, fma(f.y, f.y, accf));
  }
  __shared__ double sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    accf += __shfl_xor_sync(0xffffffffu, accf, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = acc;
    sh[1][w] = accf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += sh[0][i];
      b += sh[1][i];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// F = g, F_0 += u0 / tau
__global__ void k_pd_rhs(double2* F, const double2* g, const double2* u0, long M, int L, double inv_tau) {
  const long tot = M * (long)L;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
    double2 v = g[i];
    if (i < M) {
      v.x = fma(inv_tau, u0[i].x, v.x);
      v.y = fma(inv_tau, u0[i].y, v.y);
    }
    F[i] = v;
  }
}

int ilog2_pow2(int v) {
  if (v <= 0 || (v & (v - 1))) return -1;
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

struct csl_paradiag {
  int dim = 2, L = 0, logL = 0;
  long M = 0;
  double tau = 0, a = 0;
  cudaStream_t s = nullptr;
  csl_plan* apply_plan = nullptr;
  csl_batch* batch = nullptr;
  double2 *U = nullptr, *R = nullptr, *Rh = nullptr, *Zh = nullptr, *F = nullptr, *tw = nullptr;
  double *sf = nullptr, *sb = nullptr, *part = nullptr;
  std::vector<void*> allocs;
};

namespace {
void* pd_alloc(csl_paradiag* P, size_t bytes, cudaError_t* e) {
  if (*e != cudaSuccess) return nullptr;
  void* p = nullptr;
  *e = cudaMalloc(&p, bytes);
  if (*e == cudaSuccess) P->allocs.push_back(p);
  return p;
}

void pd_free(csl_paradiag* P) {
  if (!P) return;
  if (P->batch) csl_batch_destroy(P->batch);
  if (P->apply_plan) csl_plan_destroy(P->apply_plan);
  for (void* p : P->allocs) cudaFree(p);
  delete P;
}
}  // namespace

extern "C" {

csl_status csl_paradiag_create(csl_paradiag** out, int dim, const int64_t n[3], const double* const coef_faces[3],
                               int L, double tau, double a, const csl_plan_options* opt, void* stream) {
  if (!out) return CSL_INVALID_ARG;
  *out = nullptr;
  if (!n || !coef_faces || (dim != 2 && dim != 3)) return CSL_INVALID_ARG;
  if (!(tau > 0.0) || !isfinite(tau) || !(a > 0.0) || !(a < 1.0)) return CSL_INVALID_ARG;
  const int logL = ilog2_pow2(L);
  if (logL < 1 || L > 1024) return CSL_UNSUPPORTED_SIZE;
  csl_paradiag* P = new (std::nothrow) csl_paradiag();
  if (!P) return CSL_OUT_OF_MEMORY;
  P->dim = dim;
  P->L = L;
  P->logL = logL;
  P->tau = tau;
  P->a = a;
  P->s = (cudaStream_t)stream;
  P->M = 1;
  for (int d = 0; d < dim; ++d) P->M *= n[d];
  // (K + I/tau) for the residual
  csl_status st = csl_plan_create(&P->apply_plan, dim, n, coef_faces, 1.0 / tau, 0.0, opt, stream);
  if (st != CSL_OK) {
    pd_free(P);
    return st;
  }
  // the L shifted systems d_k I + K
  std::vector<csl_system_desc> sys(L);
  const double ra = pow(a, 1.0 / L);
  for (int k = 0; k < L; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)L;
    csl_system_desc& d = sys[k];
    memset(&d, 0, sizeof(d));
    d.dim = dim;
    for (int i = 0; i < 3; ++i) d.n[i] = i < dim ? n[i] : 1;
    for (int i = 0; i < dim; ++i) d.coef_faces[i] = coef_faces[i];
    d.alpha = (1.0 - ra * cos(ang)) / tau;
    d.beta = -ra * sin(ang) / tau;
  }
  st = csl_batch_create(&P->batch, L, sys.data(), opt, stream);
  if (st != CSL_OK) {
    pd_free(P);
    return st;
  }
  cudaError_t e = cudaSuccess;
  const size_t vb = sizeof(double2) * (size_t)P->M * L;
  P->U = (double2*)pd_alloc(P, vb, &e);
  P->R = (double2*)pd_alloc(P, vb, &e);
  P->Rh = (double2*)pd_alloc(P, vb, &e);
  P->Zh = (double2*)pd_alloc(P, vb, &e);
  P->F = (double2*)pd_alloc(P, vb, &e);
  P->tw = (double2*)pd_alloc(P, sizeof(double2) * (L / 2), &e);
  P->sf = (double*)pd_alloc(P, sizeof(double) * L, &e);
  P->sb = (double*)pd_alloc(P, sizeof(double) * L, &e);
  P->part = (double*)pd_alloc(P, sizeof(double) * 2 * kPdRedBlocks, &e);
  if (e == cudaSuccess) {
    std::vector<double2> tw(L / 2);
    std::vector<double> sf(L), sb(L);
    for (int m = 0; m < L / 2; ++m) tw[m] = make_double2(cos(2.0 * M_PI * m / L), -sin(2.0 * M_PI * m / L));
    for (int j = 0; j < L; ++j) {
      sf[j] = pow(a, (double)j / L);
      sb[j] = pow(a, -(double)j / L);
    }
    e = cudaMemcpy(P->tw, tw.data(), sizeof(double2) * (L / 2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->sf, sf.data(), sizeof(double) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->sb, sb.data(), sizeof(double) * L, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pd_time_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)(kPdTile * sizeof(double2)));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pd_time_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)(kPdTile * sizeof(double2)));
  if (e != cudaSuccess) {
    csl_internal_set_error(cudaGetErrorString(e));
    (void)cudaGetLastError();
    pd_free(P);
    return e == cudaErrorMemoryAllocation ? CSL_OUT_OF_MEMORY : CSL_CUDA_ERROR;
  }
  *out = P;
  return CSL_OK;
}

void csl_paradiag_destroy(csl_paradiag* pd) { pd_free(pd); }

csl_status csl_paradiag_solve(csl_paradiag* P, const double* u0, const double* g, double* u, double tol,
                              int maxit, double inner_tol, int inner_maxit, csl_paradiag_info* info) {
  if (!P || !u0 || !g || !u || !(tol >= 0.0) || maxit < 0 || !(inner_tol > 0.0) || inner_maxit < 1)
    return CSL_INVALID_ARG;
  const long M = P->M;
  const int L = P->L;
  const size_t vb = sizeof(double2) * (size_t)M * L;
  cudaStream_t s = P->s;
  csl_paradiag_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.status = CSL_NOT_CONVERGED;
  const long tot = M * (long)L;
  const int eblocks = (int)((tot + kPdThreads - 1) / kPdThreads < kPdRedBlocks ? (tot + kPdThreads - 1) / kPdThreads
                                                                               : kPdRedBlocks);
  const int P_pts = 4096 / L;
  const long ntiles = (M + P_pts - 1) / P_pts;
  const int fblocks = (int)(ntiles < 4096 ? ntiles : 4096);
  const size_t fsmem = kPdTile * sizeof(double2);
  cudaError_t e = cudaMemsetAsync(P->U, 0, vb, s);
  if (e == cudaSuccess) {
    k_pd_rhs<<<eblocks, kPdThreads, 0, s>>>(P->F, (const double2*)g, (const double2*)u0, M, L, 1.0 / P->tau);
    e = cudaGetLastError();
  }
  std::vector<double> part(2 * kPdRedBlocks);
  std::vector<const double*> fp(L);
  std::vector<double*> zp(L);
  for (int k = 0; k < L; ++k) {
    fp[k] = (const double*)(P->Rh + (long)k * M);
    zp[k] = (double*)(P->Zh + (long)k * M);
  }
  std::vector<csl_solve_info> infos(L);
  double fnorm = -1.0;
  csl_status result = CSL_OK;
  for (int sweep = 0; e == cudaSuccess; ++sweep) {
    // R = F - A U
    csl_status st = CSL_OK;
    for (int t = 0; t < L && st == CSL_OK; ++t)
      st = csl_apply(P->apply_plan, (const double*)(P->U + (long)t * M), (double*)(P->R + (long)t * M));
    if (st != CSL_OK) {
      result = st;
      break;
    }
    k_pd_residual<<<eblocks, kPdThreads, 0, s>>>(P->R, P->F, P->U, M, L, 1.0 / P->tau, P->part, fnorm < 0.0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), P->part, sizeof(double) * 2 * eblocks,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    double rr = 0.0, ff = 0.0;
    for (int b = 0; b < eblocks; ++b) {
      rr += part[2 * b];
      ff += part[2 * b + 1];
    }
    if (fnorm < 0.0) fnorm = sqrt(ff);
    inf.relres = fnorm > 0.0 ? sqrt(rr) / fnorm : 0.0;
    if (!(inf.relres == inf.relres)) {
      result = CSL_BREAKDOWN;
      break;
    }
    if (inf.relres <= tol) {
      inf.status = CSL_OK;
      break;
    }
    if (sweep >= maxit) break;
    // U += P_a^{-1} R
    k_pd_time_fft<true><<<fblocks, kPdThreads, fsmem, s>>>(P->R, P->Rh, M, L, P->logL, P->sf, P->tw);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    st = csl_batch_solve(P->batch, fp.data(), zp.data(), inner_tol, inner_maxit, infos.data());
    for (int k = 0; k < L; ++k)
      if (infos[k].iters > inf.inner_iters_max) inf.inner_iters_max = infos[k].iters;
    if (st != CSL_OK && st != CSL_NOT_CONVERGED) {
      result = st;
      break;
    }
    k_pd_time_fft<false><<<fblocks, kPdThreads, fsmem, s>>>(P->Zh, P->U, M, L, P->logL, P->sb, P->tw);
    e = cudaGetLastError();
    inf.sweeps = sweep + 1;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, P->U, vb, cudaMemcpyDeviceToDevice, s);
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
