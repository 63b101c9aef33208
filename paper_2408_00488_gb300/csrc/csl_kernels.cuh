// Kernels of the preconditioned MINRES solve of Eq. 2 with the preconditioner
// of Eq. 4 (arXiv 2408.00488).  One MINRES iteration j is four (2D) or six
// (3D) stream-ordered kernels:
//
//   S   k_stencil     u' = A z_j / gamma_j - (gamma_j/gamma_{j-1}) v_{j-1}     (Eq. 2)
//                     delta_j = <A zhat_j, zhat_j>;  optionally the true residual
//                     ||b - A x_j|| of the current iterate (stopping test)
//   P1  k_row<LOAD_LANCZOS>  v_{j+1} = u' - (delta_j/gamma_j) v_j; DST along x
//   (3D: k_strided along y)
//   MID k_strided<mid>   DST along the last axis, per-mode scale of P^{-1},
//                     gamma_{j+1}^2 = sum_k s_k |v^_k|^2 (Parseval), inverse DST;
//                     last block: Givens rotation and update coefficients
//   (3D: k_strided along y)
//   P3  k_row<STORE_Z_UPDATE> inverse DST along x -> z_{j+1};
//                     w_{j+1} = (zhat_j - a3 w_{j-1} - a2 w_j)/a1,  x_j = x_{j-1} + c eta w_{j+1}
//
// The grid reductions are deterministic (block sums in block order by the
// last block to finish), so repeated solves are bitwise identical.
#pragma once
#include "csl_common.cuh"
#include "csl_dst.cuh"

namespace csl {

// ---------------------------------------------------------------------------
// Stencil: (K + alpha I) applied to both blocks at point p (Eq. 1, 5/7-point
// conservative scheme with face samples pre-divided by h^2; dg = sum of the
// point's face coefficients + alpha).
// ---------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;  // nz = 1 in 2D
  long M;
};

template <int DIM, typename TZ>
__device__ __forceinline__ double2 stencil_KA(const TZ* __restrict__ z, const double* __restrict__ cx,
                                              const double* __restrict__ cy, const double* __restrict__ cz,
                                              const double* __restrict__ dg, const Grid& g, long p, int ix,
                                              int iy, int iz, double2& zc) {
  zc = to_d2(z[p]);
  const double d = dg[p];
  double ax = d * zc.x, ay = d * zc.y;
  const long rx = ((long)iz * g.ny + iy) * (g.nx + 1) + ix;
  const double cw = cx[rx], ce = cx[rx + 1];
  if (ix > 0) {
    const double2 q = to_d2(z[p - 1]);
    ax = fma(-cw, q.x, ax);
    ay = fma(-cw, q.y, ay);
  }
  if (ix < g.nx - 1) {
    const double2 q = to_d2(z[p + 1]);
    ax = fma(-ce, q.x, ax);
    ay = fma(-ce, q.y, ay);
  }
  const long ry = ((long)iz * (g.ny + 1) + iy) * g.nx + ix;
  const double cs = cy[ry], cn = cy[ry + g.nx];
  if (iy > 0) {
    const double2 q = to_d2(z[p - g.nx]);
    ax = fma(-cs, q.x, ax);
    ay = fma(-cs, q.y, ay);
  }
  if (iy < g.ny - 1) {
    const double2 q = to_d2(z[p + g.nx]);
    ax = fma(-cn, q.x, ax);
    ay = fma(-cn, q.y, ay);
  }
  if (DIM == 3) {
    const long plane = (long)g.nx * g.ny;
    const long rz = ((long)iz * g.ny + iy) * g.nx + ix;
    const double cd = cz[rz], cu = cz[rz + plane];
    if (iz > 0) {
      const double2 q = to_d2(z[p - plane]);
      ax = fma(-cd, q.x, ax);
      ay = fma(-cd, q.y, ay);
    }
    if (iz < g.nz - 1) {
      const double2 q = to_d2(z[p + plane]);
      ax = fma(-cu, q.x, ax);
      ay = fma(-cu, q.y, ay);
    }
  }
  return make_double2(ax, ay);
}

// block row of Eq. 2: A [z1; z2] = [beta z1 + (K+alpha) z2; (K+alpha) z1 - beta z2]
__device__ __forceinline__ double2 block_A(double2 KAz, double2 zc, double beta) {
  return make_double2(fma(beta, zc.x, KAz.y), fma(-beta, zc.y, KAz.x));
}

__device__ __forceinline__ void point_coords(long p, const Grid& g, int& ix, int& iy, int& iz) {
  const long row = p / g.nx;
  ix = (int)(p - row * g.nx);
  iz = (int)(row / g.ny);
  iy = (int)(row - (long)iz * g.ny);
}

struct StencilArgs {
  Grid g;
  const void* z;          // z_j (unnormalised), TZ
  double2* vold;          // in: v_{j-1}; out: u'
  const double* cx;
  const double* cy;
  const double* cz;
  const double* dg;
  const double2* x;       // current iterate (true-residual check)
  const double2* b;       // right-hand side (block form)
  DevState* st;
  double* partials;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

template <int DIM, typename TZ>
__global__ void __launch_bounds__(256) k_stencil(StencilArgs a) {
  DevState* st = a.st;
  if (st->done) {
    // keep the device-side loop closed whatever set `done` (Givens breakdown, cap, ...)
    if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
    return;
  }
  const double gam = st->gam, gam_old = st->gam_old, beta = st->beta;
  const double inv_g = 1.0 / gam, lanc = gam / gam_old;
  const int check = st->check;
  const TZ* z = (const TZ*)a.z;
  double acc[2] = {0.0, 0.0};
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < a.g.M; p += (long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    point_coords(p, a.g, ix, iy, iz);
    double2 zc;
    const double2 t = stencil_KA<DIM, TZ>(z, a.cx, a.cy, a.cz, a.dg, a.g, p, ix, iy, iz, zc);
    const double2 Az = block_A(t, zc, beta);
    acc[0] = fma(Az.x, zc.x, fma(Az.y, zc.y, acc[0]));
    const double2 vo = a.vold[p];
    a.vold[p] = make_double2(fma(Az.x, inv_g, -lanc * vo.x), fma(Az.y, inv_g, -lanc * vo.y));
    if (check) {
      double2 xc;
      const double2 tx = stencil_KA<DIM, double2>(a.x, a.cx, a.cy, a.cz, a.dg, a.g, p, ix, iy, iz, xc);
      const double2 Ax = block_A(tx, xc, beta);
      const double2 bb = a.b[p];
      const double rx = bb.x - Ax.x, ry = bb.y - Ax.y;
      acc[1] = fma(rx, rx, fma(ry, ry, acc[1]));
    }
  }
  double tot[2];
  if (!grid_sum_last_block<2>(acc, a.partials, &st->tickets[TICKET_STENCIL], tot)) return;
  if (threadIdx.x != 0) return;
  // scalar step after the stencil: delta_j and the stopping test for x_{iter}
  st->delta = tot[0] * inv_g * inv_g;
  if (check) {
    const double rnorm = sqrt(tot[1]);
    const double rel = rnorm / st->bnorm;
    st->relres = rel;
    st->checks += 1;
    st->check = 0;
    if (rel <= st->tol) {
      st->done = 1;
      st->status = ST_OK;
    } else if (st->lucky || st->iter >= st->maxit || !(rel == rel)) {
      st->done = 1;
      st->status = (rel == rel) ? ST_NOT_CONVERGED : ST_BREAKDOWN;
    } else if (st->eta_x > 0.0) {
      st->rho = rnorm / st->eta_x;  // calibrate the 2-norm / P^{-1}-norm ratio
      st->calibrated = 1;
    }
  }
  if (!st->done && !(st->delta == st->delta)) {
    st->done = 1;
    st->status = ST_BREAKDOWN;
  }
  st->loops += 1;
  if (st->iter > st->maxit + 1 || st->loops > st->maxit + 4) st->done = 1;  // hard caps (integers only)
  if (a.use_cond) cudaGraphSetConditional(a.cond, st->done ? 0u : 1u);
}

// (K + lambda I) z in complex form for csl_apply.  With x = (Re z, Im z),
// Re((K + lambda I) z) is block row 2 of A x and Im(...) is block row 1.
template <int DIM>
__global__ void __launch_bounds__(256) k_apply(Grid g, const double2* z, double2* out, const double* cx,
                                               const double* cy, const double* cz, const double* dg,
                                               double beta) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < g.M; p += (long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    point_coords(p, g, ix, iy, iz);
    double2 zc;
    const double2 t = stencil_KA<DIM, double2>(z, cx, cy, cz, dg, g, p, ix, iy, iz, zc);
    const double2 Az = block_A(t, zc, beta);
    out[p] = make_double2(Az.y, Az.x);  // Re((K+lambda)z) = row 2, Im = row 1
  }
}

// ---------------------------------------------------------------------------
// Givens step (MINRES on the tridiagonal Lanczos matrix): given
// gamma_{j+1}^2, rotate the new column (gamma_j, delta_j, gamma_{j+1}) by the
// two previous rotations, form the new rotation and the update coefficients
// of w and x, and decide whether the next stencil pass evaluates the true
// residual.
// ---------------------------------------------------------------------------
__device__ void givens_step(DevState* st, double g2) {
  if (!(g2 >= 0.0) || !(g2 < 1e300)) {
    st->done = 1;
    st->status = ST_BREAKDOWN;
    return;
  }
  const double gn = sqrt(g2);
  const double gam = st->gam, delta = st->delta;
  const double c = st->c, c_old = st->c_old, s = st->s, s_old = st->s_old;
  const double a0 = c * delta - c_old * s * gam;
  const double a1 = sqrt(a0 * a0 + gn * gn);
  const double a2 = s * delta + c_old * c * gam;
  const double a3 = s_old * gam;
  if (!(a1 > 0.0) || !(a1 < 1e300)) {
    st->done = 1;
    st->status = ST_BREAKDOWN;
    return;
  }
  const double cn = a0 / a1, sn = gn / a1;
  st->w_a = 1.0 / (a1 * gam);
  st->w_b = -a3 / a1;
  st->w_c = -a2 / a1;
  st->x_coef = cn * st->eta;
  st->eta = -sn * st->eta;
  st->c_old = c;
  st->c = cn;
  st->s_old = s;
  st->s = sn;
  st->gam_old = gam;
  st->gam = gn;
  st->iter += 1;
  // stopping-test schedule for x_iter (evaluated by the next stencil pass)
  const double e = fabs(st->eta);
  st->eta_x = e;
  const double target = st->tol * st->bnorm;
  const double pred = st->rho * e;  // predicted ||b - A x||_2
  int chk = 0;
  if (st->sqrt_pmax * e <= target) chk = 1;                       // certain convergence
  else if (st->sqrt_pmin * e <= target) {                         // convergence possible
    if (pred <= 1.05 * target) chk = 1;
    else if (!st->calibrated && pred <= 30.0 * target) chk = 1;   // calibrate rho once
  }
  if (gn <= 1e-14 * st->gam1) {  // lucky breakdown: x_iter is the exact solution
    st->lucky = 1;
    chk = 1;
  }
  if (st->iter >= st->maxit) chk = 1;
  st->check = chk;
}

// ---------------------------------------------------------------------------
// Row pass: DST along x for rows of n_x contiguous points.
// ---------------------------------------------------------------------------
enum { LOAD_V = 0, LOAD_T = 1, LOAD_LANCZOS = 2 };
enum { STORE_T = 0, STORE_D = 1, STORE_Z = 2, STORE_Z_UPDATE = 3 };

template <typename T>
struct RowArgs {
  int logn, n, nrows;   // line length n = N - 1
  int G, TL, LS;        // lines per CTA, threads per line, smem line stride
  const typename C2<T>::t* tw;
  const T* hs;
  const double2* vin;             // LOAD_V
  const typename C2<T>::t* tin;   // LOAD_T
  double2* vnew;                  // LOAD_LANCZOS: u' in, v_{j+1} out
  const double2* vcur;            // LOAD_LANCZOS: v_j
  typename C2<T>::t* tout;        // STORE_T
  double2* dout;                  // STORE_D
  typename C2<T>::t* zout;        // STORE_Z*: z_{j+1}
  const typename C2<T>::t* zcur;  // STORE_Z_UPDATE: z_j
  double2* wprev;                 // in w_{j-1}, out w_{j+1}
  const double2* wcur;            // w_j
  double2* x;
  DevState* st;                   // may be null (precondition only)
};

template <typename T>
__host__ __device__ inline size_t dst_smem_bytes(int lines, int LS, int logn, int TL) {
  // two line buffers + twiddles + half-sines + scan scratch
  const size_t H = (size_t)1 << (logn - 1);
  const int nl = lines;
  return (size_t)2 * nl * LS * sizeof(typename C2<T>::t) + H * sizeof(typename C2<T>::t) +
         (H + 2) * sizeof(T) + (size_t)nl * 32 * sizeof(typename C2<T>::t) + 64;
}

template <typename T, int LOAD, int STORE>
__global__ void __launch_bounds__(256) k_row(RowArgs<T> a) {
  typedef typename C2<T>::t c_t;
  if (a.st && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << a.logn, H = N >> 1;
  c_t* A = (c_t*)smem_raw;
  c_t* B = A + (size_t)a.G * a.LS;
  c_t* s_tw = B + (size_t)a.G * a.LS;
  c_t* s_scr = s_tw + H;
  T* s_hs = (T*)(s_scr + (size_t)a.G * 32);
  load_tables<T>(s_tw, s_hs, a.tw, a.hs, a.logn);
  double lz = 0.0, wa = 0.0, wb = 0.0, wc = 0.0, xc = 0.0;
  if (LOAD == LOAD_LANCZOS) lz = a.st->delta / a.st->gam;
  if (STORE == STORE_Z_UPDATE) {
    wa = a.st->w_a;
    wb = a.st->w_b;
    wc = a.st->w_c;
    xc = a.st->x_coef;
  }
  const int l = threadIdx.x / a.TL, t = threadIdx.x - l * a.TL;
  const int n = a.n;
  for (int row0 = blockIdx.x * a.G; row0 < a.nrows; row0 += gridDim.x * a.G) {
    const int Gh = min(a.G, a.nrows - row0);
    __syncthreads();  // tables ready / previous tile's buffers free
    if (l < Gh) {
      const long base = (long)(row0 + l) * n;
      c_t* al = A + (size_t)l * a.LS;
      for (int j = t; j < n; j += a.TL) {
        const long p = base + j;
        c_t val;
        if (LOAD == LOAD_V) {
          val = from_d2<T>(a.vin[p]);
        } else if (LOAD == LOAD_T) {
          val = a.tin[p];
        } else {
          const double2 u = a.vnew[p], vc = a.vcur[p];
          const double2 vn = make_double2(fma(-lz, vc.x, u.x), fma(-lz, vc.y, u.y));
          a.vnew[p] = vn;
          val = from_d2<T>(vn);
        }
        al[j + 1] = val;
      }
    }
    __syncthreads();
    dst_lines<T, false>(A, B, a.LS, Gh, a.TL, a.logn, s_tw, s_hs, s_scr);
    if (l < Gh) {
      const long base = (long)(row0 + l) * n;
      const c_t* al = A + (size_t)l * a.LS;
      for (int j = t; j < n; j += a.TL) {
        const long p = base + j;
        const c_t F = al[dst_out_pos(j + 1, N)];
        if (STORE == STORE_T) {
          a.tout[p] = F;
        } else if (STORE == STORE_D) {
          a.dout[p] = to_d2(F);
        } else {
          a.zout[p] = F;
          if (STORE == STORE_Z_UPDATE) {
            const double2 zo = to_d2(a.zcur[p]);
            const double2 wp = a.wprev[p], wq = a.wcur[p];
            const double2 wn = make_double2(fma(wa, zo.x, fma(wb, wp.x, wc * wq.x)),
                                            fma(wa, zo.y, fma(wb, wp.y, wc * wq.y)));
            a.wprev[p] = wn;
            const double2 xo = a.x[p];
            a.x[p] = make_double2(fma(xc, wn.x, xo.x), fma(xc, wn.y, xo.y));
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Strided pass: DST along y or z (lines of stride line_stride), C adjacent
// x-columns per tile, in place.  With MID: forward DST, per-mode scale of
// P^{-1} (Eq. 4: s_k = cnorm / sqrt((gamma mu_k + alpha)^2 + beta^2)),
// gamma^2 partial sums, inverse DST; then the scalar step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }

template <typename T>
struct StridedArgs {
  int logn, n;            // line length n = N - 1
  int ncols, nouter;      // x extent; number of outer blocks
  long outer_stride, line_stride;
  int C, TL, LS;
  const typename C2<T>::t* tw;
  const T* hs;
  typename C2<T>::t* data;
  // MID only
  const double* stab;     // FP64 per-mode scale table (data addressing) or null
  const T* mu_line;       // eigenvalues along the line axis, index k-1
  const T* mu_col;        // along x, index ix
  const T* mu_outer;      // along the outer axis (3D), index outer, or null
  T gamma, alpha, beta2, cnorm;
  DevState* st;
  double* partials;
  int scalar_mode;        // 0 none, 1 init (gamma_1), 2 MINRES iteration
};

template <typename T, bool MID>
__global__ void __launch_bounds__(256) k_strided(StridedArgs<T> a) {
  typedef typename C2<T>::t c_t;
  if (a.st && a.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << a.logn, H = N >> 1;
  c_t* A = (c_t*)smem_raw;
  c_t* B = A + (size_t)a.C * a.LS;
  c_t* s_tw = B + (size_t)a.C * a.LS;
  c_t* s_scr = s_tw + H;
  T* s_hs = (T*)(s_scr + (size_t)a.C * 32);
  load_tables<T>(s_tw, s_hs, a.tw, a.hs, a.logn);
  const int n = a.n, C = a.C;
  const int ntx = (a.ncols + C - 1) / C;
  const int ntiles = ntx * a.nouter;
  const int nthr = blockDim.x;
  int logC = 0;
  while ((1 << logC) < C) ++logC;
  double g2acc = 0.0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int o = tile / ntx;
    const int col0 = (tile - o * ntx) * C;
    const int Ch = min(C, a.ncols - col0);
    const long base = (long)o * a.outer_stride + col0;
    __syncthreads();
    for (int i = threadIdx.x; i < C * n; i += nthr) {
      const int c = i & (C - 1), j = i >> logC;
      if (c < Ch) A[(size_t)c * a.LS + j + 1] = a.data[base + (long)j * a.line_stride + c];
    }
    __syncthreads();
    dst_lines<T, false>(A, B, a.LS, Ch, a.TL, a.logn, s_tw, s_hs, s_scr);
    if (MID) {
      // per-mode scale; gamma^2 partials = sum s |F|^2 over both blocks
      const int l = threadIdx.x / a.TL, t = threadIdx.x - l * a.TL;
      if (l < Ch) {
        c_t* al = A + (size_t)l * a.LS;
        const int ix = col0 + l;
        T murest = a.mu_col ? a.mu_col[ix] : (T)0;
        if (a.mu_outer) murest += a.mu_outer[o];
        T part = (T)0;
        for (int m = 1 + t; m <= n; m += a.TL) {
          const int pos = dst_out_pos(m, N);
          c_t F = al[pos];
          T sc;
          if (a.stab) {
            sc = (T)a.stab[base + (long)(m - 1) * a.line_stride + l];
          } else {
            const T e = fma(a.gamma, murest + a.mu_line[m - 1], a.alpha);
            sc = a.cnorm * rsq(fma(e, e, a.beta2));
          }
          part = fma(sc, fma(F.x, F.x, F.y * F.y), part);
          F.x *= sc;
          F.y *= sc;
          al[pos] = F;
        }
        g2acc += (double)part;
      }
      __syncthreads();
      dst_lines<T, true>(A, B, a.LS, Ch, a.TL, a.logn, s_tw, s_hs, s_scr);
    }
    for (int i = threadIdx.x; i < C * n; i += nthr) {
      const int c = i & (C - 1), j = i >> logC;
      if (c < Ch) a.data[base + (long)j * a.line_stride + c] = A[(size_t)c * a.LS + dst_out_pos(j + 1, N)];
    }
  }
  if (!MID || a.scalar_mode == 0) return;
  double v[1] = {g2acc}, tot[1];
  if (!grid_sum_last_block<1>(v, a.partials, &a.st->tickets[TICKET_MID], tot)) return;
  if (threadIdx.x != 0) return;
  DevState* st = a.st;
  if (a.scalar_mode == 1) {  // gamma_1 = sqrt(<P^{-1} r0, r0>), start of MINRES
    const double g2 = tot[0];
    if (!(g2 > 0.0) || !(g2 < 1e300)) {
      st->done = 1;
      st->status = (g2 == 0.0) ? ST_OK : ST_BREAKDOWN;
      st->relres = (g2 == 0.0) ? 0.0 : st->relres;
      return;
    }
    st->gam = sqrt(g2);
    st->gam1 = st->gam;
    st->gam_old = 1.0;
    st->eta = st->gam;
    st->eta_x = st->gam;
    st->rho = st->bnorm / st->gam;  // exact at x_0 = 0
    return;
  }
  givens_step(st, tot[0]);
}

// ---------------------------------------------------------------------------
// Ingest: f (complex128) -> b = [Im f; Re f] (block form, Eq. 2), MINRES
// start vectors, ||b||, and the scalar state.
// ---------------------------------------------------------------------------
struct IngestArgs {
  long M;
  const double2* f;
  double2 *b, *v0, *v1, *w0, *w1, *x;
  DevState* st;
  double* partials;
  double tol, beta, sqrt_pmin, sqrt_pmax;
  int maxit;
};

__global__ void __launch_bounds__(256) k_ingest(IngestArgs a) {
  double acc[1] = {0.0};
  const double2 zero = make_double2(0.0, 0.0);
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < a.M; p += (long)gridDim.x * blockDim.x) {
    const double2 fv = a.f[p];
    const double2 bb = make_double2(fv.y, fv.x);
    a.b[p] = bb;
    a.v0[p] = bb;
    a.v1[p] = zero;
    a.w0[p] = zero;
    a.w1[p] = zero;
    a.x[p] = zero;
    acc[0] = fma(bb.x, bb.x, fma(bb.y, bb.y, acc[0]));
  }
  double tot[1];
  if (!grid_sum_last_block<1>(acc, a.partials, &a.st->tickets[TICKET_INGEST], tot)) return;
  if (threadIdx.x != 0) return;
  DevState* st = a.st;
  st->bnorm = sqrt(tot[0]);
  st->tol = a.tol;
  st->maxit = a.maxit;
  st->beta = a.beta;
  st->sqrt_pmin = a.sqrt_pmin;
  st->sqrt_pmax = a.sqrt_pmax;
  st->c = st->c_old = 1.0;
  st->s = st->s_old = 0.0;
  st->delta = 0.0;
  st->gam = st->gam_old = st->gam1 = 1.0;
  st->eta = st->eta_x = 0.0;
  st->rho = 0.0;
  st->iter = 0;
  st->check = 0;
  st->lucky = 0;
  st->checks = 0;
  st->loops = 0;
  st->calibrated = 0;
  st->status = ST_OK;
  st->relres = 1.0;
  st->done = 0;
  if (!(st->bnorm > 0.0)) {  // f = 0: z = 0 is exact (or f is not finite)
    st->done = 1;
    st->relres = 0.0;
    st->status = (st->bnorm == 0.0) ? ST_OK : ST_BREAKDOWN;
  }
}

// ---------------------------------------------------------------------------
// Plan set-up kernels
// ---------------------------------------------------------------------------
// scaled copy of one face array (a_e / h^2) and its min / max / validity
__global__ void k_scale_faces(const double* __restrict__ src, double* __restrict__ dst, long count,
                              double inv_h2, unsigned long long* minmax /* [min bits, max bits, bad] */) {
  unsigned long long lmin = ~0ull, lmax = 0ull, bad = 0ull;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const double v = src[i];
    if (!(v > 0.0) || !(v < 1e300)) bad = 1ull;
    else {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
      lmin = bits < lmin ? bits : lmin;
      lmax = bits > lmax ? bits : lmax;
    }
    dst[i] = v * inv_h2;
  }
  atomicMin(&minmax[0], lmin);
  atomicMax(&minmax[1], lmax);
  if (bad) atomicOr(&minmax[2], 1ull);
}

// diagonal of K + alpha I: sum of the (scaled) face coefficients of p, + alpha
template <int DIM>
__global__ void k_diag(Grid g, const double* cx, const double* cy, const double* cz, double* dg,
                       double alpha) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < g.M; p += (long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    point_coords(p, g, ix, iy, iz);
    const long rx = ((long)iz * g.ny + iy) * (g.nx + 1) + ix;
    const long ry = ((long)iz * (g.ny + 1) + iy) * g.nx + ix;
    double d = cx[rx] + cx[rx + 1] + cy[ry] + cy[ry + g.nx];
    if (DIM == 3) {
      const long rz = ((long)iz * g.ny + iy) * g.nx + ix;
      d += cz[rz] + cz[rz + (long)g.nx * g.ny];
    }
    dg[p] = d + alpha;
  }
}

// per-mode scale s_k = cnorm / sqrt((gamma mu_k + alpha)^2 + beta^2) in spectral
// addressing (same as the grid), and the extremes of q = (gamma mu + alpha)^2 + beta^2
template <int DIM>
__global__ void k_scale_table(Grid g, const double* mux, const double* muy, const double* muz,
                              double gamma, double alpha, double beta, double cnorm, double* stab,
                              unsigned long long* qminmax) {
  unsigned long long lmin = ~0ull, lmax = 0ull;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < g.M; p += (long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    point_coords(p, g, ix, iy, iz);
    double mu = mux[ix] + muy[iy];
    if (DIM == 3) mu += muz[iz];
    const double e = fma(gamma, mu, alpha);
    const double q = fma(e, e, beta * beta);
    if (stab) stab[p] = (q > 0.0) ? cnorm / sqrt(q) : 0.0;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(q);
    lmin = bits < lmin ? bits : lmin;
    lmax = bits > lmax ? bits : lmax;
  }
  atomicMin(&qminmax[0], lmin);
  atomicMax(&qminmax[1], lmax);
}

// dL/da_e = -h^{-2} Re(conj(dy) dz) over the faces of one axis (unscaled a_e)
template <int AXIS>
__global__ void k_coef_grad(Grid g, const double2* z, const double2* y, double* grad, double inv_h2) {
  long count;
  if (AXIS == 0) count = (long)g.nz * g.ny * (g.nx + 1);
  else if (AXIS == 1) count = (long)g.nz * (g.ny + 1) * g.nx;
  else count = (long)(g.nz + 1) * g.ny * g.nx;
  const double2 zero = make_double2(0.0, 0.0);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (long)gridDim.x * blockDim.x) {
    long hi, lo;
    bool has_hi, has_lo;
    if (AXIS == 0) {
      const long row = e / (g.nx + 1);
      const int i = (int)(e - row * (g.nx + 1));
      hi = row * g.nx + i;
      lo = hi - 1;
      has_hi = i < g.nx;
      has_lo = i > 0;
    } else if (AXIS == 1) {
      const long plane = (long)(g.ny + 1) * g.nx;
      const long iz = e / plane;
      const long r = e - iz * plane;
      const int iy = (int)(r / g.nx);
      const int ix = (int)(r - (long)iy * g.nx);
      hi = (iz * g.ny + iy) * g.nx + ix;
      lo = hi - g.nx;
      has_hi = iy < g.ny;
      has_lo = iy > 0;
    } else {
      const long plane = (long)g.ny * g.nx;
      const long iz = e / plane;
      const long r = e - iz * plane;
      hi = iz * plane + r;
      lo = hi - plane;
      has_hi = iz < g.nz;
      has_lo = iz > 0;
    }
    const double2 zh = has_hi ? z[hi] : zero, zl = has_lo ? z[lo] : zero;
    const double2 yh = has_hi ? y[hi] : zero, yl = has_lo ? y[lo] : zero;
    const double dzx = zh.x - zl.x, dzy = zh.y - zl.y;
    const double dyx = yh.x - yl.x, dyy = yh.y - yl.y;
    grad[e] = -inv_h2 * fma(dyx, dzx, dyy * dzy);
  }
}

}  // namespace csl
