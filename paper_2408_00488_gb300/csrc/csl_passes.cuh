// Sine-transform passes of P^{-1} (Eq. 4 via Section 2.3) with MINRES vector
// work fused into the first pass (the Lanczos step) and, for batches, into
// the last one (the w/x update; single solves run it beside that pass).
//
//   k_row     DST along x (contiguous rows).  Each warp owns 32/TPL rows: it
//             loads them (fusing v_{j+1} = u' - (delta_j/gamma_j) v_j when
//             LOAD_LANCZOS), transforms them in shared memory and stores them
//             (fusing z_{j+1} and the w/x update when STORE_Z_UPDATE).
//   k_strided DST along y or z: a CTA loads a tile of adjacent columns (one
//             line per column), each warp transforms its lines; with MID the
//             forward transform, per-mode scale, gamma^2 partial sums
//             (Parseval: <P^{-1}v, v> = sum_k s_k |S v|_k^2) and inverse
//             transform all happen in shared memory, and the last CTA runs
//             the Givens step.
#pragma once
#include "csl_common.cuh"
#include "csl_fft.cuh"
#include "csl_kernels.cuh"

#include <vector>

// FP32 passes: two CTAs of 256 threads per SM (at most 128 registers per
// thread); the FP64 lines need the full register file
#define CSL_PASS_MINB(T, V) (sizeof(T) == 4 && (V) < 3 ? ((V) == 2 ? 3 : 2) : 1)
// The warp-per-line row passes of length 1024 that stream MINRES vectors
// from HBM (the Lanczos step before the forward transform, the w/x update
// after the inverse one) keep many loads in flight per lane, so they take the
// whole register file: one CTA per SM, which is what their grids give (a
// 256-thread CTA of 8 lines: 128 CTAs at n = 1023).
#define CSL_ROW_STREAMS(T, N, V, LOAD_MODE, STORE_MODE) \
  (sizeof(T) == 4 && (N) == 1024 && (V) == 0 && ((LOAD_MODE) >= 2 || (STORE_MODE) >= 3))
#define CSL_ROW_MINB(T, N, V, LOAD_MODE, STORE_MODE) \
  (CSL_ROW_STREAMS(T, N, V, LOAD_MODE, STORE_MODE) ? 1 : CSL_PASS_MINB(T, V))

namespace csl {

// LOAD_LANCZOS_V64 / STORE_Z_UPDATE_V64: the FP32 transform with the MINRES
// vectors v, w and x in FP64 (CSL_PREC_FP32_PRECOND); with T = float the plain
// LOAD_LANCZOS / STORE_Z_UPDATE hold them as float pairs, with T = double in FP64
enum { LOAD_V = 0, LOAD_T = 1, LOAD_LANCZOS = 2, LOAD_LANCZOS_V64 = 3 };
enum { STORE_T = 0, STORE_D = 1, STORE_Z = 2, STORE_Z_UPDATE = 3, STORE_Z_UPDATE_V64 = 4 };

template <typename T>
struct RowArgs {
  int n, nrows;
  const typename C2<T>::t* tw;
  const T* hs;
  const typename C2<T>::t* tp;    // extra twiddle table (LineDst::TP entries)
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
struct StridedArgs {
  int n, ncols, nouter;
  long outer_stride, line_stride;
  const typename C2<T>::t* tw;
  const T* hs;
  const typename C2<T>::t* tp;
  typename C2<T>::t* data;
  // MID only
  const double* stab;  // FP64 per-mode scale table (data addressing) or null
  const T* mu_line;    // eigenvalues along the line axis, index k-1
  const T* mu_col;     // along x, index ix
  const T* mu_outer;   // along the outer axis (3D), index outer, or null
  T gamma, alpha, beta2, cnorm;
  DevState* st;
  double* partials;
  int scalar_mode;     // 0 none, 1 init (gamma_1), 2 MINRES iteration
  const void* sine_tc; // tensor-core variant: split-bf16 sine matrix in B-operand layout
};

// byte offsets of the shared-memory regions: twiddles | half sines | extra
// twiddles | scan scratch (2 per line) | lines
// (long lines, variant 3, read their tables from global memory)
template <typename T, int N, int WIDE>
__host__ __device__ constexpr size_t pass_tables_bytes() {
  return LineDst<T, N, WIDE>::GLOBAL_TABLES
             ? 0
             : (size_t)(N / 2) * sizeof(typename C2<T>::t) + (((size_t)(N / 2 + 1) * sizeof(T) + 15) / 16) * 16 +
                   (size_t)line_tp_size(N, WIDE) * sizeof(typename C2<T>::t);
}
// scan scratch per line: one complex per warp of the line (at least 4; the
// long-line variant scans in FP64, so twice as many T-complex slots)
template <typename T, int N, int WIDE>
__host__ __device__ constexpr int pass_scratch() {
  return (LineDst<T, N, WIDE>::TPL / 32 > 4 ? LineDst<T, N, WIDE>::TPL / 32 : 4) * (WIDE == 3 ? 2 : 1);
}
template <typename T, int N, int WIDE>
__host__ __device__ constexpr size_t pass_smem_bytes(int lines) {
  return pass_tables_bytes<T, N, WIDE>() + (size_t)lines * pass_scratch<T, N, WIDE>() * sizeof(typename C2<T>::t) +
         (size_t)lines * LineDst<T, N, WIDE>::LS * sizeof(typename C2<T>::t);
}
// CTA size bound of the pass kernels: 256, or one long line's lanes
template <int N, int WIDE>
__host__ __device__ constexpr int pass_max_threads() {
  return WIDE == 3 ? (N >= 8192 ? 512 : 256) : 256;
}

__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }

template <typename T, int N, int WIDE, int LOAD_MODE, int STORE_MODE>
__global__ void __launch_bounds__(pass_max_threads<N, WIDE>(), CSL_ROW_MINB(T, N, WIDE, LOAD_MODE, STORE_MODE))
    k_row(RowArgs<T> a0, const RowArgs<T>* batch, int bps) {
  // the V64 modes are the Lanczos / update modes with FP64 vectors
  constexpr int LOAD = LOAD_MODE == LOAD_LANCZOS_V64 ? LOAD_LANCZOS : LOAD_MODE;
  constexpr int STORE = STORE_MODE == STORE_Z_UPDATE_V64 ? STORE_Z_UPDATE : STORE_MODE;
  // v, w and x stored as float pairs
  constexpr bool pairs = sizeof(T) == 4 && LOAD_MODE != LOAD_LANCZOS_V64 && STORE_MODE != STORE_Z_UPDATE_V64;
  typedef typename C2<T>::t c_t;
  typedef LineDst<T, N, WIDE> D;
  const int sys = batch ? (int)(blockIdx.x / bps) : 0;
  const int bid = batch ? (int)blockIdx.x - sys * bps : (int)blockIdx.x;
  const int nblk = batch ? bps : (int)gridDim.x;
  const RowArgs<T> a = batch ? batch[sys] : a0;
  constexpr int TPL = D::TPL, LS = D::LS;
  constexpr int NL = (N + TPL - 1) / TPL;  // elements per lane
  // load batch (elements per lane in flight): the Lanczos variant holds two
  // 16-byte vector values (FP64, or float pairs) per element, the update
  // variant four; with the FP32 transform the warp-per-line form has the
  // whole register file for them (CSL_ROW_MINB)
  constexpr bool wide_batch = CSL_ROW_STREAMS(T, N, WIDE, LOAD_MODE, STORE_MODE);
  constexpr int UBMAX = STORE == STORE_Z_UPDATE ? (wide_batch ? 4 : 2) : LOAD == LOAD_LANCZOS ? (wide_batch ? 16 : 4) : 8;
  constexpr int UB = NL < UBMAX ? NL : UBMAX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c_t* w_tw = (c_t*)smem_raw;
  T* w_hs = (T*)(smem_raw + (size_t)(N / 2) * sizeof(c_t));
  c_t* w_tp = (c_t*)(smem_raw + (size_t)(N / 2) * sizeof(c_t) + (((size_t)(N / 2 + 1) * sizeof(T) + 15) / 16) * 16);
  const c_t* s_tw = w_tw;
  const T* s_hs = w_hs;
  const c_t* s_tp = w_tp;
  const int nlines = blockDim.x / TPL;
  c_t* s_scr = (c_t*)(smem_raw + pass_tables_bytes<T, N, WIDE>());
  c_t* lines = s_scr + pass_scratch<T, N, WIDE>() * nlines;
  if constexpr (D::GLOBAL_TABLES) {
    s_tw = a.tw;
    s_hs = a.hs;
  } else {
    load_tables<T>(w_tw, w_hs, w_tp, a.tw, a.hs, a.tp, N, D::TP);  // constant: may overlap the predecessor
  }
  pdl_wait();
  if (a.st && a.st->done) return;
  double lz = 0.0, wb = 0.0, wc = 0.0, xc = 0.0;
  if (LOAD == LOAD_LANCZOS) lz = a.st->delta / a.st->gam;
  // MINRES works with the normalised z_{j+1} / gamma_{j+1}; gamma_{j+1} is
  // known once the MID pass has run, so the z store applies it
  T zs = (T)1;
  if ((STORE == STORE_Z || STORE == STORE_Z_UPDATE) && a.st) zs = (T)(a.st->gam > 0.0 ? 1.0 / a.st->gam : 0.0);
  float2 wb2 = make_float2(0.f, 0.f), wc2 = wb2, xc2 = wb2;
  if (STORE == STORE_Z_UPDATE) {
    wb = a.st->w_b;
    wc = a.st->w_c;
    xc = a.st->x_coef;
    if (pairs) {
      wb2 = d_to_ff(wb);
      wc2 = d_to_ff(wc);
      xc2 = d_to_ff(xc);
    }
  }
  __syncthreads();
  const int myl = threadIdx.x / TPL, t = threadIdx.x - myl * TPL;
  const int lpb = nlines;
  c_t* line = lines + (size_t)myl * LS;
  const int n = a.n;
  for (int row0 = bid * lpb; row0 < a.nrows; row0 += nblk * lpb) {
    const int row = row0 + myl;
    const bool valid = row < a.nrows;
    const long base = (long)row * n;
    if constexpr (LOAD == LOAD_T) {
      // global -> shared copies (cp.async): every element of the lane in
      // flight at once, no registers held; rows past the end are zero-filled
#pragma unroll
      for (int k = 0; k < NL; ++k) {
        const int j = t + TPL * k;
        if (j < n) {
          if constexpr (sizeof(T) == 4)
            cp_async8(&line[D::in_pos(j + 1)], valid ? (const void*)(a.tin + base + j) : (const void*)a.tin, valid);
          else
            cp_async16(&line[D::in_pos(j + 1)], valid ? (const void*)(a.tin + base + j) : (const void*)a.tin, valid);
        }
      }
      cp_async_commit();
      cp_async_wait<0>();
    }
    // global loads in batches of UB elements per lane, all issued before use
#pragma unroll
    for (int i0 = 0; i0 < (LOAD == LOAD_T ? 0 : NL); i0 += UB) {
      if constexpr (LOAD == LOAD_LANCZOS && pairs) {
        // pair-vector forms: u' and v_j are float pairs (re.hi, re.lo, im.hi, im.lo);
        // v_{j+1} = u' - (delta/gamma) v_j in pair arithmetic, stored
        // renormalised, its hi parts (= RN of the pair) feed the transform
        float4 u[UB], vc[UB];
        const float2 lz2 = d_to_ff(lz);
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          const int j = t + TPL * (i0 + k);
          if (valid && j < n) {
            u[k] = ((const float4*)a.vnew)[base + j];
            vc[k] = ((const float4*)a.vcur)[base + j];
          }
        }
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          const int j = t + TPL * (i0 + k);
          if (j < n) {
            c_t val = mkc<T>((T)0, (T)0);
            if (valid) {
              ff2 rx = {u[k].x, u[k].y}, ry = {u[k].z, u[k].w};
              const ff2 px = ff_mul(lz2, make_float2(vc[k].x, vc[k].y));
              const ff2 py = ff_mul(lz2, make_float2(vc[k].z, vc[k].w));
              ff_acc(rx, -px.h, -px.l);
              ff_acc(ry, -py.h, -py.l);
              rx = ff_two_sum(rx.h, rx.l);
              ry = ff_two_sum(ry.h, ry.l);
              ((float4*)a.vnew)[base + j] = make_float4(rx.h, rx.l, ry.h, ry.l);
              val = mkc<T>((T)rx.h, (T)ry.h);
            }
            line[D::in_pos(j + 1)] = val;
          }
        }
      } else if (LOAD == LOAD_LANCZOS) {
        double2 u[UB], vc[UB];
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          const int j = t + TPL * (i0 + k);
          if (valid && j < n) {
            u[k] = a.vnew[base + j];
            vc[k] = a.vcur[base + j];
          }
        }
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          const int j = t + TPL * (i0 + k);
          if (j < n) {
            c_t val = mkc<T>((T)0, (T)0);
            if (valid) {
              const double2 vn = make_double2(fma(-lz, vc[k].x, u[k].x), fma(-lz, vc[k].y, u[k].y));
              a.vnew[base + j] = vn;
              val = from_d2<T>(vn);
            }
            line[D::in_pos(j + 1)] = val;
          }
        }
      } else {
        c_t val[UB];
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          const int j = t + TPL * (i0 + k);
          val[k] = mkc<T>((T)0, (T)0);
          if (valid && j < n) val[k] = (LOAD == LOAD_V) ? from_d2<T>(a.vin[base + j]) : a.tin[base + j];
        }
#pragma unroll
        for (int k = 0; k < UB; ++k) {
          const int j = t + TPL * (i0 + k);
          if (j < n) line[D::in_pos(j + 1)] = val[k];
        }
      }
    }
    D::line_sync();
    D::template run<false>(line, t, s_tw, s_hs, s_tp, s_scr);
    if (valid) {
#pragma unroll
      for (int i0 = 0; i0 < NL; i0 += UB) {
        if (STORE == STORE_Z_UPDATE) {
          c_t zo[UB];
          double2 wp[UB], wq[UB], xo[UB];
#pragma unroll
          for (int k = 0; k < UB; ++k) {
            const int j = t + TPL * (i0 + k);
            if (j < n) {
              zo[k] = a.zcur[base + j];
              wp[k] = a.wprev[base + j];
              wq[k] = a.wcur[base + j];
              xo[k] = a.x[base + j];
            }
          }
#pragma unroll
          for (int k = 0; k < UB; ++k) {
            const int j = t + TPL * (i0 + k);
            if (j < n) {
              const long p = base + j;
              const c_t F = line[D::out_pos(j + 1)];
              a.zout[p] = mkc<T>(F.x * zs, F.y * zs);
              if constexpr (pairs) {  // pair-vector forms: w and x as float pairs (see k_update)
                const float4 q = *(const float4*)&wp[k], r = *(const float4*)&wq[k], o = *(const float4*)&xo[k];
                ff2 wr, xr, wi, xi;
                ff_update(zo[k].x, make_float2(q.x, q.y), make_float2(r.x, r.y), make_float2(o.x, o.y), wb2, wc2,
                          xc2, wr, xr);
                ff_update(zo[k].y, make_float2(q.z, q.w), make_float2(r.z, r.w), make_float2(o.z, o.w), wb2, wc2,
                          xc2, wi, xi);
                ((float4*)a.wprev)[p] = make_float4(wr.h, wr.l, wi.h, wi.l);
                ((float4*)a.x)[p] = make_float4(xr.h, xr.l, xi.h, xi.l);
                continue;
              }
              const double2 zd = to_d2(zo[k]);
              // scaled w: w_a = 1 (see givens_step)
              const double2 wn = make_double2(fma(wb, wp[k].x, fma(wc, wq[k].x, zd.x)),
                                              fma(wb, wp[k].y, fma(wc, wq[k].y, zd.y)));
              a.wprev[p] = wn;
              a.x[p] = make_double2(fma(xc, wn.x, xo[k].x), fma(xc, wn.y, xo[k].y));
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < UB; ++k) {
            const int j = t + TPL * (i0 + k);
            if (j < n) {
              const long p = base + j;
              const c_t F = line[D::out_pos(j + 1)];
              if (STORE == STORE_T)
                a.tout[p] = F;
              else if (STORE == STORE_D)
                a.dout[p] = to_d2(F);
              else
                a.zout[p] = mkc<T>(F.x * zs, F.y * zs);
            }
          }
        }
      }
    }
    D::line_sync();
  }
  pdl_trigger();
}

// End of a MID pass: grid sum of the Parseval partials; the last CTA either
// starts MINRES (scalar_mode 1: gamma_1 = sqrt(<P^{-1} r0, r0>)) or runs the
// Givens step of the iteration (scalar_mode 2).
// pre: the state as the kernel found it (state_prefetch), or null
template <typename T>
__device__ void mid_scalar_tail(const StridedArgs<T>& a, double g2acc, int bid, int nblk,
                                const DevState* pre = nullptr) {
  double v[1] = {g2acc}, tot[1];
  if (!grid_sum_last_block<1>(v, a.partials, &a.st->tickets[TICKET_MID], tot, bid, nblk)) return;
  if (threadIdx.x != 0) return;
  // the scalar step runs on a register copy of the state and stores the
  // fields it sets
  DevState q = pre ? *pre : *a.st;
  if (a.scalar_mode == 1) {
    const double g2 = tot[0];
    // f = 0 never reaches this pass (the ingest closes the solve with z = 0),
    // so <P^{-1} r0, r0> = 0 for a positive definite P is an underflow
    if (!(g2 > 0.0) || !(g2 < 1e300)) {
      q.done = 1;
      q.status = ST_BREAKDOWN;
    } else {
      q.gam = sqrt(g2);
      q.gam1 = q.gam;
      q.gam_old = 1.0;
      q.eta = q.gam;
      q.eta_x = q.gam;
      q.rho = q.r0norm / q.gam;  // exact at the start vector
    }
  } else {
    givens_step(&q, tot[0]);
  }
  store_scalar_fields(a.st, q);
}

template <typename T, int N, int WIDE, bool MID>
__global__ void __launch_bounds__(pass_max_threads<N, WIDE>(), CSL_PASS_MINB(T, WIDE)) k_strided(StridedArgs<T> a0, const StridedArgs<T>* batch, int bps) {
  typedef typename C2<T>::t c_t;
  typedef LineDst<T, N, WIDE> D;
  const int sys = batch ? (int)(blockIdx.x / bps) : 0;
  const int bid = batch ? (int)blockIdx.x - sys * bps : (int)blockIdx.x;
  const int nblk = batch ? bps : (int)gridDim.x;
  const StridedArgs<T> a = batch ? batch[sys] : a0;
  constexpr int TPL = D::TPL, LS = D::LS;
  constexpr int NL = (N + TPL - 1) / TPL;
  constexpr int UB = NL < 8 ? NL : 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c_t* w_tw = (c_t*)smem_raw;
  T* w_hs = (T*)(smem_raw + (size_t)(N / 2) * sizeof(c_t));
  c_t* w_tp = (c_t*)(smem_raw + (size_t)(N / 2) * sizeof(c_t) + (((size_t)(N / 2 + 1) * sizeof(T) + 15) / 16) * 16);
  const c_t* s_tw = w_tw;
  const T* s_hs = w_hs;
  const c_t* s_tp = w_tp;
  const int C = blockDim.x / TPL;  // lines (columns) per tile, a power of two
  c_t* s_scr = (c_t*)(smem_raw + pass_tables_bytes<T, N, WIDE>());
  c_t* lines = s_scr + pass_scratch<T, N, WIDE>() * C;
  if constexpr (D::GLOBAL_TABLES) {
    s_tw = a.tw;
    s_hs = a.hs;
  } else {
    load_tables<T>(w_tw, w_hs, w_tp, a.tw, a.hs, a.tp, N, D::TP);  // constant: may overlap the predecessor
  }
  pdl_wait();
  if (a.st && a.st->done) return;
  __shared__ DevState s_pre;
  if (MID && a.scalar_mode != 0) state_prefetch(&s_pre, a.st);
  if (MID && a.scalar_mode == 2 && bid == 0 && threadIdx.x == 0) a.st->entries += 1;  // read by the next stencil pass
  int logC = 0;
  while ((1 << logC) < C) ++logC;
  const int myl = threadIdx.x / TPL, t = threadIdx.x - myl * TPL;
  c_t* line = lines + (size_t)myl * LS;
  const int n = a.n;
  const int ntx = (a.ncols + C - 1) / C;
  const int ntiles = ntx * a.nouter;
  double g2acc = 0.0;
  for (int tile = bid; tile < ntiles; tile += nblk) {
    const int o = tile / ntx;
    const int col0 = (tile - o * ntx) * C;
    const int Ch = min(C, a.ncols - col0);
    const long base = (long)o * a.outer_stride + col0;
    __syncthreads();  // tables loaded / previous tile stored
    // blockDim = C * TPL, so NL rounds per thread cover the C x n tile; the
    // elements are copied global -> shared with cp.async, all in flight at
    // once (columns past the grid's edge are zero-filled)
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int e = threadIdx.x + blockDim.x * k;
      const int c = e & (C - 1), j = e >> logC;
      if (j < n) {
        const bool ok = c < Ch;
        const c_t* src = ok ? a.data + base + (long)j * a.line_stride + c : a.data;
        if constexpr (sizeof(T) == 4)
          cp_async8(&lines[(size_t)c * LS + D::in_pos(j + 1)], src, ok);
        else
          cp_async16(&lines[(size_t)c * LS + D::in_pos(j + 1)], src, ok);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    D::template run<false>(line, t, s_tw, s_hs, s_tp, s_scr);
    if (MID) {
      if (myl < Ch) {
        const int ix = col0 + myl;
        T murest = a.mu_col ? a.mu_col[ix] : (T)0;
        if (a.mu_outer) murest += a.mu_outer[o];
        T part = (T)0;
        if (a.stab) {
          for (int m = 1 + t; m <= n; m += TPL) {
            const int pos = D::out_pos(m);
            c_t F = line[pos];
            const T sc = (T)a.stab[base + (long)(m - 1) * a.line_stride + myl];
            part = fma(sc, fma(F.x, F.x, F.y * F.y), part);
            F.x *= sc;
            F.y *= sc;
            line[pos] = F;
          }
        } else {
          // the lane's eigenvalues mu_m are loaded together before the
          // scaling, so their latencies overlap instead of adding up
          T mu[NL];
#pragma unroll
          for (int k = 0; k < NL; ++k) {
            const int m = 1 + t + TPL * k;
            mu[k] = m <= n ? a.mu_line[m - 1] : (T)0;
          }
#pragma unroll
          for (int k = 0; k < NL; ++k) {
            const int m = 1 + t + TPL * k;
            if (m <= n) {
              const int pos = D::out_pos(m);
              c_t F = line[pos];
              const T e = fma(a.gamma, murest + mu[k], a.alpha);
              const T sc = a.cnorm * rsq(fma(e, e, a.beta2));
              part = fma(sc, fma(F.x, F.x, F.y * F.y), part);
              F.x *= sc;
              F.y *= sc;
              line[pos] = F;
            }
          }
        }
        g2acc += (double)part;
      }
      D::line_sync();
      D::template run<true>(line, t, s_tw, s_hs, s_tp, s_scr);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * n; i += blockDim.x) {
      const int c = i & (C - 1), j = i >> logC;
      if (c < Ch) a.data[base + (long)j * a.line_stride + c] = lines[(size_t)c * LS + D::out_pos(j + 1)];
    }
  }
  pdl_trigger();
  if (MID && a.scalar_mode != 0) mid_scalar_tail<T>(a, g2acc, bid, nblk, &s_pre);
}

// ---------------------------------------------------------------------------
// Host-side dispatch over the transform length (one instantiation per N).
// ---------------------------------------------------------------------------
struct PassLaunch {
  int blocks, threads;
  size_t smem;
  int tc = 0;   // strided passes: 0 = FFT, 2 or 3 = tensor-core GEMM with that many bf16 terms
  int pdl = 0;  // launch with programmatic dependent launch (overlaps the predecessor's tail)
};

#define CSL_FOR_EACH_N(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

// N = 512 and 1024 exist in three variants (warp per line, 64 and 128 lanes
// per line: wide = 0, 1, 2); the autotuner picks one per pass.
inline bool pass_has_wide(int N) { return N == 512 || N == 1024; }
inline int pass_num_variants(int N) { return pass_has_wide(N) ? 3 : 1; }

// Long lines (N = 2048 .. 8192): variant 3 only, one line per CTA; their
// instantiations live in csl_pass32_big.cu / csl_pass64_big.cu.
#define CSL_FOR_EACH_BIG_N(X) X(2048) X(4096) X(8192)
inline bool pass_is_big(int N) { return N > 1024; }

template <typename T>
size_t pass_smem(int N, int wide, int lines) {
  switch (N) {
#define BIGCASE(NN) \
  case NN: return pass_smem_bytes<T, NN, 3>(lines);
    CSL_FOR_EACH_BIG_N(BIGCASE)
#undef BIGCASE
#define CASE(NN)                                                                       \
  case NN:                                                                             \
    if constexpr (NN >= 512) {                                                         \
      if (wide == 1) return pass_smem_bytes<T, NN, 1>(lines);                          \
      if (wide == 2) return pass_smem_bytes<T, NN, 2>(lines);                          \
    }                                                                                  \
    return pass_smem_bytes<T, NN, 0>(lines);
    CSL_FOR_EACH_N(CASE)
#undef CASE
  }
  return 0;
}

template <int NN>
inline int pass_tpl_n(int wide) {
  if constexpr (NN >= 512) {
    if (wide == 1) return LineDst<float, NN, 1>::TPL;
    if (wide == 2) return LineDst<float, NN, 2>::TPL;
  }
  return LineDst<float, NN, 0>::TPL;
}

inline int pass_tpl(int N, int wide) {
  switch (N) {
#define BIGCASE(NN) \
  case NN: return LineDst<float, NN, 3>::TPL;
    CSL_FOR_EACH_BIG_N(BIGCASE)
#undef BIGCASE
#define CASE(NN) \
  case NN: return pass_tpl_n<NN>(wide);
    CSL_FOR_EACH_N(CASE)
#undef CASE
  }
  return 1;
}

// batch (optional): device array of per-system arguments; the grid is then
// L.blocks blocks per system times nsys
template <typename T>
cudaError_t launch_row(int N, int wide, int load, int store, const RowArgs<T>& a, const PassLaunch& L,
                       cudaStream_t s, const RowArgs<T>* batch = nullptr, int nsys = 0);
template <typename T>
cudaError_t launch_strided(int N, int wide, bool mid, const StridedArgs<T>& a, const PassLaunch& L,
                           cudaStream_t s, const StridedArgs<T>* batch = nullptr, int nsys = 0);
// dynamic shared memory limit of one kernel = opt-in maximum - its static shared memory
inline cudaError_t allow_dyn_smem(const void* k) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

template <typename T>
cudaError_t set_pass_attrs();
template <typename T>
cudaError_t launch_row_big(int N, int load, int store, const RowArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                           const RowArgs<T>* batch, int nsys);
template <typename T>
cudaError_t launch_strided_big(int N, bool mid, const StridedArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                               const StridedArgs<T>* batch, int nsys);
template <typename T>
cudaError_t set_pass_attrs_big();
// FP64 lines of 16384 points on a two-CTA cluster (csl_cluster.cu)
size_t cluster_pass_smem();
int cluster_pass_threads();
cudaError_t launch_row_cl(int load, int store, const RowArgs<double>& a, const PassLaunch& L, cudaStream_t s);
cudaError_t launch_strided_cl(bool mid, const StridedArgs<double>& a, const PassLaunch& L, cudaStream_t s);
cudaError_t set_cluster_attrs();

// tensor-core strided passes (csl_tc.cu): lines of N = 32, 64 or 128 points
bool tc_supported(int N);
size_t tc_smem_bytes(int N, int split);
int tc_ctas_per_sm(int N, int split, bool mid);
cudaError_t launch_strided_tc(int N, int split, bool mid, const StridedArgs<float>& a, const PassLaunch& L,
                              cudaStream_t s, const StridedArgs<float>* batch, int nsys);
cudaError_t set_tc_attrs();
void build_sine_image(int N, int split, std::vector<uint16_t>& img);

}  // namespace csl
