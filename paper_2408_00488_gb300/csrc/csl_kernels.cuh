// Kernels of the preconditioned MINRES solve of Eq. 2 with the preconditioner
// of Eq. 4 (arXiv 2408.00488).  One MINRES iteration j is four (2D) or six
// (3D) stream-ordered kernels plus the update on a parallel branch:
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
//   P3  k_row<STORE_Z> inverse DST along x -> z_{j+1}, and beside it
//   UPD k_update       w_{j+1} = (zhat_j - a3 w_{j-1} - a2 w_j)/a1,  x_j = x_{j-1} + c eta w_{j+1}
//                     (batches fuse UPD into P3: k_row<STORE_Z_UPDATE>)
//
// The FP32 forms hold v, w and x as float pairs and run the per-point vector
// work in pair arithmetic; the FP64 form holds them in FP64.
//
// The grid reductions are deterministic (block sums in block order by the
// last block to finish), so repeated solves are bitwise identical.
#pragma once
#include "csl_common.cuh"

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
  double2* vold;          // in: v_{j-1}; out: u' (FP64, or float pairs in the FP32 forms)
  const double* cx;
  const double* cy;
  const double* cz;
  const double* dg;
  const float2* cxp;      // the same faces as float pairs (FF path): c = hi + lo
  const float2* cyp;
  const float2* czp;
  float2 alpha2;          // alpha as a float pair
  int strip;              // steps per warp strip along the marching axis
  const double2* x;       // current iterate (true-residual check)
  const double2* b;       // right-hand side (block form)
  DevState* st;
  double* partials;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

// ---------------------------------------------------------------------------
// Float-pair ("double-float") arithmetic for the stencil of the FP32-
// preconditioner forms.  A value is the unevaluated sum h + l of two floats.
// GB300 issues FP32 at 64 times its FP64 rate, so a pair product-sum of about
// 18 FP32 instructions costs less issue time than one FP64 FMA costs FP64
// pipe time.  The sums are error-free transformations (Knuth's TwoSum and the
// FMA product error), rounded to nearest with no contraction; the pair keeps
// about 2^-47 relative accuracy, which the difference form below spends on
// small terms.
// ---------------------------------------------------------------------------
struct ff2 {
  float h, l;
};

// a + b exactly, as s + e (Knuth's TwoSum, no ordering condition)
__device__ __forceinline__ ff2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// acc += p, p = ph + pl: the high parts summed exactly, the low parts in FP32
__device__ __forceinline__ void ff_acc(ff2& acc, float ph, float pl) {
  const ff2 t = ff_two_sum(acc.h, ph);
  acc.h = t.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(pl, t.l));
}

// c * x for a pair c and a float x (c.h * x exactly via its FMA error term)
__device__ __forceinline__ ff2 ff_mul1(float2 c, float x) {
  const float ph = __fmul_rn(c.x, x);
  return {ph, __fmaf_rn(c.y, x, __fmaf_rn(c.x, x, -ph))};
}

// acc += c * x
__device__ __forceinline__ void ff_acc_mul1(ff2& acc, float2 c, float x) {
  const ff2 p = ff_mul1(c, x);
  ff_acc(acc, p.h, p.l);
}

// The flux c * (zc - zq) across one face for one component, as a pair: the
// difference of the two floats is formed exactly, then multiplied by the
// pair c (the c.l * d.l term, below 2^-47 of the product, is dropped)
__device__ __forceinline__ ff2 ff_flux(float2 c, float zc, float zq) {
  const ff2 d = ff_two_sum(zc, -zq);
  const float ph = __fmul_rn(c.x, d.h);
  float pl = __fmaf_rn(c.x, d.h, -ph);
  pl = __fmaf_rn(c.x, d.l, pl);
  pl = __fmaf_rn(c.y, d.h, pl);
  return {ph, pl};
}

// acc += c * (zc - zq)
__device__ __forceinline__ void ff_acc_flux(ff2& acc, float2 c, float zc, float zq) {
  const ff2 f = ff_flux(c, zc, zq);
  ff_acc(acc, f.h, f.l);
}

// a * b for two pairs (the a.l * b.l term, below 2^-47 of the product, is dropped)
__device__ __forceinline__ ff2 ff_mul(float2 a, float2 b) {
  const float ph = __fmul_rn(a.x, b.x);
  float pl = __fmaf_rn(a.x, b.x, -ph);
  pl = __fmaf_rn(a.x, b.y, pl);
  pl = __fmaf_rn(a.y, b.x, pl);
  return {ph, pl};
}

__device__ __forceinline__ double ff_to_d(ff2 v) { return f2d_exact(v.h) + f2d_exact(v.l); }

// a double as a float pair hi + lo, hi = RN(d), lo = RN(d - hi) (d - hi is exact)
__device__ __forceinline__ float2 d_to_ff(double d) {
  const float h = d2f_rn(d);
  return make_float2(h, d2f_rn(d - f2d_exact(h)));
}

// Lanczos vectors v (and u'): FP64 in the FP64 form; in the FP32 forms each
// component is a float pair (re.hi, re.lo, im.hi, im.lo) in the same 16 bytes
// per point, so that the stencil and the Lanczos step run in pair arithmetic.
// VP: the vectors are stored as float pairs (CSL_PREC_FP32 and the split-BF16
// forms); otherwise as FP64 (CSL_PREC_FP64 and CSL_PREC_FP32_PRECOND).
template <bool VP>
__device__ __forceinline__ double2 v_load(const double2* v, long p) {
  if constexpr (!VP) {
    return v[p];
  } else {
    const float4 q = ((const float4*)v)[p];
    return make_double2(f2d_exact(q.x) + f2d_exact(q.y), f2d_exact(q.z) + f2d_exact(q.w));
  }
}
template <bool VP>
__device__ __forceinline__ void v_store(double2* v, long p, double2 val) {
  if constexpr (!VP) {
    v[p] = val;
  } else {
    const float2 a = d_to_ff(val.x), b = d_to_ff(val.y);
    ((float4*)v)[p] = make_float4(a.x, a.y, b.x, b.y);
  }
}


__device__ __forceinline__ float2 shfl_up_f2(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down_f2(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// Planes one warp walks per strip of the 3D FP64-arithmetic stencil; the
// float-pair stencil and the 2D FP64 one size their strips per plan
// (strip_rows).
constexpr int kStencilStrip = 16;

__device__ __forceinline__ double2 shfl_up_d2(double2 v) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ double2 shfl_down_d2(double2 v) {
  return make_double2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// Number of warp strips of k_stencil (32 x-columns by `strip` steps along
// the marching axis: y in 2D, z in 3D).
__host__ __device__ inline long stencil_strips(int dim, int nx, int ny, int nz, int strip) {
  const long nsx = (nx + 31) / 32;
  const long nm = dim == 2 ? ny : nz;
  return nsx * ((nm + strip - 1) / strip) * (dim == 3 ? ny : 1);
}

// Strip length for `warps` resident warps on each of the `sms` SMs: 24 for
// the float-pair stencil (three 8-warp CTAs at 80 registers), 16 for the 2D
// FP64-arithmetic stencil (two at 128), so that the dependent arithmetic of
// one warp hides behind the others and every SM gets the same number of
// strips; 4 .. 64 steps.
inline int strip_rows(int dim, int nx, int ny, int nz, int sms, int warps) {
  const long cols = (long)((nx + 31) / 32) * (dim == 3 ? ny : 1);
  const long nm = dim == 2 ? ny : nz;
  long per_col = (long)sms * warps / cols;
  if (per_col < 1) per_col = 1;
  const long strip = (nm + per_col - 1) / per_col;
  return (int)(strip < 4 ? 4 : strip > 64 ? 64 : strip);
}

// One value of a strip and its marching window: m-1, m, m+1 along the strip,
// x-1 / x+1 by warp shuffles (the strip's edge lanes load theirs), and in 3D
// y-1 / y+1 by direct loads.  Every value is converted to FP64 once.
template <int DIM, typename TZ>
struct StripWindow {
  double2 zm, zc, zp;
  __device__ __forceinline__ void start(const TZ* z, long base, long mstride, int m0, bool vx) {
    const double2 zero = make_double2(0.0, 0.0);
    zm = (vx && m0 > 0) ? to_d2(z[base + (long)(m0 - 1) * mstride]) : zero;
    zc = vx ? to_d2(z[base + (long)m0 * mstride]) : zero;
  }
  // (K + alpha I) applied at the current point; call with all 32 lanes
  __device__ __forceinline__ double2 KA(const TZ* z, const StencilArgs& a, long p, long mstride, int m, int nm,
                                        int x, int yfix, bool vx, int lane) {
    const double2 zero = make_double2(0.0, 0.0);
    const int nx = a.g.nx, ny = a.g.ny;
    zp = (vx && m + 1 < nm) ? to_d2(z[p + mstride]) : zero;
    double2 zl = shfl_up_d2(zc), zr = shfl_down_d2(zc);
    if (lane == 0) zl = (vx && x > 0) ? to_d2(z[p - 1]) : zero;
    if (lane == 31) zr = (x + 1 < nx) ? to_d2(z[p + 1]) : zero;
    double2 t = zero;
    if (vx) {
      const double d = a.dg[p];
      double ax = d * zc.x, ay = d * zc.y;
      long rx, ry;
      if (DIM == 2) {
        rx = (long)m * (nx + 1) + x;
        ry = (long)m * nx + x;
      } else {
        rx = ((long)m * ny + yfix) * (nx + 1) + x;
        ry = ((long)m * (ny + 1) + yfix) * nx + x;
      }
      const double cw = a.cx[rx], ce = a.cx[rx + 1];
      ax = fma(-cw, zl.x, ax);
      ay = fma(-cw, zl.y, ay);
      ax = fma(-ce, zr.x, ax);
      ay = fma(-ce, zr.y, ay);
      const double cs = a.cy[ry], cn = a.cy[ry + nx];
      if (DIM == 2) {  // y is the marching axis
        ax = fma(-cs, zm.x, ax);
        ay = fma(-cs, zm.y, ay);
        ax = fma(-cn, zp.x, ax);
        ay = fma(-cn, zp.y, ay);
      } else {
        const double2 zs = yfix > 0 ? to_d2(z[p - nx]) : zero;
        const double2 zn = yfix < ny - 1 ? to_d2(z[p + nx]) : zero;
        ax = fma(-cs, zs.x, ax);
        ay = fma(-cs, zs.y, ay);
        ax = fma(-cn, zn.x, ax);
        ay = fma(-cn, zn.y, ay);
        const double cd = a.cz[p], cu = a.cz[p + mstride];  // z-faces share the point's index
        ax = fma(-cd, zm.x, ax);
        ay = fma(-cd, zm.y, ay);
        ax = fma(-cu, zp.x, ax);
        ay = fma(-cu, zp.y, ay);
      }
      t = make_double2(ax, ay);
    }
    return t;
  }
  __device__ __forceinline__ void advance() {
    zm = zc;
    zc = zp;
  }
};

// Operands of one step m of a strip, loaded one step ahead and kept raw (TZ)
// so that the loads of step m+1 are in flight while step m computes: z at
// m+1 (the window's next value), the edge lanes' x-neighbours, in 3D the
// y-neighbours, the diagonal, the faces and v_{j-1}.
template <int DIM, typename TZ, bool VP>
struct StepOperands {
  TZ zn1, zl, zr, ys, yn;
  double d, cw, ce, cs, cn, cd, cu;
  double2 vo;
  __device__ __forceinline__ void load(const TZ* z, const StencilArgs& a, long p, long mstride, int m, int nm,
                                       int x, int yfix, bool vx, int lane) {
    const int nx = a.g.nx, ny = a.g.ny;
    TZ zero;
    zero.x = 0;
    zero.y = 0;
    zn1 = (vx && m + 1 < nm) ? z[p + mstride] : zero;
    zl = (lane == 0 && vx && x > 0) ? z[p - 1] : zero;
    zr = (lane == 31 && x + 1 < nx) ? z[p + 1] : zero;
    d = cw = ce = cs = cn = cd = cu = 0.0;
    vo = make_double2(0.0, 0.0);
    ys = yn = zero;
    if (vx) {
      long rx, ry;
      if (DIM == 2) {
        rx = (long)m * (nx + 1) + x;
        ry = (long)m * nx + x;
      } else {
        rx = ((long)m * ny + yfix) * (nx + 1) + x;
        ry = ((long)m * (ny + 1) + yfix) * nx + x;
        if (yfix > 0) ys = z[p - nx];
        if (yfix < ny - 1) yn = z[p + nx];
        cd = a.cz[p];
        cu = a.cz[p + mstride];
      }
      d = a.dg[p];
      cw = a.cx[rx];
      ce = a.cx[rx + 1];
      cs = a.cy[ry];
      cn = a.cy[ry + nx];
      vo = v_load<VP>(a.vold, p);
    }
  }
};

// Asynchronous global -> shared copies (cp.async) of 8 or 16 bytes; a false
// predicate copies nothing and zero-fills the destination (the source is
// then not read, and callers pass a valid address anyway).
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Float-pair stencil: one stage of a warp's operand ring holds what step m of
// its strip needs beyond the values carried from step m-1 (ẑ at m-1 and m,
// in 2D the south face = the previous north face, in 3D the lower z-face =
// the previous upper one).  cw[32] is the east face of lane 31; edge[0] and
// edge[1] are the x-neighbours of lanes 0 and 31 from outside the strip.
constexpr int kFFStages = 4;
template <int DIM>
struct FFStage {
  double2 v[32];     // v_{j-1} at the step's points
  float2 zp[32];     // ẑ at m+1
  float2 cn[32];     // y-face above the point
  float2 cw[33];     // x-face left of the point (+ lane 31's right face)
  float2 edge[2];
  float2 cs[DIM == 3 ? 32 : 1];  // 3D: y-face below (2D carries it)
  float2 ys[DIM == 3 ? 32 : 1];  // 3D: y-neighbours
  float2 yn[DIM == 3 ? 32 : 1];
  float2 cu[DIM == 3 ? 32 : 1];  // 3D: z-face above
};
template <int DIM>
__host__ __device__ constexpr int ff_stage_bytes() {
  return (int)((sizeof(FFStage<DIM>) + 15) / 16 * 16);
}
// dynamic shared memory of one 256-thread float-pair stencil CTA
__host__ __device__ constexpr int ff_stencil_smem(int dim) {
  return 8 * kFFStages * (dim == 2 ? ff_stage_bytes<2>() : ff_stage_bytes<3>());
}

// batch: optional per-system argument array (system = blockIdx.x / bps).
// FF (FP32 ẑ only): the non-checking steps form (K + alpha I) ẑ in the
// difference form alpha z_p + sum_e c_e (z_p - z_q) of Eq. 1 in float-pair
// arithmetic (the differences of neighbouring values are exact and small, so
// the large cancelling terms c_e z_p of the direct form never appear), and
// add the beta block term, delta and u' = A ẑ - lanc v_{j-1} (v held as float
// pairs) in pairs too: no FP64 arithmetic per point.
template <int DIM, typename TZ, bool FF, bool VP>
__global__ void __launch_bounds__(256, FF ? (DIM == 2 ? 3 : 2) : 2)
    k_stencil(StencilArgs a0, const StencilArgs* batch, int bps) {
  static_assert(!FF || (sizeof(TZ) == 8 && VP), "the float-pair stencil reads an FP32 z and pair vectors");
  static_assert(!VP || sizeof(TZ) == 8, "pair vectors go with an FP32 z");
  const int sys = batch ? (int)(blockIdx.x / bps) : 0;
  const int bid = batch ? (int)blockIdx.x - sys * bps : (int)blockIdx.x;
  const int nblk = batch ? bps : (int)gridDim.x;
  const StencilArgs a = batch ? batch[sys] : a0;
  DevState* st = a.st;
  pdl_wait();
  // `entries` counts the Givens steps (the MID pass of each iteration adds
  // one; nothing changes it while this kernel runs, so every CTA reads the
  // same value): a bound on the device-side loop that does not rely on the
  // scalar step at the end of this pass
  const bool over = st->entries > st->maxit + 8;
  if (st->done || over) {
    if (bid == 0 && threadIdx.x == 0) {
      if (!st->done) {
        st->status = ST_NOT_CONVERGED;
        st->done = 1;
      }
      // keep the device-side loop closed whatever set `done`
      if (a.use_cond) cudaGraphSetConditional(a.cond, 0u);
    }
    return;
  }
  __shared__ DevState s_pre;  // for the scalar step at the end
  state_prefetch(&s_pre, st);
  // z_j arrives normalised (z_j / gamma_j), so A z_j needs no scaling
  const double gam = st->gam, gam_old = st->gam_old, beta = st->beta;
  const double lanc = gam / gam_old;
  const int check = st->check;
  const TZ* z = (const TZ*)a.z;
  const int nx = a.g.nx, ny = a.g.ny;
  const int nm = DIM == 2 ? a.g.ny : a.g.nz;
  const long mstride = DIM == 2 ? (long)nx : (long)nx * ny;
  const int lane = threadIdx.x & 31;
  const int strip = a.strip;
  // strip indices in 32 bits (a plan has far fewer than 2^32 strips): one
  // 32-bit division per strip instead of 64-bit ones
  const unsigned nsx = (unsigned)(nx + 31) / 32u, nsm = (unsigned)(nm + strip - 1) / (unsigned)strip;
  const unsigned nstrips = (unsigned)stencil_strips(DIM, nx, ny, a.g.nz, strip);
  double acc[2] = {0.0, 0.0};
  ff2 dacc = {0.f, 0.f};
  float2 beta2 = make_float2(0.f, 0.f), lanc2 = make_float2(0.f, 0.f);
  if (FF) {
    beta2 = d_to_ff(beta);
    lanc2 = d_to_ff(lanc);
  }
  for (unsigned s = (unsigned)bid * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nstrips;
       s += (unsigned)nblk * (blockDim.x >> 5)) {
    const unsigned q = s / nsx;  // 2D: q < nsm; 3D: q = yfix * nsm + sm
    const int sx = (int)(s - q * nsx);
    const int sm = DIM == 3 ? (int)(q % nsm) : (int)q;
    const int yfix = DIM == 3 ? (int)(q / nsm) : 0;
    const int x = sx * 32 + lane;
    const bool vx = x < nx;
    const int m0 = sm * strip, m1 = min(m0 + strip, nm);
    const long base = DIM == 2 ? (long)x : (long)yfix * nx + x;
    if (FF && !check) {
      // Operands stream through the warp's ring of kFFStages stages, filled
      // kFFStages - 1 steps ahead by cp.async; ẑ at m-1 and m and the faces
      // shared with the previous step are carried in registers.
      const float2* zf = (const float2*)a.z;
      const float2 zero = make_float2(0.f, 0.f);
      const float2 nbeta2 = make_float2(-beta2.x, -beta2.y);
      extern __shared__ __align__(16) unsigned char ff_ring[];
      unsigned char* ring = ff_ring + (size_t)(threadIdx.x >> 5) * kFFStages * ff_stage_bytes<DIM>();
      const int nsteps = m1 - m0;
      auto issue = [&](int m, int slot) {
        FFStage<DIM>& S = *(FFStage<DIM>*)(ring + slot * ff_stage_bytes<DIM>());
        const long p = base + (long)m * mstride;
        long rx, ry;
        if (DIM == 2) {
          rx = (long)m * (nx + 1) + x;
          ry = (long)m * nx + x;
        } else {
          rx = ((long)m * ny + yfix) * (nx + 1) + x;
          ry = ((long)m * (ny + 1) + yfix) * nx + x;
        }
        cp_async16(&S.v[lane], vx ? (const void*)(a.vold + p) : (const void*)a.vold, vx);
        const bool hz = vx && m + 1 < nm;
        cp_async8(&S.zp[lane], hz ? zf + p + mstride : zf, hz);
        cp_async8(&S.cn[lane], vx ? a.cyp + ry + nx : a.cyp, vx);
        const bool hw = x <= nx;  // the face left of column x exists for x = nx too
        cp_async8(&S.cw[lane], hw ? a.cxp + rx : a.cxp, hw);
        if (lane == 31) cp_async8(&S.cw[32], vx ? a.cxp + rx + 1 : a.cxp, vx);
        if (lane == 0) cp_async8(&S.edge[0], (vx && x > 0) ? zf + p - 1 : zf, vx && x > 0);
        if (lane == 31) cp_async8(&S.edge[1], (x + 1 < nx) ? zf + p + 1 : zf, x + 1 < nx);
        if (DIM == 3) {
          cp_async8(&S.cs[lane], vx ? a.cyp + ry : a.cyp, vx);
          const bool hs = vx && yfix > 0, hn = vx && yfix < ny - 1;
          cp_async8(&S.ys[lane], hs ? zf + p - nx : zf, hs);
          cp_async8(&S.yn[lane], hn ? zf + p + nx : zf, hn);
          cp_async8(&S.cu[lane], vx ? a.czp + p + mstride : a.czp, vx);
        }
      };
      // prologue: stages for steps m0 .. m0 + kFFStages - 2 (one group each,
      // empty groups past the strip's end keep the group count uniform)
#pragma unroll
      for (int k = 0; k < kFFStages - 1; ++k) {
        if (k < nsteps) issue(m0 + k, k);
        cp_async_commit();
      }
      const long p0 = base + (long)m0 * mstride;
      float2 zm = (vx && m0 > 0) ? zf[p0 - mstride] : zero;
      float2 zc = vx ? zf[p0] : zero;
      // flux across the face below the point along the marching axis, carried
      // from the step before as minus its flux across the face above
      ff2 fbx = {0.f, 0.f}, fby = {0.f, 0.f};
      if (vx) {
        const float2 cb = DIM == 2 ? a.cyp[(long)m0 * nx + x] : a.czp[p0];
        fbx = ff_flux(cb, zc.x, zm.x);
        fby = ff_flux(cb, zc.y, zm.y);
      }
      for (int i = 0; i < nsteps; ++i) {
        const int m = m0 + i;
        const long p = base + (long)m * mstride;
        if (i + kFFStages - 1 < nsteps) issue(m + kFFStages - 1, (i + kFFStages - 1) % kFFStages);
        cp_async_commit();
        cp_async_wait<kFFStages - 1>();
        __syncwarp();
        const FFStage<DIM>& S = *(const FFStage<DIM>*)(ring + (i % kFFStages) * ff_stage_bytes<DIM>());
        const float2 zp = S.zp[lane];
        float2 zl = shfl_up_f2(zc), zr = shfl_down_f2(zc);
        if (lane == 0) zl = S.edge[0];
        if (lane == 31) zr = S.edge[1];
        const float2 cw = S.cw[lane], ce = S.cw[lane + 1];
        const float2 ca = DIM == 2 ? S.cn[lane] : S.cu[lane];  // face above along the marching axis
        if (vx) {
          ff2 kx = ff_mul1(a.alpha2, zc.x), ky = ff_mul1(a.alpha2, zc.y);
          ff_acc_flux(kx, cw, zc.x, zl.x);
          ff_acc_flux(ky, cw, zc.y, zl.y);
          ff_acc_flux(kx, ce, zc.x, zr.x);
          ff_acc_flux(ky, ce, zc.y, zr.y);
          ff_acc(kx, fbx.h, fbx.l);
          ff_acc(ky, fby.h, fby.l);
          const ff2 fax = ff_flux(ca, zc.x, zp.x), fay = ff_flux(ca, zc.y, zp.y);
          ff_acc(kx, fax.h, fax.l);
          ff_acc(ky, fay.h, fay.l);
          fbx = {-fax.h, -fax.l};
          fby = {-fay.h, -fay.l};
          if (DIM == 3) {
            const float2 cs = S.cs[lane], cn = S.cn[lane], ys = S.ys[lane], yn = S.yn[lane];
            ff_acc_flux(kx, cs, zc.x, ys.x);
            ff_acc_flux(ky, cs, zc.y, ys.y);
            ff_acc_flux(kx, cn, zc.x, yn.x);
            ff_acc_flux(ky, cn, zc.y, yn.y);
          }
          // block row of Eq. 2: (A z).x = beta z1 + (K+alpha) z2 in ky, (A z).y in kx
          ff_acc_mul1(ky, beta2, zc.x);
          ff_acc_mul1(kx, nbeta2, zc.y);
          ff_acc_mul1(dacc, make_float2(ky.h, ky.l), zc.x);
          ff_acc_mul1(dacc, make_float2(kx.h, kx.l), zc.y);
          // u' = A z - lanc v_{j-1}, all in pairs (v_{j-1} is stored as pairs)
          const float4 vo = *(const float4*)&S.v[lane];
          const ff2 px = ff_mul(lanc2, make_float2(vo.x, vo.y)), py = ff_mul(lanc2, make_float2(vo.z, vo.w));
          ff_acc(ky, -px.h, -px.l);
          ff_acc(kx, -py.h, -py.l);
          ((float4*)a.vold)[p] = make_float4(ky.h, ky.l, kx.h, kx.l);
        }
        __syncwarp();  // every lane is done with this slot before it is refilled
        zm = zc;
        zc = zp;
      }
      cp_async_wait<0>();
      __syncwarp();
      continue;
    }
    if (!check) {
      // u' = A z - lanc v_{j-1} and delta, operands of step m+1 loaded
      // before step m computes
      const double2 zero = make_double2(0.0, 0.0);
      double2 zm = (vx && m0 > 0) ? to_d2(z[base + (long)(m0 - 1) * mstride]) : zero;
      double2 zc = vx ? to_d2(z[base + (long)m0 * mstride]) : zero;
      StepOperands<DIM, TZ, VP> cur, nxt;
      cur.load(z, a, base + (long)m0 * mstride, mstride, m0, nm, x, yfix, vx, lane);
      for (int m = m0; m < m1; ++m) {
        const long p = base + (long)m * mstride;
        if (m + 1 < m1) nxt.load(z, a, p + mstride, mstride, m + 1, nm, x, yfix, vx, lane);
        const double2 zp = to_d2(cur.zn1);
        double2 zl = shfl_up_d2(zc), zr = shfl_down_d2(zc);
        if (lane == 0) zl = to_d2(cur.zl);
        if (lane == 31) zr = to_d2(cur.zr);
        if (vx) {
          double ax = cur.d * zc.x, ay = cur.d * zc.y;
          ax = fma(-cur.cw, zl.x, ax);
          ay = fma(-cur.cw, zl.y, ay);
          ax = fma(-cur.ce, zr.x, ax);
          ay = fma(-cur.ce, zr.y, ay);
          if (DIM == 2) {
            ax = fma(-cur.cs, zm.x, ax);
            ay = fma(-cur.cs, zm.y, ay);
            ax = fma(-cur.cn, zp.x, ax);
            ay = fma(-cur.cn, zp.y, ay);
          } else {
            const double2 zs = to_d2(cur.ys), zn = to_d2(cur.yn);
            ax = fma(-cur.cs, zs.x, ax);
            ay = fma(-cur.cs, zs.y, ay);
            ax = fma(-cur.cn, zn.x, ax);
            ay = fma(-cur.cn, zn.y, ay);
            ax = fma(-cur.cd, zm.x, ax);
            ay = fma(-cur.cd, zm.y, ay);
            ax = fma(-cur.cu, zp.x, ax);
            ay = fma(-cur.cu, zp.y, ay);
          }
          const double2 Az = block_A(make_double2(ax, ay), zc, beta);
          acc[0] = fma(Az.x, zc.x, fma(Az.y, zc.y, acc[0]));
          v_store<VP>(a.vold, p, make_double2(fma(-lanc, cur.vo.x, Az.x), fma(-lanc, cur.vo.y, Az.y)));
        }
        zm = zc;
        zc = zp;
        cur = nxt;
      }
      continue;
    }
    // x is float pairs in the pair-vector forms, else FP64
    typedef typename std::conditional<VP, float4, double2>::type TX;
    const TX* xs = (const TX*)a.x;
    StripWindow<DIM, TZ> wz;
    StripWindow<DIM, TX> wx;
    wz.start(z, base, mstride, m0, vx);
    wx.start(xs, base, mstride, m0, vx);
    for (int m = m0; m < m1; ++m) {
      const long p = base + (long)m * mstride;
      const double2 t = wz.KA(z, a, p, mstride, m, nm, x, yfix, vx, lane);
      double2 tx = make_double2(0.0, 0.0);
      if (check) tx = wx.KA(xs, a, p, mstride, m, nm, x, yfix, vx, lane);
      if (vx) {
        const double2 zc = wz.zc;
        const double2 Az = block_A(t, zc, beta);
        acc[0] = fma(Az.x, zc.x, fma(Az.y, zc.y, acc[0]));
        const double2 vo = v_load<VP>(a.vold, p);
        v_store<VP>(a.vold, p, make_double2(fma(-lanc, vo.x, Az.x), fma(-lanc, vo.y, Az.y)));
        if (check) {
          const double2 Ax = block_A(tx, wx.zc, beta);
          const double2 bb = a.b[p];
          const double rx = bb.x - Ax.x, ry = bb.y - Ax.y;
          acc[1] = fma(rx, rx, fma(ry, ry, acc[1]));
        }
      }
      wz.advance();
      if (check) wx.advance();
    }
  }
  if (FF) acc[0] += ff_to_d(dacc);
  pdl_trigger();
  double tot[2];
  if (!grid_sum_last_block<2>(acc, a.partials, &st->tickets[TICKET_STENCIL], tot, bid, nblk)) return;
  if (threadIdx.x != 0) return;
  // scalar step after the stencil: delta_j and the stopping test for x_{iter}.
  // It runs on a register copy of the state, loaded once and stored once: a
  // read-modify-write chain through global memory would cost an L2 round
  // trip per dependent access on this single thread.
  DevState q = s_pre;
  q.delta = tot[0];
  if (check) {
    const double rnorm = sqrt(tot[1]);
    const double rel = rnorm / q.bnorm;
    q.relres = rel;
    q.checks += 1;
    q.check = 0;
    if (rel <= q.tol) {
      q.done = 1;
      q.status = ST_OK;
    } else if (q.lucky || q.iter >= q.maxit || !(rel == rel)) {
      q.done = 1;
      q.status = (rel == rel) ? ST_NOT_CONVERGED : ST_BREAKDOWN;
    } else if (q.eta_x > 0.0) {
      q.rho = rnorm / q.eta_x;  // calibrate the 2-norm / P^{-1}-norm ratio
      q.calibrated = 1;
    }
  }
  if (!q.done && !(q.delta == q.delta)) {
    q.done = 1;
    q.status = ST_BREAKDOWN;
  }
  q.loops += 1;
  if (q.iter > q.maxit + 1 || q.loops > q.maxit + 4) q.done = 1;  // hard caps (integers only)
  // the fields this step sets (the copy's tickets and entry count may be stale)
  st->delta = q.delta;
  st->relres = q.relres;
  st->checks = q.checks;
  st->check = q.check;
  st->rho = q.rho;
  st->calibrated = q.calibrated;
  st->loops = q.loops;
  st->status = q.status;
  st->done = q.done;
  if (a.use_cond) cudaGraphSetConditional(a.cond, q.done ? 0u : 1u);
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
// The fields the Givens step (or the start of MINRES) sets, from the register
// copy q to the state in memory.
__device__ __forceinline__ void store_scalar_fields(DevState* st, const DevState& q) {
  st->w_a = q.w_a;
  st->w_b = q.w_b;
  st->w_c = q.w_c;
  st->x_coef = q.x_coef;
  st->a1inv_old = q.a1inv_old;
  st->a1inv_old2 = q.a1inv_old2;
  st->eta = q.eta;
  st->eta_x = q.eta_x;
  st->c_old = q.c_old;
  st->c = q.c;
  st->s_old = q.s_old;
  st->s = q.s;
  st->gam_old = q.gam_old;
  st->gam = q.gam;
  st->gam1 = q.gam1;
  st->rho = q.rho;
  st->iter = q.iter;
  st->check = q.check;
  st->lucky = q.lucky;
  st->status = q.status;
  st->done = q.done;
}

// st: the caller's register copy of the solver state (see mid_scalar_tail).
// It runs on one thread, where FP64 is latency-bound on GB300 (a dependent
// FMA about 67 cycles, a division about 440, a square root about 700), so
// the chain is kept short: a1 = sqrt(a0^2 + g2) does not wait for gn =
// sqrt(g2), one reciprocal 1/a1 serves cn, sn and the x coefficient, and the
// reciprocals of the last two a1 are kept in the state for the w coefficients.
__device__ inline void givens_step(DevState* st, double g2) {
  if (!(g2 >= 0.0) || !(g2 < 1e300)) {
    st->done = 1;
    st->status = ST_BREAKDOWN;
    return;
  }
  const double gam = st->gam, delta = st->delta;
  const double c = st->c, c_old = st->c_old, s = st->s, s_old = st->s_old;
  const double a0 = c * delta - c_old * s * gam;
  const double gn = sqrt(g2);
  const double a1 = sqrt(fma(a0, a0, g2));
  const double a2 = s * delta + c_old * c * gam;
  const double a3 = s_old * gam;
  // w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j) / a1 with z_j stored normalised
  // (z_j / gamma_j); the buffers hold w_k scaled by the a1 that made it, so
  // that the update needs no product with z: a1 w_{j+1} = z_j - (a3/a1'') (a1'' w_{j-1})
  // - (a2/a1') (a1' w_j), and x += (c_{j+1} eta / a1) (a1 w_{j+1})
  const double wb = -a3 * st->a1inv_old2, wc = -a2 * st->a1inv_old;
  if (!(a1 > 0.0) || !(a1 < 1e300)) {
    st->done = 1;
    st->status = ST_BREAKDOWN;
    return;
  }
  const double inv = 1.0 / a1;
  const double cn = a0 * inv, sn = gn * inv;
  st->w_a = 1.0;
  st->w_b = wb;
  st->w_c = wc;
  st->x_coef = cn * st->eta * inv;
  st->a1inv_old2 = st->a1inv_old;
  st->a1inv_old = inv;
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
  if (st->hist && st->iter <= st->hist_cap) st->hist[st->iter - 1] = e / st->gam1;
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
// Ingest: f (complex128) -> b = [Im f; Re f] (block form, Eq. 2), MINRES
// start vectors, ||b||, and the scalar state.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// MINRES direction and iterate update of iteration j as a streaming kernel
// (run beside the inverse x transform of the same iteration, which does not
// touch these vectors): w_{j+1} = ẑ_j + w_b w_{j-1} + w_c w_j (the w buffers
// hold w scaled by its a1, so w_a = 1) over w_{j-1}'s buffer, and
// x_j = x_{j-1} + x_coef w_{j+1}; the coefficients come from the Givens step
// in the MID pass.  Per point: ẑ_j, w_{j-1}, w_j, x read, w_{j+1}, x written.
// ---------------------------------------------------------------------------
struct UpdateArgs {
  const void* z;     // ẑ_j (TZ)
  double2* wprev;    // in: w_{j-1}; out: w_{j+1}
  const double2* wcur;
  double2* x;
  const DevState* st;
  long M;
};

constexpr int kUpdateUnroll = 2;

// one component of the pair update: w_{j+1} = z + wb w_{j-1} + wc w_j and
// x_j = x_{j-1} + xc w_{j+1}, all float pairs (renormalised on store)
__device__ __forceinline__ void ff_update(float z, float2 wp, float2 wq, float2 xo, float2 wb2, float2 wc2,
                                          float2 xc2, ff2& wn, ff2& xn) {
  ff2 acc = {z, 0.f};
  const ff2 p1 = ff_mul(wc2, wq), p2 = ff_mul(wb2, wp);
  ff_acc(acc, p1.h, p1.l);
  ff_acc(acc, p2.h, p2.l);
  wn = ff_two_sum(acc.h, acc.l);
  const ff2 p3 = ff_mul(xc2, make_float2(wn.h, wn.l));
  ff2 xa = {xo.x, xo.y};
  ff_acc(xa, p3.h, p3.l);
  xn = ff_two_sum(xa.h, xa.l);
}

template <typename TZ, bool VP>
__global__ void __launch_bounds__(256) k_update(UpdateArgs a) {
  if (a.st->done) return;
  const double wb = a.st->w_b, wc = a.st->w_c, xc = a.st->x_coef;
  const TZ* z = (const TZ*)a.z;
  constexpr int U = kUpdateUnroll;
  if constexpr (VP) {  // pair-vector forms: w and x as float pairs
    const float2 wb2 = d_to_ff(wb), wc2 = d_to_ff(wc), xc2 = d_to_ff(xc);
    const float4* wq4 = (const float4*)a.wcur;
    float4* wp4 = (float4*)a.wprev;
    float4* x4 = (float4*)a.x;
    for (long c0 = (long)blockIdx.x * 256 * U; c0 < a.M; c0 += (long)gridDim.x * 256 * U) {
      float2 zj[U];
      float4 wp[U], wq[U], xo[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const long p = c0 + threadIdx.x + 256 * k;
        if (p < a.M) {
          zj[k] = ((const float2*)z)[p];
          wp[k] = wp4[p];
          wq[k] = wq4[p];
          xo[k] = x4[p];
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const long p = c0 + threadIdx.x + 256 * k;
        if (p < a.M) {
          ff2 wr, xr, wi, xi;
          ff_update(zj[k].x, make_float2(wp[k].x, wp[k].y), make_float2(wq[k].x, wq[k].y),
                    make_float2(xo[k].x, xo[k].y), wb2, wc2, xc2, wr, xr);
          ff_update(zj[k].y, make_float2(wp[k].z, wp[k].w), make_float2(wq[k].z, wq[k].w),
                    make_float2(xo[k].z, xo[k].w), wb2, wc2, xc2, wi, xi);
          wp4[p] = make_float4(wr.h, wr.l, wi.h, wi.l);
          x4[p] = make_float4(xr.h, xr.l, xi.h, xi.l);
        }
      }
    }
  } else {
    for (long c0 = (long)blockIdx.x * 256 * U; c0 < a.M; c0 += (long)gridDim.x * 256 * U) {
      TZ zj[U];
      double2 wp[U], wq[U], xo[U];
  #pragma unroll
      for (int k = 0; k < U; ++k) {
        const long p = c0 + threadIdx.x + 256 * k;
        if (p < a.M) {
          zj[k] = z[p];
          wp[k] = a.wprev[p];
          wq[k] = a.wcur[p];
          xo[k] = a.x[p];
        }
      }
  #pragma unroll
      for (int k = 0; k < U; ++k) {
        const long p = c0 + threadIdx.x + 256 * k;
        if (p < a.M) {
          const double2 zd = to_d2(zj[k]);
          const double2 wn = make_double2(fma(wb, wp[k].x, fma(wc, wq[k].x, zd.x)),
                                          fma(wb, wp[k].y, fma(wc, wq[k].y, zd.y)));
          a.wprev[p] = wn;
          a.x[p] = make_double2(fma(xc, wn.x, xo[k].x), fma(xc, wn.y, xo[k].y));
        }
      }
    }
  }
}

// the FP32 forms' iterate (float pairs) as FP64 values for the caller
static __global__ void k_x_out(const float4* __restrict__ x, double2* __restrict__ out, long M) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x)
    out[p] = to_d2(x[p]);
}

struct IngestArgs {
  long M;
  const double2* f;
  double2 *b, *v0, *v1, *w0, *w1, *x;
  DevState* st;
  double* partials;
  double tol, beta, sqrt_pmin, sqrt_pmax;
  int maxit;
  int vpair;  // FP32 forms: v stored as float pairs
};

static __global__ void __launch_bounds__(256) k_ingest(IngestArgs a0, const IngestArgs* batch, int bps) {
  const int sys = batch ? (int)(blockIdx.x / bps) : 0;
  const int bid = batch ? (int)blockIdx.x - sys * bps : (int)blockIdx.x;
  const int nblk = batch ? bps : (int)gridDim.x;
  const IngestArgs a = batch ? batch[sys] : a0;
  double acc[1] = {0.0};
  const double2 zero = make_double2(0.0, 0.0);
  for (long p = (long)bid * blockDim.x + threadIdx.x; p < a.M; p += (long)nblk * blockDim.x) {
    const double2 fv = a.f[p];
    const double2 bb = make_double2(fv.y, fv.x);
    a.b[p] = bb;
    if (a.vpair) {  // FP32 forms: v as float pairs (see v_store)
      const float2 re = d_to_ff(bb.x), im = d_to_ff(bb.y);
      ((float4*)a.v0)[p] = make_float4(re.x, re.y, im.x, im.y);
    } else {
      a.v0[p] = bb;
    }
    a.v1[p] = zero;
    a.w0[p] = zero;
    a.w1[p] = zero;
    a.x[p] = zero;
    acc[0] = fma(bb.x, bb.x, fma(bb.y, bb.y, acc[0]));
  }
  double tot[1];
  if (!grid_sum_last_block<1>(acc, a.partials, &a.st->tickets[TICKET_INGEST], tot, bid, nblk)) return;
  if (threadIdx.x != 0) return;
  DevState* st = a.st;
  st->bnorm = sqrt(tot[0]);
  st->r0norm = st->bnorm;
  st->tol = a.tol;
  st->maxit = a.maxit;
  st->beta = a.beta;
  st->sqrt_pmin = a.sqrt_pmin;
  st->sqrt_pmax = a.sqrt_pmax;
  st->c = st->c_old = 1.0;
  st->s = st->s_old = 0.0;
  st->delta = 0.0;
  st->gam = st->gam_old = st->gam1 = 1.0;
  st->a1inv_old = st->a1inv_old2 = 1.0;
  st->eta = st->eta_x = 0.0;
  st->rho = 0.0;
  st->iter = 0;
  st->entries = 0;
  st->check = 0;
  st->lucky = 0;
  st->checks = 0;
  st->loops = 0;
  st->calibrated = 0;
  st->status = ST_OK;
  st->relres = 1.0;
  st->done = 0;
  if (st->bnorm == 0.0) {  // f = 0: z = 0 is exact
    st->done = 1;
    st->relres = 0.0;
    st->status = ST_OK;
  } else if (!(st->bnorm < INFINITY)) {  // f holds a NaN or an infinity
    st->done = 1;
    st->relres = __longlong_as_double(0x7ff8000000000000ll);
    st->status = ST_BREAKDOWN;
  }
}

// Warm start: with the initial guess x_0, MINRES runs on the correction
// A d = b - A x_0 from d = 0 (x = x_0 + d), so the block right-hand side and
// v_1 become r_0 = b - A x_0 (Eq. 2's operator in FP64); ||r_0|| calibrates
// the residual estimate, while the stopping test stays relative to ||b||.
// x_0 already meeting the tolerance ends the solve at once with x = x_0.
struct WarmArgs {
  Grid g;
  const double2* x0;  // block pairs (Re, Im) of the caller's initial guess
  double2 *b, *v0;
  const double *cx, *cy, *cz, *dg;
  DevState* st;
  double* partials;
  int vpair;
};

template <int DIM>
__global__ void __launch_bounds__(256) k_warm_start(WarmArgs a) {
  DevState* st = a.st;
  if (st->done) return;  // f = 0 or not finite: decided by the ingest
  const double beta = st->beta;
  double acc[1] = {0.0};
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < a.g.M; p += (long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    point_coords(p, a.g, ix, iy, iz);
    double2 xc;
    const double2 Ax = block_A(stencil_KA<DIM, double2>(a.x0, a.cx, a.cy, a.cz, a.dg, a.g, p, ix, iy, iz, xc), xc, beta);
    const double2 bb = a.b[p];
    const double2 r = make_double2(bb.x - Ax.x, bb.y - Ax.y);
    a.b[p] = r;
    if (a.vpair) {
      const float2 re = d_to_ff(r.x), im = d_to_ff(r.y);
      ((float4*)a.v0)[p] = make_float4(re.x, re.y, im.x, im.y);
    } else {
      a.v0[p] = r;
    }
    acc[0] = fma(r.x, r.x, fma(r.y, r.y, acc[0]));
  }
  double tot[1];
  if (!grid_sum_last_block<1>(acc, a.partials, &st->tickets[TICKET_AUX], tot, blockIdx.x, gridDim.x)) return;
  if (threadIdx.x != 0) return;
  st->r0norm = sqrt(tot[0]);
  st->relres = st->r0norm / st->bnorm;
  if (!(st->r0norm < INFINITY)) {
    st->done = 1;
    st->status = ST_BREAKDOWN;
  } else if (st->r0norm <= st->tol * st->bnorm) {
    st->done = 1;
    st->status = ST_OK;
  }
}

// egress with a warm start: z = x_0 + d (d as float pairs or FP64)
static __global__ void k_x_out_add(const double2* __restrict__ d, int pairs, const double2* __restrict__ x0,
                                   double2* __restrict__ out, long M) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
    const double2 dd = pairs ? to_d2(((const float4*)d)[p]) : d[p];
    const double2 x = x0[p];
    out[p] = make_double2(x.x + dd.x, x.y + dd.y);
  }
}

// ---------------------------------------------------------------------------
// Plan set-up kernels
// ---------------------------------------------------------------------------
// scaled copy of one face array (a_e / h^2) and its min / max / validity
static __global__ void k_scale_faces(const double* __restrict__ src, double* __restrict__ dst, long count,
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

// scaled faces as float pairs for the float-pair stencil: hi = RN(c), lo = RN(c - hi)
static __global__ void k_pair_faces(const double* __restrict__ c, float2* __restrict__ out, long count) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const double v = c[i];
    const float h = __double2float_rn(v);
    out[i] = make_float2(h, __double2float_rn(v - (double)h));
  }
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
