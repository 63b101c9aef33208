// Shared device types for the complex-shifted Laplacian solver (arXiv 2408.00488).
//
// Vector layout in HBM: one 16-byte double2 per grid point holding the pair
// (block-1, block-2) of the 2x2 block real system of Eq. 2, C order with x
// fastest.  Both blocks always travel together, so every sine transform is a
// complex FFT of the pair and every stencil load serves both blocks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace csl {

template <typename T> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

template <typename T>
__device__ __forceinline__ typename C2<T>::t mkc(T x, T y) {
  typename C2<T>::t r;
  r.x = x;
  r.y = y;
  return r;
}

// Exact float -> double by moving the sign, exponent and mantissa fields with
// integer instructions.  On GB300 the hardware conversion issues on the FP64
// pipe (about two per SM per clock), which the FP64 stencil and vector
// updates already saturate; the integer pipe is idle.  Zero, infinities and
// NaN are handled; subnormal floats (exponent field 0) take the hardware path.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) {
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
  }
  const unsigned ex = (e == 255u) ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
  const unsigned hi = (u & 0x80000000u) | (ex << 20) | ((u >> 3) & 0xfffffu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// Double -> float with round-to-nearest-even by integer field moves, for the
// same reason (the hardware conversion issues on the FP64 pipe): the 52-bit
// mantissa is cut to 23 bits and rounded up when the 29 dropped bits exceed
// half an ulp, or equal it with an odd kept mantissa; a carry out of the
// mantissa increments the exponent (and overflows to infinity at the top).
// Results that would be zero or subnormal, and infinities / NaN, take the
// hardware path.
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 897u || e > 1150u) return __double2float_rn(d);  // float exponent 1..254 only
  unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
  return __uint_as_float(f);
}

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(f2d_exact(v.x), f2d_exact(v.y)); }
// a complex value held as two float pairs (re.hi, re.lo, im.hi, im.lo): the
// FP32 forms' storage of the MINRES vectors v, w and x
__device__ __forceinline__ double2 to_d2(float4 v) {
  return make_double2(f2d_exact(v.x) + f2d_exact(v.y), f2d_exact(v.z) + f2d_exact(v.w));
}
template <typename T> __device__ __forceinline__ typename C2<T>::t from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float>(double2 v) {
  return make_float2(d2f_rn(v.x), d2f_rn(v.y));
}
template <typename TZ> __device__ __forceinline__ TZ store_as(double2 v);
template <> __device__ __forceinline__ double2 store_as<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 store_as<float2>(double2 v) {
  return make_float2(d2f_rn(v.x), d2f_rn(v.y));
}

// Scalars of one MINRES solve, resident in device memory so that the whole
// iteration (including the Givens step and the stopping decision) runs
// without host round trips.
struct DevState {
  // Lanczos recurrence: gam = gamma_j, gam_old = gamma_{j-1}, delta = delta_j
  double gam, gam_old, gam1, delta;
  // Givens rotations (c_j, c_{j-1}, s_j, s_{j-1}) and the rotated right-hand side eta
  double c, c_old, s, s_old, eta;
  // coefficients of the update w_{j+1} = w_a z_j + w_b w_{j-1} + w_c w_j, x += x_coef w_{j+1};
  // the w vectors are kept scaled by the a1 of the step that made them
  // (w_a = 1); a1inv_old / a1inv_old2 are the reciprocals of the a1 of the
  // last two steps
  double w_a, w_b, w_c, x_coef, a1inv_old, a1inv_old2;
  double bnorm, tol;
  double rho;     // calibrated ratio ||b - A x||_2 / |eta| (residual 2-norm per P^{-1}-norm)
  double relres;  // last explicitly evaluated true relative residual
  double eta_x;   // |eta| belonging to the current iterate x
  double beta;    // coupling coefficient of this solve (beta, or -beta for the adjoint)
  double sqrt_pmin, sqrt_pmax;  // sqrt of extreme eigenvalues of one block of P
  double r0norm;  // ||b - A x_0||_2 of the start vector (= bnorm for x_0 = 0)
  double* hist;   // optional: |eta_j| / gamma_1 of every iteration j (hist_cap entries), or null
  int hist_cap;
  int entries;    // Givens steps started (MID passes): a loop bound that needs no reduction
  int iter;       // completed iterations = index of the current iterate x
  int maxit, done, status, check, lucky, checks, calibrated, loops;
  unsigned int tickets[4];
};

static_assert(sizeof(DevState) % 4 == 0, "DevState is copied as 32-bit words");

// Copy of the solver state into shared memory, taken when a kernel starts
// (after its predecessor completed), so that the scalar step at its end does
// not wait on a global round trip.  Only that step changes the scalars while
// the kernel runs; the reduction tickets do change (other CTAs may have
// arrived before this one started), so a scalar step writes back the fields
// it sets, never the whole copy.  Block-wide; a barrier must separate it from
// the reads.
__device__ __forceinline__ void state_prefetch(DevState* dst, const DevState* st) {
  constexpr int W = (int)(sizeof(DevState) / 4);
  for (int i = threadIdx.x; i < W; i += blockDim.x) ((unsigned*)dst)[i] = ((const unsigned*)st)[i];
}

enum { TICKET_STENCIL = 0, TICKET_MID = 1, TICKET_INGEST = 2, TICKET_AUX = 3 };  // TICKET_AUX: warm start

// status codes mirrored from csl.h
enum {
  ST_OK = 0, ST_INVALID_ARG = 1, ST_UNSUPPORTED = 2, ST_SINGULAR = 3, ST_BREAKDOWN = 4,
  ST_NOT_CONVERGED = 5, ST_TIMEOUT = 6, ST_CUDA = 7, ST_OOM = 8
};

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may start while its predecessor in the
// stream is still running: pdl_wait() blocks until the predecessor grid has
// completed and its memory is visible (a no-op after a normal launch), so it
// precedes every read of data an earlier kernel wrote; pdl_trigger() lets
// the next grid launch once every CTA of this grid has triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV per-thread values over the block; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* >= 32*NV */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[wid * NV + i] = v[i];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = (lane < nw) ? sh[lane * NV + i] : 0.0;
      v[i] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Deterministic grid reduction: every block deposits its block sum in
// partials[blockIdx.x*NV + i]; the last block to arrive (atomic ticket) sums
// the deposits in block order and returns true with the totals in tot[]
// (valid in all threads of that block).  The ticket is re-armed for reuse.
// bid / nblk: the block's index and the number of blocks working on the same
// system (the whole grid for a single system; one slice of a batched launch).
template <int NV>
__device__ bool grid_sum_last_block(double (&v)[NV], double* partials, unsigned int* ticket,
                                    double (&tot)[NV], int bid, int nblk) {
  __shared__ double sh[32 * NV];
  __shared__ int s_last;
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[bid * NV + i] = v[i];
    // one acquire-release arrival: the release orders this thread's partial
    // stores before it, and the last arrival's acquire orders every other
    // CTA's partials before this CTA's reads below (the CTA barrier passes
    // that order on to the other threads)
    unsigned int t;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(t) : "l"(ticket) : "memory");
    s_last = (t == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += ((volatile double*)partials)[b * NV + i];
  }
  block_sum<NV>(acc, sh);
  __shared__ double s_tot[NV];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) s_tot[i] = acc[i];
    *ticket = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) tot[i] = s_tot[i];
  return true;
}

// Launch k<<<grid, block, smem, s>>>(args...), with the programmatic
// stream-serialisation attribute when pdl is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

}  // namespace csl
