// Sine transforms along y and z as split-BF16 GEMMs on the fifth-generation
// tensor cores (tcgen05.mma, FP32 accumulators in tensor memory).
//
// For lines of N = n+1 <= 128 points, the unnormalised DST-I of Section 2.3
// (y_k = sum_j sin(pi k j / N) x_j, j, k = 1..n) is a dense N x N contraction
// with the sine matrix S[k][j] = sin(pi (k+1)(j+1) / N) (0-based; row and
// column N-1 are zero padding).  A CTA takes a tile of 64 adjacent complex
// columns of the strided pass.  With the real and imaginary parts as separate
// rows, the tile is the 128 x N matrix X^T (row = one real line, K = position
// along the line), and
//     D = X^T S^T        (M = 128, N_mma = N, K = N)
// leaves every transformed line in one TMEM lane.
//
// Precision: the FP32 data are split on the fly into bf16 terms
// x = x_0 + x_1 (+ x_2), S likewise once on the host, and D accumulates the
// products x_a S_b with a + b < SPLIT in FP32: 3 products for SPLIT = 2
// (about 2^-16 relative), 6 products for SPLIT = 3 (about FP32 rounding).
//
// The MID variant then scales D by the per-mode factor of Eq. 4, accumulates
// the Parseval sum sum_k s_k |S v|_k^2 for gamma_{j+1}^2, splits the scaled
// spectrum into the A operand again and runs the inverse transform as a
// second GEMM before the store; its last CTA runs the Givens step exactly as
// the FFT variant does.
//
// Shared-memory operands use the no-swizzle K-major layout of tcgen05: core
// matrices of 8 rows x 16 bytes (8 bf16 along K), 128 bytes each.  A
// (128 rows): core (row/8, k/8) at ((k/8)*16 + row/8)*128, i.e. leading
// (K-direction) byte offset 2048 and stride (row-group) byte offset 128.
// B = S (N rows): core (row/8, k/8) at ((k/8)*(N/8) + row/8)*128, leading
// offset 16N, stride offset 128.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "csl_passes.cuh"

namespace csl {
namespace {

constexpr int kTcThreads = 256;
constexpr long long kTcWaitCycles = 1ll << 31;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major
template <int NN>
__host__ __device__ constexpr uint32_t umma_idesc_m128() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait for the mbarrier phase `parity`; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (true) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
}

// 32 lanes x KC columns of FP32 from TMEM (this warp's lane quarter)
template <int KC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[KC]);

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x (8 consecutive K elements) = sum of SPLIT bf16 terms, each packed as one
// 16-byte core-matrix row (element e at byte 2e)
template <int SPLIT>
__device__ __forceinline__ void split_pack(const float* x, uint4 (&out)[SPLIT]) {
  float r[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = x[i];
#pragma unroll
  for (int t = 0; t < SPLIT; ++t) {
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * p], r[2 * p + 1]);
      w[p] = *reinterpret_cast<const uint32_t*>(&h);
      if (t + 1 < SPLIT) {
        r[2 * p] -= __low2float(h);
        r[2 * p + 1] -= __high2float(h);
      }
    }
    out[t] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// byte offset of the 16-byte row (row, K chunk kc) in the 128-row A operand
__device__ __forceinline__ uint32_t a_off(int row, int kc) {
  return (uint32_t)(((kc << 4) + (row >> 3)) * 128 + (row & 7) * 16);
}

// D (+)= sum_{a+b<SPLIT} A_a B_b^T over K = N, issued by one thread.  The
// descriptors differ only in their start-address field (low 14 bits, in
// 16-byte units, no carry below 256 KB), so each is a base plus an offset.
template <int N, int SPLIT>
__device__ __forceinline__ void issue_gemm(uint32_t tmem_d, uint32_t sA, uint32_t sB) {
  constexpr uint32_t A_BYTES = 128u * N * 2u, B_BYTES = (uint32_t)N * N * 2u;
  constexpr uint32_t idesc = umma_idesc_m128<N>();
  const uint64_t da0 = umma_desc(sA, 2048u, 128u);
  const uint64_t db0 = umma_desc(sB, 16u * N, 128u);
  uint32_t acc = 0;
#pragma unroll 1
  for (int s = 0; s < N / 16; ++s) {
#pragma unroll
    for (int ta = 0; ta < SPLIT; ++ta)
#pragma unroll
      for (int tb = 0; tb < SPLIT - ta; ++tb) {
        const uint64_t da = da0 + (uint64_t)((ta * A_BYTES + (uint32_t)s * 4096u) >> 4);
        const uint64_t db = db0 + (uint64_t)((tb * B_BYTES + (uint32_t)s * 32u * N) >> 4);
        umma_bf16(tmem_d, da, db, idesc, acc);
        acc = 1;
      }
  }
}

template <int NC>
__host__ __device__ constexpr uint32_t tmem_cols_pow2() {
  return NC <= 32 ? 32u : NC <= 64 ? 64u : NC <= 128 ? 128u : NC <= 256 ? 256u : 512u;
}

}  // namespace

template <int N, bool MID, int SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_strided_tc(StridedArgs<float> a0, const StridedArgs<float>* batch, int bps) {
  constexpr uint32_t A_BYTES = 128u * N * 2u, B_BYTES = (uint32_t)N * N * 2u;
  constexpr uint32_t TCOLS = tmem_cols_pow2<MID ? 2 * N : N>();
  constexpr int KC = (N / 2) < 32 ? (N / 2) : 32;  // TMEM columns per load
  constexpr int CPT = N / 32;                      // K chunks of 8 per thread in the load phase
  const int sys = batch ? (int)(blockIdx.x / bps) : 0;
  const int bid = batch ? (int)blockIdx.x - sys * bps : (int)blockIdx.x;
  const int nblk = batch ? bps : (int)gridDim.x;
  const StridedArgs<float> a = batch ? batch[sys] : a0;
  pdl_wait();
  if (a.st && a.st->done) return;
  if (MID && a.scalar_mode == 2 && bid == 0 && threadIdx.x == 0) a.st->entries += 1;  // read by the next stencil pass

  extern __shared__ __align__(128) unsigned char tc_smem[];
  unsigned char* sB = tc_smem;                  // SPLIT sine-matrix terms
  unsigned char* sA = tc_smem + SPLIT * B_BYTES;  // SPLIT data terms
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_bar;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const uint4* src = (const uint4*)a.sine_tc;
    uint4* dst = (uint4*)sB;
    for (int i = tid; i < (int)(SPLIT * B_BYTES / 16); i += kTcThreads) dst[i] = src[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t bar = smem_u32(&s_bar);
  const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
  uint32_t phase = 0;

  const int n = a.n;
  const int ntx = (a.ncols + 63) / 64;
  const int ntiles = ntx * a.nouter;
  // load phase: complex column lc of the tile, K chunks lg, lg+4, ...
  const int lc = tid & 63, lg = tid >> 6;
  // epilogue: TMEM lane (= A row) er holds the real (er < 64) or imaginary
  // part of column ec; warps w and w+4 share the lane quarter and split the
  // columns (modes) into halves eh
  const int er = 32 * (warp & 3) + lane, eh = warp >> 2;
  const int ecomp = er >> 6, ec = er & 63;
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  float* fdata = (float*)a.data;
  double g2acc = 0.0;
  int ok = 1;
  uint32_t pending = 0;  // after a wait gave up: the parity of the commit still outstanding

  for (int tile = bid; tile < ntiles; tile += nblk) {
    const int o = tile / ntx;
    const int col0 = (tile - o * ntx) * 64;
    const long base = (long)o * a.outer_stride + col0;
    {
      // element offsets j * line_stride stay below 2^31 (at most 1023 * 1024^2)
      const bool cv = col0 + lc < a.ncols;
      const float2* src = a.data + base + lc;
      const int ls = (int)a.line_stride;
      constexpr int QB = CPT < 2 ? CPT : 2;  // K chunks loaded together
#pragma unroll
      for (int q0 = 0; q0 < CPT; q0 += QB) {
        float2 v[QB][8];
#pragma unroll
        for (int q = 0; q < QB; ++q)
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int j = (lg + 4 * (q0 + q)) * 8 + i;
            v[q][i] = (cv && j < n) ? src[j * ls] : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int q = 0; q < QB; ++q) {
          const int kc = lg + 4 * (q0 + q);
          float re[8], im[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            re[i] = v[q][i].x;
            im[i] = v[q][i].y;
          }
          uint4 pr[SPLIT], pi[SPLIT];
          split_pack<SPLIT>(re, pr);
          split_pack<SPLIT>(im, pi);
#pragma unroll
          for (int t = 0; t < SPLIT; ++t) {
            *(uint4*)(sA + t * A_BYTES + a_off(lc, kc)) = pr[t];
            *(uint4*)(sA + t * A_BYTES + a_off(64 + lc, kc)) = pi[t];
          }
        }
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_gemm<N, SPLIT>(tmem, sA_u, sB_u);
      umma_commit(bar);
    }
    ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0);
    if (!ok) {
      pending = phase;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    if (MID) {
      const bool cvalid = col0 + ec < a.ncols;
      float murest = 0.f;
      if (cvalid) {
        murest = a.mu_col[col0 + ec];
        if (a.mu_outer) murest += a.mu_outer[o];
      }
      float part = 0.f;
#pragma unroll
      for (int ch = 0; ch < (N / 2) / KC; ++ch) {
        const int k0 = eh * (N / 2) + ch * KC;
        float F[KC];
        tmem_ld<KC>(tmem + tlane + (uint32_t)k0, F);
#pragma unroll
        for (int i = 0; i < KC; ++i) {
          const int k = k0 + i;
          float fsc = 0.f;
          if (cvalid && k < n) {
            const float e = fmaf(a.gamma, murest + a.mu_line[k], a.alpha);
            const float sc = a.cnorm * rsqrtf(fmaf(e, e, a.beta2));
            fsc = sc * F[i];
            part = fmaf(fsc, F[i], part);
          }
          F[i] = fsc;
        }
#pragma unroll
        for (int q = 0; q < KC / 8; ++q) {
          uint4 pk[SPLIT];
          split_pack<SPLIT>(&F[8 * q], pk);
#pragma unroll
          for (int t = 0; t < SPLIT; ++t) *(uint4*)(sA + t * A_BYTES + a_off(er, (k0 >> 3) + q)) = pk[t];
        }
      }
      g2acc += (double)part;
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        issue_gemm<N, SPLIT>(tmem + (uint32_t)N, sA_u, sB_u);
        umma_commit(bar);
      }
      ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0);
      if (!ok) {
        pending = phase;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
    }
    {
      const uint32_t dcol = MID ? (uint32_t)N : 0u;
      const bool cvalid = col0 + ec < a.ncols;
#pragma unroll
      for (int ch = 0; ch < (N / 2) / KC; ++ch) {
        const int k0 = eh * (N / 2) + ch * KC;
        float D[KC];
        tmem_ld<KC>(tmem + tlane + dcol + (uint32_t)k0, D);
        if (cvalid) {
          float* dst = fdata + 2 * (base + ec) + ecomp;
          const int ls2 = 2 * (int)a.line_stride;
#pragma unroll
          for (int i = 0; i < KC; ++i) {
            const int k = k0 + i;
            if (k < n) dst[k * ls2] = D[i];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // operands and TMEM free for the next tile
  }
  if (!ok) {
    // A wait gave up (about a second without the commit's arrival).  The
    // MMAs of that commit may still be in flight, reading this CTA's shared
    // memory and writing its TMEM: wait for the same commit once more,
    // again bounded, before the TMEM is freed and the CTA exits.  No thread
    // issues further MMAs or writes the operands after the break, so a
    // commit that arrives within this second wait leaves nothing in flight.
    (void)mbar_wait(bar, pending);
    tc_fence_after();
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  if (!ok && tid == 0 && a.st) {
    a.st->status = ST_TIMEOUT;
    a.st->done = 1;
  }
  if (MID && a.scalar_mode != 0) mid_scalar_tail<float>(a, g2acc, bid, nblk);
}

// ---------------------------------------------------------------------------
size_t tc_smem_bytes(int N, int split) { return (size_t)split * ((size_t)128 * N * 2 + (size_t)N * N * 2); }

int tc_ctas_per_sm(int N, int split, bool mid) {
  const size_t smem = tc_smem_bytes(N, split);
  int by_smem = (int)((220 * 1024) / (smem + 1024));
  const int cols = mid ? 2 * N : N;
  const int tcols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
  // registers: the N >= 64 variants use close to 255 per thread
  const int by_regs = N >= 64 ? 1 : 65536 / (kTcThreads * 160);
  int c = by_smem < 512 / tcols ? by_smem : 512 / tcols;
  if (c > by_regs) c = by_regs;
  return c < 1 ? 1 : c;
}

bool tc_supported(int N) { return N == 32 || N == 64 || N == 128; }

namespace {
template <int N, bool MID, int SPLIT>
cudaError_t launch_tc_n(const StridedArgs<float>& a, const PassLaunch& L, cudaStream_t s,
                        const StridedArgs<float>* batch, int nsys) {
  const int grid = batch ? L.blocks * nsys : L.blocks;
  return launch_k(L.pdl != 0, k_strided_tc<N, MID, SPLIT>, grid, kTcThreads, L.smem, s, a, batch, L.blocks);
}

template <int N, bool MID, int SPLIT>
cudaError_t tc_attr_n() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_strided_tc<N, MID, SPLIT>);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_strided_tc<N, MID, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}
}  // namespace

cudaError_t launch_strided_tc(int N, int split, bool mid, const StridedArgs<float>& a, const PassLaunch& L,
                              cudaStream_t s, const StridedArgs<float>* batch, int nsys) {
#define TC_CASE(NN)                                                                         \
  if (N == NN) {                                                                            \
    if (split == 2) return mid ? launch_tc_n<NN, true, 2>(a, L, s, batch, nsys)             \
                               : launch_tc_n<NN, false, 2>(a, L, s, batch, nsys);           \
    if (split == 3) return mid ? launch_tc_n<NN, true, 3>(a, L, s, batch, nsys)             \
                               : launch_tc_n<NN, false, 3>(a, L, s, batch, nsys);           \
  }
  TC_CASE(32)
  TC_CASE(64)
  TC_CASE(128)
#undef TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t set_tc_attrs() {
  cudaError_t e = cudaSuccess;
#define TC_ATTR(NN)                                           \
  if (e == cudaSuccess) e = tc_attr_n<NN, true, 2>();         \
  if (e == cudaSuccess) e = tc_attr_n<NN, false, 2>();        \
  if (e == cudaSuccess) e = tc_attr_n<NN, true, 3>();         \
  if (e == cudaSuccess) e = tc_attr_n<NN, false, 3>();
  TC_ATTR(32)
  TC_ATTR(64)
  TC_ATTR(128)
#undef TC_ATTR
  return e;
}

// ---- host: the sine matrix as SPLIT bf16 terms in the B-operand layout ----
namespace {
uint16_t bf16_rn(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}
}  // namespace

void build_sine_image(int N, int split, std::vector<uint16_t>& img) {
  img.assign((size_t)split * N * N, 0);
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j) {
      double r = 0.0;
      if (k < N - 1 && j < N - 1) r = sin(M_PI * (double)(((long)(k + 1) * (j + 1)) % (2L * N)) / (double)N);
      // element (row k, K index j): core (k/8, j/8) at ((j/8)*(N/8) + k/8)*128 bytes
      const size_t off = ((size_t)((j >> 3) * (N >> 3) + (k >> 3)) * 128 + (size_t)(k & 7) * 16) / 2 + (j & 7);
      for (int t = 0; t < split; ++t) {
        const uint16_t b = bf16_rn((float)r);
        img[(size_t)t * N * N + off] = b;
        r -= bf16_value(b);
      }
    }
}

}  // namespace csl
