// FP64 sine transforms of lines of N = 16384 points (2D grids of n = 16383,
// the paper's largest tables) on a thread-block cluster of two CTAs.
//
// One FP64 line is 256 KB, more than one CTA's shared memory, so each CTA of
// a cluster holds half of it and reaches the other half through distributed
// shared memory (generic pointers from cluster.map_shared_rank), with cluster
// barriers between the transform's passes.  The transform is the long-line
// algorithm of csl_fft.cuh: sine pre-twiddle, a four-pass Stockham FFT
// (radices 8, 8, 16, 16) with twiddles from the length-N table, the split
// into C_k / S_k and the FP64 prefix scan of the odd outputs; 1024 lanes
// (2 x 512 threads) per line.
//
// The line is addressed as a virtual array of VIRT = N + 1026 complex
// entries (the FFT range plus the scan layout of the output): entry v lives in
// CTA v / HALF at padded offset wpad(v mod HALF).
#include <cooperative_groups.h>

#include "csl_passes.cuh"

namespace cg = cooperative_groups;

namespace csl {
namespace {

constexpr int kCN = 16384, kCH = kCN / 2;
constexpr int kCThreads = 512, kCTPL = 2 * kCThreads;
constexpr int kCVirt = kCN + kCTPL + 2;
constexpr int kCHalf = (kCVirt + 1) / 2;
constexpr int kCLocal = wpad(kCHalf) + 1;  // shared-memory entries of one CTA
constexpr int kCChunk = kCH / kCTPL;       // scan chunk per lane
constexpr int kCSBase = kCH + kCTPL - 1;
constexpr int kCNW = kCTPL / 32;           // warps of a line

struct CLine {
  double2* b[2];
  __device__ __forceinline__ double2& operator[](int v) const {
    const int r = v >= kCHalf;
    return b[r][wpad(v - r * kCHalf)];
  }
};

// output order of the transform (odd modes in the scan layout, even after it)
__device__ __forceinline__ int c_out_pos(int m) {
  if (m & 1) {
    const int k = m >> 1;
    return k + k / kCChunk;
  }
  return kCSBase + (m >> 1) - 1;
}

template <bool PERM_IN>
__device__ __forceinline__ double2 c_pre_twiddle(const CLine& L, const double* hs, int j) {
  if (j == 0) return make_double2(0.0, 0.0);
  const int jm = kCN - j;
  const double2 zj = L[PERM_IN ? c_out_pos(j) : j];
  const double2 zm = L[PERM_IN ? c_out_pos(jm) : jm];
  const double h = hs[j < jm ? j : jm];
  const double dx = (zj.x - zm.x) * 0.25, dy = (zj.y - zm.y) * 0.25;
  return make_double2(fma(h, zj.x + zm.x, dx), fma(h, zj.y + zm.y, dy));
}

template <int R, int LSP, bool FIRST, bool PERM_IN>
__device__ __forceinline__ void c_pass(const CLine& L, int t, const double* hs, const double2* tw,
                                       const cg::cluster_group& cl) {
  constexpr int G = kCN / R, PER = (G + kCTPL - 1) / kCTPL;
  constexpr bool FULL = (G % kCTPL) == 0;
  constexpr int TSTEP = kCN / (LSP * R);
  double2 x[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int l = t + kCTPL * i;
    if (FULL || l < G) {
      const int k = l & (LSP - 1);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int idx = l + q * G;
        double2 v = FIRST ? c_pre_twiddle<PERM_IN>(L, hs, idx) : L[idx];
        if (!FIRST && q > 0) v = cmul<double>(v, tw_full<double>(tw, (q * k * TSTEP) & (kCN - 1), kCH));
        x[i][q] = v;
      }
      dft_reg<double, R, kCN / R>(x[i], tw);
    }
  }
  cl.sync();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int l = t + kCTPL * i;
    if (FULL || l < G) {
      const int j = l / LSP, k = l & (LSP - 1);
#pragma unroll
      for (int s = 0; s < R; ++s) L[j * LSP * R + k + s * LSP] = x[i][s];
    }
  }
  cl.sync();
}

// unnormalised DST-I of the cluster's line: input at 1..N-1 (or at c_out_pos
// when PERM_IN), output at c_out_pos; scr0 is rank 0's scan scratch (kCNW entries)
template <bool PERM_IN>
__device__ void c_dst(const CLine& L, int t, const double2* tw, const double* hs, double2* scr0,
                      const cg::cluster_group& cl) {
  c_pass<8, 1, true, PERM_IN>(L, t, hs, tw, cl);
  c_pass<8, 8, false, false>(L, t, hs, tw, cl);
  c_pass<16, 64, false, false>(L, t, hs, tw, cl);
  c_pass<16, 1024, false, false>(L, t, hs, tw, cl);
  double2 cc[kCChunk], ss[kCChunk];
#pragma unroll
  for (int i = 0; i < kCChunk; ++i) {
    const int k = t + kCTPL * i;
    const double2 Yk = L[k];
    if (k == 0) {
      cc[i] = Yk;
      ss[i] = Yk;
    } else {
      const double2 Ym = L[kCN - k];
      cc[i] = make_double2(Yk.x + Ym.x, Yk.y + Ym.y);
      ss[i] = make_double2(Ym.y - Yk.y, Yk.x - Ym.x);
    }
  }
  cl.sync();
#pragma unroll
  for (int i = 0; i < kCChunk; ++i) {
    const int k = t + kCTPL * i;
    L[k + k / kCChunk] = cc[i];
    if (k != 0) L[kCSBase + k - 1] = ss[i];
  }
  cl.sync();
  double2 v[kCChunk];
  double2 sum = make_double2(0.0, 0.0);
#pragma unroll
  for (int i = 0; i < kCChunk; ++i) {
    v[i] = L[t * (kCChunk + 1) + i];
    sum.x += v[i].x;
    sum.y += v[i].y;
  }
  double2 inc = sum;
  const int lw = t & 31, w = t >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double ux = __shfl_up_sync(0xffffffffu, inc.x, d);
    const double uy = __shfl_up_sync(0xffffffffu, inc.y, d);
    if (lw >= d) {
      inc.x += ux;
      inc.y += uy;
    }
  }
  if (lw == 31) scr0[w] = inc;
  cl.sync();
  for (int u = 0; u < w; ++u) {
    const double2 s = scr0[u];
    inc.x += s.x;
    inc.y += s.y;
  }
  double2 run = make_double2(inc.x - sum.x, inc.y - sum.y);
#pragma unroll
  for (int i = 0; i < kCChunk; ++i) {
    run.x += v[i].x;
    run.y += v[i].y;
    L[t * (kCChunk + 1) + i] = run;
  }
  cl.sync();
}

constexpr int kCElem = kCN / kCTPL;  // line elements per lane (16)

template <int LOAD, int STORE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kCThreads, 1) k_row_cl(RowArgs<double> a) {
  cg::cluster_group cl = cg::this_cluster();
  if (a.st && a.st->done) return;  // the state is read-only here: both CTAs agree
  extern __shared__ __align__(16) unsigned char cl_smem[];
  double2* line = (double2*)cl_smem;
  double2* scr = line + kCLocal;
  CLine L;
  L.b[0] = cl.map_shared_rank(line, 0);
  L.b[1] = cl.map_shared_rank(line, 1);
  double2* scr0 = cl.map_shared_rank(scr, 0);
  const int rank = (int)cl.block_rank();
  const int t = rank * kCThreads + (int)threadIdx.x;
  const int cid = (int)blockIdx.x / 2, ncl = (int)gridDim.x / 2;
  const double lz = LOAD == LOAD_LANCZOS ? a.st->delta / a.st->gam : 0.0;
  const double zs = ((STORE == STORE_Z || STORE == STORE_Z_UPDATE) && a.st) ? (a.st->gam > 0.0 ? 1.0 / a.st->gam : 0.0)
                                                                               : 1.0;
  const double wb = STORE == STORE_Z_UPDATE ? a.st->w_b : 0.0, wc = STORE == STORE_Z_UPDATE ? a.st->w_c : 0.0;
  const double xc = STORE == STORE_Z_UPDATE ? a.st->x_coef : 0.0;
  const int n = a.n;
  cl.sync();  // both CTAs running before any access to the other's shared memory
  for (int row = cid; row < a.nrows; row += ncl) {
    const long base = (long)row * n;
#pragma unroll 4
    for (int i = 0; i < kCElem; ++i) {
      const int j = t + kCTPL * i;
      if (j < n) {
        double2 val;
        if (LOAD == LOAD_LANCZOS) {
          const double2 u = a.vnew[base + j], vc = a.vcur[base + j];
          val = make_double2(fma(-lz, vc.x, u.x), fma(-lz, vc.y, u.y));
          a.vnew[base + j] = val;
        } else {
          val = LOAD == LOAD_V ? a.vin[base + j] : a.tin[base + j];
        }
        L[j + 1] = val;
      }
    }
    cl.sync();
    c_dst<false>(L, t, a.tw, a.hs, scr0, cl);
#pragma unroll 4
    for (int i = 0; i < kCElem; ++i) {
      const int j = t + kCTPL * i;
      if (j < n) {
        const long p = base + j;
        const double2 F = L[c_out_pos(j + 1)];
        if (STORE == STORE_T) {
          a.tout[p] = F;
        } else if (STORE == STORE_D) {
          a.dout[p] = F;
        } else {
          a.zout[p] = make_double2(F.x * zs, F.y * zs);
          if (STORE == STORE_Z_UPDATE) {
            const double2 zd = a.zcur[p], wp = a.wprev[p], wq = a.wcur[p], xo = a.x[p];
            const double2 wn = make_double2(fma(wb, wp.x, fma(wc, wq.x, zd.x)), fma(wb, wp.y, fma(wc, wq.y, zd.y)));
            a.wprev[p] = wn;
            a.x[p] = make_double2(fma(xc, wn.x, xo.x), fma(xc, wn.y, xo.y));
          }
        }
      }
    }
    cl.sync();
  }
}

template <bool MID>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kCThreads, 1) k_strided_cl(StridedArgs<double> a) {
  cg::cluster_group cl = cg::this_cluster();
  if (a.st && a.st->done) return;
  if (MID && a.scalar_mode == 2 && blockIdx.x == 0 && threadIdx.x == 0) a.st->entries += 1;  // read by the next stencil pass
  extern __shared__ __align__(16) unsigned char cl_smem[];
  double2* line = (double2*)cl_smem;
  double2* scr = line + kCLocal;
  CLine L;
  L.b[0] = cl.map_shared_rank(line, 0);
  L.b[1] = cl.map_shared_rank(line, 1);
  double2* scr0 = cl.map_shared_rank(scr, 0);
  const int rank = (int)cl.block_rank();
  const int t = rank * kCThreads + (int)threadIdx.x;
  const int cid = (int)blockIdx.x / 2, ncl = (int)gridDim.x / 2;
  const int n = a.n;
  const long ncolumns = (long)a.ncols * a.nouter;
  double g2acc = 0.0;
  cl.sync();
  for (long col = cid; col < ncolumns; col += ncl) {
    const int o = (int)(col / a.ncols);
    const int c = (int)(col - (long)o * a.ncols);
    const long base = (long)o * a.outer_stride + c;
#pragma unroll 4
    for (int i = 0; i < kCElem; ++i) {
      const int j = t + kCTPL * i;
      if (j < n) L[j + 1] = a.data[base + (long)j * a.line_stride];
    }
    cl.sync();
    c_dst<false>(L, t, a.tw, a.hs, scr0, cl);
    if (MID) {
      double part = 0.0;
      for (int m = 1 + t; m <= n; m += kCTPL) {
        double2 F = L[c_out_pos(m)];
        const double sc = a.stab[base + (long)(m - 1) * a.line_stride];
        part = fma(sc, fma(F.x, F.x, F.y * F.y), part);
        F.x *= sc;
        F.y *= sc;
        L[c_out_pos(m)] = F;
      }
      g2acc += part;
      cl.sync();
      c_dst<true>(L, t, a.tw, a.hs, scr0, cl);
    }
#pragma unroll 4
    for (int i = 0; i < kCElem; ++i) {
      const int j = t + kCTPL * i;
      if (j < n) a.data[base + (long)j * a.line_stride] = L[c_out_pos(j + 1)];
    }
    cl.sync();
  }
  if (MID && a.scalar_mode != 0) mid_scalar_tail<double>(a, g2acc, (int)blockIdx.x, (int)gridDim.x);
}

constexpr size_t kCSmem = (size_t)(kCLocal + kCNW) * sizeof(double2);

}  // namespace

size_t cluster_pass_smem() { return kCSmem; }
int cluster_pass_threads() { return kCThreads; }

cudaError_t launch_row_cl(int load, int store, const RowArgs<double>& a, const PassLaunch& L, cudaStream_t s) {
  const int grid = L.blocks;  // a multiple of 2 (one cluster per line in flight)
  if (load == LOAD_V && store == STORE_T)
    k_row_cl<LOAD_V, STORE_T><<<grid, kCThreads, kCSmem, s>>>(a);
  else if (load == LOAD_LANCZOS && store == STORE_T)
    k_row_cl<LOAD_LANCZOS, STORE_T><<<grid, kCThreads, kCSmem, s>>>(a);
  else if (load == LOAD_T && store == STORE_Z)
    k_row_cl<LOAD_T, STORE_Z><<<grid, kCThreads, kCSmem, s>>>(a);
  else if (load == LOAD_T && store == STORE_Z_UPDATE)
    k_row_cl<LOAD_T, STORE_Z_UPDATE><<<grid, kCThreads, kCSmem, s>>>(a);
  else if (load == LOAD_T && store == STORE_D)
    k_row_cl<LOAD_T, STORE_D><<<grid, kCThreads, kCSmem, s>>>(a);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_strided_cl(bool mid, const StridedArgs<double>& a, const PassLaunch& L, cudaStream_t s) {
  if (mid)
    k_strided_cl<true><<<L.blocks, kCThreads, kCSmem, s>>>(a);
  else
    k_strided_cl<false><<<L.blocks, kCThreads, kCSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t set_cluster_attrs() {
  cudaError_t e = cudaSuccess;
#define SETA(k) \
  if (e == cudaSuccess) e = allow_dyn_smem((const void*)k);
  SETA((k_row_cl<LOAD_V, STORE_T>))
  SETA((k_row_cl<LOAD_LANCZOS, STORE_T>))
  SETA((k_row_cl<LOAD_T, STORE_Z>))
  SETA((k_row_cl<LOAD_T, STORE_Z_UPDATE>))
  SETA((k_row_cl<LOAD_T, STORE_D>))
  SETA((k_strided_cl<true>))
  SETA((k_strided_cl<false>))
#undef SETA
  return e;
}

}  // namespace csl
