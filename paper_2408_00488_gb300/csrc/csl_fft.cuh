// Sine transform DST-I of length n = N - 1 (N = 2^k <= 1024) on one line held
// in shared memory, computed by the TPL lanes of one warp (Section 2.3:
// W_{jk} = sqrt(2/N) sin(pi j k/N) is real, symmetric and orthogonal, so the
// unnormalised S_{jk} = sin(pi j k/N) serves forward and inverse; the factor
// 2/N per axis and pair of transforms is folded into the per-mode scale).
//
// One complex line carries both real blocks of the 2x2 system (real part =
// block 1, imaginary part = block 2); S is real, so S(x + i y) = Sx + i Sy.
//
// Algorithm: one length-N complex FFT per line.
//   y_j = s_j (z_j + z_{N-j})/2 + (z_j - z_{N-j})/4,  s_j = sin(pi j/N), z_0 = z_N = 0
//   Y = FFT_N(y)   (exp(-2 pi i jk/N))
//   C_k = Y_k + Y_{N-k},  S_k = i (Y_k - Y_{N-k})
//   (S z)_{2k}   = S_k                      k = 1 .. N/2-1
//   (S z)_{2k+1} = Y_0 + C_1 + ... + C_k    k = 0 .. N/2-1   (prefix sum)
// (2 sin a cos b = sin(a+b) - sin(b-a) applied to the cosine and sine sums of y.)
//
// The FFT is a four-step transform N = R1 * R2: lane g computes a radix-R1
// DFT over the samples j = g + R2 r held in registers, multiplies by
// w_N^{g k1} and writes them to shared memory; lanes then take radix-R2 DFTs
// over g.  Each radix-R DFT is unrolled in registers (radix-2 stages with the
// trivial twiddles 1 and -i removed at compile time).  All lanes of a line sit
// in one warp, so only __syncwarp() orders the shared-memory exchanges.
//
// The result is left in the line buffer in a padded order: element m at
// out_pos(m) (odd m in a scan layout with one pad slot per chunk, even m in a
// separate region), so that the prefix scan and the split are free of bank
// conflicts.
#pragma once
#include "csl_common.cuh"

namespace csl {

template <int N> struct DstShape;
template <> struct DstShape<4> { enum { R1 = 4, R2 = 1, TPL = 1 }; };
template <> struct DstShape<8> { enum { R1 = 8, R2 = 1, TPL = 1 }; };
template <> struct DstShape<16> { enum { R1 = 16, R2 = 1, TPL = 1 }; };
template <> struct DstShape<32> { enum { R1 = 32, R2 = 1, TPL = 1 }; };
template <> struct DstShape<64> { enum { R1 = 8, R2 = 8, TPL = 8 }; };
template <> struct DstShape<128> { enum { R1 = 16, R2 = 8, TPL = 8 }; };
template <> struct DstShape<256> { enum { R1 = 16, R2 = 16, TPL = 16 }; };
template <> struct DstShape<512> { enum { R1 = 32, R2 = 16, TPL = 16 }; };
template <> struct DstShape<1024> { enum { R1 = 32, R2 = 32, TPL = 32 }; };

// shared-memory line stride (complex elements); odd, so that column-wise tile
// loads (consecutive threads -> consecutive lines) hit distinct banks
template <int N>
__host__ __device__ constexpr int dst_line_stride() {
  return N + DstShape<N>::R2 + 1;
}

template <int N>
__device__ __forceinline__ int dst_out_pos(int m) {
  constexpr int H = N / 2, TPL = DstShape<N>::TPL, CH = H / TPL;
  constexpr int SBASE = H + TPL - 1;
  if (m & 1) {
    const int k = m >> 1;
    return k + k / CH;
  }
  return SBASE + (m >> 1) - 1;
}

template <typename T>
__device__ __forceinline__ typename C2<T>::t cmul(typename C2<T>::t a, typename C2<T>::t b) {
  return mkc<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename T>
__device__ __forceinline__ typename C2<T>::t cadd(typename C2<T>::t a, typename C2<T>::t b) {
  return mkc<T>(a.x + b.x, a.y + b.y);
}
template <typename T>
__device__ __forceinline__ typename C2<T>::t csub(typename C2<T>::t a, typename C2<T>::t b) {
  return mkc<T>(a.x - b.x, a.y - b.y);
}

template <int R>
__host__ __device__ constexpr int bit_reverse(int i) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// w_N^m for 0 <= m < N from the half table tw[m] = exp(-2 pi i m/N), m < N/2
template <typename T>
__device__ __forceinline__ typename C2<T>::t tw_full(const typename C2<T>::t* tw, int m, int H) {
  if (m < H) return tw[m];
  const typename C2<T>::t v = tw[m - H];
  return mkc<T>(-v.x, -v.y);
}

// In-register forward DFT of length R (natural order in and out).  The table
// holds w_N^m, and w_R^k = w_N^{k * TWS} with TWS = N/R.
template <typename T, int R, int TWS>
__device__ __forceinline__ void dft_reg(typename C2<T>::t (&x)[R], const typename C2<T>::t* tw) {
  typedef typename C2<T>::t c_t;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bit_reverse<R>(i);
    if (j > i) {
      const c_t t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
#pragma unroll
  for (int s = 1; s < R; s <<= 1) {
#pragma unroll
    for (int k = 0; k < s; ++k) {
      c_t w = mkc<T>((T)1, (T)0);
      if (k != 0 && 2 * k != s) w = tw[k * (R / (2 * s)) * TWS];  // w_{2s}^k
#pragma unroll
      for (int b = 0; b < R; b += 2 * s) {
        const c_t u = x[b + k], v = x[b + k + s];
        c_t t;
        if (k == 0)
          t = v;
        else if (2 * k == s)
          t = mkc<T>(v.y, -v.x);  // times -i
        else
          t = cmul<T>(w, v);
        x[b + k] = cadd<T>(u, t);
        x[b + k + s] = csub<T>(u, t);
      }
    }
  }
}

// y_j of the pre-twiddle, from the line input (natural or out_pos order)
template <typename T, int N, bool PERM_IN>
__device__ __forceinline__ typename C2<T>::t pre_twiddle(const typename C2<T>::t* a, const T* hs, int j) {
  typedef typename C2<T>::t c_t;
  if (j == 0) return mkc<T>((T)0, (T)0);
  const int jm = N - j;
  const c_t zj = a[PERM_IN ? dst_out_pos<N>(j) : j];
  const c_t zm = a[PERM_IN ? dst_out_pos<N>(jm) : jm];
  const T h = hs[j < jm ? j : jm];
  const T dx = (zj.x - zm.x) * (T)0.25, dy = (zj.y - zm.y) * (T)0.25;
  return mkc<T>(fma(h, zj.x + zm.x, dx), fma(h, zj.y + zm.y, dy));
}

// Unnormalised DST-I of one line in place: input at natural positions 1..N-1
// (or at out_pos when PERM_IN), output at out_pos.  Called by all TPL lanes of
// the line (lane index t); every lane of the warp must call it.
template <typename T, int N, bool PERM_IN>
__device__ __forceinline__ void dst_line(typename C2<T>::t* a, int t, const typename C2<T>::t* tw, const T* hs,
                                         const typename C2<T>::t* t4) {
  typedef typename C2<T>::t c_t;
  typedef DstShape<N> S;
  constexpr int R1 = S::R1, R2 = S::R2, TPL = S::TPL, H = N / 2, CH = H / TPL;
  constexpr int SBASE = H + TPL - 1;
  if (R2 == 1) {
    // whole line in one thread
    c_t x[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) x[j] = pre_twiddle<T, N, PERM_IN>(a, hs, j);
    dft_reg<T, R1, N / R1>(x, tw);
    c_t run = x[0];
    a[0] = run;  // (S z)_1
#pragma unroll
    for (int k = 1; k < H; ++k) {
      const c_t Yk = x[k], Ym = x[N - k];
      run = cadd<T>(run, cadd<T>(Yk, Ym));
      a[k] = run;                                               // (S z)_{2k+1} at k
      a[SBASE + k - 1] = mkc<T>(Ym.y - Yk.y, Yk.x - Ym.x);   // (S z)_{2k}
    }
    return;
  }
  // ---- pass 1: lane g, radix-R1 DFT over j = g + R2 r, twiddle w_N^{g k1}
  //      (read from the [k1][g] table t4 so that the lanes hit distinct banks)
  {
    const int g = t;
    c_t x[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) x[r] = pre_twiddle<T, N, PERM_IN>(a, hs, g + R2 * r);
    dft_reg<T, R1, N / R1>(x, tw);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) x[k1] = cmul<T>(x[k1], t4[k1 * R2 + g]);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[g * (R1 + 1) + k1] = x[k1];
    __syncwarp();
  }
  // ---- pass 2: lane takes k1 = t + TPL i, radix-R2 DFT over g
  {
    constexpr int NG = R1 / TPL;
    c_t x[NG][R2];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      const int k1 = t + TPL * i;
#pragma unroll
      for (int g = 0; g < R2; ++g) x[i][g] = a[g * (R1 + 1) + k1];
      dft_reg<T, R2, N / R2>(x[i], tw);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      const int k1 = t + TPL * i;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = x[i][k2];  // Y natural order
    }
    __syncwarp();
  }
  // ---- split into C_k (scan layout) and S_k
  {
    c_t cc[CH], ss[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int k = t + TPL * i;
      const c_t Yk = a[k];
      if (k == 0) {
        cc[i] = Yk;
        ss[i] = Yk;
      } else {
        const c_t Ym = a[N - k];
        cc[i] = cadd<T>(Yk, Ym);
        ss[i] = mkc<T>(Ym.y - Yk.y, Yk.x - Ym.x);
      }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int k = t + TPL * i;
      a[k + k / CH] = cc[i];
      if (k != 0) a[SBASE + k - 1] = ss[i];
    }
    __syncwarp();
  }
  // ---- prefix sum of C over k (chunk of CH per lane, segmented warp scan)
  {
    c_t* c = a + t * (CH + 1);
    c_t v[CH];
    c_t sum = mkc<T>((T)0, (T)0);
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      v[i] = c[i];
      sum = cadd<T>(sum, v[i]);
    }
    c_t inc = sum;
#pragma unroll
    for (int d = 1; d < TPL; d <<= 1) {
      const T ux = __shfl_up_sync(0xffffffffu, inc.x, d, TPL);
      const T uy = __shfl_up_sync(0xffffffffu, inc.y, d, TPL);
      if (t >= d) {
        inc.x += ux;
        inc.y += uy;
      }
    }
    c_t run = csub<T>(inc, sum);
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      run = cadd<T>(run, v[i]);
      c[i] = run;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Wide paths (N = 512, 1024): TPL = 64 or 128 lanes (two or four warps) per
// line, a three-pass Stockham autosort FFT with radices R0 x R1 x R2,
// CTA-wide barriers.  On a 2D grid there are only n lines per pass, so one
// warp per line leaves most of the GPU idle; more lanes per line cut the
// per-line latency and multiply the warps in flight.  Pass p (Ls =
// R0..R_{p-1}, radix r) takes butterfly l = j Ls + k (l < N/r; lanes beyond
// that idle in the pass), reads x[l + q N/r] (q < r), multiplies by
// w_{Ls r}^{q k} (table [q][k], conflict-free), transforms over q and writes
// x[j Ls r + k + s Ls].  Shared-memory indices are padded by one slot per 32
// (wpad) so the strided stores of the early passes spread over the banks.
// ---------------------------------------------------------------------------
template <int N> struct WideShape;
template <> struct WideShape<512> { enum { R0 = 8, R1 = 8, R2 = 8 }; };
template <> struct WideShape<1024> { enum { R0 = 8, R1 = 8, R2 = 16 }; };

// lanes per line of wide variant v (1: two warps, 2: four warps)
__host__ __device__ constexpr int wide_tpl(int v) { return v == 2 ? 128 : 64; }

__host__ __device__ constexpr int wpad(int i) { return i + (i >> 5); }

template <int N, int TPL>
__host__ __device__ constexpr int wide_line_stride() {
  return wpad(N + TPL + 2) | 1;
}

// size of the per-pass twiddle table: passes 2 and 3 ([q][k] blocks)
template <int N>
__host__ __device__ constexpr int wide_tp_size() {
  return WideShape<N>::R0 * WideShape<N>::R1 + WideShape<N>::R0 * WideShape<N>::R1 * WideShape<N>::R2;
}

template <int N, int TPL>
__device__ __forceinline__ int wide_out_pos(int m) {
  constexpr int H = N / 2, CH = H / TPL, SBASE = H + TPL - 1;
  if (m & 1) {
    const int k = m >> 1;
    return wpad(k + k / CH);
  }
  return wpad(SBASE + (m >> 1) - 1);
}

template <typename T, int N, int TPL, bool PERM_IN>
__device__ __forceinline__ typename C2<T>::t wide_pre_twiddle(const typename C2<T>::t* a, const T* hs, int j) {
  typedef typename C2<T>::t c_t;
  if (j == 0) return mkc<T>((T)0, (T)0);
  const int jm = N - j;
  const c_t zj = a[PERM_IN ? wide_out_pos<N, TPL>(j) : wpad(j)];
  const c_t zm = a[PERM_IN ? wide_out_pos<N, TPL>(jm) : wpad(jm)];
  const T h = hs[j < jm ? j : jm];
  const T dx = (zj.x - zm.x) * (T)0.25, dy = (zj.y - zm.y) * (T)0.25;
  return mkc<T>(fma(h, zj.x + zm.x, dx), fma(h, zj.y + zm.y, dy));
}

template <typename T, int N, int TPL, int R, int LSP, bool FIRST, bool PERM_IN>
__device__ __forceinline__ void wide_pass(typename C2<T>::t* a, int lane, const typename C2<T>::t* tp, const T* hs,
                                          const typename C2<T>::t* tw) {
  typedef typename C2<T>::t c_t;
  constexpr int G = N / R, PER = (G + TPL - 1) / TPL;
  constexpr bool FULL = (G % TPL) == 0;
  c_t x[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int l = lane + TPL * i;
    if (FULL || l < G) {
      const int k = l & (LSP - 1);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int idx = l + q * G;
        c_t v = FIRST ? wide_pre_twiddle<T, N, TPL, PERM_IN>(a, hs, idx) : a[wpad(idx)];
        if (!FIRST && q > 0) v = cmul<T>(v, tp[q * LSP + k]);
        x[i][q] = v;
      }
      dft_reg<T, R, N / R>(x[i], tw);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int l = lane + TPL * i;
    if (FULL || l < G) {
      const int j = l / LSP, k = l & (LSP - 1);
#pragma unroll
      for (int s = 0; s < R; ++s) a[wpad(j * LSP * R + k + s * LSP)] = x[i][s];
    }
  }
  __syncthreads();
}

// Wide-path DST-I of the lines of a CTA (line = threadIdx / TPL); every thread
// of the CTA must call it (CTA-wide barriers).  scratch: TPL/32 complex per line.
template <typename T, int N, int TPL, bool PERM_IN>
__device__ __forceinline__ void dst_line_wide(typename C2<T>::t* a, int t, const typename C2<T>::t* tw,
                                              const T* hs, const typename C2<T>::t* tp,
                                              typename C2<T>::t* scratch) {
  typedef typename C2<T>::t c_t;
  typedef WideShape<N> S;
  constexpr int R0 = S::R0, R1 = S::R1, R2 = S::R2, H = N / 2, CH = H / TPL, NW = TPL / 32;
  constexpr int SBASE = H + TPL - 1;
  wide_pass<T, N, TPL, R0, 1, true, PERM_IN>(a, t, nullptr, hs, tw);
  wide_pass<T, N, TPL, R1, R0, false, false>(a, t, tp, hs, tw);
  wide_pass<T, N, TPL, R2, R0 * R1, false, false>(a, t, tp + R0 * R1, hs, tw);
  // split into C_k (scan layout) and S_k
  c_t cc[CH], ss[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const int k = t + TPL * i;
    const c_t Yk = a[wpad(k)];
    if (k == 0) {
      cc[i] = Yk;
      ss[i] = Yk;
    } else {
      const c_t Ym = a[wpad(N - k)];
      cc[i] = cadd<T>(Yk, Ym);
      ss[i] = mkc<T>(Ym.y - Yk.y, Yk.x - Ym.x);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const int k = t + TPL * i;
    a[wpad(k + k / CH)] = cc[i];
    if (k != 0) a[wpad(SBASE + k - 1)] = ss[i];
  }
  __syncthreads();
  // prefix sum of C: chunk of CH per lane, warp scan, then across the NW warps
  c_t v[CH];
  c_t sum = mkc<T>((T)0, (T)0);
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    v[i] = a[wpad(t * (CH + 1) + i)];
    sum = cadd<T>(sum, v[i]);
  }
  c_t inc = sum;
  const int lw = t & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T ux = __shfl_up_sync(0xffffffffu, inc.x, d);
    const T uy = __shfl_up_sync(0xffffffffu, inc.y, d);
    if (lw >= d) {
      inc.x += ux;
      inc.y += uy;
    }
  }
  const int line = threadIdx.x / TPL, w = t >> 5;
  if (lw == 31) scratch[line * NW + w] = inc;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NW - 1; ++u)
    if (u < w) inc = cadd<T>(inc, scratch[line * NW + u]);
  c_t run = csub<T>(inc, sum);
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    run = cadd<T>(run, v[i]);
    a[wpad(t * (CH + 1) + i)] = run;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One interface for the paths, used by the pass kernels.  V = 0: warp per
// line; V = 1, 2: wide path with 64 or 128 lanes per line.
//   TPL       lanes per line (lines = threadIdx / TPL)
//   LS        shared-memory line stride (complex elements)
//   TP        size of the extra twiddle table (four-step [k1][g] table, or the
//             wide path's per-pass tables; 0 for single-thread lines)
//   BLOCK_SYNC whether the transform uses CTA-wide barriers
// ---------------------------------------------------------------------------
template <typename T, int N, int V = 0>
struct LineDst;

template <typename T, int N>
struct LineDst<T, N, 0> {
  typedef typename C2<T>::t c_t;
  enum { TPL = DstShape<N>::TPL, LS = dst_line_stride<N>(), BLOCK_SYNC = 0,
         TP = DstShape<N>::R2 == 1 ? 0 : N, GLOBAL_TABLES = 0 };
  static __device__ __forceinline__ int in_pos(int j) { return j; }
  static __device__ __forceinline__ int out_pos(int m) { return dst_out_pos<N>(m); }
  template <bool PERM_IN>
  static __device__ __forceinline__ void run(c_t* a, int t, const c_t* tw, const T* hs, const c_t* tp, c_t*) {
    dst_line<T, N, PERM_IN>(a, t, tw, hs, tp);
  }
  static __device__ __forceinline__ void line_sync() { __syncwarp(); }
};

template <typename T, int N, int V>
struct LineDst {
  typedef typename C2<T>::t c_t;
  enum { TPL = wide_tpl(V), LS = wide_line_stride<N, wide_tpl(V)>(), BLOCK_SYNC = 1, TP = wide_tp_size<N>(),
         GLOBAL_TABLES = 0 };
  static __device__ __forceinline__ int in_pos(int j) { return wpad(j); }
  static __device__ __forceinline__ int out_pos(int m) { return wide_out_pos<N, TPL>(m); }
  template <bool PERM_IN>
  static __device__ __forceinline__ void run(c_t* a, int t, const c_t* tw, const T* hs, const c_t* tp,
                                             c_t* scratch) {
    dst_line_wide<T, N, TPL, PERM_IN>(a, t, tw, hs, tp, scratch);
  }
  static __device__ __forceinline__ void line_sync() { __syncthreads(); }
};

// ---------------------------------------------------------------------------
// Long lines (N = 2048 .. 8192, 2D grids of the paper's large tables): one
// CTA of TPL lanes per line, an NP-pass Stockham autosort FFT (radices R0..R3)
// whose inter-pass twiddles w_{Ls r}^{q k} = w_N^{q k N/(Ls r)} come from the
// length-N table itself, so no per-pass tables exist; the line (up to 128 KB
// in FP64) fills shared memory and the tables are read from global memory
// through the cache.  Pre-twiddle, split and prefix scan as in the wide path.
// ---------------------------------------------------------------------------
template <int N> struct BigShape;
template <> struct BigShape<2048> { enum { TPL = 256, NP = 3, R0 = 8, R1 = 16, R2 = 16, R3 = 1 }; };
template <> struct BigShape<4096> { enum { TPL = 256, NP = 3, R0 = 16, R1 = 16, R2 = 16, R3 = 1 }; };
template <> struct BigShape<8192> { enum { TPL = 512, NP = 4, R0 = 8, R1 = 8, R2 = 8, R3 = 16 }; };

template <typename T, int N, int TPL, int R, int LSP, bool FIRST, bool PERM_IN>
__device__ __forceinline__ void big_pass(typename C2<T>::t* a, int lane, const T* hs, const typename C2<T>::t* tw) {
  typedef typename C2<T>::t c_t;
  constexpr int G = N / R, PER = (G + TPL - 1) / TPL, H = N / 2;
  constexpr bool FULL = (G % TPL) == 0;
  constexpr int TSTEP = N / (LSP * R);  // w_{LSP R} = w_N^{TSTEP}
  c_t x[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int l = lane + TPL * i;
    if (FULL || l < G) {
      const int k = l & (LSP - 1);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int idx = l + q * G;
        c_t v = FIRST ? wide_pre_twiddle<T, N, TPL, PERM_IN>(a, hs, idx) : a[wpad(idx)];
        if (!FIRST && q > 0) v = cmul<T>(v, tw_full<T>(tw, (q * k * TSTEP) & (N - 1), H));
        x[i][q] = v;
      }
      dft_reg<T, R, N / R>(x[i], tw);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int l = lane + TPL * i;
    if (FULL || l < G) {
      const int j = l / LSP, k = l & (LSP - 1);
#pragma unroll
      for (int s = 0; s < R; ++s) a[wpad(j * LSP * R + k + s * LSP)] = x[i][s];
    }
  }
  __syncthreads();
}

template <typename T, int N, bool PERM_IN>
__device__ __forceinline__ void dst_line_big(typename C2<T>::t* a, int t, const typename C2<T>::t* tw, const T* hs,
                                             typename C2<T>::t* scratch) {
  typedef typename C2<T>::t c_t;
  typedef BigShape<N> S;
  constexpr int TPL = S::TPL, R0 = S::R0, R1 = S::R1, R2 = S::R2, R3 = S::R3, H = N / 2, CH = H / TPL,
                NW = TPL / 32, SBASE = H + TPL - 1;
  big_pass<T, N, TPL, R0, 1, true, PERM_IN>(a, t, hs, tw);
  big_pass<T, N, TPL, R1, R0, false, false>(a, t, hs, tw);
  big_pass<T, N, TPL, R2, R0 * R1, false, false>(a, t, hs, tw);
  if constexpr (S::NP == 4) big_pass<T, N, TPL, R3, R0 * R1 * R2, false, false>(a, t, hs, tw);
  c_t cc[CH], ss[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const int k = t + TPL * i;
    const c_t Yk = a[wpad(k)];
    if (k == 0) {
      cc[i] = Yk;
      ss[i] = Yk;
    } else {
      const c_t Ym = a[wpad(N - k)];
      cc[i] = cadd<T>(Yk, Ym);
      ss[i] = mkc<T>(Ym.y - Yk.y, Yk.x - Ym.x);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const int k = t + TPL * i;
    a[wpad(k + k / CH)] = cc[i];
    if (k != 0) a[wpad(SBASE + k - 1)] = ss[i];
  }
  __syncthreads();
  // prefix sum of C in FP64 whatever T is (the odd outputs are partial sums
  // of up to N/2 terms); the inputs and outputs stay in T
  double2 v[CH];
  double2 sum = make_double2(0.0, 0.0);
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    v[i] = to_d2(a[wpad(t * (CH + 1) + i)]);
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
  double2* dscr = reinterpret_cast<double2*>(scratch);
  if (lw == 31) dscr[w] = inc;
  __syncthreads();
  for (int u = 0; u < w; ++u) {
    inc.x += dscr[u].x;
    inc.y += dscr[u].y;
  }
  double2 run = make_double2(inc.x - sum.x, inc.y - sum.y);
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    run.x += v[i].x;
    run.y += v[i].y;
    a[wpad(t * (CH + 1) + i)] = from_d2<T>(run);
  }
  __syncthreads();
}

template <typename T, int N>
struct LineDst<T, N, 3> {
  typedef typename C2<T>::t c_t;
  enum { TPL = BigShape<N>::TPL, LS = wide_line_stride<N, BigShape<N>::TPL>(), BLOCK_SYNC = 1, TP = 0,
         GLOBAL_TABLES = 1 };
  static __device__ __forceinline__ int in_pos(int j) { return wpad(j); }
  static __device__ __forceinline__ int out_pos(int m) { return wide_out_pos<N, TPL>(m); }
  template <bool PERM_IN>
  static __device__ __forceinline__ void run(c_t* a, int t, const c_t* tw, const T* hs, const c_t*, c_t* scratch) {
    dst_line_big<T, N, PERM_IN>(a, t, tw, hs, scratch);
  }
  static __device__ __forceinline__ void line_sync() { __syncthreads(); }
};

// Host-side size of the extra twiddle table of length N (matches LineDst::TP).
__host__ __device__ constexpr int line_tp_size(int N, int wide) {
  return wide ? (N >= 1024 ? wide_tp_size<1024>() : N >= 512 ? wide_tp_size<512>() : 0) : (N >= 64 ? N : 0);
}

// Copy the transform tables of length N into shared memory (block-wide).
template <typename T>
__device__ __forceinline__ void load_tables(typename C2<T>::t* s_tw, T* s_hs, typename C2<T>::t* s_tp,
                                            const typename C2<T>::t* g_tw, const T* g_hs,
                                            const typename C2<T>::t* g_tp, int N, int ntp) {
  const int H = N >> 1;
  for (int i = threadIdx.x; i < H; i += blockDim.x) s_tw[i] = g_tw[i];
  for (int i = threadIdx.x; i <= H; i += blockDim.x) s_hs[i] = g_hs[i];
  for (int i = threadIdx.x; i < ntp; i += blockDim.x) s_tp[i] = g_tp[i];
}

}  // namespace csl
