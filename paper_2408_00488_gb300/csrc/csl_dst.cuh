// Sine transform DST-I of length n = N - 1 (N = 2^logn) on lines held in
// shared memory (Section 2.3: W_{jk} = sqrt(2/N) sin(pi j k / N) is real,
// symmetric and orthogonal, so the same unnormalised transform
// S_{jk} = sin(pi j k / N) serves forward and inverse; the factor 2/N per axis
// and pair of transforms is folded into the per-mode scale).
//
// One complex line carries the two real blocks of the 2x2 system (real part =
// block 1, imaginary part = block 2); S is real, so S(x + i y) = Sx + i Sy.
//
// Algorithm (one length-N complex FFT per line instead of the length-2N FFT of
// the odd extension):
//   y_j     = s_j (z_j + z_{N-j})/2 + (z_j - z_{N-j})/4,  s_j = sin(pi j / N),
//   y_{N-j} = s_j (z_j + z_{N-j})/2 - (z_j - z_{N-j})/4,  (z_0 = z_N = 0)
//   Y = FFT_N(y)   (exp(-2 pi i jk/N), radix-2^2 DIT on bit-reversed input)
//   C_k = Y_k + Y_{N-k},  S_k = i (Y_k - Y_{N-k}),
//   (S z)_{2k}   = S_k                     (k = 1 .. N/2-1)
//   (S z)_{2k+1} = Y_0 + C_1 + ... + C_k   (k = 0 .. N/2-1, prefix sum)
// which follows from 2 sin(a) cos(b) = sin(a+b) - sin(b-a) applied to the
// cosine and sine sums of y.  The output is left in place in a permuted order:
// element m at out_pos(m) = (m-1)/2 for odd m, N - m/2 for even m.
#pragma once
#include "csl_common.cuh"

namespace csl {

__device__ __forceinline__ int dst_out_pos(int m, int N) {
  return (m & 1) ? (m >> 1) : (N - (m >> 1));
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

// Exclusive prefix sum of one complex value per thread over the TL threads
// that own one line (TL a power of two <= 1024, TL threads contiguous in the
// block).  scratch: 32 complex per line.  Must be called by all threads.
template <typename T>
__device__ typename C2<T>::t line_exclusive_scan(typename C2<T>::t v, int l, int t, int TL,
                                                 typename C2<T>::t* scratch) {
  typedef typename C2<T>::t c_t;
  const int W = TL < 32 ? TL : 32;
  c_t inc = v;
  for (int d = 1; d < W; d <<= 1) {
    T ux = __shfl_up_sync(0xffffffffu, inc.x, d, W);
    T uy = __shfl_up_sync(0xffffffffu, inc.y, d, W);
    if ((t & (W - 1)) >= d) {
      inc.x += ux;
      inc.y += uy;
    }
  }
  if (TL > 32) {
    // combine the warp totals of this line (TL/32 <= 32 of them)
    const int w = t >> 5;
    if ((t & 31) == 31) scratch[l * 32 + w] = inc;
    __syncthreads();
    c_t add = mkc<T>((T)0, (T)0);
    for (int k = 0; k < w; ++k) add = cadd<T>(add, scratch[l * 32 + k]);
    inc = cadd<T>(inc, add);
    __syncthreads();
  }
  return csub<T>(inc, v);
}

// Unnormalised DST-I of G lines, in place in A (B is FFT workspace).
// Line l lives at A + l*LS (LS >= N).  Input element j (1..N-1) is read from
// A[j] (natural order) or A[dst_out_pos(j)] (PERM_IN, i.e. the output of a
// previous dst_lines call); the output is left in permuted order.
// Threads: line l = threadIdx / TL, lane t = threadIdx % TL; threads with
// l >= G only take part in the barriers.  All threads must call it.
template <typename T, bool PERM_IN>
__device__ void dst_lines(typename C2<T>::t* A, typename C2<T>::t* B, int LS, int G, int TL,
                          int logn, const typename C2<T>::t* tw, const T* hs,
                          typename C2<T>::t* scratch) {
  typedef typename C2<T>::t c_t;
  const int N = 1 << logn, H = N >> 1;
  const int l = threadIdx.x / TL, t = threadIdx.x - (threadIdx.x / TL) * TL;
  const bool act = l < G;
  c_t* a = A + (size_t)l * LS;
  c_t* b = B + (size_t)l * LS;
  const int sh = 32 - logn;
  const T q = (T)0.25;
  // 1. pre-twiddle into bit-reversed order
  if (act) {
    for (int j = t; j <= H; j += TL) {
      c_t zj, zm;
      if (j == 0) {
        zj = mkc<T>((T)0, (T)0);
        zm = zj;
      } else {
        zj = a[PERM_IN ? dst_out_pos(j, N) : j];
        zm = (j == H) ? zj : a[PERM_IN ? dst_out_pos(N - j, N) : (N - j)];
      }
      const T h = hs[j];
      const T sx = zj.x + zm.x, sy = zj.y + zm.y;
      const T dx = (zj.x - zm.x) * q, dy = (zj.y - zm.y) * q;
      b[__brev((unsigned)j) >> sh] = mkc<T>(fma(h, sx, dx), fma(h, sy, dy));
      if (j != 0 && j != H) b[__brev((unsigned)(N - j)) >> sh] = mkc<T>(fma(h, sx, -dx), fma(h, sy, -dy));
    }
  }
  __syncthreads();
  // 2. FFT: radix-2 first stage if logn is odd, then radix-2^2 pairs of stages
  int s = 0;
  if (logn & 1) {
    if (act) {
      for (int g = t; g < H; g += TL) {
        c_t x0 = b[2 * g], x1 = b[2 * g + 1];
        b[2 * g] = cadd<T>(x0, x1);
        b[2 * g + 1] = csub<T>(x0, x1);
      }
    }
    __syncthreads();
    s = 1;
  }
  for (; s < logn; s += 2) {
    const int h = 1 << s;
    if (act) {
      for (int g = t; g < (N >> 2); g += TL) {
        const int r = g & (h - 1);
        const int i0 = ((g >> s) << (s + 2)) + r;
        c_t x0 = b[i0], x1 = b[i0 + h], x2 = b[i0 + 2 * h], x3 = b[i0 + 3 * h];
        const c_t W = tw[r << (logn - s - 1)];
        const c_t V = tw[r << (logn - s - 2)];
        const c_t t1 = cmul<T>(W, x1), t3 = cmul<T>(W, x3);
        const c_t a0 = cadd<T>(x0, t1), a1 = csub<T>(x0, t1);
        const c_t a2 = cadd<T>(x2, t3), a3 = csub<T>(x2, t3);
        const c_t u2 = cmul<T>(V, a2);
        c_t u3 = cmul<T>(V, a3);
        u3 = mkc<T>(u3.y, -u3.x);  // times -i = w_{4h}^h
        b[i0] = cadd<T>(a0, u2);
        b[i0 + 2 * h] = csub<T>(a0, u2);
        b[i0 + h] = cadd<T>(a1, u3);
        b[i0 + 3 * h] = csub<T>(a1, u3);
      }
    }
    __syncthreads();
  }
  // 3. split into cosine sums C_k (at k) and sine sums S_k (at N-k)
  if (act) {
    for (int k = t; k < H; k += TL) {
      if (k == 0) {
        a[0] = b[0];
      } else {
        const c_t Yk = b[k], Ym = b[N - k];
        a[k] = cadd<T>(Yk, Ym);
        a[N - k] = mkc<T>(Ym.y - Yk.y, Yk.x - Ym.x);
      }
    }
  }
  __syncthreads();
  // 4. odd outputs: inclusive prefix sum over positions 0..H-1
  const int CH = (H + TL - 1) / TL;
  const int k0 = t * CH, k1 = min(k0 + CH, H);
  c_t sum = mkc<T>((T)0, (T)0);
  if (act)
    for (int k = k0; k < k1; ++k) sum = cadd<T>(sum, a[k]);
  c_t run = line_exclusive_scan<T>(sum, l, t, TL, scratch);
  if (act) {
    for (int k = k0; k < k1; ++k) {
      run = cadd<T>(run, a[k]);
      a[k] = run;
    }
  }
  __syncthreads();
}

// Copy the transform tables of length N into shared memory.
template <typename T>
__device__ __forceinline__ void load_tables(typename C2<T>::t* s_tw, T* s_hs,
                                            const typename C2<T>::t* g_tw, const T* g_hs, int logn) {
  const int H = 1 << (logn - 1);
  for (int i = threadIdx.x; i < H; i += blockDim.x) s_tw[i] = g_tw[i];
  for (int i = threadIdx.x; i <= H; i += blockDim.x) s_hs[i] = g_hs[i];
}

}  // namespace csl
