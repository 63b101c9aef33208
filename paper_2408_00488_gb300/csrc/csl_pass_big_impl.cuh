// Launch wrappers of the long-line sine-transform passes (N = 2048 .. 8192,
// variant 3: one CTA of 256 or 512 lanes per line) for one real type CSL_T,
// instantiated by csl_pass32_big.cu and csl_pass64_big.cu so that they compile
// in parallel with the other passes.
#pragma once
#include "csl_passes.cuh"

namespace csl {

template <typename T, int N>
cudaError_t launch_row_big_n(int load, int store, const RowArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                             const RowArgs<T>* batch, int nsys) {
  const int grid = batch ? L.blocks * nsys : L.blocks;
  const int bps = L.blocks;
  if constexpr (sizeof(T) == 8) {  // the FP64 form's vectors are FP64 in the plain modes
    if (load == LOAD_LANCZOS_V64) load = LOAD_LANCZOS;
    if (store == STORE_Z_UPDATE_V64) store = STORE_Z_UPDATE;
  }
  if constexpr (sizeof(T) == 4) {  // FP32 transform, FP64 vectors
    if (load == LOAD_LANCZOS_V64 && store == STORE_T) {
      k_row<T, N, 3, LOAD_LANCZOS_V64, STORE_T><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
      return cudaGetLastError();
    }
    if (load == LOAD_T && store == STORE_Z_UPDATE_V64) {
      k_row<T, N, 3, LOAD_T, STORE_Z_UPDATE_V64><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
      return cudaGetLastError();
    }
  }
  if (load == LOAD_V && store == STORE_T)
    k_row<T, N, 3, LOAD_V, STORE_T><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
  else if (load == LOAD_LANCZOS && store == STORE_T)
    k_row<T, N, 3, LOAD_LANCZOS, STORE_T><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
  else if (load == LOAD_T && store == STORE_Z)
    k_row<T, N, 3, LOAD_T, STORE_Z><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
  else if (load == LOAD_T && store == STORE_Z_UPDATE)
    k_row<T, N, 3, LOAD_T, STORE_Z_UPDATE><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
  else if (load == LOAD_T && store == STORE_D)
    k_row<T, N, 3, LOAD_T, STORE_D><<<grid, L.threads, L.smem, s>>>(a, batch, bps);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_big(int N, int load, int store, const RowArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                           const RowArgs<T>* batch, int nsys) {
  if (N == 16384) {  // FP64 only, single systems: two-CTA cluster per line
    if constexpr (sizeof(T) == 8) {
      // the FP64 form's vectors are FP64 in the plain modes
      if (load == LOAD_LANCZOS_V64) load = LOAD_LANCZOS;
      if (store == STORE_Z_UPDATE_V64) store = STORE_Z_UPDATE;
      if (!batch) return launch_row_cl(load, store, a, L, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (N) {
#define CASE(NN) \
  case NN: return launch_row_big_n<T, NN>(load, store, a, L, s, batch, nsys);
    CSL_FOR_EACH_BIG_N(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_strided_big(int N, bool mid, const StridedArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                               const StridedArgs<T>* batch, int nsys) {
  if (N == 16384) {
    if constexpr (sizeof(T) == 8) {
      if (!batch) return launch_strided_cl(mid, a, L, s);
    }
    return cudaErrorInvalidValue;
  }
  const int grid = batch ? L.blocks * nsys : L.blocks;
  switch (N) {
#define CASE(NN)                                                                              \
  case NN:                                                                                    \
    if (mid)                                                                                  \
      k_strided<T, NN, 3, true><<<grid, L.threads, L.smem, s>>>(a, batch, L.blocks);          \
    else                                                                                      \
      k_strided<T, NN, 3, false><<<grid, L.threads, L.smem, s>>>(a, batch, L.blocks);         \
    return cudaGetLastError();
    CSL_FOR_EACH_BIG_N(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t set_pass_attrs_big() {
  cudaError_t e = cudaSuccess;
#define SETA(k) \
  if (e == cudaSuccess) e = allow_dyn_smem((const void*)k);
#define CASE(NN)                                  \
  SETA((k_row<T, NN, 3, LOAD_V, STORE_T>))        \
  SETA((k_row<T, NN, 3, LOAD_LANCZOS, STORE_T>))  \
  SETA((k_row<T, NN, 3, LOAD_T, STORE_Z>))        \
  SETA((k_row<T, NN, 3, LOAD_T, STORE_Z_UPDATE>)) \
  SETA((k_row<T, NN, 3, LOAD_T, STORE_D>))        \
  SETA((k_strided<T, NN, 3, true>))               \
  SETA((k_strided<T, NN, 3, false>))             \
  if constexpr (sizeof(T) == 4) {                 \
    SETA((k_row<T, NN, 3, LOAD_LANCZOS_V64, STORE_T>)) \
    SETA((k_row<T, NN, 3, LOAD_T, STORE_Z_UPDATE_V64>)) \
  }
  CSL_FOR_EACH_BIG_N(CASE)
#undef CASE
#undef SETA
  if constexpr (sizeof(T) == 8) {
    if (e == cudaSuccess) e = set_cluster_attrs();
  }
  return e;
}

template cudaError_t launch_row_big<CSL_T>(int, int, int, const RowArgs<CSL_T>&, const PassLaunch&, cudaStream_t,
                                           const RowArgs<CSL_T>*, int);
template cudaError_t launch_strided_big<CSL_T>(int, bool, const StridedArgs<CSL_T>&, const PassLaunch&, cudaStream_t,
                                               const StridedArgs<CSL_T>*, int);
template cudaError_t set_pass_attrs_big<CSL_T>();

}  // namespace csl
