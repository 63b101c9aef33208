// Launch wrappers of the sine-transform passes for one real type CSL_T
// (instantiated by csl_pass64.cu and csl_pass32.cu so that the two
// precisions compile in parallel).
#pragma once
#include "csl_passes.cuh"

namespace csl {

template <typename T, int N, int W>
cudaError_t launch_row_n(int load, int store, const RowArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                         const RowArgs<T>* batch, int nsys) {
  const int grid = batch ? L.blocks * nsys : L.blocks;
  const int bps = L.blocks;
  if constexpr (sizeof(T) == 4) {  // FP32 transform, FP64 vectors
    if (load == LOAD_LANCZOS_V64 && store == STORE_T)
      return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_LANCZOS_V64, STORE_T>, grid, L.threads, L.smem, s, a, batch,
                      bps);
    if (load == LOAD_T && store == STORE_Z_UPDATE_V64)
      return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_T, STORE_Z_UPDATE_V64>, grid, L.threads, L.smem, s, a, batch,
                      bps);
  } else {  // the FP64 form's vectors are FP64 in the plain modes
    if (load == LOAD_LANCZOS_V64) load = LOAD_LANCZOS;
    if (store == STORE_Z_UPDATE_V64) store = STORE_Z_UPDATE;
  }
  if (load == LOAD_V && store == STORE_T)
    return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_V, STORE_T>, grid, L.threads, L.smem, s, a, batch, bps);
  else if (load == LOAD_LANCZOS && store == STORE_T)
    return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_LANCZOS, STORE_T>, grid, L.threads, L.smem, s, a, batch, bps);
  else if (load == LOAD_T && store == STORE_Z)
    return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_T, STORE_Z>, grid, L.threads, L.smem, s, a, batch, bps);
  else if (load == LOAD_T && store == STORE_Z_UPDATE)
    return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_T, STORE_Z_UPDATE>, grid, L.threads, L.smem, s, a, batch, bps);
  else if (load == LOAD_T && store == STORE_D)
    return launch_k(L.pdl != 0, k_row<T, N, W, LOAD_T, STORE_D>, grid, L.threads, L.smem, s, a, batch, bps);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_row(int N, int wide, int load, int store, const RowArgs<T>& a, const PassLaunch& L,
                       cudaStream_t s, const RowArgs<T>* batch, int nsys) {
  if (pass_is_big(N)) return launch_row_big<T>(N, load, store, a, L, s, batch, nsys);
  switch (N) {
#define CASE(NN)                                                                    \
  case NN:                                                                          \
    if constexpr (NN >= 512) {                                                      \
      if (wide == 1) return launch_row_n<T, NN, 1>(load, store, a, L, s, batch, nsys); \
      if (wide == 2) return launch_row_n<T, NN, 2>(load, store, a, L, s, batch, nsys); \
    }                                                                               \
    return launch_row_n<T, NN, 0>(load, store, a, L, s, batch, nsys);
    CSL_FOR_EACH_N(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T, int N, int W>
cudaError_t launch_strided_n(bool mid, const StridedArgs<T>& a, const PassLaunch& L, cudaStream_t s,
                             const StridedArgs<T>* batch, int nsys) {
  const int grid = batch ? L.blocks * nsys : L.blocks;
  if (mid) return launch_k(L.pdl != 0, k_strided<T, N, W, true>, grid, L.threads, L.smem, s, a, batch, L.blocks);
  return launch_k(L.pdl != 0, k_strided<T, N, W, false>, grid, L.threads, L.smem, s, a, batch, L.blocks);
}

template <typename T>
cudaError_t launch_strided(int N, int wide, bool mid, const StridedArgs<T>& a, const PassLaunch& L,
                           cudaStream_t s, const StridedArgs<T>* batch, int nsys) {
  if constexpr (sizeof(T) == 4) {
    if (L.tc) return launch_strided_tc(N, L.tc, mid, a, L, s, batch, nsys);
  }
  if (pass_is_big(N)) return launch_strided_big<T>(N, mid, a, L, s, batch, nsys);
  switch (N) {
#define CASE(NN)                                                                  \
  case NN:                                                                        \
    if constexpr (NN >= 512) {                                                    \
      if (wide == 1) return launch_strided_n<T, NN, 1>(mid, a, L, s, batch, nsys); \
      if (wide == 2) return launch_strided_n<T, NN, 2>(mid, a, L, s, batch, nsys); \
    }                                                                             \
    return launch_strided_n<T, NN, 0>(mid, a, L, s, batch, nsys);
    CSL_FOR_EACH_N(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t set_pass_attrs() {
  cudaError_t e = cudaSuccess;
#define SETA(k) \
  if (e == cudaSuccess) e = allow_dyn_smem((const void*)k);
#define VARIANT(NN, W)                                 \
  SETA((k_row<T, NN, W, LOAD_V, STORE_T>))             \
  SETA((k_row<T, NN, W, LOAD_LANCZOS, STORE_T>))       \
  SETA((k_row<T, NN, W, LOAD_T, STORE_Z>))             \
  SETA((k_row<T, NN, W, LOAD_T, STORE_Z_UPDATE>))      \
  SETA((k_row<T, NN, W, LOAD_T, STORE_D>))             \
  SETA((k_strided<T, NN, W, true>))                    \
  SETA((k_strided<T, NN, W, false>))                   \
  if constexpr (sizeof(T) == 4) {                      \
    SETA((k_row<T, NN, W, LOAD_LANCZOS_V64, STORE_T>)) \
    SETA((k_row<T, NN, W, LOAD_T, STORE_Z_UPDATE_V64>)) \
  }
#define CASE(NN) VARIANT(NN, 0)
  CSL_FOR_EACH_N(CASE)
#undef CASE
  VARIANT(512, 1)
  VARIANT(1024, 1)
  VARIANT(512, 2)
  VARIANT(1024, 2)
#undef VARIANT
#undef SETA
  if (e == cudaSuccess) e = set_pass_attrs_big<T>();
  return e;
}

template cudaError_t launch_row<CSL_T>(int, int, int, int, const RowArgs<CSL_T>&, const PassLaunch&,
                                       cudaStream_t, const RowArgs<CSL_T>*, int);
template cudaError_t launch_strided<CSL_T>(int, int, bool, const StridedArgs<CSL_T>&, const PassLaunch&,
                                           cudaStream_t, const StridedArgs<CSL_T>*, int);
template cudaError_t set_pass_attrs<CSL_T>();

}  // namespace csl
