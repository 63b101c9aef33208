// csl_probe.cu -- measurement hook (declared in include/csl_testing.h): what
// one synchronisation point between two dependent stages of a MINRES
// iteration costs on this GPU, in the two forms a device-resident solver can
// take.
//
//  * a kernel boundary: `kernels` kernels without work, captured in a CUDA
//    graph, each launched with programmatic dependent launch (the form the
//    solver's graph uses) and without it; every kernel has the grid of a
//    transform pass (2 CTAs per SM, 256 threads, 48 KB of dynamic shared
//    memory), waits for its predecessor (griddepcontrol.wait) and triggers
//    its dependents;
//  * a grid barrier inside one persistent kernel: a cooperative launch of
//    (resident CTAs per SM, at most 2) x SMs CTAs crossing `barriers`
//    barriers; each barrier is an arrival counter in global memory and a
//    spin of thread 0 of every CTA until the counter reaches the barrier's
//    target.
//
// The spin is bounded by a clock64 budget.  When it runs out, the CTA records
// the time-out in a flag and returns; nothing else is in flight in this
// kernel (no asynchronous copies, no tensor memory), so returning early is
// safe, and the host reads the flag and returns CSL_TIMEOUT.  With
// `unreachable` set, every barrier target is one arrival above what the grid
// provides, so every wait runs out after a short budget (about 1 ms): the
// bounded-wait path, exercised without any fault.
#include <cuda_runtime.h>
#include <stdio.h>

#include "../../include/csl_testing.h"
#include "csl_common.cuh"

void csl_internal_set_error(const char* msg);  // csl_api.cu

namespace {

constexpr int kProbeThreads = 256;
constexpr size_t kProbeSmem = 48 * 1024;

__global__ void __launch_bounds__(kProbeThreads) k_probe_stage(int* sink, int k) {
  extern __shared__ int probe_smem[];
  csl::pdl_wait();
  if (threadIdx.x == 0) probe_smem[0] = k;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) sink[0] = probe_smem[0];
  csl::pdl_trigger();
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_barriers(unsigned* counter, int nbar, unsigned extra,
                                                                 long long budget, int* timed_out) {
  __shared__ int give_up;
  if (threadIdx.x == 0) give_up = 0;
  __syncthreads();
  for (int b = 1; b <= nbar; ++b) {
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(counter, 1u);
      const unsigned target = (unsigned)b * gridDim.x + extra;
      const long long t0 = clock64();
      while (*((volatile unsigned*)counter) < target) {
        if (clock64() - t0 > budget) {
          give_up = 1;
          atomicExch(timed_out, 1);
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    if (give_up) return;
  }
}

struct ProbeRes {
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  int* dbuf = nullptr;  // [0] sink, [1] counter, [2] time-out flag
  ~ProbeRes() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dbuf) cudaFree(dbuf);
    if (s) cudaStreamDestroy(s);
  }
};

csl_status probe_fail(cudaError_t e, const char* what) {
  char msg[256];
  snprintf(msg, sizeof(msg), "csl_probe_sync_cost: %s: %s", what, cudaGetErrorString(e));
  csl_internal_set_error(msg);
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? CSL_OUT_OF_MEMORY : CSL_CUDA_ERROR;
}

#define PROBE_TRY(call)                                \
  do {                                                 \
    const cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return probe_fail(e_, #call); \
  } while (0)

// microseconds per kernel of a graph of `kernels` stage kernels
csl_status time_graph(ProbeRes& R, int kernels, bool pdl, int grid, double* us) {
  PROBE_TRY(cudaStreamBeginCapture(R.s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kernels && e == cudaSuccess; ++k)
    e = csl::launch_k(pdl, k_probe_stage, dim3(grid), dim3(kProbeThreads), kProbeSmem, R.s, R.dbuf, k);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(R.s, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return probe_fail(e, "stage kernel launch");
  }
  PROBE_TRY(e2);
  R.g = g;
  PROBE_TRY(cudaGraphInstantiate(&R.ge, R.g, 0));
  PROBE_TRY(cudaGraphLaunch(R.ge, R.s));  // warm-up
  PROBE_TRY(cudaEventRecord(R.e0, R.s));
  PROBE_TRY(cudaGraphLaunch(R.ge, R.s));
  PROBE_TRY(cudaEventRecord(R.e1, R.s));
  PROBE_TRY(cudaEventSynchronize(R.e1));
  float ms = 0.f;
  PROBE_TRY(cudaEventElapsedTime(&ms, R.e0, R.e1));
  *us = 1e3 * ms / kernels;
  PROBE_TRY(cudaGraphExecDestroy(R.ge));
  R.ge = nullptr;
  PROBE_TRY(cudaGraphDestroy(R.g));
  R.g = nullptr;
  return CSL_OK;
}

}  // namespace

extern "C" csl_status csl_probe_sync_cost(int kernels, int barriers, int unreachable, double out[3]) {
  if (!out || kernels < 1 || kernels > 100000 || barriers < 1 || barriers > 1000000) return CSL_INVALID_ARG;
  out[0] = out[1] = out[2] = 0.0;
  int dev = 0, sms = 0, clock_khz = 0, per_sm = 0, coop = 0;
  PROBE_TRY(cudaGetDevice(&dev));
  PROBE_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PROBE_TRY(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
  PROBE_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    csl_internal_set_error("csl_probe_sync_cost: the device has no cooperative launch");
    return CSL_UNSUPPORTED_SIZE;
  }
  ProbeRes R;
  PROBE_TRY(cudaStreamCreateWithFlags(&R.s, cudaStreamNonBlocking));
  PROBE_TRY(cudaEventCreate(&R.e0));
  PROBE_TRY(cudaEventCreate(&R.e1));
  PROBE_TRY(cudaMalloc(&R.dbuf, 4 * sizeof(int)));
  PROBE_TRY(cudaMemsetAsync(R.dbuf, 0, 4 * sizeof(int), R.s));

  const int grid_stage = 2 * sms;
  csl_status st = time_graph(R, kernels, true, grid_stage, &out[0]);
  if (st == CSL_OK) st = time_graph(R, kernels, false, grid_stage, &out[1]);
  if (st != CSL_OK) return st;

  PROBE_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_barriers, kProbeThreads, 0));
  if (per_sm < 1) {
    csl_internal_set_error("csl_probe_sync_cost: the barrier kernel does not fit on an SM");
    return CSL_UNSUPPORTED_SIZE;
  }
  const int grid_bar = (per_sm < 2 ? per_sm : 2) * sms;
  // about one second per wait (a safety net), or about 1 ms when the waits
  // are meant to run out
  const long long cycles_per_ms = (long long)(clock_khz > 0 ? clock_khz : 2000000);
  long long budget = unreachable ? cycles_per_ms : 1000 * cycles_per_ms;
  unsigned extra = unreachable ? 1u : 0u;
  unsigned* counter = (unsigned*)(R.dbuf + 1);
  int* timed_out = R.dbuf + 2;
  int nbar = barriers;
  void* args[] = {&counter, &nbar, &extra, &budget, &timed_out};
  PROBE_TRY(cudaEventRecord(R.e0, R.s));
  PROBE_TRY(cudaLaunchCooperativeKernel((const void*)k_probe_barriers, dim3(grid_bar), dim3(kProbeThreads), args, 0,
                                        R.s));
  PROBE_TRY(cudaEventRecord(R.e1, R.s));
  PROBE_TRY(cudaEventSynchronize(R.e1));
  float ms = 0.f;
  PROBE_TRY(cudaEventElapsedTime(&ms, R.e0, R.e1));
  int flag = 0;
  PROBE_TRY(cudaMemcpy(&flag, timed_out, sizeof(int), cudaMemcpyDeviceToHost));
  out[2] = 1e3 * ms / barriers;
  if (flag) {
    csl_internal_set_error("csl_probe_sync_cost: a grid-barrier wait ran out of its budget");
    return CSL_TIMEOUT;
  }
  return CSL_OK;
}
