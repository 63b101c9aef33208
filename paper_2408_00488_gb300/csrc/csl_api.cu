// Host side of the C ABI declared in include/csl.h: plan set-up (Eq. 4 and
// the Section 2.3 tables), launch configurations, the MINRES driver (a CUDA
// graph whose WHILE node is closed from the device once the true residual
// meets the tolerance), and the remaining entry points.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/csl.h"
#include "../../include/csl_testing.h"
#include "csl_kernels.cuh"
#include "csl_passes.cuh"

using namespace csl;

namespace {
thread_local char g_last_error[512] = "";

// NVTX range for the life of a scope (named per entry point and phase, so
// that a profiler can select a solve, its prologue or its loop)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
void record_error(cudaError_t e, const char* what, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s failed at csl_api.cu:%d: %s (%s)", what, line,
           cudaGetErrorName(e), cudaGetErrorString(e));
}
}  // namespace

#define CSL_TRY(call)                                                               \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      record_error(e_, #call, __LINE__);                                            \
      (void)cudaGetLastError();                                                     \
      return e_ == cudaErrorMemoryAllocation ? CSL_OUT_OF_MEMORY : CSL_CUDA_ERROR; \
    }                                                                               \
  } while (0)
#define CSL_NOTE(e, what)                                        \
  do {                                                           \
    if ((e) != cudaSuccess) record_error((e), (what), __LINE__); \
  } while (0)

namespace {

const int kSMs = 152;
const int kMaxRedBlocks = 4096;
const double kNaN = __builtin_nan("");

// one sine-transform pass: line length N = n + 1, CTA shape and grid
struct PassCfg {
  int N = 0, n = 0, lines = 0;  // lines per CTA
  int wide = 0;                  // N = 512, 1024: 0 warp per line, 1 / 2 Stockham with 64 / 128 lanes per line
  int ncols = 0, nouter = 0;     // strided: x extent and outer blocks; row: nouter = rows
  long outer_stride = 0, line_stride = 0;
  PassLaunch L = {1, 32, 0};
};

int ilog2_exact(long v) {
  if (v <= 0 || (v & (v - 1))) return -1;
  int l = 0;
  while ((1L << l) < v) ++l;
  return l;
}

// exp(-2 pi i num/den) as interleaved (re, im)
void push_root(std::vector<double>& out, long num, long den) {
  const double a = 2.0 * M_PI * (double)(num % den) / (double)den;
  out.push_back(cos(a));
  out.push_back(-sin(a));
}

// The extra twiddle tables of a transform of length N: first the four-step
// table of the warp-per-line path (N >= 64: [k1][g] = w_N^{g k1}, k1 < R1,
// g < R2; line_tp_size(N, false) entries), then, for N = 512 and 1024, the
// Stockham passes 2 and 3 of the two-warp path ([q][k] = w_{Ls r}^{q k}).
void make_tp_table(int N, std::vector<double>& out) {
  out.clear();
  int R1 = 0, R2 = 0;
  switch (N) {
    case 64: R1 = DstShape<64>::R1; R2 = DstShape<64>::R2; break;
    case 128: R1 = DstShape<128>::R1; R2 = DstShape<128>::R2; break;
    case 256: R1 = DstShape<256>::R1; R2 = DstShape<256>::R2; break;
    case 512: R1 = DstShape<512>::R1; R2 = DstShape<512>::R2; break;
    case 1024: R1 = DstShape<1024>::R1; R2 = DstShape<1024>::R2; break;
    default: return;
  }
  for (int k1 = 0; k1 < R1; ++k1)
    for (int g = 0; g < R2; ++g) push_root(out, (long)g * k1, N);
  if (N < 512) return;
  const int R0 = N == 1024 ? WideShape<1024>::R0 : WideShape<512>::R0;
  const int W1 = N == 1024 ? WideShape<1024>::R1 : WideShape<512>::R1;
  const int W2 = N == 1024 ? WideShape<1024>::R2 : WideShape<512>::R2;
  const int passes[2][2] = {{R0, W1}, {R0 * W1, W2}};  // (Ls, r) of passes 2 and 3
  for (int p = 0; p < 2; ++p) {
    const int Ls = passes[p][0], r = passes[p][1];
    for (int q = 0; q < r; ++q)
      for (int k = 0; k < Ls; ++k) push_root(out, (long)q * k, (long)Ls * r);
  }
}

}  // namespace

struct csl_plan {
  int dim = 2;
  int n[3] = {1, 1, 1};
  long M = 0;
  double h[3] = {1, 1, 1};
  double alpha = 0, beta = 0, gamma = 0, amin = 0, amax = 0, sqrt_pmin = 0, sqrt_pmax = 0;
  double sigma = 1.0;  // FP32 forms: power-of-two prescale of the per-mode scale arguments
  int precision = CSL_PREC_FP64;
  int use_graph = 1;
  int use_pdl = 1;  // programmatic dependent launch of the iteration's kernels
  int ff = 0;       // FP32-preconditioner forms: float-pair stencil (faces in cxp/cyp/czp)
  int vpair = 0;    // v, w and x stored as float pairs (CSL_PREC_FP32 and the split-BF16 forms)
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  // the w/x update of an iteration runs on a side branch beside the inverse
  // x transform (fork after MID, join before the next stencil)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int split_update = 1;
  int serial_update = 0;  // update_mode 3: the update kernel after the inverse x transform, same stream
  int body_iters = 2;     // MINRES iterations per WHILE body of the graph
  int upd_blocks = 1;
  std::vector<void*> allocs;
  size_t bytes = 0;
  double *cx = nullptr, *cy = nullptr, *cz = nullptr, *dg = nullptr, *stab = nullptr;
  float2 *cxp = nullptr, *cyp = nullptr, *czp = nullptr;
  float2 alpha2 = {0.f, 0.f};
  double* mu_d[3] = {nullptr, nullptr, nullptr};
  float* mu_f[3] = {nullptr, nullptr, nullptr};
  void* tw[3] = {nullptr, nullptr, nullptr};
  void* hs[3] = {nullptr, nullptr, nullptr};
  void* tp[3] = {nullptr, nullptr, nullptr};
  void* sine_tc[3] = {nullptr, nullptr, nullptr};  // tensor-core passes: split-bf16 sine matrix per axis
  int tc_split = 0;                                // 2 or 3 bf16 terms (CSL_PREC_BF16X3 / X6), else 0
  double2 *b = nullptr, *x = nullptr, *io = nullptr;
  double2* x0 = nullptr;       // warm start: the caller's initial guess
  int warm = 0;
  double* hist = nullptr;      // residual history (plan option `history`)
  int hist_cap = 0;
  double2* v[2] = {nullptr, nullptr};
  double2* w[2] = {nullptr, nullptr};
  void* z[2] = {nullptr, nullptr};
  void* T = nullptr;
  DevState* st = nullptr;
  DevState* st_prof = nullptr;  // scratch state for csl_time_kernels
  double* partials = nullptr;
  unsigned long long* u64 = nullptr;
  PassCfg row, sy, sz;
  int sten_blocks = 1, ew_blocks = 1;
  int sten_strip = kStencilStrip;  // steps per warp strip of the stencil
  double cnorm = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int graph_state = 0;  // 0 not built, 1 ready, -1 failed (host-driven loop)
  char config[512] = "";
};

namespace {

void* dalloc(csl_plan* P, size_t bytes, cudaError_t* err) {
  void* p = nullptr;
  if (*err != cudaSuccess) return nullptr;
  *err = cudaMalloc(&p, bytes ? bytes : 16);
  if (*err == cudaSuccess) {
    P->allocs.push_back(p);
    P->bytes += bytes;
  }
  return p;
}

void free_plan(csl_plan* P) {
  if (!P) return;
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (void* p : P->allocs) cudaFree(p);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->side) cudaStreamDestroy(P->side);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  delete P;
}

cudaError_t set_attrs_once() {
  static int done = 0;
  static cudaError_t err = cudaSuccess;
  if (!done) {
    err = set_pass_attrs<double>();
    if (err == cudaSuccess) err = set_pass_attrs<float>();
    if (err == cudaSuccess) err = set_tc_attrs();
    done = 1;
  }
  return err;
}

// ---- launch configuration -------------------------------------------------
// CTA of `threads` lanes holds threads/TPL lines; shrink the CTA until its
// shared memory fits ~100 KB (two or more CTAs per SM).
template <typename T>
void choose_cta(PassCfg& c, int want_threads) {
  const int tpl = pass_tpl(c.N, c.wide);
  int threads = want_threads;
  while (threads > 32 && threads > tpl && pass_smem<T>(c.N, c.wide, threads / tpl) > 100 * 1024) threads >>= 1;
  c.lines = threads / tpl;
  c.L.threads = threads;
  c.L.smem = pass_smem<T>(c.N, c.wide, c.lines);
}

template <typename T>
void config_row(PassCfg& c, int n, int nrows) {
  c.n = n;
  c.N = n + 1;
  c.nouter = nrows;
  c.ncols = n;
  if (c.N == 16384) {  // FP64: one two-CTA cluster per row
    c.wide = 4;
    c.lines = 1;
    c.L.threads = cluster_pass_threads();
    c.L.smem = cluster_pass_smem();
    c.L.blocks = 2 * (nrows < 456 ? nrows : 456);
    return;
  }
  if (pass_is_big(c.N)) {  // one CTA of all the line's lanes per row
    c.wide = 3;
    c.lines = 1;
    c.L.threads = pass_tpl(c.N, 3);
    c.L.smem = pass_smem<T>(c.N, 3, 1);
    c.L.blocks = nrows < kSMs * 8 ? nrows : kSMs * 8;
    return;
  }
  int threads = 256;
  const int tpl = pass_tpl(c.N, c.wide);
  // few rows: smaller CTAs so that every SM gets work
  while (threads > 32 && threads / tpl > 1 && (nrows + threads / tpl - 1) / (threads / tpl) < 2 * kSMs) threads >>= 1;
  choose_cta<T>(c, threads);
  const long tiles = (nrows + c.lines - 1) / c.lines;
  c.L.blocks = (int)(tiles < (long)kSMs * 16 ? tiles : (long)kSMs * 16);
}

template <typename T>
void config_strided(PassCfg& c, int n, int ncols, int nouter, long outer_stride, long line_stride, int want_lines) {
  c.n = n;
  c.N = n + 1;
  c.ncols = ncols;
  c.nouter = nouter;
  c.outer_stride = outer_stride;
  c.line_stride = line_stride;
  if (c.N == 16384) {  // FP64: one two-CTA cluster per column
    c.wide = 4;
    c.lines = 1;
    c.L.threads = cluster_pass_threads();
    c.L.smem = cluster_pass_smem();
    const long cols = (long)ncols * nouter;
    c.L.blocks = (int)(2 * (cols < kMaxRedBlocks / 2 ? cols : kMaxRedBlocks / 2));
    return;
  }
  if (pass_is_big(c.N)) {  // one column per CTA
    c.wide = 3;
    c.lines = 1;
    c.L.threads = pass_tpl(c.N, 3);
    c.L.smem = pass_smem<T>(c.N, 3, 1);
    const long tiles = (long)ncols * nouter;
    c.L.blocks = (int)(tiles < kMaxRedBlocks ? tiles : kMaxRedBlocks);
    return;
  }
  const int tpl = pass_tpl(c.N, c.wide);
  int threads = 256;
  if (want_lines > 0) {
    int l = 1;
    while (l < want_lines) l <<= 1;
    threads = l * tpl < 32 ? 32 : l * tpl;
    if (threads > 1024) threads = 1024;
  }
  // no wider than the grid's x extent needs
  while (threads > 32 && threads > tpl && (threads / tpl) / 2 >= ncols) threads >>= 1;
  // few tiles: smaller CTAs so that every SM gets work
  while (want_lines <= 0 && threads > 32 && threads / tpl > 2 &&
         (long)((ncols + threads / tpl - 1) / (threads / tpl)) * nouter < 2 * kSMs)
    threads >>= 1;
  choose_cta<T>(c, threads);
  const long tiles = (long)((ncols + c.lines - 1) / c.lines) * nouter;
  c.L.blocks = (int)(tiles < kMaxRedBlocks ? tiles : kMaxRedBlocks);
}

// ---- launches ---------------------------------------------------------------
template <typename T>
RowArgs<T> row_args(csl_plan* P) {
  RowArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.n = P->row.n;
  a.nrows = P->row.nouter;
  a.tw = (const typename C2<T>::t*)P->tw[0];
  a.hs = (const T*)P->hs[0];
  a.tp = (const typename C2<T>::t*)P->tp[0] + (P->row.wide ? line_tp_size(P->row.N, false) : 0);
  return a;
}

// row-pass modes of the Lanczos step and the fused update for the plan's vector storage
inline int lanczos_load(const csl_plan* P) { return P->vpair ? LOAD_LANCZOS : LOAD_LANCZOS_V64; }
inline int update_store(const csl_plan* P) { return P->vpair ? STORE_Z_UPDATE : STORE_Z_UPDATE_V64; }

template <typename T>
StridedArgs<T> strided_args(csl_plan* P, const PassCfg& c, int axis) {
  StridedArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.n = c.n;
  a.ncols = c.ncols;
  a.nouter = c.nouter;
  a.outer_stride = c.outer_stride;
  a.line_stride = c.line_stride;
  a.tw = (const typename C2<T>::t*)P->tw[axis];
  a.hs = (const T*)P->hs[axis];
  a.tp = (const typename C2<T>::t*)P->tp[axis] + (c.wide ? line_tp_size(c.N, false) : 0);
  a.data = (typename C2<T>::t*)P->T;
  a.sine_tc = P->sine_tc[axis];
  return a;
}

template <typename T>
void fill_mid(csl_plan* P, StridedArgs<T>& a, int axis) {
  a.stab = (sizeof(T) == 8) ? P->stab : nullptr;
  if (sizeof(T) == 4) {
    a.mu_line = (const T*)P->mu_f[axis];
    a.mu_col = (const T*)P->mu_f[0];
    a.mu_outer = (axis == 2) ? (const T*)P->mu_f[1] : nullptr;
  }
  // s_k = cnorm / sqrt(e^2 + beta^2), e = gamma mu_k + alpha: every factor
  // times sigma leaves s_k unchanged and keeps e^2 + beta^2 inside FP32 range
  const double sg = sizeof(T) == 4 ? P->sigma : 1.0;
  a.gamma = (T)(P->gamma * sg);
  a.alpha = (T)(P->alpha * sg);
  a.beta2 = (T)((P->beta * sg) * (P->beta * sg));
  a.cnorm = (T)(P->cnorm * sg);
  a.partials = P->partials;
}

template <typename T>
cudaError_t run_row(csl_plan* P, int load, int store, const RowArgs<T>& a, cudaStream_t s) {
  return launch_row<T>(P->row.N, P->row.wide, load, store, a, P->row.L, s);
}

// P^{-1} applied to the plan's T buffer after the x pass: [y fwd,] mid, [y inv]
template <typename T>
cudaError_t launch_mid_chain(csl_plan* P, cudaStream_t s, DevState* st, int scalar_mode) {
  cudaError_t e;
  if (P->dim == 2) {
    StridedArgs<T> m = strided_args<T>(P, P->sy, 1);
    fill_mid<T>(P, m, 1);
    m.st = st;
    m.scalar_mode = scalar_mode;
    return launch_strided<T>(P->sy.N, P->sy.wide, true, m, P->sy.L, s);
  }
  StridedArgs<T> y = strided_args<T>(P, P->sy, 1);
  y.st = st;
  e = launch_strided<T>(P->sy.N, P->sy.wide, false, y, P->sy.L, s);
  if (e != cudaSuccess) return e;
  StridedArgs<T> m = strided_args<T>(P, P->sz, 2);
  fill_mid<T>(P, m, 2);
  m.st = st;
  m.scalar_mode = scalar_mode;
  e = launch_strided<T>(P->sz.N, P->sz.wide, true, m, P->sz.L, s);
  if (e != cudaSuccess) return e;
  return launch_strided<T>(P->sy.N, P->sy.wide, false, y, P->sy.L, s);
}

// stencil arguments of one plan for the buffer parity par
StencilArgs stencil_args(const csl_plan* P, int par) {
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.g.nx = P->n[0];
  a.g.ny = P->n[1];
  a.g.nz = P->dim == 3 ? P->n[2] : 1;
  a.g.M = P->M;
  a.z = P->z[par];
  a.vold = P->v[1 - par];
  a.cx = P->cx;
  a.cy = P->cy;
  a.cz = P->cz;
  a.dg = P->dg;
  a.cxp = P->cxp;
  a.cyp = P->cyp;
  a.czp = P->czp;
  a.alpha2 = P->alpha2;
  a.strip = P->sten_strip;
  a.x = P->x;
  a.b = P->b;
  a.st = P->st;
  a.partials = P->partials;
  return a;
}

typedef void (*StencilFn)(StencilArgs, const StencilArgs*, int);

// the stencil kernel for the plan's form: float-pair arithmetic (ff) and
// pair-stored vectors (vp) only with an FP32 ẑ
template <typename TZ>
StencilFn stencil_fn(int dim, bool ff, bool vp) {
  if constexpr (sizeof(TZ) == 8) {
    if (ff) return dim == 2 ? k_stencil<2, TZ, true, true> : k_stencil<3, TZ, true, true>;
    if (vp) return dim == 2 ? k_stencil<2, TZ, false, true> : k_stencil<3, TZ, false, true>;
  }
  return dim == 2 ? k_stencil<2, TZ, false, false> : k_stencil<3, TZ, false, false>;
}

template <typename T>
cudaError_t launch_stencil(csl_plan* P, int par, cudaStream_t s, bool use_cond) {
  StencilArgs a = stencil_args(P, par);
  a.cond = P->cond;
  a.use_cond = use_cond ? 1 : 0;
  typedef typename C2<T>::t TZ;
  const StencilArgs* nob = nullptr;
  const size_t smem = (sizeof(TZ) == 8 && P->ff) ? ff_stencil_smem(P->dim) : 0;
  return launch_k(P->use_pdl != 0, stencil_fn<TZ>(P->dim, P->ff != 0, P->vpair != 0), P->sten_blocks, 256, smem, s, a,
                  nob, 0);
}

template <typename T>
RowArgs<T> p1_args(csl_plan* P, int par) {
  RowArgs<T> r = row_args<T>(P);
  r.vnew = P->v[1 - par];
  r.vcur = P->v[par];
  r.tout = (typename C2<T>::t*)P->T;
  r.st = P->st;
  return r;
}

template <typename T>
RowArgs<T> p3_args(csl_plan* P, int par) {
  RowArgs<T> r = row_args<T>(P);
  r.tin = (const typename C2<T>::t*)P->T;
  r.zout = (typename C2<T>::t*)P->z[1 - par];
  r.zcur = (const typename C2<T>::t*)P->z[par];
  r.wprev = P->w[par];
  r.wcur = P->w[1 - par];
  r.x = P->x;
  r.st = P->st;
  return r;
}

// the w/x update of the iteration with parity par (see k_update)
template <typename T>
cudaError_t launch_update(csl_plan* P, int par, cudaStream_t s) {
  UpdateArgs u;
  u.z = P->z[par];
  u.wprev = P->w[par];
  u.wcur = P->w[1 - par];
  u.x = P->x;
  u.st = P->st;
  u.M = P->M;
  if constexpr (sizeof(T) == 4) {
    if (P->vpair) {
      k_update<float2, true><<<P->upd_blocks, 256, 0, s>>>(u);
      return cudaGetLastError();
    }
  }
  k_update<typename C2<T>::t, false><<<P->upd_blocks, 256, 0, s>>>(u);
  return cudaGetLastError();
}

// one MINRES iteration with buffer parity `par` (v_j in v[par], z_j in z[par])
template <typename T>
cudaError_t launch_iteration_T(csl_plan* P, int par, cudaStream_t s, bool use_cond) {
  cudaError_t e = launch_stencil<T>(P, par, s, use_cond);
  if (e == cudaSuccess) e = run_row<T>(P, lanczos_load(P), STORE_T, p1_args<T>(P, par), s);
  if (e == cudaSuccess) e = launch_mid_chain<T>(P, s, P->st, 2);
  if (!P->split_update) {
    if (e == cudaSuccess) e = run_row<T>(P, LOAD_T, update_store(P), p3_args<T>(P, par), s);
    return e;
  }
  if (P->serial_update) {
    if (e == cudaSuccess) e = run_row<T>(P, LOAD_T, STORE_Z, p3_args<T>(P, par), s);
    if (e == cudaSuccess) e = launch_update<T>(P, par, s);
    return e;
  }
  // fork: the update on the side stream, the inverse x transform (z_{j+1})
  // on s; join before the next stencil, which reads both
  if (e == cudaSuccess) e = cudaEventRecord(P->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->side, P->ev_fork, 0);
  if (e == cudaSuccess) e = launch_update<T>(P, par, P->side);
  if (e == cudaSuccess) e = run_row<T>(P, LOAD_T, STORE_Z, p3_args<T>(P, par), s);
  if (e == cudaSuccess) e = cudaEventRecord(P->ev_join, P->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P->ev_join, 0);
  return e;
}

cudaError_t launch_iteration(csl_plan* P, int par, cudaStream_t s, bool use_cond) {
  if (P->precision != CSL_PREC_FP64) return launch_iteration_T<float>(P, par, s, use_cond);
  return launch_iteration_T<double>(P, par, s, use_cond);
}

// ingest f and compute z_1 = P^{-1} b, gamma_1
template <typename T>
cudaError_t launch_prologue_T(csl_plan* P, const double2* f, double tol, int maxit, double beta, cudaStream_t s) {
  IngestArgs ia;
  memset(&ia, 0, sizeof(ia));
  ia.M = P->M;
  ia.f = f;
  ia.b = P->b;
  ia.v0 = P->v[0];
  ia.v1 = P->v[1];
  ia.w0 = P->w[0];
  ia.w1 = P->w[1];
  ia.x = P->x;
  ia.st = P->st;
  ia.partials = P->partials;
  ia.tol = tol;
  ia.beta = beta;
  ia.maxit = maxit;
  ia.sqrt_pmin = P->sqrt_pmin;
  ia.sqrt_pmax = P->sqrt_pmax;
  ia.vpair = P->vpair;
  k_ingest<<<P->ew_blocks, 256, 0, s>>>(ia, nullptr, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && P->warm) {
    WarmArgs wa;
    wa.g.nx = P->n[0];
    wa.g.ny = P->n[1];
    wa.g.nz = P->dim == 3 ? P->n[2] : 1;
    wa.g.M = P->M;
    wa.x0 = P->x0;
    wa.b = P->b;
    wa.v0 = P->v[0];
    wa.cx = P->cx;
    wa.cy = P->cy;
    wa.cz = P->cz;
    wa.dg = P->dg;
    wa.st = P->st;
    wa.partials = P->partials;
    wa.vpair = P->vpair;
    if (P->dim == 2)
      k_warm_start<2><<<P->ew_blocks, 256, 0, s>>>(wa);
    else
      k_warm_start<3><<<P->ew_blocks, 256, 0, s>>>(wa);
    e = cudaGetLastError();
  }
  RowArgs<T> r1 = row_args<T>(P);
  r1.vin = P->b;  // v_1 = b (v[0] holds it as pairs in the FP32 forms)
  r1.tout = (typename C2<T>::t*)P->T;
  r1.st = P->st;
  if (e == cudaSuccess) e = run_row<T>(P, LOAD_V, STORE_T, r1, s);
  if (e == cudaSuccess) e = launch_mid_chain<T>(P, s, P->st, 1);
  RowArgs<T> r3 = row_args<T>(P);
  r3.tin = (const typename C2<T>::t*)P->T;
  r3.zout = (typename C2<T>::t*)P->z[0];
  r3.st = P->st;
  if (e == cudaSuccess) e = run_row<T>(P, LOAD_T, STORE_Z, r3, s);
  return e;
}

cudaError_t launch_prologue(csl_plan* P, const double2* f, double tol, int maxit, double beta, cudaStream_t s) {
  if (P->precision != CSL_PREC_FP64) return launch_prologue_T<float>(P, f, tol, maxit, beta, s);
  return launch_prologue_T<double>(P, f, tol, maxit, beta, s);
}

template <typename T>
cudaError_t launch_precondition_T(csl_plan* P, const double2* v, double2* out, cudaStream_t s) {
  RowArgs<T> r1 = row_args<T>(P);
  r1.vin = v;
  r1.tout = (typename C2<T>::t*)P->T;
  cudaError_t e = run_row<T>(P, LOAD_V, STORE_T, r1, s);
  if (e == cudaSuccess) e = launch_mid_chain<T>(P, s, nullptr, 0);
  RowArgs<T> r3 = row_args<T>(P);
  r3.tin = (const typename C2<T>::t*)P->T;
  r3.dout = out;
  if (e == cudaSuccess) e = run_row<T>(P, LOAD_T, STORE_D, r3, s);
  return e;
}

// one kernel (index k of the iteration's sequence) of the MINRES iteration
// with buffer parity par, on the plan's stream (measurement and tuning);
// mid_mode: the MID pass's scalar tail (2: Givens step, 0: none)
cudaError_t launch_iteration_kernel(csl_plan* P, int k, int par, int mid_mode) {
  const bool fp32 = P->precision != CSL_PREC_FP64;
  const int nkb = P->dim == 2 ? 4 : 6;  // kernels of the main chain
  const int st3 = P->split_update ? STORE_Z : update_store(P);
  if (k == 0) return fp32 ? launch_stencil<float>(P, par, P->stream, false) : launch_stencil<double>(P, par, P->stream, false);
  if (k == 1)
    return fp32 ? run_row<float>(P, lanczos_load(P), STORE_T, p1_args<float>(P, par), P->stream)
                : run_row<double>(P, LOAD_LANCZOS, STORE_T, p1_args<double>(P, par), P->stream);
  if (k == nkb) return fp32 ? launch_update<float>(P, par, P->stream) : launch_update<double>(P, par, P->stream);
  if (k == nkb - 1)
    return fp32 ? run_row<float>(P, LOAD_T, st3, p3_args<float>(P, par), P->stream)
                : run_row<double>(P, LOAD_T, st3, p3_args<double>(P, par), P->stream);
  const bool mid = (P->dim == 2) || (k == 3);
  const PassCfg& c = (P->dim == 3 && k == 3) ? P->sz : P->sy;
  const int axis = (P->dim == 3 && k == 3) ? 2 : 1;
  if (fp32) {
    StridedArgs<float> a = strided_args<float>(P, c, axis);
    a.st = P->st;
    if (mid) {
      fill_mid<float>(P, a, axis);
      a.scalar_mode = mid_mode;
    }
    return launch_strided<float>(c.N, c.wide, mid, a, c.L, P->stream);
  }
  StridedArgs<double> a = strided_args<double>(P, c, axis);
  a.st = P->st;
  if (mid) {
    fill_mid<double>(P, a, axis);
    a.scalar_mode = mid_mode;
  }
  return launch_strided<double>(c.N, c.wide, mid, a, c.L, P->stream);
}


// Number of kernels of one iteration in csl_time_kernels' order: stencil,
// P1, [3D: y fwd,] MID, [3D: y inv,] P3, and the update when it is its own kernel
int iteration_kernels(const csl_plan* P) { return (P->dim == 2 ? 4 : 6) + (P->split_update ? 1 : 0); }

// The iteration's kernel sequence, `reps` iterations in a row on the plan's
// stream after one untimed iteration, an event between consecutive kernels
// (the update after the inverse x transform); ms[k] = mean duration of
// kernel k.  The caller points P->st at a scratch state.  ev: at least
// (reps + 1) * (iteration_kernels(P) + 1) created events.
cudaError_t time_sequence(csl_plan* P, int reps, int mid_mode, cudaEvent_t* ev, double* ms) {
  const int nk = iteration_kernels(P);
  cudaError_t err = cudaSuccess;
  for (int r = 0; r <= reps && err == cudaSuccess; ++r) {
    cudaEvent_t* er = ev + (size_t)r * (nk + 1);
    err = cudaEventRecord(er[0], P->stream);
    for (int k = 0; k < nk && err == cudaSuccess; ++k) {
      err = launch_iteration_kernel(P, k, r & 1, mid_mode);
      if (err == cudaSuccess) err = cudaEventRecord(er[k + 1], P->stream);
    }
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(P->stream);
  for (int k = 0; k < nk && err == cudaSuccess; ++k) {
    double tot = 0.0;
    for (int r = 1; r <= reps && err == cudaSuccess; ++r) {
      float t = 0.f;
      err = cudaEventElapsedTime(&t, ev[(size_t)r * (nk + 1) + k], ev[(size_t)r * (nk + 1) + k + 1]);
      tot += t;
    }
    ms[k] = tot / reps;
  }
  return err;
}

// scratch solver state for timing: a Lanczos run with the stopping schedule
// disabled (no true-residual pass, no exit)
DevState scratch_state(const csl_plan* P) {
  DevState h;
  memset(&h, 0, sizeof(h));
  h.gam = h.gam_old = h.gam1 = 1.0;
  h.a1inv_old = h.a1inv_old2 = 1.0;
  h.c = h.c_old = 1.0;
  h.eta = h.eta_x = h.bnorm = h.r0norm = 1.0;
  h.tol = 1e-300;
  h.maxit = 1 << 30;
  h.beta = P->beta;
  h.sqrt_pmin = h.sqrt_pmax = 1e300;
  return h;
}

// ---- autotuner ---------------------------------------------------------------
// Each sine-transform pass tries every CTA size and, for N = 512 and 1024,
// every transform variant.  A candidate is timed inside the iteration's own
// kernel sequence (time_sequence: three iterations after a warm-up, on
// zeroed vectors and a scratch state, the MID pass without its scalar tail),
// so that its cost includes the caches and the predecessor it really has;
// the candidate with the smallest summed duration of the pass's kernels is
// kept.  Results are cached per (precision, pass, geometry) for the life of
// the process, and can be saved to and loaded from a file.
struct TuneKey {
  int prec, kind, N, ncols, nouter;
  bool operator<(const TuneKey& o) const {
    if (prec != o.prec) return prec < o.prec;
    if (kind != o.kind) return kind < o.kind;
    if (N != o.N) return N < o.N;
    if (ncols != o.ncols) return ncols < o.ncols;
    return nouter < o.nouter;
  }
};
std::map<TuneKey, PassCfg> g_tune_cache;
std::mutex g_tune_mu;

// One candidate shape of a pass: transform variant w with `lines` lines per
// CTA; false when the shape is not allowed (CTA size, shared memory, tile
// wider than twice the grid's x extent).  Used by the tuner and by the cache
// loader, so a shape read from a file is rebuilt and checked the same way.
template <typename T>
bool make_candidate(const PassCfg& c, int kind, int w, int lines, PassCfg& cand) {
  if (w < 0 || w >= pass_num_variants(c.N) || lines < 1 || (lines & (lines - 1))) return false;
  const int tpl = pass_tpl(c.N, w);
  if (lines * tpl < 32 || lines * tpl > 256) return false;
  cand = c;
  cand.wide = w;
  cand.lines = lines;
  cand.L.threads = lines * tpl;
  cand.L.smem = pass_smem<T>(c.N, cand.wide, lines);
  if (cand.L.smem > 200 * 1024) return false;
  long tiles;
  if (kind == 0) {
    tiles = (c.nouter + lines - 1) / lines;
    cand.L.blocks = (int)(tiles < (long)kSMs * 16 ? tiles : (long)kSMs * 16);
  } else {
    if (lines > 2 * c.ncols) return false;
    tiles = (long)((c.ncols + lines - 1) / lines) * c.nouter;
    cand.L.blocks = (int)(tiles < kMaxRedBlocks ? tiles : kMaxRedBlocks);
  }
  return true;
}

// the kernels of the sequence that a pass's shape governs (kind 0: the row
// passes P1 and P3; kind 1: the 3D y passes; kind 2: the MID pass)
int pass_kernels(const csl_plan* P, int kind, int idx[2]) {
  const int nkb = P->dim == 2 ? 4 : 6;
  if (kind == 0) {
    idx[0] = 1;
    idx[1] = nkb - 1;
    return 2;
  }
  if (kind == 1) {
    idx[0] = 2;
    idx[1] = 4;
    return 2;
  }
  idx[0] = P->dim == 2 ? 2 : 3;
  return 1;
}

template <typename T>
cudaError_t tune_pass(csl_plan* P, PassCfg& c, int kind, cudaEvent_t* ev, const DevState& hst) {
  if (c.L.tc || c.wide >= 3) return cudaSuccess;  // the tensor-core and long-line variants have one shape
  const TuneKey key = {(int)sizeof(T), kind, c.N, c.ncols, c.nouter};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      PassCfg hit;
      // a cached shape is rebuilt from (variant, lines) for this plan's pass
      if (make_candidate<T>(c, kind, it->second.wide, it->second.lines, hit)) {
        c = hit;
        return cudaSuccess;
      }
    }
  }
  int idx[2];
  const int nidx = pass_kernels(P, kind, idx);
  const PassCfg keep = c;
  PassCfg best = c;
  double best_ms = 1e30;
  double ms[8];
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < pass_num_variants(keep.N) && e == cudaSuccess; ++w) {
    for (int lines = 1; lines <= 256 && e == cudaSuccess; lines <<= 1) {
      PassCfg cand;
      if (!make_candidate<T>(keep, kind, w, lines, cand)) continue;
      c = cand;  // c is the plan's own pass configuration
      double t = 1e30;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the faster of two measurements
        e = cudaMemcpyAsync(P->st, &hst, sizeof(hst), cudaMemcpyHostToDevice, P->stream);
        if (e == cudaSuccess) e = time_sequence(P, 3, 0, ev, ms);
        double sum = 0.0;
        for (int i = 0; i < nidx; ++i) sum += ms[idx[i]];
        if (e == cudaSuccess && sum < t) t = sum;
      }
      if (e == cudaSuccess && t < best_ms) {
        best_ms = t;
        best = cand;
      }
    }
  }
  c = best;
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return cudaSuccess;
}

template <typename T>
cudaError_t autotune(csl_plan* P) {
  const DevState h = scratch_state(P);
  DevState* keep = P->st;
  P->st = P->st_prof;
  std::vector<cudaEvent_t> ev((size_t)4 * (iteration_kernels(P) + 1), nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  // the vectors are uninitialised here: zero them (finite inputs for every pass)
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemsetAsync(P->v[i], 0, sizeof(double2) * P->M, P->stream);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemsetAsync(P->w[i], 0, sizeof(double2) * P->M, P->stream);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(P->z[i], 0, sizeof(typename C2<T>::t) * P->M, P->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->x, 0, sizeof(double2) * P->M, P->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->b, 0, sizeof(double2) * P->M, P->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->T, 0, sizeof(typename C2<T>::t) * P->M, P->stream);
  if (e == cudaSuccess) e = tune_pass<T>(P, P->row, 0, ev.data(), h);
  if (P->dim == 2) {
    if (e == cudaSuccess) e = tune_pass<T>(P, P->sy, 2, ev.data(), h);
  } else {
    if (e == cudaSuccess) e = tune_pass<T>(P, P->sy, 1, ev.data(), h);
    if (e == cudaSuccess) e = tune_pass<T>(P, P->sz, 2, ev.data(), h);
  }
  P->st = keep;
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  return e;
}

// The tuner's cache as a text file: a header line, then one line per tuned
// pass "prec kind N ncols nouter variant lines".  Only (variant, lines) are
// kept; the launch shape is rebuilt from them when a plan asks for that pass.
const char* kTuneHeader = "csl-tune-cache 1";

bool tune_entry_valid(const TuneKey& k, int wide, int lines) {
  if (k.prec != 4 && k.prec != 8) return false;
  if (k.kind < 0 || k.kind > 2) return false;
  if (k.N < 4 || k.N > 1024 || ilog2_exact(k.N) < 0) return false;
  if (k.ncols < 1 || k.nouter < 1) return false;
  if (wide < 0 || wide >= pass_num_variants(k.N)) return false;
  return lines >= 1 && lines <= 256 && !(lines & (lines - 1));
}

// Build the graph: one WHILE node whose body is two MINRES iterations (both
// buffer parities); the stencil kernel's last block sets the condition.
void build_graph(csl_plan* P) {
  if (P->graph_state != 0) return;
  P->graph_state = -1;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&P->cond, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    cp.conditional.handle = P->cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(P->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaSuccess;
      for (int k = 0; k < P->body_iters && e1 == cudaSuccess; ++k) e1 = launch_iteration(P, k & 1, P->cap, true);
      cudaGraph_t captured = body;
      e = cudaStreamEndCapture(P->cap, &captured);
      if (e == cudaSuccess) e = e1;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->gexec, g, 0);
  if (e != cudaSuccess) {
    CSL_NOTE(e, "graph build (falling back to the host-driven loop)");
    (void)cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    P->gexec = nullptr;
    return;
  }
  P->graph = g;
  P->graph_state = 1;
}

csl_status run_loop(csl_plan* P, int maxit) {
  if (P->use_graph) build_graph(P);
  if (P->graph_state == 1) {
    CSL_TRY(cudaGraphLaunch(P->gexec, P->stream));
    return CSL_OK;
  }
  // host-driven loop: batches of 8 iterations, then read the done flag
  int done = 0;
  for (int it = 0; it < maxit + 4 && !done; it += 8) {
    for (int k = 0; k < 8; ++k) {
      NvtxRange r("csl:iteration");
      CSL_TRY(launch_iteration(P, k & 1, P->stream, false));
    }
    CSL_TRY(cudaMemcpyAsync(&done, &P->st->done, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    CSL_TRY(cudaStreamSynchronize(P->stream));
  }
  return CSL_OK;
}

csl_status read_info(csl_plan* P, csl_solve_info* info, csl_status* solve_status) {
  DevState h;
  CSL_TRY(cudaMemcpyAsync(&h, P->st, sizeof(DevState), cudaMemcpyDeviceToHost, P->stream));
  CSL_TRY(cudaStreamSynchronize(P->stream));
  *solve_status = h.done ? (csl_status)h.status : CSL_NOT_CONVERGED;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = h.iter;
    info->status = (int)*solve_status;
    info->relres = h.relres;
    info->pnorm = h.eta_x;
    info->gamma = P->gamma;
    info->checks = h.checks;
    // prologue kernels + every launched WHILE body (two iterations each)
    const int per_iter = P->dim == 2 ? 4 : 6;
    const int prologue = 1 + per_iter;
    const int it_launches = per_iter + (P->split_update ? 1 : 0);  // + k_update on the side branch
    const int B = P->body_iters;
    const int bodies = (h.loops + B - 1) / B;
    info->launches =
        prologue + (P->graph_state == 1 ? bodies * B * it_launches : ((h.loops + 7) / 8) * 8 * it_launches);
  }
  return CSL_OK;
}

// the iterate x to the caller's FP64 vector (the FP32 forms hold it as float
// pairs; with a warm start x is the correction to x_0)
cudaError_t copy_out(csl_plan* P, double2* dst, cudaStream_t s) {
  if (P->warm) {
    k_x_out_add<<<P->ew_blocks, 256, 0, s>>>(P->x, P->vpair, P->x0, dst, P->M);
    return cudaGetLastError();
  }
  if (!P->vpair) return cudaMemcpyAsync(dst, P->x, sizeof(double2) * P->M, cudaMemcpyDeviceToDevice, s);
  k_x_out<<<P->ew_blocks, 256, 0, s>>>((const float4*)P->x, dst, P->M);
  return cudaGetLastError();
}

// x0: the caller's initial guess (device, warm-start plans), copied before the
// prologue because the caller's buffer is also the output
csl_status solve_impl(csl_plan* P, const double2* f, double tol, int maxit, double beta, const double2* x0) {
  if (!(tol > 0.0) || maxit < 1) return CSL_INVALID_ARG;
  if (P->warm && x0 && x0 != P->x0)
    CSL_TRY(cudaMemcpyAsync(P->x0, x0, sizeof(double2) * P->M, cudaMemcpyDeviceToDevice, P->stream));
  {
    NvtxRange r("csl:prologue");
    CSL_TRY(launch_prologue(P, f, tol, maxit, beta, P->stream));
  }
  NvtxRange r("csl:minres-loop");
  return run_loop(P, maxit);
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* csl_version(void) { return "csl 0.2 (sm_103a)"; }

const char* csl_last_error(void) { return g_last_error; }

}  // extern "C"

// message for csl_last_error() from the other translation units of the library
void csl_internal_set_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

extern "C" {

const char* csl_status_string(csl_status s) {
  switch (s) {
    case CSL_OK: return "CSL_OK";
    case CSL_INVALID_ARG: return "CSL_INVALID_ARG";
    case CSL_UNSUPPORTED_SIZE: return "CSL_UNSUPPORTED_SIZE";
    case CSL_SINGULAR_PRECOND: return "CSL_SINGULAR_PRECOND";
    case CSL_BREAKDOWN: return "CSL_BREAKDOWN";
    case CSL_NOT_CONVERGED: return "CSL_NOT_CONVERGED";
    case CSL_TIMEOUT: return "CSL_TIMEOUT";
    case CSL_CUDA_ERROR: return "CSL_CUDA_ERROR";
    case CSL_OUT_OF_MEMORY: return "CSL_OUT_OF_MEMORY";
  }
  return "CSL_UNKNOWN_STATUS";
}

csl_status csl_plan_options_init(csl_plan_options* opt) {
  if (!opt) return CSL_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->precision = CSL_PREC_FP64;
  opt->gamma_override = kNaN;
  opt->lines_per_cta = 0;
  opt->use_graph = 1;
  opt->autotune = 1;
  opt->programmatic_launch = 1;
  opt->float_pair_stencil = 1;
  return CSL_OK;
}

csl_status csl_plan_create(csl_plan** out, int dim, const int64_t n[3], const double* const coef_faces[3],
                           double alpha, double beta, const csl_plan_options* opt, void* stream) {
  if (!out) return CSL_INVALID_ARG;
  *out = nullptr;
  if (!n || !coef_faces || (dim != 2 && dim != 3)) return CSL_INVALID_ARG;
  if (!isfinite(alpha) || !isfinite(beta)) return CSL_INVALID_ARG;
  csl_plan_options o;
  csl_plan_options_init(&o);
  if (opt) o = *opt;
  if (o.history < 0 || o.history > (1 << 24)) return CSL_INVALID_ARG;
  NvtxRange nv("csl_plan_create");
  // transform lengths: 4 .. 1024 in 2D and 3D; 2D grids up to 16384 in FP64
  // (lines of 16384 on two-CTA clusters) and 4096 in the FP32 forms, whose
  // P^{-1} error grows like eps_32 kappa(P), kappa(P) ~ n^2
  const long nmax = dim == 3 ? 1024 : (o.precision == CSL_PREC_FP64 ? 16384 : 4096);
  for (int d = 0; d < dim; ++d) {
    if (!coef_faces[d] || n[d] < 1) return CSL_INVALID_ARG;
    if (n[d] + 1 < 4 || n[d] + 1 > nmax || ilog2_exact(n[d] + 1) < 0) return CSL_UNSUPPORTED_SIZE;
  }
  if (o.precision != CSL_PREC_FP64 && o.precision != CSL_PREC_FP32 && o.precision != CSL_PREC_BF16X3 &&
      o.precision != CSL_PREC_BF16X6 && o.precision != CSL_PREC_FP32_PRECOND)
    return CSL_INVALID_ARG;
  CSL_TRY(set_attrs_once());

  csl_plan* P = new (std::nothrow) csl_plan();
  if (!P) return CSL_OUT_OF_MEMORY;
  P->dim = dim;
  P->precision = o.precision;
  P->vpair = (o.precision == CSL_PREC_FP32 || o.precision == CSL_PREC_BF16X3 || o.precision == CSL_PREC_BF16X6) ? 1 : 0;
  P->use_graph = o.use_graph;
  P->use_pdl = o.programmatic_launch;
  if (o.update_mode < 0 || o.update_mode > 3 ||
      !(o.body_iters == 0 || o.body_iters == 2 || o.body_iters == 4 || o.body_iters == 8)) {
    delete P;
    return CSL_INVALID_ARG;
  }
  P->split_update = o.update_mode == 2 ? 0 : 1;
  P->serial_update = o.update_mode == 3 ? 1 : 0;
  P->body_iters = o.body_iters ? o.body_iters : 2;
  P->warm = o.warm_start ? 1 : 0;
  P->hist_cap = o.history;
  P->stream = (cudaStream_t)stream;
  P->alpha = alpha;
  P->beta = beta;
  P->M = 1;
  for (int d = 0; d < 3; ++d) P->n[d] = d < dim ? (int)n[d] : 1;
  for (int d = 0; d < dim; ++d) {
    P->M *= n[d];
    P->h[d] = 1.0 / (double)(n[d] + 1);
  }
  const long M = P->M;
  const int nx = P->n[0], ny = P->n[1], nz = P->n[2];
  const size_t tsz = o.precision != CSL_PREC_FP64 ? sizeof(float) : sizeof(double);
  long nface[3];
  nface[0] = (long)nz * ny * (nx + 1);
  nface[1] = (long)nz * (ny + 1) * nx;
  nface[2] = dim == 3 ? (long)(nz + 1) * ny * nx : 0;

  cudaError_t err = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming);
  P->cx = (double*)dalloc(P, nface[0] * 8, &err);
  P->cy = (double*)dalloc(P, nface[1] * 8, &err);
  if (dim == 3) P->cz = (double*)dalloc(P, nface[2] * 8, &err);
  P->dg = (double*)dalloc(P, M * 8, &err);
  if (o.precision == CSL_PREC_FP64) P->stab = (double*)dalloc(P, M * 8, &err);
  if (P->vpair && o.float_pair_stencil) {
    P->cxp = (float2*)dalloc(P, nface[0] * 8, &err);
    P->cyp = (float2*)dalloc(P, nface[1] * 8, &err);
    if (dim == 3) P->czp = (float2*)dalloc(P, nface[2] * 8, &err);
  }
  for (int d = 0; d < dim; ++d) {
    const int N = P->n[d] + 1;
    P->mu_d[d] = (double*)dalloc(P, (size_t)P->n[d] * 8, &err);
    P->mu_f[d] = (float*)dalloc(P, (size_t)P->n[d] * 4, &err);
    P->tw[d] = dalloc(P, (size_t)(N / 2) * 2 * tsz, &err);
    P->hs[d] = dalloc(P, (size_t)(N / 2 + 1) * tsz, &err);
    P->tp[d] = dalloc(P, (size_t)(line_tp_size(N, false) + line_tp_size(N, true) + 1) * 2 * tsz, &err);
  }
  P->b = (double2*)dalloc(P, M * 16, &err);
  P->x = (double2*)dalloc(P, M * 16, &err);
  P->io = (double2*)dalloc(P, M * 16, &err);
  if (P->warm) P->x0 = (double2*)dalloc(P, M * 16, &err);
  if (P->hist_cap > 0) P->hist = (double*)dalloc(P, (size_t)P->hist_cap * 8, &err);
  for (int i = 0; i < 2; ++i) {
    P->v[i] = (double2*)dalloc(P, M * 16, &err);
    P->w[i] = (double2*)dalloc(P, M * 16, &err);
    P->z[i] = dalloc(P, M * 2 * tsz, &err);
  }
  P->T = dalloc(P, M * 2 * tsz, &err);
  P->st = (DevState*)dalloc(P, sizeof(DevState), &err);
  P->st_prof = (DevState*)dalloc(P, sizeof(DevState), &err);
  P->partials = (double*)dalloc(P, (size_t)kMaxRedBlocks * 4 * 8, &err);
  P->u64 = (unsigned long long*)dalloc(P, 8 * 8, &err);
  if (err != cudaSuccess) {
    CSL_NOTE(err, "device allocation");
    (void)cudaGetLastError();
    free_plan(P);
    return err == cudaErrorMemoryAllocation ? CSL_OUT_OF_MEMORY : CSL_CUDA_ERROR;
  }
  cudaStream_t s = P->stream;
  P->ew_blocks = (int)((M + 255) / 256 < kSMs * 8 ? (M + 255) / 256 : kSMs * 8);
  {
    const long chunks = (M + 256 * kUpdateUnroll - 1) / (256 * kUpdateUnroll);
    P->upd_blocks = (int)(chunks < kSMs * 8 ? chunks : kSMs * 8);
  }

  // coefficient faces: a_e / h^2, min / max / validity (Eq. 1 and Eq. 4's a_min, a_max)
  {
    unsigned long long init[3] = {~0ull, 0ull, 0ull};
    double* dst[3] = {P->cx, P->cy, P->cz};
    double amin = INFINITY, amax = 0.0;
    for (int d = 0; d < dim; ++d) {
      err = cudaMemcpyAsync(P->u64, init, sizeof(init), cudaMemcpyHostToDevice, s);
      if (err == cudaSuccess) {
        const long cnt = nface[d];
        const int blocks = (int)((cnt + 255) / 256 < 1024 ? (cnt + 255) / 256 : 1024);
        k_scale_faces<<<blocks, 256, 0, s>>>(coef_faces[d], dst[d], cnt, 1.0 / (P->h[d] * P->h[d]), P->u64);
        err = cudaGetLastError();
      }
      unsigned long long res[3] = {0, 0, 0};
      if (err == cudaSuccess) err = cudaMemcpyAsync(res, P->u64, sizeof(res), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err != cudaSuccess) {
        CSL_NOTE(err, "coefficient set-up");
        (void)cudaGetLastError();
        free_plan(P);
        return CSL_CUDA_ERROR;
      }
      if (res[2]) {
        free_plan(P);
        return CSL_INVALID_ARG;
      }
      double lo, hi;
      memcpy(&lo, &res[0], 8);
      memcpy(&hi, &res[1], 8);
      amin = lo < amin ? lo : amin;
      amax = hi > amax ? hi : amax;
    }
    P->amin = amin;
    P->amax = amax;
    P->gamma = (o.gamma_override > 0.0 && isfinite(o.gamma_override)) ? o.gamma_override : sqrt(amin * amax);
    // Float-pair stencil: every scaled face, alpha and beta inside [2^-60, 2^60]
    // (zero allowed for alpha and beta), so that both halves of each pair and
    // their products with an FP32 ẑ stay normal floats.
    if (P->cxp) {
      double smin = INFINITY, smax = 0.0;
      for (int d = 0; d < dim; ++d) {
        const double s2 = 1.0 / (P->h[d] * P->h[d]);
        smin = s2 < smin ? s2 : smin;
        smax = s2 > smax ? s2 : smax;
      }
      const double lo = ldexp(1.0, -60), hi = ldexp(1.0, 60);
      auto ok_shift = [&](double v) { return v == 0.0 || (fabs(v) >= lo && fabs(v) <= hi); };
      P->ff = (amin * smin >= lo && amax * smax <= hi && ok_shift(alpha) && ok_shift(beta)) ? 1 : 0;
      const float ah = (float)alpha;
      P->alpha2 = make_float2(ah, (float)(alpha - (double)ah));
      float2* pdst[3] = {P->cxp, P->cyp, P->czp};
      if (P->ff) err = allow_dyn_smem((const void*)stencil_fn<float2>(dim, true, true));
      for (int d = 0; d < dim && err == cudaSuccess; ++d) {
        const int blocks = (int)((nface[d] + 255) / 256 < 1024 ? (nface[d] + 255) / 256 : 1024);
        k_pair_faces<<<blocks, 256, 0, s>>>(dst[d], pdst[d], nface[d]);
        err = cudaGetLastError();
      }
      if (err != cudaSuccess) {
        CSL_NOTE(err, "float-pair faces");
        (void)cudaGetLastError();
        free_plan(P);
        return CSL_CUDA_ERROR;
      }
    }
  }
  {
    // one warp per strip, 8 warps per CTA
    P->sten_strip = P->ff ? strip_rows(dim, nx, ny, nz, kSMs, 24)
                    : dim == 2 ? strip_rows(dim, nx, ny, nz, kSMs, 16) : kStencilStrip;
    const long blocks = (stencil_strips(dim, nx, ny, nz, P->sten_strip) + 7) / 8;
    P->sten_blocks = (int)(blocks < kSMs * 8 ? blocks : kSMs * 8);
  }
  Grid g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.M = M;
  if (dim == 2)
    k_diag<2><<<P->ew_blocks, 256, 0, s>>>(g, P->cx, P->cy, P->cz, P->dg, alpha);
  else
    k_diag<3><<<P->ew_blocks, 256, 0, s>>>(g, P->cx, P->cy, P->cz, P->dg, alpha);

  // Section 2.3 tables: 1D Laplacian eigenvalues, FFT twiddles, half sines
  P->cnorm = 1.0;
  for (int d = 0; d < dim && err == cudaSuccess; ++d) {
    const int nd = P->n[d], N = nd + 1;
    P->cnorm *= 2.0 / (double)N;
    std::vector<double> mu(nd);
    std::vector<float> muf(nd);
    for (int k = 1; k <= nd; ++k) {
      const double sn = sin(M_PI * (double)k / (2.0 * N));
      mu[k - 1] = 4.0 / (P->h[d] * P->h[d]) * sn * sn;
      muf[k - 1] = (float)mu[k - 1];
    }
    std::vector<double> twd(N), hsd(N / 2 + 1);
    for (int m = 0; m < N / 2; ++m) {
      twd[2 * m] = cos(2.0 * M_PI * (double)m / N);
      twd[2 * m + 1] = -sin(2.0 * M_PI * (double)m / N);
    }
    for (int j = 0; j <= N / 2; ++j) hsd[j] = 0.5 * sin(M_PI * (double)j / N);
    hsd[N / 2] = 0.5;
    std::vector<double> tpd;
    make_tp_table(N, tpd);
    const size_t ntp = tpd.size();
    if (ntp) {
      if (o.precision != CSL_PREC_FP64) {
        std::vector<float> tpf(ntp);
        for (size_t i = 0; i < ntp; ++i) tpf[i] = (float)tpd[i];
        err = cudaMemcpy(P->tp[d], tpf.data(), ntp * 4, cudaMemcpyHostToDevice);
      } else {
        err = cudaMemcpy(P->tp[d], tpd.data(), ntp * 8, cudaMemcpyHostToDevice);
      }
      if (err != cudaSuccess) break;
    }
    err = cudaMemcpy(P->mu_d[d], mu.data(), nd * 8, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(P->mu_f[d], muf.data(), nd * 4, cudaMemcpyHostToDevice);
    if (o.precision != CSL_PREC_FP64) {
      std::vector<float> twf(N), hsf(N / 2 + 1);
      for (int i = 0; i < N; ++i) twf[i] = (float)twd[i];
      for (int j = 0; j <= N / 2; ++j) hsf[j] = (float)hsd[j];
      if (err == cudaSuccess) err = cudaMemcpy(P->tw[d], twf.data(), N * 4, cudaMemcpyHostToDevice);
      if (err == cudaSuccess) err = cudaMemcpy(P->hs[d], hsf.data(), (N / 2 + 1) * 4, cudaMemcpyHostToDevice);
    } else {
      if (err == cudaSuccess) err = cudaMemcpy(P->tw[d], twd.data(), N * 8, cudaMemcpyHostToDevice);
      if (err == cudaSuccess) err = cudaMemcpy(P->hs[d], hsd.data(), (N / 2 + 1) * 8, cudaMemcpyHostToDevice);
    }
  }
  // per-mode scale of P^{-1} (Eq. 4) and the extremes of its eigenvalues
  if (err == cudaSuccess) {
    unsigned long long init[2] = {~0ull, 0ull};
    err = cudaMemcpyAsync(P->u64, init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) {
      if (dim == 2)
        k_scale_table<2><<<P->ew_blocks, 256, 0, s>>>(g, P->mu_d[0], P->mu_d[1], nullptr, P->gamma, alpha, beta,
                                                      P->cnorm, P->stab, P->u64);
      else
        k_scale_table<3><<<P->ew_blocks, 256, 0, s>>>(g, P->mu_d[0], P->mu_d[1], P->mu_d[2], P->gamma, alpha,
                                                      beta, P->cnorm, P->stab, P->u64);
      err = cudaGetLastError();
    }
    unsigned long long res[2] = {0, 0};
    if (err == cudaSuccess) err = cudaMemcpyAsync(res, P->u64, sizeof(res), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(P->st, 0, sizeof(DevState), s);
    if (err == cudaSuccess && P->hist) {  // the history buffer, once per plan (the ingest leaves it alone)
      DevState hs;
      memset(&hs, 0, sizeof(hs));
      hs.hist = P->hist;
      hs.hist_cap = P->hist_cap;
      err = cudaMemcpyAsync(P->st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, s);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess) {
      double qmin, qmax;
      memcpy(&qmin, &res[0], 8);
      memcpy(&qmax, &res[1], 8);
      if (!(qmin > 0.0)) {
        free_plan(P);
        return CSL_SINGULAR_PRECOND;
      }
      P->sqrt_pmin = sqrt(sqrt(qmin));
      P->sqrt_pmax = sqrt(sqrt(qmax));
      if (o.precision != CSL_PREC_FP64) {
        // FP32 scale: |e + i beta| is brought to at most 2^40 when it leaves
        // [2^-40, 2^60]; the scales s_k themselves must be normal floats
        const double mmin = sqrt(qmin), mmax = sqrt(qmax);
        if (mmax > ldexp(1.0, 60) || mmin < ldexp(1.0, -40)) P->sigma = ldexp(1.0, 40 - (int)ceil(log2(mmax)));
        const double smin = P->cnorm / mmax, smax = P->cnorm / mmin;
        if (!(smin >= ldexp(1.0, -120)) || !(smax <= ldexp(1.0, 120)) ||
            !(mmin * P->sigma >= ldexp(1.0, -60))) {
          csl_internal_set_error(
              "csl_plan_create: the per-mode scales of P^-1 lie outside the FP32 range; use CSL_PREC_FP64");
          free_plan(P);
          return CSL_INVALID_ARG;
        }
      }
    }
  }
  if (err != cudaSuccess) {
    CSL_NOTE(err, "table / scale set-up");
    (void)cudaGetLastError();
    free_plan(P);
    return CSL_CUDA_ERROR;
  }
  // launch configurations of the sine-transform passes
  const long nrows = M / nx;
  if (o.precision != CSL_PREC_FP64) {
    config_row<float>(P->row, nx, (int)nrows);
    if (dim == 2) {
      config_strided<float>(P->sy, ny, nx, 1, 0, nx, o.lines_per_cta);
    } else {
      config_strided<float>(P->sy, ny, nx, nz, (long)nx * ny, nx, o.lines_per_cta);
      config_strided<float>(P->sz, nz, nx, ny, nx, (long)nx * ny, o.lines_per_cta);
    }
  } else {
    config_row<double>(P->row, nx, (int)nrows);
    if (dim == 2) {
      config_strided<double>(P->sy, ny, nx, 1, 0, nx, o.lines_per_cta);
    } else {
      config_strided<double>(P->sy, ny, nx, nz, (long)nx * ny, nx, o.lines_per_cta);
      config_strided<double>(P->sz, nz, nx, ny, nx, (long)nx * ny, o.lines_per_cta);
    }
  }
  // split-BF16 tensor-core variant of the strided passes (lines of N <= 128)
  if (o.precision == CSL_PREC_BF16X3 || o.precision == CSL_PREC_BF16X6) {
    P->tc_split = o.precision == CSL_PREC_BF16X3 ? 2 : 3;
    PassCfg* sc[3] = {nullptr, &P->sy, &P->sz};
    for (int d = 1; d < dim && err == cudaSuccess; ++d) {
      PassCfg& c = *sc[d];
      if (!tc_supported(c.N)) continue;
      const bool mid = (d == dim - 1);
      void* img_dev = nullptr;
      for (int e2 = 1; e2 < d; ++e2)
        if (P->sine_tc[e2] && sc[e2]->N == c.N) img_dev = P->sine_tc[e2];
      if (!img_dev) {
        std::vector<uint16_t> img;
        build_sine_image(c.N, P->tc_split, img);
        img_dev = dalloc(P, img.size() * sizeof(uint16_t), &err);
        if (err == cudaSuccess)
          err = cudaMemcpy(img_dev, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
      }
      P->sine_tc[d] = img_dev;
      const long tiles = (long)((c.ncols + 63) / 64) * c.nouter;
      long cap = (long)kSMs * tc_ctas_per_sm(c.N, P->tc_split, mid);
      if (cap > kMaxRedBlocks) cap = kMaxRedBlocks;
      c.L.blocks = (int)(tiles < cap ? tiles : cap);
      c.L.threads = 256;
      c.L.smem = tc_smem_bytes(c.N, P->tc_split);
      c.L.tc = P->tc_split;
      c.lines = 64;
      c.wide = 0;
    }
    if (err != cudaSuccess) {
      CSL_NOTE(err, "tensor-core sine tables");
      (void)cudaGetLastError();
      free_plan(P);
      return CSL_CUDA_ERROR;
    }
  }
  P->row.L.pdl = P->sy.L.pdl = P->sz.L.pdl = P->use_pdl;
  if (o.autotune && o.lines_per_cta <= 0) {
    // (the chosen shapes are described in P->config below)
    err = o.precision != CSL_PREC_FP64 ? autotune<float>(P) : autotune<double>(P);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
      CSL_NOTE(err, "autotune");
      (void)cudaGetLastError();
      free_plan(P);
      return CSL_CUDA_ERROR;
    }
  }
  {
    const PassCfg* cs[3] = {&P->row, &P->sy, &P->sz};
    const char* nm[3] = {"x", "y", "z"};
    const char* pname = o.precision == CSL_PREC_FP64            ? "fp64"
                        : o.precision == CSL_PREC_FP32          ? "fp32"
                        : o.precision == CSL_PREC_FP32_PRECOND  ? "fp32-precond"
                        : o.precision == CSL_PREC_BF16X3        ? "bf16x3"
                                                                : "bf16x6";
    int off = snprintf(P->config, sizeof(P->config), "%s%s stencil[%s strip=%d blocks=%d]", pname,
                       o.autotune ? " autotuned" : "", P->ff ? "float-pair" : "fp64", P->sten_strip, P->sten_blocks);
    for (int d = 0; d < dim && off < (int)sizeof(P->config); ++d)
      off += snprintf(P->config + off, sizeof(P->config) - off, " %s[N=%d %s lines=%d threads=%d blocks=%d smem=%zu]",
                      nm[d], cs[d]->N,
                      cs[d]->L.tc == 2   ? "tcgen05-bf16x3"
                      : cs[d]->L.tc == 3 ? "tcgen05-bf16x6"
                      : cs[d]->wide == 4 ? "cluster2"
                      : cs[d]->wide == 3 ? "long-line"
                      : cs[d]->wide == 2 ? "stockham128"
                      : cs[d]->wide == 1 ? "stockham64"
                                         : "warp",
                      cs[d]->lines, cs[d]->L.threads, cs[d]->L.blocks, cs[d]->L.smem);
  }
  *out = P;
  return CSL_OK;
}

const char* csl_plan_config(const csl_plan* plan) { return plan ? plan->config : ""; }

csl_status csl_tune_cache_save(const char* path) {
  if (!path) return CSL_INVALID_ARG;
  FILE* fh = fopen(path, "w");
  if (!fh) {
    csl_internal_set_error("csl_tune_cache_save: cannot open the file for writing");
    return CSL_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  fprintf(fh, "%s\n", kTuneHeader);
  for (const auto& kv : g_tune_cache)
    fprintf(fh, "%d %d %d %d %d %d %d\n", kv.first.prec, kv.first.kind, kv.first.N, kv.first.ncols,
            kv.first.nouter, kv.second.wide, kv.second.lines);
  const int bad = ferror(fh);
  fclose(fh);
  return bad ? CSL_INVALID_ARG : CSL_OK;
}

csl_status csl_tune_cache_load(const char* path) {
  if (!path) return CSL_INVALID_ARG;
  FILE* fh = fopen(path, "r");
  if (!fh) {
    csl_internal_set_error("csl_tune_cache_load: cannot open the file");
    return CSL_INVALID_ARG;
  }
  char line[256];
  if (!fgets(line, sizeof(line), fh) || strncmp(line, kTuneHeader, strlen(kTuneHeader)) != 0) {
    fclose(fh);
    csl_internal_set_error("csl_tune_cache_load: not a csl tuner cache file");
    return CSL_INVALID_ARG;
  }
  std::vector<std::pair<TuneKey, PassCfg>> entries;
  while (fgets(line, sizeof(line), fh)) {
    TuneKey k;
    int wide = 0, lines = 0;
    if (sscanf(line, "%d %d %d %d %d %d %d", &k.prec, &k.kind, &k.N, &k.ncols, &k.nouter, &wide, &lines) != 7 ||
        !tune_entry_valid(k, wide, lines)) {
      fclose(fh);
      csl_internal_set_error("csl_tune_cache_load: malformed entry; nothing was loaded");
      return CSL_INVALID_ARG;
    }
    PassCfg c;
    c.N = k.N;
    c.wide = wide;
    c.lines = lines;
    entries.push_back({k, c});
  }
  fclose(fh);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& e : entries) g_tune_cache[e.first] = e.second;
  return CSL_OK;
}

void csl_plan_destroy(csl_plan* plan) {
  if (!plan) return;
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
}

csl_status csl_plan_set_stream(csl_plan* plan, void* stream) {
  if (!plan) return CSL_INVALID_ARG;
  plan->stream = (cudaStream_t)stream;
  return CSL_OK;
}

size_t csl_plan_workspace_bytes(const csl_plan* plan) { return plan ? plan->bytes : 0; }

double csl_plan_gamma(const csl_plan* plan) { return plan ? plan->gamma : kNaN; }

csl_status csl_apply(csl_plan* P, const double* z, double* out) {
  if (!P || !z || !out) return CSL_INVALID_ARG;
  NvtxRange r("csl_apply");
  Grid g;
  g.nx = P->n[0];
  g.ny = P->n[1];
  g.nz = P->dim == 3 ? P->n[2] : 1;
  g.M = P->M;
  if (P->dim == 2)
    k_apply<2><<<P->ew_blocks, 256, 0, P->stream>>>(g, (const double2*)z, (double2*)out, P->cx, P->cy, P->cz,
                                                    P->dg, P->beta);
  else
    k_apply<3><<<P->ew_blocks, 256, 0, P->stream>>>(g, (const double2*)z, (double2*)out, P->cx, P->cy, P->cz,
                                                    P->dg, P->beta);
  CSL_TRY(cudaGetLastError());
  return CSL_OK;
}

csl_status csl_precondition(csl_plan* P, const double* v, double* out) {
  if (!P || !v || !out) return CSL_INVALID_ARG;
  NvtxRange r("csl_precondition");
  if (P->precision != CSL_PREC_FP64)
    CSL_TRY(launch_precondition_T<float>(P, (const double2*)v, (double2*)out, P->stream));
  else
    CSL_TRY(launch_precondition_T<double>(P, (const double2*)v, (double2*)out, P->stream));
  return CSL_OK;
}

csl_status csl_solve(csl_plan* P, const double* f, double* z, double tol, int maxit, csl_solve_info* info) {
  if (!P || !f || !z) return CSL_INVALID_ARG;
  NvtxRange r("csl_solve");
  csl_status s = solve_impl(P, (const double2*)f, tol, maxit, P->beta, (const double2*)z);
  if (s != CSL_OK) return s;
  CSL_TRY(copy_out(P, (double2*)z, P->stream));
  csl_status st = CSL_OK;
  s = read_info(P, info, &st);
  return s != CSL_OK ? s : st;
}

csl_status csl_adjoint(csl_plan* P, const double* g, double* y, double tol, int maxit, csl_solve_info* info) {
  if (!P || !g || !y) return CSL_INVALID_ARG;
  NvtxRange r("csl_adjoint");
  csl_status s = solve_impl(P, (const double2*)g, tol, maxit, -P->beta, (const double2*)y);
  if (s != CSL_OK) return s;
  CSL_TRY(copy_out(P, (double2*)y, P->stream));
  csl_status st = CSL_OK;
  s = read_info(P, info, &st);
  return s != CSL_OK ? s : st;
}

csl_status csl_solve_host(csl_plan* P, const double* f_host, double* z_host, double tol, int maxit,
                          csl_solve_info* info) {
  if (!P || !f_host || !z_host) return CSL_INVALID_ARG;
  if (!(tol > 0.0) || maxit < 1) return CSL_INVALID_ARG;
  const size_t bytes = sizeof(double2) * P->M;
  NvtxRange r("csl_solve_host");
  CSL_TRY(cudaMemcpyAsync(P->io, f_host, bytes, cudaMemcpyHostToDevice, P->stream));
  if (P->warm) CSL_TRY(cudaMemcpyAsync(P->x0, z_host, bytes, cudaMemcpyHostToDevice, P->stream));
  csl_status s = solve_impl(P, P->io, tol, maxit, P->beta, P->x0);
  if (s != CSL_OK) return s;
  CSL_TRY(copy_out(P, P->io, P->stream));  // f is no longer needed
  CSL_TRY(cudaMemcpyAsync(z_host, P->io, bytes, cudaMemcpyDeviceToHost, P->stream));
  csl_status st = CSL_OK;
  s = read_info(P, info, &st);
  return s != CSL_OK ? s : st;
}

csl_status csl_solve_history(csl_plan* P, double* out_host, int cap, int* count) {
  if (!P || !out_host || !count || cap < 0) return CSL_INVALID_ARG;
  *count = 0;
  if (!P->hist) return CSL_INVALID_ARG;
  DevState h;
  CSL_TRY(cudaMemcpyAsync(&h, P->st, sizeof(DevState), cudaMemcpyDeviceToHost, P->stream));
  CSL_TRY(cudaStreamSynchronize(P->stream));
  int n = h.iter < P->hist_cap ? h.iter : P->hist_cap;
  if (n > cap) n = cap;
  if (n > 0) {
    CSL_TRY(cudaMemcpyAsync(out_host, P->hist, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream));
    CSL_TRY(cudaStreamSynchronize(P->stream));
  }
  *count = n;
  return CSL_OK;
}

csl_status csl_coef_grad(csl_plan* P, const double* z, const double* y, double* const grad_faces[3]) {
  if (!P || !z || !y || !grad_faces) return CSL_INVALID_ARG;
  for (int d = 0; d < P->dim; ++d)
    if (!grad_faces[d]) return CSL_INVALID_ARG;
  Grid g;
  g.nx = P->n[0];
  g.ny = P->n[1];
  g.nz = P->dim == 3 ? P->n[2] : 1;
  g.M = P->M;
  const double2* zz = (const double2*)z;
  const double2* yy = (const double2*)y;
  const int blocks = P->ew_blocks;
  k_coef_grad<0><<<blocks, 256, 0, P->stream>>>(g, zz, yy, grad_faces[0], 1.0 / (P->h[0] * P->h[0]));
  k_coef_grad<1><<<blocks, 256, 0, P->stream>>>(g, zz, yy, grad_faces[1], 1.0 / (P->h[1] * P->h[1]));
  if (P->dim == 3)
    k_coef_grad<2><<<blocks, 256, 0, P->stream>>>(g, zz, yy, grad_faces[2], 1.0 / (P->h[2] * P->h[2]));
  CSL_TRY(cudaGetLastError());
  return CSL_OK;
}

csl_status csl_time_kernels(csl_plan* P, int reps, double ms[8], const char* names[8], int* count) {
  if (!P || !ms || !names || !count || reps < 1 || reps > 1000) return CSL_INVALID_ARG;
  *count = 0;
  const DevState h = scratch_state(P);
  DevState* keep = P->st;
  P->st = P->st_prof;  // all launches below read the scratch state
  const int nkb = P->dim == 2 ? 4 : 6;  // kernels of the main chain
  const int nk = iteration_kernels(P);
  static const char* n2[5] = {"k_stencil", "k_row<LOAD_LANCZOS,STORE_T>", "k_strided<mid>",
                              "k_row<LOAD_T,STORE_Z_UPDATE>", "k_update"};
  static const char* n3[7] = {"k_stencil", "k_row<LOAD_LANCZOS,STORE_T>", "k_strided<y>", "k_strided<mid>",
                              "k_strided<y>(inverse)", "k_row<LOAD_T,STORE_Z_UPDATE>", "k_update"};
  static const char* p3split = "k_row<LOAD_T,STORE_Z>";
  std::vector<cudaEvent_t> ev((size_t)(reps + 1) * (nk + 1), nullptr);
  cudaError_t err = cudaMemcpyAsync(P->st_prof, &h, sizeof(h), cudaMemcpyHostToDevice, P->stream);
  for (size_t i = 0; i < ev.size() && err == cudaSuccess; ++i) err = cudaEventCreate(&ev[i]);
  if (err == cudaSuccess) err = time_sequence(P, reps, 2, ev.data(), ms);
  // the scratch run must not have ended (a breakdown would let kernels exit at entry)
  DevState after;
  if (err == cudaSuccess) err = cudaMemcpyAsync(&after, P->st_prof, sizeof(after), cudaMemcpyDeviceToHost, P->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(P->stream);
  P->st = keep;
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (err != cudaSuccess) {
    record_error(err, "csl_time_kernels", __LINE__);
    (void)cudaGetLastError();
    return CSL_CUDA_ERROR;
  }
  if (after.done) {
    csl_internal_set_error("csl_time_kernels: the scratch iteration ended early; the timings are not valid");
    return CSL_BREAKDOWN;
  }
  for (int k = 0; k < nk; ++k) names[k] = (P->split_update && k == nkb - 1) ? p3split : P->dim == 2 ? n2[k] : n3[k];
  *count = nk;
  return CSL_OK;
}

}  // extern "C"

// ============================================================================
// Batched solves: many independent systems (shifts lambda_k, and grids of
// different sizes) in one graph launch.  Systems of the same grid form a group;
// each kernel of an iteration is launched once per group with a device array
// of per-system arguments (system = blockIdx / blocks-per-system), so a group
// of small grids fills the GPU.  Groups run on parallel branches of the
// graph; a one-CTA control kernel closes the WHILE node once every system has
// met its stopping test (or an integer iteration cap is reached).  Converged
// systems' CTAs exit at entry.
// ============================================================================
namespace {

struct BatchGroup {
  int n[3] = {1, 1, 1};
  std::vector<int> sys;  // indices of the group's systems
  csl_plan* proto = nullptr;
  int ff = 1;  // all systems of the group take the float-pair stencil
  StencilArgs* d_sten[2] = {nullptr, nullptr};
  void* d_p1[2] = {nullptr, nullptr};   // RowArgs<T>
  void* d_p3[2] = {nullptr, nullptr};   // RowArgs<T>
  void* d_mid = nullptr;                // StridedArgs<T> (mid pass, iteration)
  void* d_y = nullptr;                  // StridedArgs<T> (3D y pass)
  IngestArgs* d_ing = nullptr;
  void* d_pro1 = nullptr;               // RowArgs<T> prologue x-fwd
  void* d_pro_mid = nullptr;            // StridedArgs<T> prologue mid (scalar mode 1)
  void* d_pro3 = nullptr;               // RowArgs<T> prologue x-inv -> z[0]
  std::vector<IngestArgs> h_ing;
  cudaStream_t branch = nullptr;
  cudaEvent_t ev = nullptr;
};

// loops[0]: WHILE bodies run so far; loops[1]: cap on them (set per solve)
__global__ void k_batch_control(DevState* states, int nsys, int* loops, cudaGraphConditionalHandle cond) {
  __shared__ int remaining;
  if (threadIdx.x == 0) remaining = 0;
  __syncthreads();
  int mine = 0;
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) mine += states[s].done ? 0 : 1;
  atomicAdd(&remaining, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int l = ++loops[0];
    cudaGraphSetConditional(cond, (remaining > 0 && l <= loops[1]) ? 1u : 0u);
  }
}

// egress of a batch: x of every system to its z (pairs = FP32 forms, x held as float pairs)
__global__ void k_batch_copy(const double2* const* src, double2* const* dst, const long* count, int pairs) {
  const int s = blockIdx.y;
  const double2* a = src[s];
  double2* b = dst[s];
  const long M = count[s];
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (long)gridDim.x * blockDim.x)
    b[i] = pairs ? to_d2(((const float4*)a)[i]) : a[i];
}

}  // namespace

struct csl_batch {
  int nsys = 0, precision = CSL_PREC_FP64, dim = 2;
  std::vector<csl_plan*> plans;
  std::vector<BatchGroup> groups;
  DevState* states = nullptr;
  int* d_loops = nullptr;
  int h_loops[2] = {0, 0};
  const double2** d_src = nullptr;
  double2** d_dst = nullptr;
  long* d_count = nullptr;
  long maxM = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int graph_state = 0;
  std::vector<void*> allocs;
  size_t bytes = 0;
};

namespace {

cudaError_t balloc(csl_batch* B, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    B->allocs.push_back(*p);
    B->bytes += bytes;
  }
  return e;
}

template <typename A>
cudaError_t upload_array(csl_batch* B, void** d, const std::vector<A>& h) {
  cudaError_t e = balloc(B, d, sizeof(A) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), sizeof(A) * h.size(), cudaMemcpyHostToDevice);
  return e;
}

void free_batch(csl_batch* B) {
  if (!B) return;
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto& g : B->groups) {
    if (g.branch) cudaStreamDestroy(g.branch);
    if (g.ev) cudaEventDestroy(g.ev);
  }
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->cap) cudaStreamDestroy(B->cap);
  for (void* p : B->allocs) cudaFree(p);
  for (csl_plan* P : B->plans) free_plan(P);
  delete B;
}

// per-system argument arrays of one group
template <typename T>
cudaError_t build_group_args(csl_batch* B, BatchGroup& G) {
  const int ns = (int)G.sys.size();
  cudaError_t e = cudaSuccess;
  for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
    std::vector<StencilArgs> sa(ns);
    std::vector<RowArgs<T>> p1(ns), p3(ns);
    for (int i = 0; i < ns; ++i) {
      csl_plan* P = B->plans[G.sys[i]];
      StencilArgs a = stencil_args(P, par);
      a.use_cond = 0;
      sa[i] = a;
      if (!P->ff) G.ff = 0;
      p1[i] = p1_args<T>(P, par);
      p3[i] = p3_args<T>(P, par);
    }
    e = upload_array(B, (void**)&G.d_sten[par], sa);
    if (e == cudaSuccess) e = upload_array(B, &G.d_p1[par], p1);
    if (e == cudaSuccess) e = upload_array(B, &G.d_p3[par], p3);
  }
  std::vector<StridedArgs<T>> mid(ns), y(ns), pmid(ns);
  std::vector<RowArgs<T>> pro1(ns), pro3(ns);
  G.h_ing.resize(ns);
  for (int i = 0; i < ns && e == cudaSuccess; ++i) {
    csl_plan* P = B->plans[G.sys[i]];
    const int ax = P->dim == 2 ? 1 : 2;
    const PassCfg& cm = P->dim == 2 ? P->sy : P->sz;
    StridedArgs<T> m = strided_args<T>(P, cm, ax);
    fill_mid<T>(P, m, ax);
    m.st = P->st;
    m.scalar_mode = 2;
    mid[i] = m;
    m.scalar_mode = 1;
    pmid[i] = m;
    StridedArgs<T> yy = strided_args<T>(P, P->sy, 1);
    yy.st = P->st;
    y[i] = yy;
    RowArgs<T> r1 = row_args<T>(P);
    r1.vin = P->b;  // v_1 = b
    r1.tout = (typename C2<T>::t*)P->T;
    r1.st = P->st;
    pro1[i] = r1;
    RowArgs<T> r3 = row_args<T>(P);
    r3.tin = (const typename C2<T>::t*)P->T;
    r3.zout = (typename C2<T>::t*)P->z[0];
    r3.st = P->st;
    pro3[i] = r3;
    IngestArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.M = P->M;
    ia.b = P->b;
    ia.v0 = P->v[0];
    ia.v1 = P->v[1];
    ia.w0 = P->w[0];
    ia.w1 = P->w[1];
    ia.x = P->x;
    ia.st = P->st;
    ia.partials = P->partials;
    ia.sqrt_pmin = P->sqrt_pmin;
    ia.sqrt_pmax = P->sqrt_pmax;
    ia.beta = P->beta;
    ia.vpair = P->vpair;
    G.h_ing[i] = ia;
  }
  if (e == cudaSuccess) e = upload_array(B, &G.d_mid, mid);
  if (e == cudaSuccess) e = upload_array(B, &G.d_y, y);
  if (e == cudaSuccess) e = upload_array(B, &G.d_pro_mid, pmid);
  if (e == cudaSuccess) e = upload_array(B, &G.d_pro1, pro1);
  if (e == cudaSuccess) e = upload_array(B, &G.d_pro3, pro3);
  if (e == cudaSuccess) e = upload_array(B, (void**)&G.d_ing, G.h_ing);
  return e;
}

// P^{-1} chain of a group after the x pass: [y fwd,] mid, [y inv]
template <typename T>
cudaError_t group_mid_chain(csl_batch* B, BatchGroup& G, cudaStream_t s, const void* d_mid) {
  csl_plan* P = G.proto;
  const int ns = (int)G.sys.size();
  StridedArgs<T> dummy;
  memset(&dummy, 0, sizeof(dummy));
  if (P->dim == 2)
    return launch_strided<T>(P->sy.N, P->sy.wide, true, dummy, P->sy.L, s, (const StridedArgs<T>*)d_mid, ns);
  cudaError_t e =
      launch_strided<T>(P->sy.N, P->sy.wide, false, dummy, P->sy.L, s, (const StridedArgs<T>*)G.d_y, ns);
  if (e == cudaSuccess)
    e = launch_strided<T>(P->sz.N, P->sz.wide, true, dummy, P->sz.L, s, (const StridedArgs<T>*)d_mid, ns);
  if (e == cudaSuccess)
    e = launch_strided<T>(P->sy.N, P->sy.wide, false, dummy, P->sy.L, s, (const StridedArgs<T>*)G.d_y, ns);
  return e;
}

template <typename T>
cudaError_t group_iteration(csl_batch* B, BatchGroup& G, int par, cudaStream_t s) {
  csl_plan* P = G.proto;
  const int ns = (int)G.sys.size();
  typedef typename C2<T>::t TZ;
  StencilArgs sd;
  memset(&sd, 0, sizeof(sd));
  const StencilArgs* sb = (const StencilArgs*)G.d_sten[par];
  const size_t smem = (sizeof(TZ) == 8 && G.ff) ? ff_stencil_smem(P->dim) : 0;
  cudaError_t e = launch_k(P->use_pdl != 0, stencil_fn<TZ>(P->dim, G.ff != 0, P->vpair != 0), P->sten_blocks * ns, 256,
                           smem, s,
                           sd, sb, P->sten_blocks);
  RowArgs<T> rd;
  memset(&rd, 0, sizeof(rd));
  if (e == cudaSuccess)
    e = launch_row<T>(P->row.N, P->row.wide, lanczos_load(P), STORE_T, rd, P->row.L, s,
                      (const RowArgs<T>*)G.d_p1[par], ns);
  if (e == cudaSuccess) e = group_mid_chain<T>(B, G, s, G.d_mid);
  if (e == cudaSuccess)
    e = launch_row<T>(P->row.N, P->row.wide, LOAD_T, update_store(P), rd, P->row.L, s,
                      (const RowArgs<T>*)G.d_p3[par], ns);
  return e;
}

template <typename T>
cudaError_t group_prologue(csl_batch* B, BatchGroup& G, cudaStream_t s) {
  csl_plan* P = G.proto;
  const int ns = (int)G.sys.size();
  IngestArgs id;
  memset(&id, 0, sizeof(id));
  k_ingest<<<P->ew_blocks * ns, 256, 0, s>>>(id, G.d_ing, P->ew_blocks);
  cudaError_t e = cudaGetLastError();
  RowArgs<T> rd;
  memset(&rd, 0, sizeof(rd));
  if (e == cudaSuccess)
    e = launch_row<T>(P->row.N, P->row.wide, LOAD_V, STORE_T, rd, P->row.L, s, (const RowArgs<T>*)G.d_pro1, ns);
  if (e == cudaSuccess) e = group_mid_chain<T>(B, G, s, G.d_pro_mid);
  if (e == cudaSuccess)
    e = launch_row<T>(P->row.N, P->row.wide, LOAD_T, STORE_Z, rd, P->row.L, s, (const RowArgs<T>*)G.d_pro3, ns);
  return e;
}

template <typename T>
void build_batch_graph(csl_batch* B) {
  if (B->graph_state != 0) return;
  B->graph_state = -1;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&B->cond, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    cp.conditional.handle = B->cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaEventRecord(B->ev_fork, B->cap);
      for (auto& G : B->groups) {
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(G.branch, B->ev_fork, 0);
        for (int par = 0; par < 2 && e1 == cudaSuccess; ++par) e1 = group_iteration<T>(B, G, par, G.branch);
        if (e1 == cudaSuccess) e1 = cudaEventRecord(G.ev, G.branch);
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(B->cap, G.ev, 0);
      }
      if (e1 == cudaSuccess) {
        k_batch_control<<<1, 256, 0, B->cap>>>(B->states, B->nsys, B->d_loops, B->cond);
        e1 = cudaGetLastError();
      }
      cudaGraph_t captured = body;
      e = cudaStreamEndCapture(B->cap, &captured);
      if (e == cudaSuccess) e = e1;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->gexec, g, 0);
  if (e != cudaSuccess) {
    CSL_NOTE(e, "batch graph build");
    (void)cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    B->gexec = nullptr;
    return;
  }
  B->graph = g;
  B->graph_state = 1;
}

template <typename T>
csl_status batch_solve_T(csl_batch* B, const double* const* f, double* const* z, double tol, int maxit,
                         csl_solve_info* infos) {
  cudaStream_t s = B->stream;
  // per-call inputs: right-hand side pointers and the stopping parameters
  for (auto& G : B->groups) {
    for (size_t i = 0; i < G.sys.size(); ++i) {
      IngestArgs& ia = G.h_ing[i];
      ia.f = (const double2*)f[G.sys[i]];
      ia.tol = tol;
      ia.maxit = maxit;
    }
    CSL_TRY(cudaMemcpyAsync(G.d_ing, G.h_ing.data(), sizeof(IngestArgs) * G.h_ing.size(), cudaMemcpyHostToDevice, s));
    CSL_TRY(group_prologue<T>(B, G, s));
  }
  build_batch_graph<T>(B);
  B->h_loops[0] = 0;
  B->h_loops[1] = maxit / 2 + 4;
  CSL_TRY(cudaMemcpyAsync(B->d_loops, B->h_loops, sizeof(B->h_loops), cudaMemcpyHostToDevice, s));
  if (B->graph_state == 1) {
    CSL_TRY(cudaGraphLaunch(B->gexec, s));
  } else {
    int done = 0;
    for (int it = 0; it < maxit + 4 && !done; it += 8) {
      for (int k = 0; k < 8; ++k)
        for (auto& G : B->groups) CSL_TRY(group_iteration<T>(B, G, k & 1, s));
      std::vector<DevState> h(B->nsys);
      CSL_TRY(cudaMemcpyAsync(h.data(), B->states, sizeof(DevState) * B->nsys, cudaMemcpyDeviceToHost, s));
      CSL_TRY(cudaStreamSynchronize(s));
      done = 1;
      for (auto& st : h) done &= st.done;
    }
  }
  // egress: x of every system to its z
  std::vector<const double2*> src(B->nsys);
  std::vector<double2*> dst(B->nsys);
  std::vector<long> cnt(B->nsys);
  for (int i = 0; i < B->nsys; ++i) {
    src[i] = B->plans[i]->x;
    dst[i] = (double2*)z[i];
    cnt[i] = B->plans[i]->M;
  }
  CSL_TRY(cudaMemcpyAsync(B->d_src, src.data(), sizeof(void*) * B->nsys, cudaMemcpyHostToDevice, s));
  CSL_TRY(cudaMemcpyAsync(B->d_dst, dst.data(), sizeof(void*) * B->nsys, cudaMemcpyHostToDevice, s));
  CSL_TRY(cudaMemcpyAsync(B->d_count, cnt.data(), sizeof(long) * B->nsys, cudaMemcpyHostToDevice, s));
  dim3 grid((unsigned)((B->maxM + 255) / 256 < 256 ? (B->maxM + 255) / 256 : 256), (unsigned)B->nsys);
  k_batch_copy<<<grid, 256, 0, s>>>(B->d_src, B->d_dst, B->d_count, B->plans[0]->vpair);
  CSL_TRY(cudaGetLastError());
  std::vector<DevState> h(B->nsys);
  CSL_TRY(cudaMemcpyAsync(h.data(), B->states, sizeof(DevState) * B->nsys, cudaMemcpyDeviceToHost, s));
  CSL_TRY(cudaStreamSynchronize(s));
  csl_status worst = CSL_OK;
  for (int i = 0; i < B->nsys; ++i) {
    const csl_status st = h[i].done ? (csl_status)h[i].status : CSL_NOT_CONVERGED;
    if (st != CSL_OK && worst == CSL_OK) worst = st;
    if (infos) {
      memset(&infos[i], 0, sizeof(csl_solve_info));
      infos[i].iters = h[i].iter;
      infos[i].status = (int)st;
      infos[i].relres = h[i].relres;
      infos[i].pnorm = h[i].eta_x;
      infos[i].gamma = B->plans[i]->gamma;
      infos[i].checks = h[i].checks;
    }
  }
  return worst;
}

}  // namespace

extern "C" {

csl_status csl_batch_create(csl_batch** out, int nsys, const csl_system_desc* sys, const csl_plan_options* opt,
                            void* stream) {
  if (!out || nsys < 1 || !sys) return CSL_INVALID_ARG;
  *out = nullptr;
  csl_plan_options o;
  csl_plan_options_init(&o);
  if (opt) o = *opt;
  for (int i = 0; i < nsys; ++i)
    if (sys[i].dim != sys[0].dim) return CSL_INVALID_ARG;
  if (o.warm_start || o.history) return CSL_INVALID_ARG;  // single plans only
  NvtxRange nv("csl_batch_create");
  csl_batch* B = new (std::nothrow) csl_batch();
  if (!B) return CSL_OUT_OF_MEMORY;
  B->nsys = nsys;
  B->precision = o.precision;
  B->dim = sys[0].dim;
  B->stream = (cudaStream_t)stream;
  // one plan per system (its workspace and tables); shapes are tuned once per
  // grid size (the tuner's cache) and shared by the group
  for (int i = 0; i < nsys; ++i) {
    csl_plan* P = nullptr;
    const csl_status st = csl_plan_create(&P, sys[i].dim, sys[i].n, sys[i].coef_faces, sys[i].alpha, sys[i].beta,
                                          &o, stream);
    if (st != CSL_OK) {
      free_batch(B);
      return st;
    }
    B->plans.push_back(P);
    B->maxM = P->M > B->maxM ? P->M : B->maxM;
  }
  cudaError_t e = balloc(B, (void**)&B->states, sizeof(DevState) * nsys);
  if (e == cudaSuccess) e = cudaMemset(B->states, 0, sizeof(DevState) * nsys);
  if (e == cudaSuccess) e = balloc(B, (void**)&B->d_loops, 2 * sizeof(int));
  if (e == cudaSuccess) e = balloc(B, (void**)&B->d_src, sizeof(void*) * nsys);
  if (e == cudaSuccess) e = balloc(B, (void**)&B->d_dst, sizeof(void*) * nsys);
  if (e == cudaSuccess) e = balloc(B, (void**)&B->d_count, sizeof(long) * nsys);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
  // the systems' scalar states live side by side so one copy reads them all
  for (int i = 0; i < nsys; ++i) B->plans[i]->st = B->states + i;
  // groups: systems with the same grid
  for (int i = 0; i < nsys && e == cudaSuccess; ++i) {
    csl_plan* P = B->plans[i];
    BatchGroup* G = nullptr;
    for (auto& g : B->groups)
      if (g.n[0] == P->n[0] && g.n[1] == P->n[1] && g.n[2] == P->n[2]) G = &g;
    if (!G) {
      B->groups.emplace_back();
      G = &B->groups.back();
      for (int d = 0; d < 3; ++d) G->n[d] = P->n[d];
      G->proto = P;
    }
    G->sys.push_back(i);
  }
  for (auto& G : B->groups) {
    // the group shares its prototype's launch shapes
    for (int i : G.sys) {
      csl_plan* P = B->plans[i];
      P->row = G.proto->row;
      P->sy = G.proto->sy;
      P->sz = G.proto->sz;
      P->sten_blocks = G.proto->sten_blocks;
      P->ew_blocks = G.proto->ew_blocks;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.branch, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = o.precision != CSL_PREC_FP64 ? build_group_args<float>(B, G) : build_group_args<double>(B, G);
  }
  if (e != cudaSuccess) {
    CSL_NOTE(e, "csl_batch_create");
    (void)cudaGetLastError();
    free_batch(B);
    return e == cudaErrorMemoryAllocation ? CSL_OUT_OF_MEMORY : CSL_CUDA_ERROR;
  }
  *out = B;
  return CSL_OK;
}

csl_status csl_batch_solve(csl_batch* B, const double* const* f, double* const* z, double tol, int maxit,
                           csl_solve_info* infos) {
  if (!B || !f || !z || !(tol > 0.0) || maxit < 1) return CSL_INVALID_ARG;
  for (int i = 0; i < B->nsys; ++i)
    if (!f[i] || !z[i]) return CSL_INVALID_ARG;
  NvtxRange nv("csl_batch_solve");
  return B->precision != CSL_PREC_FP64 ? batch_solve_T<float>(B, f, z, tol, maxit, infos)
                                       : batch_solve_T<double>(B, f, z, tol, maxit, infos);
}

void csl_batch_destroy(csl_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  free_batch(B);
}

size_t csl_batch_workspace_bytes(const csl_batch* B) {
  if (!B) return 0;
  size_t t = B->bytes;
  for (csl_plan* P : B->plans) t += P->bytes;
  return t;
}

}  // extern "C"

// ---- test hooks (include/csl_testing.h) -------------------------------------
namespace {
__global__ void k_test_d2f(const double* in, float* out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = csl::d2f_rn(in[i]);
}
__global__ void k_test_f2d(const float* in, double* out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = csl::f2d_exact(in[i]);
}
}  // namespace

csl_status csl_test_convert_d2f(const double* in, float* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return CSL_INVALID_ARG;
  if (n == 0) return CSL_OK;
  const long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_test_d2f<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(in, out, (long)n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    CSL_NOTE(e, "csl_test_convert_d2f");
    return CSL_CUDA_ERROR;
  }
  return CSL_OK;
}

csl_status csl_test_convert_f2d(const float* in, double* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return CSL_INVALID_ARG;
  if (n == 0) return CSL_OK;
  const long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_test_f2d<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(in, out, (long)n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    CSL_NOTE(e, "csl_test_convert_f2d");
    return CSL_CUDA_ERROR;
  }
  return CSL_OK;
}

