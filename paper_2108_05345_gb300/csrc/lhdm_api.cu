// lhdm_api.cu -- the C ABI (include/lhdm.h) of the GB300 LHDM nonnegative
// least-squares solver: contexts, workspaces and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "lhdm.h"
#include "lhdm_kernels.cuh"

using namespace lhdm;

// ======================================================================= host side
struct lhdm_ctx {
  int device = 0;
  int nsm = 0;
  int max_m = 0, max_n = 0, cap = 0, ldr = 0;
  ScratchLayout L{};
  double* dscr = nullptr;
  int* iscr = nullptr;
  double* R = nullptr;
  int* rslot = nullptr;
  int* order = nullptr;
  double* xP = nullptr;
  double* r = nullptr;
  int* nP = nullptr;
  unsigned int* bar = nullptr;
  int* err = nullptr;
  lhdm_info* d_info = nullptr;
  double* d_phase = nullptr;
  int* d_trace = nullptr;
  int trace_cap = 0;
  // host-buffer path staging (allocated on first use)
  double* hA = nullptr;
  double* hb = nullptr;
  double* hx = nullptr;
  int* hp = nullptr;
  // state for the adjoint
  bool have_state = false;
  int last_m = 0, last_n = 0;
  // bounded waits (0 = default) and the failure-detection test's stall
  long long wait_ns = 0;
  bool stall_next = false;
  int guard_force = 0;  // test aid for the tensor-core commit's accuracy guard
  // batched solves: the plan of the last lhdm_solve_batched and the
  // arguments it was made for (reused while they repeat)
  int max_batch = 0;
  lhdm_batch* plan = nullptr;
  std::vector<int32_t> pm, pn, plda;
  std::vector<const void*> pptr;  // A, b, x, passive of every instance, then info
  lhdm_params pprm{};
  bool batch_state = false;
  int* d_zero = nullptr;  // one int 0: the work-queue order of a one-instance adjoint
  // l1-NNLS: the stacked system (allocated by the first lhdm_solve_l1)
  double* l1A = nullptr;  // max_m x max_n, ld = L.ldw
  double* l1b = nullptr;  // max_m
};

struct lhdm_batch {
  int device = 0;
  int batch = 0;
  int nblocks = 0;
  ScratchLayout L{};
  double* dscr = nullptr;
  int* iscr = nullptr;
  double* pers_d = nullptr;
  int* pers_i = nullptr;
  BatchItem* d_items = nullptr;
  int* d_perm = nullptr;
  int* d_queue = nullptr;
  BatchItem* d_adj = nullptr;
  std::vector<BatchItem> items;
  std::vector<int> kmax;
  DevParams prm{};
  bool ran = false;
};

// Kernel attributes are per device context: a flag per device records that
// they were set on it (set under a mutex, read without one).
constexpr int MAX_DEVICES = 64;
static std::mutex g_attr_mu;
static std::atomic<bool> g_attr_done[MAX_DEVICES];

static int cuda_ok(cudaError_t e) { return e == cudaSuccess ? LHDM_OK : LHDM_ERR_CUDA; }

static int set_attrs() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LHDM_ERR_CUDA;
  if (g_attr_done[dev].load(std::memory_order_acquire)) return LHDM_OK;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (g_attr_done[dev].load(std::memory_order_relaxed)) return LHDM_OK;
  cudaError_t e = cudaFuncSetAttribute(lhdm_solve_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DYN_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lhdm_backward_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DYN_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lhdm_solve_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DYN_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(lhdm_backward_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DYN_SMEM);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  g_attr_done[dev].store(true, std::memory_order_release);
  return LHDM_OK;
}

static int check_params(const lhdm_params* p, bool allow_auto_k) {
  if (!(p->tau1 > 0.0 && p->tau1 <= 1.0)) return LHDM_ERR_INVALID_ARG;
  if (!(p->tau2 > 0.0 && p->tau2 <= 1.0)) return LHDM_ERR_INVALID_ARG;
  if (!(p->delta > 0.0 && p->delta <= 1.0)) return LHDM_ERR_INVALID_ARG;
  if (std::isnan(p->tol_w)) return LHDM_ERR_INVALID_ARG;
  if (p->k_max > LHDM_KMAX_LIMIT) return LHDM_ERR_INVALID_ARG;
  if (p->k_max < 1 && !allow_auto_k) return LHDM_ERR_INVALID_ARG;
  if (p->mode < LHDM_MODE_NNLS || p->mode > LHDM_MODE_SIGNED_FLIP) return LHDM_ERR_INVALID_ARG;
  return LHDM_OK;
}

static DevParams to_dev(const lhdm_params& p) {
  DevParams d;
  d.tau1 = p.tau1;
  d.tau2 = p.tau2;
  d.delta = p.delta;
  d.tol_w = p.tol_w;
  d.k_max = p.k_max;
  d.max_outer = p.max_outer;
  d.mode = p.mode;
  return d;
}

extern "C" {

int lhdm_default_params(lhdm_params* p) {
  if (!p) return LHDM_ERR_INVALID_ARG;
  p->tau1 = 0.6;
  p->tau2 = 0.15;
  p->delta = 0.9;
  p->tol_w = -1.0;
  p->k_max = 32;
  p->max_outer = 0;
  p->mode = LHDM_MODE_NNLS;
  p->reserved = 0;
  return LHDM_OK;
}

const char* lhdm_status_string(int s) {
  switch (s) {
    case LHDM_OK: return "ok";
    case LHDM_ERR_INVALID_ARG: return "invalid argument";
    case LHDM_ERR_MAX_ITER: return "outer-iteration cap reached";
    case LHDM_ERR_NONFINITE: return "non-finite value in A or b";
    case LHDM_ERR_CUDA: return "CUDA runtime error";
    case LHDM_ERR_TIMEOUT: return "a bounded device-side wait expired";
    case LHDM_ERR_ALLOC: return "allocation failed";
    case LHDM_ERR_NO_STATE: return "no solve state for the adjoint";
    case LHDM_ERR_TOO_LARGE: return "problem larger than the static workspace of lhdm_solve_noalloc";
    default: return "unknown status";
  }
}

int lhdm_create(lhdm_ctx** out, int32_t max_m, int32_t max_n, int32_t max_batch) {
  if (!out || max_m < 1 || max_n < 1 || max_batch < 0) return LHDM_ERR_INVALID_ARG;
  *out = nullptr;
  lhdm_ctx* c = new (std::nothrow) lhdm_ctx();
  if (!c) return LHDM_ERR_ALLOC;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return LHDM_ERR_CUDA;
  }
  int rc = set_attrs();
  if (rc) { delete c; return rc; }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lhdm_solve_grid_kernel, NT, DYN_SMEM) != cudaSuccess ||
      nb < 1) {
    delete c;
    return LHDM_ERR_CUDA;
  }
  c->max_m = max_m;
  c->max_n = max_n;
  c->max_batch = max_batch;
  c->cap = std::max(std::min(max_m, max_n), 1);
  c->ldr = (c->cap + 1) & ~1;
  if ((max_n + c->nsm - 1) / c->nsm > CAND_LOCAL_MAX) { delete c; return LHDM_ERR_INVALID_ARG; }
  c->L = make_layout(max_m, max_n, c->nsm);
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&c->dscr, c->L.dtotal * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->iscr, c->L.itotal * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->R, (size_t)c->ldr * c->cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->rslot, (size_t)c->cap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->order, (size_t)c->cap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->xP, (size_t)c->cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->r, (size_t)std::max(max_m, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->nP, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->bar, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_info, sizeof(lhdm_info));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_phase, (2 * NPHASE + 2) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_phase, 0, (2 * NPHASE + 2) * sizeof(double));
  c->trace_cap = 3 * max_n + 8;
  if (e == cudaSuccess) e = cudaMalloc(&c->d_trace, (size_t)6 * c->trace_cap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_zero, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_zero, 0, sizeof(int));
  if (e != cudaSuccess) {
    lhdm_destroy(c);
    return e == cudaErrorMemoryAllocation ? LHDM_ERR_ALLOC : LHDM_ERR_CUDA;
  }
  *out = c;
  return LHDM_OK;
}

int lhdm_destroy(lhdm_ctx* c) {
  if (!c) return LHDM_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  cudaFree(c->dscr);
  cudaFree(c->iscr);
  cudaFree(c->R);
  cudaFree(c->rslot);
  cudaFree(c->order);
  cudaFree(c->xP);
  cudaFree(c->r);
  cudaFree(c->nP);
  cudaFree(c->bar);
  cudaFree(c->err);
  cudaFree(c->d_info);
  cudaFree(c->d_phase);
  cudaFree(c->d_trace);
  cudaFree(c->hA);
  cudaFree(c->hb);
  cudaFree(c->hx);
  cudaFree(c->hp);
  cudaFree(c->d_zero);
  cudaFree(c->l1A);
  cudaFree(c->l1b);
  if (c->plan) lhdm_batch_destroy(c->plan);
  delete c;
  return LHDM_OK;
}

static void fill_ctx_inst(lhdm_ctx* c, Inst& I) {
  bind_scratch(I, c->L, c->dscr, c->iscr);
  I.cap = std::min(I.m, I.n);
  I.ldr = c->ldr;
  I.R = c->R;
  I.rslot = c->rslot;
  I.order = c->order;
  I.xP = c->xP;
  I.r = c->r;
  I.nP_out = c->nP;
  I.info_out = c->d_info;
  I.phase_ns = c->d_phase;
  I.trace = c->d_trace;
  I.trace_cap = c->trace_cap;
  I.wait_ns = c->wait_ns > 0 ? c->wait_ns : WAIT_NS;
  I.guard_force = c->guard_force;
}

int lhdm_solve(lhdm_ctx* c, int32_t m, int32_t n, const double* A, int32_t lda, const double* b,
               const lhdm_params* prm, double* x, int32_t* passive, lhdm_info* info, void* stream) {
  if (!c || m < 0 || n < 0 || m > c->max_m || n > c->max_n || lda < std::max(1, m)) return LHDM_ERR_INVALID_ARG;
  if ((m > 0 && n > 0 && !A) || (m > 0 && !b) || (n > 0 && (!x || !passive))) return LHDM_ERR_INVALID_ARG;
  lhdm_params p;
  lhdm_default_params(&p);
  if (prm) p = *prm;
  int rc = check_params(&p, false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Inst I;
  std::memset(&I, 0, sizeof(I));
  I.m = m;
  I.n = n;
  I.lda = lda;
  I.A = A;
  I.b = b;
  I.x_out = x;
  I.passive_out = passive;
  I.prm = to_dev(p);
  fill_ctx_inst(c, I);
  I.bar_extra = c->stall_next ? 1 : 0;
  c->stall_next = false;
  c->have_state = false;
  cudaError_t e = cudaMemsetAsync(c->bar, 0, 4 * sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  void* args[] = {(void*)&I, (void*)&c->bar, (void*)&c->err};
  e = cudaLaunchCooperativeKernel((const void*)lhdm_solve_grid_kernel, dim3(c->nsm), dim3(NT), args, DYN_SMEM, st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  c->have_state = p.mode == LHDM_MODE_NNLS;  // the adjoint covers problem (1) only
  c->last_m = m;
  c->last_n = n;
  if (info) {
    e = cudaMemcpyAsync(info, c->d_info, sizeof(lhdm_info), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LHDM_ERR_CUDA;
  }
  return LHDM_OK;
}

int lhdm_solve_host(lhdm_ctx* c, int32_t m, int32_t n, const double* A, int32_t lda, const double* b,
                    const lhdm_params* prm, double* x, int32_t* passive, lhdm_info* info, void* stream) {
  if (!c || m < 0 || n < 0 || m > c->max_m || n > c->max_n || lda < std::max(1, m)) return LHDM_ERR_INVALID_ARG;
  if ((m > 0 && n > 0 && !A) || (m > 0 && !b) || (n > 0 && (!x || !passive))) return LHDM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!c->hA) {
    e = cudaMalloc(&c->hA, (size_t)c->L.ldw * std::max(c->max_n, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->hb, (size_t)std::max(c->max_m, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->hx, (size_t)2 * std::max(c->max_n, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->hp, (size_t)2 * std::max(c->max_n, 1) * sizeof(int));
    if (e != cudaSuccess) return LHDM_ERR_ALLOC;
  }
  const int ld = c->L.ldw;
  if (m > 0 && n > 0)
    e = cudaMemcpy2DAsync(c->hA, (size_t)ld * sizeof(double), A, (size_t)lda * sizeof(double),
                          (size_t)m * sizeof(double), n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(c->hb, b, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  int rc = lhdm_solve(c, m, n, c->hA, ld, c->hb, prm, c->hx, c->hp, nullptr, stream);
  if (rc) return rc;
  const size_t nx = (size_t)n * ((prm && prm->mode != LHDM_MODE_NNLS) ? 2 : 1);
  if (n > 0) {
    e = cudaMemcpyAsync(x, c->hx, nx * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(passive, c->hp, nx * sizeof(int), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, c->d_info, sizeof(lhdm_info), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_ok(e);
}

int lhdm_get_info(lhdm_ctx* c, lhdm_info* info, void* stream) {
  if (!c || !info) return LHDM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(info, c->d_info, sizeof(lhdm_info), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_ok(e);
}

int lhdm_phase_times(lhdm_ctx* c, double* ms, int32_t n, void* stream) {
  static_assert(NPHASE == 12, "phase list documented in lhdm.h");
  if (!c || !ms || n < 0) return -LHDM_ERR_INVALID_ARG;
  double h[2 * NPHASE + 1];
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h, c->d_phase, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return -LHDM_ERR_CUDA;
  const int k = std::min<int>(n, 2 * NPHASE + 1);
  for (int i = 0; i < k; ++i) ms[i] = (i < NPHASE) ? h[i] * 1e-6 : h[i];
  return k;
}

int lhdm_trace(lhdm_ctx* c, int32_t* out, int32_t max_rows, void* stream) {
  if (!c || !out || max_rows < 0) return -LHDM_ERR_INVALID_ARG;
  lhdm_info inf;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&inf, c->d_info, sizeof(inf), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return -LHDM_ERR_CUDA;
  const int rows = std::min(std::min(inf.n_outer, c->trace_cap), max_rows);
  if (rows > 0) {
    e = cudaMemcpyAsync(out, c->d_trace, (size_t)6 * rows * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return -LHDM_ERR_CUDA;
  }
  return rows;
}

int lhdm_debug_state(lhdm_ctx* c, const char* name, void* host, int64_t count, void* stream) {
  if (!c || !name || !host || count < 0) return LHDM_ERR_INVALID_ARG;
  struct Entry { const char* nm; const void* ptr; size_t elem; size_t cap; };
  const size_t n = (size_t)std::max(c->max_n, 1), m = (size_t)std::max(c->max_m, 1), cp = (size_t)c->cap;
  const Entry table[] = {
      {"w", c->dscr + c->L.w, 8, n},          {"u", c->dscr + c->L.u, 8, n},
      {"anorm", c->dscr + c->L.anorm, 8, n},  {"bt", c->dscr + c->L.bt, 8, m},
      {"yP", c->dscr + c->L.yP, 8, cp},       {"xP", c->xP, 8, cp},
      {"r", c->r, 8, m},                      {"W", c->dscr + c->L.W, 8, (size_t)c->L.ldw * n},
      {"R", c->R, 8, (size_t)c->ldr * cp},    {"order", c->order, 4, cp},
      {"rslot", c->rslot, 4, cp},             {"pos", c->iscr + c->L.pos, 4, n},
      {"ctl", c->iscr + c->L.ctl, 4, 16},
  };
  for (const Entry& e : table) {
    if (std::strcmp(e.nm, name) != 0) continue;
    if ((size_t)count > e.cap) return LHDM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaMemcpyAsync(host, e.ptr, (size_t)count * e.elem, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    return cuda_ok(err);
  }
  return LHDM_ERR_INVALID_ARG;
}

static int batch_adjoint(lhdm_batch* B, std::vector<BatchItem>& it, const int* d_perm, int count, int nblocks,
                         cudaStream_t st);

int lhdm_backward(lhdm_ctx* c, int32_t idx, const double* A, int32_t lda, const double* dLdx, double* dLdb,
                  double* dLdA, int32_t ld_dA, void* stream) {
  if (!c) return LHDM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (idx >= 0) {
    // one instance of the last batched solve: the batch adjoint kernel on a
    // one-entry table, one CTA
    if (!c->batch_state || !c->plan || c->plan->prm.mode != LHDM_MODE_NNLS) return LHDM_ERR_NO_STATE;
    lhdm_batch* B = c->plan;
    if (idx >= B->batch) return LHDM_ERR_INVALID_ARG;
    BatchItem it = B->items[idx];
    const int m = it.m, n = it.n;
    if ((m > 0 && n > 0 && A != it.A) || (n > 0 && !dLdx)) return LHDM_ERR_INVALID_ARG;
    if (dLdA && ld_dA < std::max(1, m)) return LHDM_ERR_INVALID_ARG;
    (void)lda;
    it.g = dLdx;
    it.dLdb = dLdb;
    it.dLdA = dLdA;
    it.ld_dA = ld_dA;
    std::vector<BatchItem> one(1, it);
    return batch_adjoint(B, one, c->d_zero, 1, 1, st);
  }
  if (!c->have_state) return LHDM_ERR_NO_STATE;
  const int m = c->last_m, n = c->last_n;
  if ((m > 0 && n > 0 && !A) || lda < std::max(1, m) || (n > 0 && !dLdx)) return LHDM_ERR_INVALID_ARG;
  if (dLdA && ld_dA < std::max(1, m)) return LHDM_ERR_INVALID_ARG;
  Inst I;
  std::memset(&I, 0, sizeof(I));
  I.m = m;
  I.n = n;
  I.lda = lda;
  I.A = A;
  fill_ctx_inst(c, I);
  double* apu = c->dscr + c->L.apu;
  cudaError_t e = cudaMemsetAsync(c->bar, 0, 4 * sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  double* apu_arg = dLdb ? dLdb : apu;
  void* args[] = {(void*)&I, (void*)&c->bar, (void*)&c->err, (void*)&dLdx, (void*)&dLdb,
                  (void*)&dLdA, (void*)&ld_dA, (void*)&apu_arg};
  e = cudaLaunchCooperativeKernel((const void*)lhdm_backward_grid_kernel, dim3(c->nsm), dim3(NT), args, DYN_SMEM, st);
  return cuda_ok(e);
}

// ----------------------------------------------------------------------- l1-NNLS
// The system of eq. (l1_NNLS): column j of [1^T 1^T; lam A  -lam A] for j < n
// and its partner n + j, from column j of A (one read of A, two writes);
// the right-hand side [0; lam b] by the first column block.
__global__ void lhdm_l1_stack_kernel(int m, int n, const double* __restrict__ A, int lda,
                                     const double* __restrict__ b, double lam, double* __restrict__ S, int lds,
                                     double* __restrict__ rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // row of the stacked system
  if (i > m) return;
  for (int j = blockIdx.y; j < n; j += gridDim.y) {
    const double v = (i == 0) ? 0.0 : lam * A[(size_t)j * lda + i - 1];
    S[(size_t)j * lds + i] = (i == 0) ? 1.0 : v;
    S[(size_t)(n + j) * lds + i] = (i == 0) ? 1.0 : -v;
  }
  if (blockIdx.y == 0) rhs[i] = (i == 0) ? 0.0 : lam * b[i - 1];
}

int lhdm_solve_l1(lhdm_ctx* c, int32_t m, int32_t n, const double* A, int32_t lda, const double* b, double lambda,
                  const lhdm_params* prm, double* x, int32_t* passive, lhdm_info* info, void* stream) {
  if (!c || m < 0 || n < 0 || m + 1 > c->max_m || 2 * (int64_t)n > c->max_n || lda < std::max(1, m))
    return LHDM_ERR_INVALID_ARG;
  if ((m > 0 && n > 0 && !A) || (m > 0 && !b) || (n > 0 && (!x || !passive))) return LHDM_ERR_INVALID_ARG;
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return LHDM_ERR_INVALID_ARG;
  if (prm && prm->mode != LHDM_MODE_NNLS) return LHDM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!c->l1A) {
    e = cudaMalloc(&c->l1A, (size_t)c->L.ldw * std::max(c->max_n, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->l1b, (size_t)std::max(c->max_m, 1) * sizeof(double));
    if (e != cudaSuccess) {
      cudaFree(c->l1A);
      cudaFree(c->l1b);
      c->l1A = nullptr;
      c->l1b = nullptr;
      return LHDM_ERR_ALLOC;
    }
  }
  const int ld = c->L.ldw;
  const dim3 grid((unsigned)((m + 1 + 255) / 256), (unsigned)std::max(1, std::min(n, 65535)));
  lhdm_l1_stack_kernel<<<grid, 256, 0, st>>>(m, n, A, lda, b, lambda, c->l1A, ld, c->l1b);
  if (cudaGetLastError() != cudaSuccess) return LHDM_ERR_CUDA;
  const int rc = lhdm_solve(c, m + 1, 2 * n, c->l1A, ld, c->l1b, prm, x, passive, info, stream);
  c->have_state = false;  // the adjoint of lhdm_backward is for the caller's own A
  return rc;
}

int lhdm_set_wait_limit(lhdm_ctx* c, int64_t ns) {
  if (!c) return LHDM_ERR_INVALID_ARG;
  c->wait_ns = ns > 0 ? (long long)ns : 0;
  return LHDM_OK;
}

int lhdm_debug_commit_guard(lhdm_ctx* c, int32_t mode) {
  if (!c || mode < 0 || mode > 1) return LHDM_ERR_INVALID_ARG;
  c->guard_force = mode;
  return LHDM_OK;
}

int lhdm_debug_stall_next_solve(lhdm_ctx* c) {
  if (!c) return LHDM_ERR_INVALID_ARG;
  c->stall_next = true;
  return LHDM_OK;
}

__global__ void lhdm_fast_math_kernel(const double* __restrict__ x, double* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i], a = fabs(v);
  out[4 * i] = rcp_nr(v);
  out[4 * i + 1] = 1.0 / v;
  out[4 * i + 2] = sqrt_gm(a);
  out[4 * i + 3] = sqrt(a);
}

int lhdm_debug_fast_math(const double* x, double* out, int32_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return LHDM_ERR_INVALID_ARG;
  if (n == 0) return LHDM_OK;
  lhdm_fast_math_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? LHDM_OK : LHDM_ERR_CUDA;
}

// ----------------------------------------------------------------------- allocation-free solve
// Callers that cannot allocate device memory (see lhdm_solve_noalloc) use one
// workspace that lives in a file-scope device array for the life of the
// process: its address is taken once per device, every call reuses it.
constexpr int NOALLOC_MAX_M = 256;
constexpr int NOALLOC_MAX_N = 512;
constexpr int NOALLOC_MAX_TEAM = 160;                // SMs the workspace is sized for
constexpr size_t NOALLOC_WORDS = (size_t)640 * 1024;  // 8-byte words: 5 MiB
static __device__ __align__(256) double g_lhdm_noalloc_scratch[NOALLOC_WORDS];

struct NoallocDevice {
  bool ready = false;
  int nsm = 0;
  double* base = nullptr;  // device address of g_lhdm_noalloc_scratch
  ScratchLayout L{};
  int cap = 0, ldr = 0;
  size_t oR = 0, oxP = 0, oR2 = 0, oI = 0;  // word offsets
};
static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc[MAX_DEVICES];

// Per-device set-up (first call on the device, with it current): the symbol's
// device address, kernel attributes and the fixed workspace layout.
static int noalloc_setup(NoallocDevice& d) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_lhdm_noalloc_scratch) != cudaSuccess || !ptr) return LHDM_ERR_CUDA;
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LHDM_ERR_CUDA;
  int rc = set_attrs();
  if (rc) return rc;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lhdm_solve_grid_kernel, NT, DYN_SMEM) != cudaSuccess ||
      occ < 1)
    return LHDM_ERR_CUDA;
  if (nsm > NOALLOC_MAX_TEAM) return LHDM_ERR_TOO_LARGE;
  d.nsm = nsm;
  d.base = static_cast<double*>(ptr);
  d.L = make_layout(NOALLOC_MAX_M, NOALLOC_MAX_N, nsm);
  d.cap = std::min(NOALLOC_MAX_M, NOALLOC_MAX_N);
  d.ldr = (d.cap + 1) & ~1;
  size_t o = d.L.dtotal;
  d.oR = o;
  o += up8((size_t)d.ldr * d.cap);
  d.oxP = o;
  o += up8(d.cap);
  d.oR2 = o;  // residual r
  o += up8(NOALLOC_MAX_M);
  d.oI = o;   // int region: scratch ints, rslot, order, nP, barrier words, error flag
  const size_t ints = d.L.itotal + 2 * up8(d.cap) + 3 * 32;
  o += (ints + 1) / 2;
  if (o > NOALLOC_WORDS) return LHDM_ERR_TOO_LARGE;
  d.ready = true;
  return LHDM_OK;
}

extern "C" int lhdm_solve_noalloc(int32_t m, int32_t n, const double* A, int32_t lda, const double* b,
                                  const lhdm_params* prm, double* x, int32_t* passive, lhdm_info* info,
                                  void* stream) {
  if (m < 0 || n < 0 || lda < std::max(1, m) || !info) return LHDM_ERR_INVALID_ARG;
  if ((m > 0 && n > 0 && !A) || (m > 0 && !b) || (n > 0 && (!x || !passive))) return LHDM_ERR_INVALID_ARG;
  if (m > NOALLOC_MAX_M || n > NOALLOC_MAX_N) return LHDM_ERR_TOO_LARGE;
  lhdm_params p;
  lhdm_default_params(&p);
  if (prm) p = *prm;
  int rc = check_params(&p, false);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LHDM_ERR_CUDA;
  NoallocDevice* d = &g_noalloc[dev];
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!d->ready) {
      rc = noalloc_setup(*d);
      if (rc) return rc;
    }
  }
  double* base = d->base;
  int* ib = reinterpret_cast<int*>(base + d->oI);
  Inst I;
  std::memset(&I, 0, sizeof(I));
  bind_scratch(I, d->L, base, ib);
  I.m = m;
  I.n = n;
  I.lda = lda;
  I.A = A;
  I.b = b;
  I.x_out = x;
  I.passive_out = passive;
  I.info_out = info;
  I.cap = std::min(m, n);
  I.ldr = d->ldr;
  I.R = base + d->oR;
  I.xP = base + d->oxP;
  I.r = base + d->oR2;
  int* tail = ib + d->L.itotal;
  I.rslot = tail;
  I.order = tail + up8(d->cap);
  I.nP_out = tail + 2 * up8(d->cap);
  unsigned int* bar = reinterpret_cast<unsigned int*>(tail + 2 * up8(d->cap) + 32);
  int* err = tail + 2 * up8(d->cap) + 64;
  I.phase_ns = nullptr;
  I.trace = nullptr;
  I.trace_cap = 0;
  I.prm = to_dev(p);
  cudaStream_t st = (cudaStream_t)stream;
  // the barrier words and the error flag must start at zero; everything
  // else is (re)initialised by the kernel itself
  cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  void* args[] = {(void*)&I, (void*)&bar, (void*)&err};
  e = cudaLaunchCooperativeKernel((const void*)lhdm_solve_grid_kernel, dim3(d->nsm), dim3(NT), args, DYN_SMEM, st);
  return cuda_ok(e);
}

// ----------------------------------------------------------------------- batches
// Block size per instance when the caller asks the tuner (k_max <= 0):
// the choice for each size bucket of n, from timing sweeps kept with the
// project's benchmark data (k_max in {4, 8, 16, 32}).
// ---------------------------------------------------------------- autotuner
// k_max per size bucket for batched solves with prm->k_max <= 0: a
// process-wide table filled by lhdm_batch_autotune (0 = untuned, which falls
// back to a rule from the benchmark sizes).
static std::mutex g_tune_mu;
static int g_tune_kmax[LHDM_TUNE_BUCKETS] = {0, 0, 0, 0, 0, 0};
static const int kTuneCands[] = {4, 8, 16, 32};

static int tune_bucket(int n) {
  int bkt = 0;
  for (long long lim = 128; bkt < LHDM_TUNE_BUCKETS - 1 && n > lim; lim <<= 1) ++bkt;
  return bkt;
}

static int tuned_kmax(int m, int n) {
  (void)m;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    const int k = g_tune_kmax[tune_bucket(n)];
    if (k > 0) return k;
  }
  if (n <= 256) return 8;
  if (n <= 512) return 16;
  return 32;
}

int lhdm_batch_create(lhdm_batch** out, int32_t batch, const int32_t* m, const int32_t* n, const int32_t* lda,
                      const double* const* A, const double* const* b, double* const* x,
                      int32_t* const* passive, lhdm_info* info, const lhdm_params* prm, void* stream) {
  if (!out || batch < 0 || (batch > 0 && (!m || !n || !lda || !A || !b || !x || !passive || !info)))
    return LHDM_ERR_INVALID_ARG;
  *out = nullptr;
  lhdm_params p;
  lhdm_default_params(&p);
  if (prm) p = *prm;
  int rc = check_params(&p, true);
  if (rc) return rc;
  int max_m = 1, max_n = 1;
  for (int i = 0; i < batch; ++i) {
    if (m[i] < 0 || n[i] < 0 || lda[i] < std::max(1, m[i])) return LHDM_ERR_INVALID_ARG;
    if ((m[i] > 0 && n[i] > 0 && !A[i]) || (m[i] > 0 && !b[i]) || (n[i] > 0 && (!x[i] || !passive[i])))
      return LHDM_ERR_INVALID_ARG;
    max_m = std::max(max_m, m[i]);
    max_n = std::max(max_n, n[i]);
  }
  if (max_n > CAND_LOCAL_MAX) return LHDM_ERR_INVALID_ARG;
  rc = set_attrs();
  if (rc) return rc;
  lhdm_batch* B = new (std::nothrow) lhdm_batch();
  if (!B) return LHDM_ERR_ALLOC;
  cudaStream_t st = (cudaStream_t)stream;
  int nsm = 0, occ = 0;
  cudaGetDevice(&B->device);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lhdm_solve_batch_kernel, NT, DYN_SMEM);
  B->batch = batch;
  B->nblocks = std::max(1, std::min(batch, nsm * std::max(occ, 1)));
  B->L = make_layout(max_m, max_n, 1);
  B->prm = to_dev(p);
  // persistent per-instance state
  size_t dtot = 0, itot = 0;
  std::vector<size_t> doff(batch), ioff(batch);
  for (int i = 0; i < batch; ++i) {
    const int cap = std::max(std::min(m[i], n[i]), 1), ldr = (cap + 1) & ~1;
    doff[i] = dtot;
    dtot += up8((size_t)ldr * cap) + up8(cap) + up8(std::max(m[i], 1));
    ioff[i] = itot;
    itot += up8(cap) * 2 + up8(1);
  }
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&B->dscr, B->L.dtotal * B->nblocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&B->iscr, B->L.itotal * B->nblocks * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B->pers_d, std::max<size_t>(dtot, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&B->pers_i, std::max<size_t>(itot, 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_items, std::max(batch, 1) * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_perm, std::max(batch, 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_queue, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_adj, std::max(batch, 1) * sizeof(BatchItem));
  if (e != cudaSuccess) {
    lhdm_batch_destroy(B);
    return LHDM_ERR_ALLOC;
  }
  B->items.resize(batch);
  B->kmax.resize(batch);
  for (int i = 0; i < batch; ++i) {
    BatchItem& it = B->items[i];
    std::memset(&it, 0, sizeof(it));
    const int cap = std::max(std::min(m[i], n[i]), 1), ldr = (cap + 1) & ~1;
    it.m = m[i];
    it.n = n[i];
    it.lda = lda[i];
    it.cap = std::min(m[i], n[i]);
    it.ldr = ldr;
    it.k_max = p.k_max > 0 ? p.k_max : tuned_kmax(m[i], n[i]);
    B->kmax[i] = it.k_max;
    it.A = A[i];
    it.b = b[i];
    it.x = x[i];
    it.passive = passive[i];
    it.info = info + i;
    double* pd = B->pers_d + doff[i];
    it.R = pd;
    it.xP = pd + up8((size_t)ldr * cap);
    it.r = it.xP + up8(cap);
    int* pi = B->pers_i + ioff[i];
    it.rslot = pi;
    it.order = pi + up8(cap);
    it.nP = pi + 2 * up8(cap);
  }
  // largest work first (about m * n * min(m, n) flops per instance)
  std::vector<int> perm(batch);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int c) {
    const double wa = (double)m[a] * n[a] * std::min(m[a], n[a]);
    const double wc = (double)m[c] * n[c] * std::min(m[c], n[c]);
    return wa > wc;
  });
  if (batch > 0) {
    e = cudaMemcpyAsync(B->d_items, B->items.data(), batch * sizeof(BatchItem), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_perm, perm.data(), batch * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      lhdm_batch_destroy(B);
      return LHDM_ERR_CUDA;
    }
  }
  *out = B;
  return LHDM_OK;
}

int lhdm_batch_run(lhdm_batch* B, void* stream) {
  if (!B) return LHDM_ERR_INVALID_ARG;
  if (B->batch == 0) return LHDM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(B->d_queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  lhdm_solve_batch_kernel<<<B->nblocks, NT, DYN_SMEM, st>>>(B->d_items, B->d_perm, B->batch, B->d_queue, B->L,
                                                             B->dscr, B->iscr, B->prm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  B->ran = true;
  return LHDM_OK;
}

int lhdm_batch_backward(lhdm_batch* B, const double* const* dLdx, double* const* dLdb, double* const* dLdA,
                        const int32_t* ld_dA, void* stream) {
  if (!B || (B->batch > 0 && !dLdx)) return LHDM_ERR_INVALID_ARG;
  if (!B->ran || B->prm.mode != LHDM_MODE_NNLS) return LHDM_ERR_NO_STATE;
  if (B->batch == 0) return LHDM_OK;
  std::vector<BatchItem> it = B->items;
  for (int i = 0; i < B->batch; ++i) {
    it[i].g = dLdx[i];
    it[i].dLdb = dLdb ? dLdb[i] : nullptr;
    it[i].dLdA = dLdA ? dLdA[i] : nullptr;
    it[i].ld_dA = ld_dA ? ld_dA[i] : std::max(1, it[i].m);
    if (it[i].dLdA && it[i].ld_dA < std::max(1, it[i].m)) return LHDM_ERR_INVALID_ARG;
  }
  int rc = batch_adjoint(B, it, B->d_perm, B->batch, B->nblocks, (cudaStream_t)stream);
  if (rc) return rc;
  return cuda_ok(cudaStreamSynchronize((cudaStream_t)stream));
}

int lhdm_batch_kmax(const lhdm_batch* B, int32_t i) {
  if (!B || i < 0 || i >= B->batch) return -1;
  return B->kmax[i];
}

int lhdm_batch_destroy(lhdm_batch* B) {
  if (!B) return LHDM_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  cudaFree(B->dscr);
  cudaFree(B->iscr);
  cudaFree(B->pers_d);
  cudaFree(B->pers_i);
  cudaFree(B->d_items);
  cudaFree(B->d_perm);
  cudaFree(B->d_queue);
  cudaFree(B->d_adj);
  delete B;
  return LHDM_OK;
}

}  // extern "C"

// The adjoint kernel of a batch over the descriptors `it` (count entries,
// visited in the order d_perm gives), on nblocks CTAs.  The descriptors go to
// the plan's second table, so the forward table stays intact; the table is
// uploaded from a host buffer that stays alive until the copy has run.
static int batch_adjoint(lhdm_batch* B, std::vector<BatchItem>& it, const int* d_perm, int count, int nblocks,
                         cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(B->d_adj, it.data(), count * sizeof(BatchItem), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `it` is a pageable host buffer
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return LHDM_ERR_CUDA;
  lhdm_backward_batch_kernel<<<nblocks, NT, DYN_SMEM, st>>>(B->d_adj, d_perm, count, B->d_queue, B->L, B->dscr,
                                                            B->iscr);
  return cuda_ok(cudaGetLastError());
}

// lhdm_solve_batched: the batch plan of the context is made on the first call
// with a given argument set and reused while the arguments repeat.
static bool same_batch_args(const lhdm_ctx* c, int batch, const int32_t* m, const int32_t* n, const int32_t* lda,
                            const double* const* A, const double* const* b, double* const* x,
                            int32_t* const* passive, const lhdm_info* info, const lhdm_params& p) {
  if (!c->plan || (int)c->pm.size() != batch) return false;
  if (std::memcmp(&c->pprm, &p, sizeof(p)) != 0) return false;
  for (int i = 0; i < batch; ++i) {
    if (c->pm[i] != m[i] || c->pn[i] != n[i] || c->plda[i] != lda[i]) return false;
    if (c->pptr[4 * i] != A[i] || c->pptr[4 * i + 1] != b[i] || c->pptr[4 * i + 2] != x[i] ||
        c->pptr[4 * i + 3] != passive[i])
      return false;
  }
  return c->pptr[4 * batch] == (const void*)info;
}

extern "C" int lhdm_solve_batched(lhdm_ctx* c, int32_t batch, const int32_t* m, const int32_t* n,
                                  const double* const* A, const int32_t* lda, const double* const* b,
                                  const lhdm_params* prm, double* const* x, int32_t* const* passive,
                                  lhdm_info* info, void* stream) {
  if (!c || batch < 0 || batch > c->max_batch) return LHDM_ERR_INVALID_ARG;
  if (batch > 0 && (!m || !n || !A || !lda || !b || !x || !passive || !info)) return LHDM_ERR_INVALID_ARG;
  for (int i = 0; i < batch; ++i)
    if (m[i] > c->max_m || n[i] > c->max_n) return LHDM_ERR_INVALID_ARG;
  lhdm_params p;
  lhdm_default_params(&p);
  if (prm) p = *prm;
  int rc = check_params(&p, true);
  if (rc) return rc;
  if (!same_batch_args(c, batch, m, n, lda, A, b, x, passive, info, p)) {
    if (c->plan) {
      lhdm_batch_destroy(c->plan);
      c->plan = nullptr;
    }
    c->batch_state = false;
    c->pm.assign(m, m + batch);
    c->pn.assign(n, n + batch);
    c->plda.assign(lda, lda + batch);
    c->pptr.resize(4 * (size_t)batch + 1);
    for (int i = 0; i < batch; ++i) {
      c->pptr[4 * i] = A[i];
      c->pptr[4 * i + 1] = b[i];
      c->pptr[4 * i + 2] = x[i];
      c->pptr[4 * i + 3] = passive[i];
    }
    c->pptr[4 * batch] = info;
    c->pprm = p;
    rc = lhdm_batch_create(&c->plan, batch, m, n, lda, A, b, x, passive, info, &p, stream);
    if (rc) {
      c->plan = nullptr;
      c->pm.clear();
      return rc;
    }
  }
  rc = lhdm_batch_run(c->plan, stream);
  c->batch_state = rc == LHDM_OK;
  return rc;
}

extern "C" int lhdm_backward_batched(lhdm_ctx* c, const double* const* dLdx, double* const* dLdb,
                                     double* const* dLdA, const int32_t* ld_dA, void* stream) {
  if (!c) return LHDM_ERR_INVALID_ARG;
  if (!c->batch_state || !c->plan) return LHDM_ERR_NO_STATE;
  return lhdm_batch_backward(c->plan, dLdx, dLdb, dLdA, ld_dA, stream);
}

extern "C" int lhdm_batch_autotune(int32_t batch, const int32_t* m, const int32_t* n, const int32_t* lda,
                                   const double* const* A, const double* const* b, const lhdm_params* prm,
                                   int32_t* table, void* stream) {
  if (batch < 0 || (batch > 0 && (!m || !n || !lda || !A || !b))) return LHDM_ERR_INVALID_ARG;
  lhdm_params p;
  lhdm_default_params(&p);
  if (prm) p = *prm;
  p.k_max = 1;
  int rc = check_params(&p, true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> idx[LHDM_TUNE_BUCKETS];
  for (int i = 0; i < batch; ++i) {
    if (m[i] < 0 || n[i] < 0 || lda[i] < std::max(1, m[i])) return LHDM_ERR_INVALID_ARG;
    if ((m[i] > 0 && n[i] > 0 && !A[i]) || (m[i] > 0 && !b[i])) return LHDM_ERR_INVALID_ARG;
    idx[tune_bucket(n[i])].push_back(i);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return LHDM_ERR_CUDA;
  }
  int result = LHDM_OK;
  for (int bkt = 0; bkt < LHDM_TUNE_BUCKETS && result == LHDM_OK; ++bkt) {
    const int cnt = (int)idx[bkt].size();
    if (cnt == 0) continue;
    std::vector<int32_t> sm(cnt), sn(cnt), sl(cnt);
    std::vector<const double*> sA(cnt), sb(cnt);
    std::vector<double*> sx(cnt);
    std::vector<int32_t*> sp(cnt);
    size_t nx = 0;
    for (int k = 0; k < cnt; ++k) {
      const int i = idx[bkt][k];
      sm[k] = m[i];
      sn[k] = n[i];
      sl[k] = lda[i];
      sA[k] = A[i];
      sb[k] = b[i];
      nx += (size_t)std::max(n[i], 1);
    }
    // trial outputs: one x / passive buffer for the bucket, carved per instance
    double* dx = nullptr;
    int32_t* dp = nullptr;
    lhdm_info* dinfo = nullptr;
    cudaError_t e = cudaMalloc(&dx, nx * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dp, nx * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&dinfo, (size_t)cnt * sizeof(lhdm_info));
    if (e != cudaSuccess) result = LHDM_ERR_ALLOC;
    size_t o = 0;
    for (int k = 0; k < cnt && result == LHDM_OK; ++k) {
      sx[k] = dx + o;
      sp[k] = dp + o;
      o += (size_t)std::max(sn[k], 1);
    }
    int best_k = 0;
    float best_ms = 0.0f;
    for (int kc : kTuneCands) {
      if (result != LHDM_OK) break;
      lhdm_params pk = p;
      pk.k_max = kc;
      lhdm_batch* B = nullptr;
      rc = lhdm_batch_create(&B, cnt, sm.data(), sn.data(), sl.data(), sA.data(), sb.data(), sx.data(), sp.data(),
                             dinfo, &pk, stream);
      if (rc) { result = rc; break; }
      rc = lhdm_batch_run(B, stream);  // warm-up
      if (!rc && (cudaEventRecord(e0, st) != cudaSuccess)) rc = LHDM_ERR_CUDA;
      if (!rc) rc = lhdm_batch_run(B, stream);
      if (!rc && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)) rc = LHDM_ERR_CUDA;
      float ms = 0.0f;
      if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = LHDM_ERR_CUDA;
      lhdm_batch_destroy(B);
      if (rc) { result = rc; break; }
      if (best_k == 0 || ms < best_ms) {
        best_k = kc;
        best_ms = ms;
      }
    }
    cudaFree(dx);
    cudaFree(dp);
    cudaFree(dinfo);
    if (result == LHDM_OK) {
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tune_kmax[bkt] = best_k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result == LHDM_OK && table) lhdm_tuning_get(table);
  return result;
}

extern "C" int lhdm_tuning_get(int32_t* table) {
  if (!table) return LHDM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (int i = 0; i < LHDM_TUNE_BUCKETS; ++i) table[i] = g_tune_kmax[i];
  return LHDM_OK;
}

extern "C" int lhdm_tuning_set(const int32_t* table) {
  if (!table) return LHDM_ERR_INVALID_ARG;
  for (int i = 0; i < LHDM_TUNE_BUCKETS; ++i)
    if (table[i] < 0 || table[i] > LHDM_KMAX_LIMIT) return LHDM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (int i = 0; i < LHDM_TUNE_BUCKETS; ++i) g_tune_kmax[i] = table[i];
  return LHDM_OK;
}
