// lhdm_kernels.cuh -- what the kernels and the host side of the C ABI
// share: the batch descriptor, the scratch layout and the kernel
// declarations.  Each kernel is compiled in a translation unit of its own
// (lhdm_grid_solve.cu, lhdm_batch_solve.cu, lhdm_backward.cu) so the library
// builds in parallel.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "lhdm.h"
#include "lhdm_solve.cuh"

namespace lhdm {

// Per-instance descriptor of a batch (device array).
struct BatchItem {
  int m, n, lda, cap, ldr, k_max;
  const double* A;
  const double* b;
  double* x;
  int* passive;
  lhdm_info* info;
  double* R;
  int* rslot;
  int* order;
  double* xP;
  double* r;
  int* nP;
  const double* g;   // adjoint inputs/outputs (set per backward call)
  double* dLdb;
  double* dLdA;
  int ld_dA;
};

// Offsets of one team's scratch inside a double region and an int region.
struct ScratchLayout {
  size_t W, bt, yP, rhs, w, u, anorm, V, vtop, beta, T, R22, Gm, yJ, pr, part, pacc, candw, rotc, rots, apu;
  size_t Dinv, accb;  // pipelined triangular solve (teams of more than one CTA)
  size_t dtotal;
  size_t Vd;  // reflector digits of the tensor-core commit
  size_t pos, J, candi, candn, ipart, ctl, qlist, tflag, Ver, csign;
  size_t itotal;
  int ldw;
  bool pipelined;
};

inline size_t up8(size_t x) { return (x + 31) & ~(size_t)31; }  // 256-byte granules of doubles/ints

inline ScratchLayout make_layout(int max_m, int max_n, int team) {
  ScratchLayout L;
  const int m = std::max(max_m, 1), n = std::max(max_n, 1);
  const int cap = std::max(std::min(max_m, max_n), 1);
  L.ldw = (m + 1) & ~1;
  size_t o = 0;
  auto take = [&](size_t cnt) { size_t r = o; o += up8(std::max<size_t>(cnt, 1)); return r; };
  L.W = take((size_t)L.ldw * n);
  L.bt = take(m);
  L.yP = take(cap);
  L.rhs = take(std::max(m, cap));
  L.w = take(n);
  L.u = take(n);
  L.anorm = take(n);
  L.V = take((size_t)m * KM);
  L.vtop = take(KM);
  L.beta = take(KM);
  L.T = take(KM * KM);
  L.R22 = take(KM * KM);
  L.Gm = take(KM * KM);
  L.yJ = take(KM);
  L.pr = take(KM);
  L.part = take((size_t)team * PW);
  L.pacc = take(3 * PACC_W);
  L.candw = take((size_t)team * KM);
  L.rotc = take(cap);
  L.rots = take(cap);
  L.apu = take(m);
  // diagonal-block inverses and slab accumulators of the pipelined solve
  const size_t nbk = (size_t)(cap + TB - 1) / TB;
  L.pipelined = team > 1;
  L.Dinv = take(L.pipelined ? nbk * TB * TB : 1);
  L.accb = take(L.pipelined ? nbk * TB : 1);
  L.Vd = take((size_t)ND * m * 8);  // m x ND x 16 words
  L.dtotal = o;
  o = 0;
  L.pos = take(n);
  L.J = take(KM);
  L.candi = take((size_t)team * KM);
  L.candn = take(team);
  L.ipart = take((size_t)team * 8);
  L.ctl = take(16);
  L.qlist = take(cap);
  L.tflag = take(L.pipelined ? nbk * (1 + TB / SLAB + INV_PARTS) : 1);
  L.Ver = take(m);
  L.csign = take(n);
  L.itotal = o;
  return L;
}

inline __host__ __device__ void bind_scratch(Inst& I, const ScratchLayout& L, double* d, int* ip) {
  I.ldw = L.ldw;
  I.W = d + L.W;
  I.bt = d + L.bt;
  I.yP = d + L.yP;
  I.rhs = d + L.rhs;
  I.w = d + L.w;
  I.u = d + L.u;
  I.anorm = d + L.anorm;
  I.V = d + L.V;
  I.vtop = d + L.vtop;
  I.beta = d + L.beta;
  I.T = d + L.T;
  I.R22 = d + L.R22;
  I.Gm = d + L.Gm;
  I.yJ = d + L.yJ;
  I.pr = d + L.pr;
  I.part = d + L.part;
  I.pacc = reinterpret_cast<long long*>(d + L.pacc);
  I.candw = d + L.candw;
  I.rotc = d + L.rotc;
  I.rots = d + L.rots;
  I.pos = ip + L.pos;
  I.J = ip + L.J;
  I.candi = ip + L.candi;
  I.candn = ip + L.candn;
  I.ipart = ip + L.ipart;
  I.ctl = ip + L.ctl;
  I.qlist = ip + L.qlist;
  I.csign = ip + L.csign;
  I.Dinv = L.pipelined ? d + L.Dinv : nullptr;
  I.accb = L.pipelined ? d + L.accb : nullptr;
  I.tflag = L.pipelined ? ip + L.tflag : nullptr;
  I.Vd = reinterpret_cast<unsigned*>(d + L.Vd);
  I.Ver = ip + L.Ver;
  I.amask = nullptr;
  I.wait_ns = WAIT_NS;
  I.bar_extra = 0;
  I.guard_force = 0;
}

inline __device__ void bind_item(Inst& I, const BatchItem& it) {
  I.m = it.m;
  I.n = it.n;
  I.lda = it.lda;
  I.cap = it.cap;
  I.ldr = it.ldr;
  I.A = it.A;
  I.b = it.b;
  I.x_out = it.x;
  I.passive_out = it.passive;
  I.info_out = it.info;
  I.R = it.R;
  I.rslot = it.rslot;
  I.order = it.order;
  I.xP = it.xP;
  I.r = it.r;
  I.nP_out = it.nP;
  I.prm.k_max = it.k_max;
}

}  // namespace lhdm

// One solve on the whole GPU: one CTA per SM, cooperative launch.
__global__ void __launch_bounds__(lhdm::NT, 1) lhdm_solve_grid_kernel(lhdm::Inst I, unsigned int* bar, int* err);
// Adjoint of a solve on the whole GPU (cooperative launch).
__global__ void __launch_bounds__(lhdm::NT, 1) lhdm_backward_grid_kernel(lhdm::Inst I, unsigned int* bar, int* err,
                                                                         const double* g, double* dLdb,
                                                                         double* dLdA, int ld_dA, double* apu);
// Many instances in one persistent launch, one instance per CTA at a time.
__global__ void __launch_bounds__(lhdm::NT, 1) lhdm_solve_batch_kernel(const lhdm::BatchItem* items,
                                                                       const int* perm, int batch, int* queue,
                                                                       lhdm::ScratchLayout L, double* dscr,
                                                                       int* iscr, lhdm::DevParams prm);
__global__ void __launch_bounds__(lhdm::NT, 1) lhdm_backward_batch_kernel(const lhdm::BatchItem* items,
                                                                          const int* perm, int batch, int* queue,
                                                                          lhdm::ScratchLayout L, double* dscr,
                                                                          int* iscr);
