// lhdm_backward.cu -- adjoint kernels (one instance on the whole GPU, and a
// batch of instances one per CTA).
#include "lhdm_kernels.cuh"
#include "lhdm_adjoint.cuh"

using namespace lhdm;

__global__ void __launch_bounds__(NT, 1) lhdm_backward_grid_kernel(Inst I, unsigned int* bar, int* err,
                                                                   const double* g, double* dLdb,
                                                                   double* dLdA, int ld_dA, double* apu) {
  extern __shared__ double dyn[];
  GridTeam tm{(int)blockIdx.x, (int)gridDim.x, bar, err, I.wait_ns, I.bar_extra};
  Engine<GridTeam> e(tm, I, dyn);
  Adjoint<GridTeam> adj(e);
  adj.run(g, dLdb, dLdA, ld_dA, apu);
}

__global__ void __launch_bounds__(NT, 1) lhdm_backward_batch_kernel(const BatchItem* items, const int* perm,
                                                                    int batch, int* queue, ScratchLayout L,
                                                                    double* dscr, int* iscr) {
  extern __shared__ double dyn[];
  __shared__ int s_k;
  Inst I;
  I.prm = DevParams{};  // plain NNLS: the adjoint reads no solver parameter
  const size_t dbase = (size_t)blockIdx.x * L.dtotal;
  bind_scratch(I, L, dscr + dbase, iscr + (size_t)blockIdx.x * L.itotal);
  I.phase_ns = nullptr;
  I.trace = nullptr;
  I.trace_cap = 0;
  double* apu = dscr + dbase + L.apu;
  for (;;) {
    if (threadIdx.x == 0) s_k = atomicAdd(queue, 1);
    __syncthreads();
    const int k = s_k;
    __syncthreads();
    if (k >= batch) break;
    const BatchItem it = items[perm[k]];
    bind_item(I, it);
    CtaTeam tm{0, 1};
    Engine<CtaTeam> e(tm, I, dyn);
    if (it.g) {
      Adjoint<CtaTeam> adj(e);
      adj.run(it.g, it.dLdb, it.dLdA, it.ld_dA, it.dLdb ? it.dLdb : apu);
    }
    __syncthreads();
  }
}
