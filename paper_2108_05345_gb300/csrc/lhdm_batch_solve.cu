// lhdm_batch_solve.cu -- the persistent solve kernel of a batch of instances.
#include "lhdm_kernels.cuh"

using namespace lhdm;

// Many instances in one persistent launch: each CTA takes the next instance
// (largest first) from a device queue and solves it alone.
__global__ void __launch_bounds__(NT, 1) lhdm_solve_batch_kernel(const BatchItem* items, const int* perm,
                                                                 int batch, int* queue, ScratchLayout L,
                                                                 double* dscr, int* iscr, DevParams prm) {
  extern __shared__ double dyn[];
  __shared__ int s_k;
  Inst I;
  bind_scratch(I, L, dscr + (size_t)blockIdx.x * L.dtotal, iscr + (size_t)blockIdx.x * L.itotal);
  I.phase_ns = nullptr;
  I.trace = nullptr;
  I.trace_cap = 0;
  for (;;) {
    if (threadIdx.x == 0) s_k = atomicAdd(queue, 1);
    __syncthreads();
    const int k = s_k;
    __syncthreads();
    if (k >= batch) break;
    const BatchItem it = items[perm[k]];
    I.prm = prm;
    bind_item(I, it);
    CtaTeam tm{0, 1};
    Engine<CtaTeam> e(tm, I, dyn);
    e.run();
    __syncthreads();
  }
}
