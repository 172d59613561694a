// lhdm_grid_solve.cu -- the solve kernel of one instance on the whole GPU.
#include "lhdm_kernels.cuh"

using namespace lhdm;

// One solve on the whole GPU: one CTA per SM, cooperative launch.
__global__ void __launch_bounds__(NT, 1) lhdm_solve_grid_kernel(Inst I, unsigned int* bar, int* err) {
  extern __shared__ double dyn[];
  GridTeam tm{(int)blockIdx.x, (int)gridDim.x, bar, err, I.wait_ns, I.bar_extra};
  Engine<GridTeam> e(tm, I, dyn);
  e.run();
}
