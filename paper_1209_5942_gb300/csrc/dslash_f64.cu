// dslash_f64.cu -- FP64 instantiations of the hop kernels (one translation
// unit per precision, so the build compiles them in parallel).
#include "hop_kernels.cuh"

namespace lqcd {

void hop_launch_f64(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (recon == 12) launch_t<LQCD_F64, 12>(A, grid, block, dag, red, st);
  else launch_t<LQCD_F64, 18>(A, grid, block, dag, red, st);
}

void hop_batched_f64(int recon, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st) {
  if (recon == 12) batched_t<LQCD_F64, 12>(dag, red, d, tl, ntiles, grid, halt, st);
  else batched_t<LQCD_F64, 18>(dag, red, d, tl, ntiles, grid, halt, st);
}

}  // namespace lqcd
