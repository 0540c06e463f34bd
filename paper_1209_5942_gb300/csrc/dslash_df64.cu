// dslash_df64.cu -- float-float instantiations of the hop kernels: the
// two-threads-per-site kernel for 18-real links and the one-thread kernel for
// REC12 links.
#include "hop_kernels.cuh"

namespace lqcd {

void hop_launch_df64(const HopArgs &A, int recon, bool pair, dim3 grid, dim3 block, bool dag, bool red,
                     cudaStream_t st) {
  if (pair) {
    if (dag) {
      if (red) hop_df64_pair_kernel<true, true><<<grid, block, 0, st>>>(A);
      else hop_df64_pair_kernel<true, false><<<grid, block, 0, st>>>(A);
    } else {
      if (red) hop_df64_pair_kernel<false, true><<<grid, block, 0, st>>>(A);
      else hop_df64_pair_kernel<false, false><<<grid, block, 0, st>>>(A);
    }
    return;
  }
  if (recon == 12) launch_t<LQCD_DF64, 12>(A, grid, block, dag, red, st);
  else launch_t<LQCD_DF64, 18>(A, grid, block, dag, red, st);
}

void hop_batched_df64(int recon, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                      const int *halt, cudaStream_t st) {
  if (recon == 12) batched_t<LQCD_DF64, 12>(dag, red, d, tl, ntiles, grid, halt, st);
  else batched_t<LQCD_DF64, 18>(dag, red, d, tl, ntiles, grid, halt, st);
}

}  // namespace lqcd
