// dslash_df64.cu -- float-float instantiations of the hop kernels: the
// two-threads-per-site kernel for 18-real links (scalar or packed FP32x2
// arithmetic, the packed one also with its operands staged through shared
// memory; all three give the same bits) and the one-thread kernel for REC12
// links.
#include "hop_kernels.cuh"

namespace lqcd {

template <bool PK>
static void launch_pair(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) launch_pdl(hop_df64_pair_kernel<true, true, PK>, grid, block, 0, st, A);
    else launch_pdl(hop_df64_pair_kernel<true, false, PK>, grid, block, 0, st, A);
  } else {
    if (red) launch_pdl(hop_df64_pair_kernel<false, true, PK>, grid, block, 0, st, A);
    else launch_pdl(hop_df64_pair_kernel<false, false, PK>, grid, block, 0, st, A);
  }
}

void hop_launch_df64(const HopArgs &A, int recon, bool pair, int mode, dim3 grid, dim3 block, bool dag,
                     bool red, cudaStream_t st) {
  if (pair && (mode == 2 || mode == 3)) {
    const size_t smem = (size_t)block.y * df_staged_words(block.x) * sizeof(float4);
    if (mode == 3) {
      if (dag) {
        if (red) launch_pdl(hop_df64_staged_kernel<true, true, 5>, grid, block, smem, st, A);
        else launch_pdl(hop_df64_staged_kernel<true, false, 5>, grid, block, smem, st, A);
      } else {
        if (red) launch_pdl(hop_df64_staged_kernel<false, true, 5>, grid, block, smem, st, A);
        else launch_pdl(hop_df64_staged_kernel<false, false, 5>, grid, block, smem, st, A);
      }
      return;
    }
    if (dag) {
      if (red) launch_pdl(hop_df64_staged_kernel<true, true>, grid, block, smem, st, A);
      else launch_pdl(hop_df64_staged_kernel<true, false>, grid, block, smem, st, A);
    } else {
      if (red) launch_pdl(hop_df64_staged_kernel<false, true>, grid, block, smem, st, A);
      else launch_pdl(hop_df64_staged_kernel<false, false>, grid, block, smem, st, A);
    }
    return;
  }
  if (pair) {
    if (mode == 1) launch_pair<true>(A, grid, block, dag, red, st);
    else launch_pair<false>(A, grid, block, dag, red, st);
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
