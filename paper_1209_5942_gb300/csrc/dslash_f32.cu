// dslash_f32.cu -- FP32 instantiations of the hop kernels (both load orders,
// the register-blocked multi-RHS kernel, the multi-RHS kernel with links
// staged in shared memory and the one with RHS interleaved with the site
// blocks).
#include "hop_kernels.cuh"

namespace lqcd {

void hop_launch_f32(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, cudaStream_t st) {
  if (two) {
    if (recon == 12) launch_pair2<LQCD_F32, 12>(A, grid, block, dag, red, st);
    else launch_pair2<LQCD_F32, 18>(A, grid, block, dag, red, st);
    return;
  }
  if (rt > 1) {
    if (recon == 12) launch_rt<LQCD_F32, 12>(A, rt, grid, block, dag, red, st);
    else launch_rt<LQCD_F32, 18>(A, rt, grid, block, dag, red, st);
    return;
  }
  if (recon == 12) launch_t<LQCD_F32, 12>(A, grid, block, dag, red, st, lf);
  else launch_t<LQCD_F32, 18>(A, grid, block, dag, red, st, lf);
}

void hop_launch_f32_ri(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (recon == 12) launch_ri<LQCD_F32, 12>(A, grid, block, dag, red, st);
  else launch_ri<LQCD_F32, 18>(A, grid, block, dag, red, st);
}

void hop_launch_mrhs_f32(const HopArgs &A, int recon, int srec, int rg, dim3 grid, dim3 block, bool dag, bool red,
                         cudaStream_t st) {
  if (recon == 12) {
    if (srec == 12) launch_mrhs2<LQCD_F32, 12, 12>(A, rg, grid, block, dag, red, st);
    else launch_mrhs2<LQCD_F32, 12, 18>(A, rg, grid, block, dag, red, st);
  } else {
    launch_mrhs2<LQCD_F32, 18, 18>(A, rg, grid, block, dag, red, st);
  }
}

void hop_batched_f32(int recon, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st) {
  if (recon == 12) batched_t<LQCD_F32, 12>(dag, red, d, tl, ntiles, grid, halt, st);
  else batched_t<LQCD_F32, 18>(dag, red, d, tl, ntiles, grid, halt, st);
}

}  // namespace lqcd
