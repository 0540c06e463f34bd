// dslash_h16.cu -- BF16 / FP16 (per-site scaled spinors, REC12 links)
// instantiations of the hop kernels (both load orders, and the
// register-blocked multi-RHS kernel).
#include "hop_kernels.cuh"

namespace lqcd {

void hop_launch_h16(const HopArgs &A, int prec, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, cudaStream_t st) {
  if (two) {
    if (prec == LQCD_BF16S) launch_pair2<LQCD_BF16S, 12>(A, grid, block, dag, red, st);
    else launch_pair2<LQCD_F16S, 12>(A, grid, block, dag, red, st);
    return;
  }
  if (rt > 1) {
    if (prec == LQCD_BF16S) launch_rt<LQCD_BF16S, 12>(A, rt, grid, block, dag, red, st);
    else launch_rt<LQCD_F16S, 12>(A, rt, grid, block, dag, red, st);
    return;
  }
  if (prec == LQCD_BF16S) launch_t<LQCD_BF16S, 12>(A, grid, block, dag, red, st, lf);
  else launch_t<LQCD_F16S, 12>(A, grid, block, dag, red, st, lf);
}

void hop_batched_h16(int prec, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st) {
  if (prec == LQCD_BF16S) batched_t<LQCD_BF16S, 12>(dag, red, d, tl, ntiles, grid, halt, st);
  else batched_t<LQCD_F16S, 12>(dag, red, d, tl, ntiles, grid, halt, st);
}

}  // namespace lqcd
