// dslash_h16.cu -- BF16 / FP16 (per-site scaled spinors, REC12 links)
// instantiations of the hop kernels (both load orders, the register-blocked
// multi-RHS kernel, the multi-RHS kernel with links staged in shared memory,
// and the two-site packed kernel with direct loads or with
// its operands staged through shared memory).
#include "hop_kernels.cuh"

namespace lqcd {

template <int PREC>
static void launch_h16_staged(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  const size_t smem = (size_t)h16_staged_bytes(block.x);
  if (dag) {
    if (red) launch_pdl(hop_h16_staged_kernel<PREC, true, true>, grid, block, smem, st, A);
    else launch_pdl(hop_h16_staged_kernel<PREC, true, false>, grid, block, smem, st, A);
  } else {
    if (red) launch_pdl(hop_h16_staged_kernel<PREC, false, true>, grid, block, smem, st, A);
    else launch_pdl(hop_h16_staged_kernel<PREC, false, false>, grid, block, smem, st, A);
  }
}

void hop_launch_h16(const HopArgs &A, int prec, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, bool staged, cudaStream_t st) {
  if (two && staged) {
    if (prec == LQCD_BF16S) launch_h16_staged<LQCD_BF16S>(A, grid, block, dag, red, st);
    else launch_h16_staged<LQCD_F16S>(A, grid, block, dag, red, st);
    return;
  }
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

void hop_launch_mrhs_h16(const HopArgs &A, int prec, int srec, int rg, dim3 grid, dim3 block, bool dag, bool red,
                         cudaStream_t st) {
  if (prec == LQCD_BF16S) {
    if (srec == 12) launch_mrhs2<LQCD_BF16S, 12, 12>(A, rg, grid, block, dag, red, st);
    else launch_mrhs2<LQCD_BF16S, 12, 18>(A, rg, grid, block, dag, red, st);
  } else {
    if (srec == 12) launch_mrhs2<LQCD_F16S, 12, 12>(A, rg, grid, block, dag, red, st);
    else launch_mrhs2<LQCD_F16S, 12, 18>(A, rg, grid, block, dag, red, st);
  }
}

void hop_batched_h16(int prec, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st) {
  if (prec == LQCD_BF16S) batched_t<LQCD_BF16S, 12>(dag, red, d, tl, ntiles, grid, halt, st);
  else batched_t<LQCD_F16S, 12>(dag, red, d, tl, ntiles, grid, halt, st);
}

}  // namespace lqcd
