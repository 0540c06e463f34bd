// dd_z.cu -- the domain hop instances for a lattice split along z as well as
// t (kernels in dd_kernels.cuh), a translation unit of their own so that they
// compile in parallel with the t-only set in dd.cu.
#include "dd_kernels.cuh"

namespace lqcd {

bool dd_hop_dispatch_z(int prec, int recon, bool dag, const HopArgs &A, const DdFaces &F, cudaStream_t st) {
  return dd_hop_dispatch<true>(prec, recon, dag, A, F, st);
}

}  // namespace lqcd
