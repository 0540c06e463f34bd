// dd_kernels.cuh -- kernels of the half hop on one domain of a lattice split
// along t, and optionally along z as well (the paper's Sec. 6 outlook: Dslash
// over several GPUs).  Each domain keeps its own links and spinors in the
// library's layouts on its local geometry (Lz / nz and Lt / nt even, so local
// and global parities agree).  Only the hops along a split direction mu that
// cross a domain boundary need data from a neighbour, and they need only a
// spin-projected half spinor per boundary site (6 complex instead of 12):
//   - the +mu hop of a site at local x_mu = L_mu - 1 reads (1 - S gamma_mu)
//     psi(y) of the site y at x_mu = 0 of the next domain along mu, and
//     multiplies it by its own link U_mu(x);
//   - the -mu hop of a site at local x_mu = 0 reads U_mu(y)^+ (1 + S gamma_mu)
//     psi(y) of the site y at x_mu = L_mu - 1 of the previous domain, whose
//     link U_mu(y) that domain holds, so the product is formed there.
// dd_pack_kernel writes both faces of a domain along one direction (the t
// faces with the fermion boundary sign of the global lattice when their hop
// crosses the global t boundary; z is periodic), the caller moves them to the
// neighbours, and dd_hop_kernel computes the half hop with the received faces
// in place of those hops.  Face layout: [6][n] words of the spinor precision
// (complex128, float-float or complex64), n = the sites of one parity in a
// boundary slice, indexed by the site's checkerboard index within its slice:
// (x/2) + Lx/2 (y + Ly z) for a t slice, (x/2) + Lx/2 (y + Ly t) for a z
// slice (a hop along mu keeps the other three coordinates, so both domains
// give a site and its neighbour the same index).
#pragma once
#include "hop_kernels.cuh"

namespace lqcd {

// received faces of a domain hop; z_next == nullptr: z is not split
struct DdFaces {
  const void *t_next, *t_prev, *z_next, *z_prev;
  int n_t, n_z;  // sites per face along t and z
};

template <int PREC> struct FaceIO;
template <> struct FaceIO<LQCD_F64> {
  using R = double;
  static LQCD_DEV Cx<R> load(const void *f, int n, int k, int j) {
    const double2 w = ((const double2 *)f)[(size_t)k * n + j];
    return {w.x, w.y};
  }
  static LQCD_DEV void store(void *f, int n, int k, int j, Cx<R> v) {
    ((double2 *)f)[(size_t)k * n + j] = make_double2(v.re, v.im);
  }
};
template <> struct FaceIO<LQCD_DF64> {
  using R = df;
  static LQCD_DEV Cx<R> load(const void *f, int n, int k, int j) {
    const float4 w = ((const float4 *)f)[(size_t)k * n + j];
    return {{w.x, w.z}, {w.y, w.w}};
  }
  static LQCD_DEV void store(void *f, int n, int k, int j, Cx<R> v) {
    ((float4 *)f)[(size_t)k * n + j] = make_float4(v.re.hi, v.im.hi, v.re.lo, v.im.lo);
  }
};
template <> struct FaceIO<LQCD_F32> {
  using R = float;
  static LQCD_DEV Cx<R> load(const void *f, int n, int k, int j) {
    const float2 w = ((const float2 *)f)[(size_t)k * n + j];
    return {w.x, w.y};
  }
  static LQCD_DEV void store(void *f, int n, int k, int j, Cx<R> v) {
    ((float2 *)f)[(size_t)k * n + j] = make_float2(v.re, v.im);
  }
};

// index of a site within its boundary slice along MU (2: z, 3: t)
template <int MU> LQCD_DEV int face_index(const Geom &g, const Site &s) {
  static_assert(MU == 2 || MU == 3, "faces along z or t");
  return (s.x >> 1) + g.Lh0 * (s.y + g.L[1] * (MU == 3 ? s.z : s.t));
}

// checkerboard index of face site j in the slice x_MU = c
template <int MU> LQCD_DEV int face_site(const Geom &g, int j, int c) {
  if (MU == 3) return j + c * (g.Lh0 * g.L[1] * g.L[2]);
  const int xh = j % g.Lh0, r = j / g.Lh0;
  const int y = r % g.L[1], t = r / g.L[1];
  return xh + g.Lh0 * (y + g.L[1] * (c + g.L[2] * t));
}

// blockIdx.y = 0: the face for the previous domain along MU (sites at
// x_MU = 0), 1: the face for the next domain (sites at x_MU = L_MU - 1,
// times their links U_MU^+)
template <int PREC, int RECON, int MU, int S>
__global__ void __launch_bounds__(128) dd_pack_kernel(HopArgs A, int n, void *to_prev, void *to_next,
                                                      int neg_prev, int neg_next) {
  pdl_wait();
  using R = typename SpinorIO<PREC>::R;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int q = A.out_parity ^ 1;  // parity of the input sites
  const SpinorView vin{A.in, A.in_scale, A.g.Vh};
  Cx<R> ps[12], h[6];
  if (blockIdx.y == 0) {
    SpinorIO<PREC>::load(vin, face_site<MU>(A.g, j, 0), ps);
    project<MU, S>(ps, h);
    negate_if(h, neg_prev != 0);
#pragma unroll
    for (int k = 0; k < 6; k++) FaceIO<PREC>::store(to_prev, n, k, j, h[k]);
  } else {
    const int cb = face_site<MU>(A.g, j, A.g.L[MU] - 1);
    SpinorIO<PREC>::load(vin, cb, ps);
    project<MU, -S>(ps, h);
    Cx<R> u[9], v[6];
    LinkIO<PREC, RECON>::load(A.U, q, MU, cb, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link_dag(u, h, v);
    negate_if(v, neg_next != 0);
#pragma unroll
    for (int k = 0; k < 6; k++) FaceIO<PREC>::store(to_next, n, k, j, v[k]);
  }
}

// the two hops along a split direction MU: inside the domain from the input
// field, across its boundary from the received faces
template <int PREC, int RECON, int MU, int S>
LQCD_DEV void dd_dir(const HopArgs &A, const Site &s, int p, int cb, const SpinorView &vin, const void *from_next,
                     const void *from_prev, int n, Cx<typename SpinorIO<PREC>::R> acc[12]) {
  using R = typename SpinorIO<PREC>::R;
  const int c = MU == 2 ? s.z : s.t;
  Cx<R> ps[12], h[6], u[9], v[6];
  // forward: (1 - S gamma_mu) U_mu(x) psi(x + mu)
  if (c == A.g.L[MU] - 1) {
    const int j = face_index<MU>(A.g, s);
#pragma unroll
    for (int k = 0; k < 6; k++) h[k] = FaceIO<PREC>::load(from_next, n, k, j);
  } else {
    SpinorIO<PREC>::load(vin, neighbour_cb(A.g, s, MU, +1), ps);
    project<MU, S>(ps, h);
  }
  LinkIO<PREC, RECON>::load(A.U, p, MU, cb, u);
  if (RECON == 12) reconstruct_row2(u);
  mul_link(u, h, v);
  accumulate<MU, S>(v, acc);
  // backward: (1 + S gamma_mu) U_mu(x - mu)^+ psi(x - mu)
  if (c == 0) {
    const int j = face_index<MU>(A.g, s);
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = FaceIO<PREC>::load(from_prev, n, k, j);
  } else {
    const int jb = neighbour_cb(A.g, s, MU, -1);
    SpinorIO<PREC>::load(vin, jb, ps);
    project<MU, -S>(ps, h);
    LinkIO<PREC, RECON>::load(A.U, p ^ 1, MU, jb, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link_dag(u, h, v);
  }
  accumulate<MU, -S>(v, acc);
}

// The half hop on a domain: x and y hops as in hop_site, z likewise unless
// SZ (z split), t and (SZ) z from the input field inside the domain and from
// the faces across its boundary.  REDUCE: also the per-warp |out|^2 partials
// of hop_warp_partial (all lanes of a warp reach it, so inactive lanes do not
// return early).
template <int PREC, int RECON, bool DAG, bool REDUCE, bool SZ>
__global__ void __launch_bounds__(128) dd_hop_kernel(HopArgs A, DdFaces F) {
  pdl_wait();
  using R = typename SpinorIO<PREC>::R;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  double nrm = 0.0;
  if (cb < A.g.Vh) {
    constexpr int S = DAG ? -1 : 1;
    const int p = A.out_parity;
    const Site s = site_of(A.g, p, cb);
    const SpinorView vin{A.in, A.in_scale, A.g.Vh};
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = czero<R>();
    hop_dir<PREC, RECON, 0, S, false>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 1, S, false>(A, s, p, cb, vin, acc);
    if constexpr (SZ) dd_dir<PREC, RECON, 2, S>(A, s, p, cb, vin, F.z_next, F.z_prev, F.n_z, acc);
    else hop_dir<PREC, RECON, 2, S, false>(A, s, p, cb, vin, acc);
    dd_dir<PREC, RECON, 3, S>(A, s, p, cb, vin, F.t_next, F.t_prev, F.n_t, acc);
    nrm = hop_epilogue<PREC, REDUCE>(A, cb, 0, acc);
  }
  if (REDUCE) hop_warp_partial(A, cb, 0, nrm);
}

template <int PREC, int RECON, bool SZ>
void dd_hop_launch(bool dag, const HopArgs &A, const DdFaces &F, cudaStream_t st) {
  const unsigned grid = (unsigned)((A.g.Vh + 127) / 128);
  // programmatic dependent launches (the kernels wait for their predecessor
  // in pdl_wait), so a launch overlaps the tail of the kernel before it
  if (A.partials) {  // the reducing form (norms of the domain-decomposed CG)
    if (dag) launch_pdl(dd_hop_kernel<PREC, RECON, true, true, SZ>, dim3(grid), dim3(128), 0, st, A, F);
    else launch_pdl(dd_hop_kernel<PREC, RECON, false, true, SZ>, dim3(grid), dim3(128), 0, st, A, F);
  } else {
    if (dag) launch_pdl(dd_hop_kernel<PREC, RECON, true, false, SZ>, dim3(grid), dim3(128), 0, st, A, F);
    else launch_pdl(dd_hop_kernel<PREC, RECON, false, false, SZ>, dim3(grid), dim3(128), 0, st, A, F);
  }
}

// all precisions and link formats of the domain hop for one SZ (false: dd.cu,
// true: dd_z.cu, so that the two sets compile in parallel); false for a
// precision without a domain hop
template <bool SZ> bool dd_hop_dispatch(int prec, int recon, bool dag, const HopArgs &A, const DdFaces &F,
                                        cudaStream_t st) {
  switch (prec) {
    case LQCD_F64:
      if (recon == 12) dd_hop_launch<LQCD_F64, 12, SZ>(dag, A, F, st);
      else dd_hop_launch<LQCD_F64, 18, SZ>(dag, A, F, st);
      return true;
    case LQCD_DF64:
      if (recon == 12) dd_hop_launch<LQCD_DF64, 12, SZ>(dag, A, F, st);
      else dd_hop_launch<LQCD_DF64, 18, SZ>(dag, A, F, st);
      return true;
    case LQCD_F32:
      if (recon == 12) dd_hop_launch<LQCD_F32, 12, SZ>(dag, A, F, st);
      else dd_hop_launch<LQCD_F32, 18, SZ>(dag, A, F, st);
      return true;
    default: return false;
  }
}

// the z-split set (dd_z.cu)
bool dd_hop_dispatch_z(int prec, int recon, bool dag, const HopArgs &A, const DdFaces &F, cudaStream_t st);

}  // namespace lqcd
