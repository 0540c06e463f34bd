// dd.cu -- the half hop on one domain of a lattice split along t (the paper's
// Sec. 6 outlook: Dslash over several GPUs).  Each domain keeps its own links
// and spinors in the library's layouts, with the local extent Lt / nt (even,
// so local and global parities agree).  Only the t hops that cross a domain
// boundary need data from a neighbour, and they need only a spin-projected
// half spinor per boundary site (6 complex instead of 12):
//   - the +t hop of a site at local t = Lt-1 reads (1 - S gamma_t) psi(y) of
//     the site y at t = 0 of the next domain, and multiplies it by its own
//     link U_t(x);
//   - the -t hop of a site at local t = 0 reads U_t(y)^+ (1 + S gamma_t) psi(y)
//     of the site y at t = Lt-1 of the previous domain, whose link U_t(y) that
//     domain holds, so the product is formed there.
// dd_pack_kernel writes both faces of a domain (each with the fermion boundary
// sign of the global lattice when its hop crosses the global t boundary),
// the caller moves them to the neighbours, and dd_hop_kernel computes the half
// hop with the received faces in place of those two hops.  Face layout:
// [6][Vs/2] words of the spinor precision (complex128, float-float or
// complex64), Vs/2 = the sites of one parity in a t slice, indexed by the
// site's checkerboard index within its slice.
#include "hop_kernels.cuh"

namespace lqcd {

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

// blockIdx.y = 0: the face for the previous domain (sites at t = 0), 1: the
// face for the next domain (sites at t = Lt - 1, times their links U_t^+)
template <int PREC, int RECON, int S>
__global__ void __launch_bounds__(128) dd_pack_kernel(HopArgs A, int vsh, void *to_prev, void *to_next,
                                                      int neg_prev, int neg_next) {
  using R = typename SpinorIO<PREC>::R;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= vsh) return;
  const int q = A.out_parity ^ 1;  // parity of the input sites
  const SpinorView vin{A.in, A.in_scale, A.g.Vh};
  Cx<R> ps[12], h[6];
  if (blockIdx.y == 0) {
    SpinorIO<PREC>::load(vin, j, ps);
    project<3, S>(ps, h);
    negate_if(h, neg_prev != 0);
#pragma unroll
    for (int k = 0; k < 6; k++) FaceIO<PREC>::store(to_prev, vsh, k, j, h[k]);
  } else {
    const int cb = j + (A.g.L[3] - 1) * vsh;
    SpinorIO<PREC>::load(vin, cb, ps);
    project<3, -S>(ps, h);
    Cx<R> u[9], v[6];
    LinkIO<PREC, RECON>::load(A.U, q, 3, cb, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link_dag(u, h, v);
    negate_if(v, neg_next != 0);
#pragma unroll
    for (int k = 0; k < 6; k++) FaceIO<PREC>::store(to_next, vsh, k, j, v[k]);
  }
}

// The half hop on a domain: x, y, z hops as in hop_site, t hops inside the
// domain from the input field, the two boundary ones from the faces.
// REDUCE: also the per-warp |out|^2 partials of hop_warp_partial (all lanes
// of a warp reach it, so inactive lanes do not return early).
template <int PREC, int RECON, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(128) dd_hop_kernel(HopArgs A, int vsh, const void *from_next,
                                                     const void *from_prev) {
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
    hop_dir<PREC, RECON, 2, S, false>(A, s, p, cb, vin, acc);
    const int Lt = A.g.L[3];
    Cx<R> ps[12], h[6], u[9], v[6];
    // forward: (1 - S gamma_t) U_t(x) psi(x + t)
    if (s.t == Lt - 1) {
      const int j = cb - (Lt - 1) * vsh;
#pragma unroll
      for (int k = 0; k < 6; k++) h[k] = FaceIO<PREC>::load(from_next, vsh, k, j);
    } else {
      SpinorIO<PREC>::load(vin, neighbour_cb(A.g, s, 3, +1), ps);
      project<3, S>(ps, h);
    }
    LinkIO<PREC, RECON>::load(A.U, p, 3, cb, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link(u, h, v);
    accumulate<3, S>(v, acc);
    // backward: (1 + S gamma_t) U_t(x - t)^+ psi(x - t)
    if (s.t == 0) {
#pragma unroll
      for (int k = 0; k < 6; k++) v[k] = FaceIO<PREC>::load(from_prev, vsh, k, cb);
    } else {
      const int jb = neighbour_cb(A.g, s, 3, -1);
      SpinorIO<PREC>::load(vin, jb, ps);
      project<3, -S>(ps, h);
      LinkIO<PREC, RECON>::load(A.U, p ^ 1, 3, jb, u);
      if (RECON == 12) reconstruct_row2(u);
      mul_link_dag(u, h, v);
    }
    accumulate<3, -S>(v, acc);
    nrm = hop_epilogue<PREC, REDUCE>(A, cb, 0, acc);
  }
  if (REDUCE) hop_warp_partial(A, cb, 0, nrm);
}

template <int PREC, int RECON>
static void dd_launch(bool pack, bool dag, const HopArgs &A, int vsh, void *f0, void *f1, int n0, int n1,
                      cudaStream_t st) {
  if (pack) {
    const dim3 grid((unsigned)((vsh + 127) / 128), 2);
    if (dag) dd_pack_kernel<PREC, RECON, -1><<<grid, 128, 0, st>>>(A, vsh, f0, f1, n0, n1);
    else dd_pack_kernel<PREC, RECON, 1><<<grid, 128, 0, st>>>(A, vsh, f0, f1, n0, n1);
  } else {
    const unsigned grid = (unsigned)((A.g.Vh + 127) / 128);
    if (A.partials) {  // the reducing form (norms of the domain-decomposed CG)
      if (dag) dd_hop_kernel<PREC, RECON, true, true><<<grid, 128, 0, st>>>(A, vsh, f0, f1);
      else dd_hop_kernel<PREC, RECON, false, true><<<grid, 128, 0, st>>>(A, vsh, f0, f1);
      return;
    }
    if (dag) dd_hop_kernel<PREC, RECON, true, false><<<grid, 128, 0, st>>>(A, vsh, f0, f1);
    else dd_hop_kernel<PREC, RECON, false, false><<<grid, 128, 0, st>>>(A, vsh, f0, f1);
  }
}

size_t dd_face_word_bytes(int prec) { return prec == LQCD_F32 ? 8 : 16; }

// pack = true: faces (f0 = to_prev, f1 = to_next, n0/n1 = negate flags);
// pack = false: the hop (f0 = from_next, f1 = from_prev)
lqcd_status dd_run(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, bool pack, void *f0, void *f1, int n0,
                   int n1) {
  HopArgs A;
  hop_args_fill(g, L, &A);
  const int vsh = g.Lh0 * g.L[1] * g.L[2];
  const bool dag = L.dagger != 0;
  cudaStream_t st = ctx->stream;
  switch (L.prec) {
    case LQCD_F64:
      if (L.recon == 12) dd_launch<LQCD_F64, 12>(pack, dag, A, vsh, f0, f1, n0, n1, st);
      else dd_launch<LQCD_F64, 18>(pack, dag, A, vsh, f0, f1, n0, n1, st);
      break;
    case LQCD_DF64:
      if (L.recon == 12) dd_launch<LQCD_DF64, 12>(pack, dag, A, vsh, f0, f1, n0, n1, st);
      else dd_launch<LQCD_DF64, 18>(pack, dag, A, vsh, f0, f1, n0, n1, st);
      break;
    case LQCD_F32:
      if (L.recon == 12) dd_launch<LQCD_F32, 12>(pack, dag, A, vsh, f0, f1, n0, n1, st);
      else dd_launch<LQCD_F32, 18>(pack, dag, A, vsh, f0, f1, n0, n1, st);
      break;
    default: return fail(ctx, LQCD_ERR_UNSUPPORTED, "domain-decomposed hop: precision %d", L.prec);
  }
  LQCD_CUDA(ctx, cudaGetLastError());
  // algorithmic bytes: pack reads a boundary spinor (and, for the next
  // domain's face, a link) and writes 6 face words per face site; the hop is
  // counted as a half hop (8 links, input and output spinor per site)
  const double fw = 6.0 * dd_face_word_bytes(L.prec), sb = spinor_site_bytes(L.prec);
  const double lb = link_bytes_per_site(L.prec, L.recon);
  count_launch(ctx, pack ? vsh * (2.0 * (sb + fw) + lb) : (double)g.Vh * (8.0 * lb + 2.0 * sb));
  return LQCD_OK;
}

}  // namespace lqcd
