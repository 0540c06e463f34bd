// dd.cu -- the face packs and the half hop on one domain of a lattice split
// along t (and optionally z); the kernels are in dd_kernels.cuh, the z-split
// hop instances in dd_z.cu.
#include "dd_kernels.cuh"

namespace lqcd {

template <int PREC, int RECON>
static void dd_pack_launch(int mu, bool dag, const HopArgs &A, int n, void *f0, void *f1, int n0, int n1,
                           cudaStream_t st) {
  const dim3 grid((unsigned)((n + 127) / 128), 2), block(128);
  if (mu == 3) {
    if (dag) launch_pdl(dd_pack_kernel<PREC, RECON, 3, -1>, grid, block, 0, st, A, n, f0, f1, n0, n1);
    else launch_pdl(dd_pack_kernel<PREC, RECON, 3, 1>, grid, block, 0, st, A, n, f0, f1, n0, n1);
  } else {
    if (dag) launch_pdl(dd_pack_kernel<PREC, RECON, 2, -1>, grid, block, 0, st, A, n, f0, f1, n0, n1);
    else launch_pdl(dd_pack_kernel<PREC, RECON, 2, 1>, grid, block, 0, st, A, n, f0, f1, n0, n1);
  }
}

size_t dd_face_word_bytes(int prec) { return prec == LQCD_F32 ? 8 : 16; }

int dd_face_sites(const Geom &g, int mu) { return g.Lh0 * g.L[1] * (mu == 3 ? g.L[2] : g.L[3]); }

// the two faces along mu (2: z, 3: t) of a domain: f0 = to_prev, f1 =
// to_next, n0 / n1 = negate them
lqcd_status dd_pack(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, int mu, void *f0, void *f1, int n0,
                    int n1) {
  if (mu != 2 && mu != 3) return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed hop: faces along z or t");
  HopArgs A;
  hop_args_fill(g, L, &A);
  const int n = dd_face_sites(g, mu);
  const bool dag = L.dagger != 0;
  cudaStream_t st = ctx->stream;
  switch (L.prec) {
    case LQCD_F64:
      if (L.recon == 12) dd_pack_launch<LQCD_F64, 12>(mu, dag, A, n, f0, f1, n0, n1, st);
      else dd_pack_launch<LQCD_F64, 18>(mu, dag, A, n, f0, f1, n0, n1, st);
      break;
    case LQCD_DF64:
      if (L.recon == 12) dd_pack_launch<LQCD_DF64, 12>(mu, dag, A, n, f0, f1, n0, n1, st);
      else dd_pack_launch<LQCD_DF64, 18>(mu, dag, A, n, f0, f1, n0, n1, st);
      break;
    case LQCD_F32:
      if (L.recon == 12) dd_pack_launch<LQCD_F32, 12>(mu, dag, A, n, f0, f1, n0, n1, st);
      else dd_pack_launch<LQCD_F32, 18>(mu, dag, A, n, f0, f1, n0, n1, st);
      break;
    default: return fail(ctx, LQCD_ERR_UNSUPPORTED, "domain-decomposed hop: precision %d", L.prec);
  }
  LQCD_CUDA(ctx, cudaGetLastError());
  // algorithmic bytes: a boundary spinor read (and, for the next domain's
  // face, a link) and 6 face words written per face site
  const double fw = 6.0 * dd_face_word_bytes(L.prec), sb = spinor_site_bytes(L.prec);
  count_launch(ctx, n * (2.0 * (sb + fw) + link_bytes_per_site(L.prec, L.recon)));
  return LQCD_OK;
}

// the domain's half hop with the received faces (z_next == nullptr: z is not
// split), counted as a half hop (8 links, input and output spinor per site)
lqcd_status dd_hop(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, const void *t_next, const void *t_prev,
                   const void *z_next, const void *z_prev) {
  HopArgs A;
  hop_args_fill(g, L, &A);
  const DdFaces F{t_next, t_prev, z_next, z_prev, dd_face_sites(g, 3), dd_face_sites(g, 2)};
  const bool dag = L.dagger != 0;
  const bool ok = z_next ? dd_hop_dispatch_z(L.prec, L.recon, dag, A, F, ctx->stream)
                         : dd_hop_dispatch<false>(L.prec, L.recon, dag, A, F, ctx->stream);
  if (!ok) return fail(ctx, LQCD_ERR_UNSUPPORTED, "domain-decomposed hop: precision %d", L.prec);
  LQCD_CUDA(ctx, cudaGetLastError());
  count_launch(ctx, (double)g.Vh * (8.0 * link_bytes_per_site(L.prec, L.recon) + 2.0 * spinor_site_bytes(L.prec)));
  return LQCD_OK;
}

}  // namespace lqcd
