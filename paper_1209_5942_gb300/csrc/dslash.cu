// dslash.cu -- the hopping term of the twisted-mass Wilson matrix (Sec. 2.1,
// eq. "D_tm") on one checkerboard parity, with the site-diagonal factors
// fused into its epilogue.  This file is the host side: launch shapes, the
// autotuner hook and the work counters; the device code is in
// hop_kernels.cuh, instantiated per precision in dslash_{f64,df64,f32,h16}.cu.
//
//   out(x) = c_chi * (H in)(x) + d_chi * aux(x),   x of parity p,
//   (H in)(x) = sum_mu (1 - s gamma_mu) U_mu(x) in(x + mu)
//                    + (1 + s gamma_mu) U_mu(x - mu)^+ in(x - mu)
// with s = +1 for H and s = -1 for H^+ (dagger), the fermion boundary factor
// on hops across the time boundary, and chi = upper (spins 0,1) / lower
// (spins 2,3) chirality (gamma_5 = diag(1,1,-1,-1)).  The epilogue gives
//   t_o = A_o^-1 H_oe psi_e            (c = A^-1, no aux)
//   y_e = A_e psi_e - kappa^2 H_eo t_o (c = -kappa^2, d = A, aux = psi_e)
//   y   = A psi - kappa H psi          (full M, one launch per parity)
//   source preparation and reconstruction of the even-odd solve.
//
// Design (GB300): one thread per output site and right-hand side (two for the
// float-float kernel with 18-real links); all loads are 16-byte words of
// site-ordered SoA planes, so each warp load is fully coalesced; neighbour
// spinors are reused through the 126 MB L2.  For nrhs > 1 the block is
// (32 sites) x (RHS), so the warps of all right-hand sides fetch the same link
// words back to back and L1 serves all but the first; for the memory-bound
// formats a thread may also own 2 or 4 right-hand sides and apply each loaded
// link to all of them (register blocking).  The spin projection
// uses the chiral basis: (1 - s gamma_mu) psi = [h; -s B^+ h] with
// h = psi_up - s B psi_dn, gamma_mu = [[0, B], [B^+, 0]], so only the two
// upper spin components are multiplied by the link.
#include <cstdio>

#include "hop_kernels.cuh"

namespace lqcd {

// number of reduction partials per right-hand side written by a reducing hop
int hop_blocks(const Geom &g, int nrhs) {
  (void)nrhs;
  return (g.Vh + 31) / 32;
}

lqcd_status launch_hop(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, int *nblocks_out) {
  HopArgs A;
  hop_args_fill(g, L, &A);
  A.nrhs = L.out.nrhs;
  A.halt = L.halt;
  const int nrhs = L.out.nrhs;
  if (nblocks_out) *nblocks_out = hop_blocks(g, nrhs);
  const bool dag = L.dagger != 0, red = L.partials != nullptr;
  if (L.prec < LQCD_F64 || L.prec > LQCD_F16S)
    return fail(ctx, LQCD_ERR_INVALID, "launch_hop: bad precision %d", L.prec);
  if (nrhs < 1) return fail(ctx, LQCD_ERR_INVALID, "launch_hop: nrhs %d", nrhs);
  // Candidate launches (results never depend on the choice):
  //  - one RHS: blocks of 64/128/256 sites;
  //  - several RHS: blocks of 32 sites x {1,2,4,8} RHS, one RHS per thread,
  //    and for the memory-bound formats also 32 sites x {1,2,4} groups of
  //    rt = 2 or 4 RHS per thread (the register-blocked kernel);
  //  each with a full grid (one site per thread) or a persistent grid of 4 or
  //  8 blocks per SM, and for the memory-bound one-RHS-per-thread kernels both
  //  load orders.  The float-float kernel with 18-real links runs two threads
  //  per site and is bounded to 128 threads per block; it comes in scalar
  //  and in packed FP32x2 arithmetic, the packed form also with its operands
  //  staged through shared memory (bounded to 128 or to 96 registers).
  struct Cand {
    short bx, by, gm, rt;
    bool lf, two;  // two: two sites per thread in packed FP32x2
    char pk;       // float-float pair kernel: 0 scalar, 1 packed FP32x2, 2 packed + shared-memory
                   // staging; 16-bit two-site kernel: 1 = operands staged in shared memory
    char mr;       // links staged in shared memory for a group of RHS: 0 no, else the
                   // reals kept per link (18, or 12 with the third row rebuilt per RHS)
    short rg;      // with mr: right-hand sides per block
    bool ri;       // F32, several RHS: RHS interleaved with the site blocks (hop_ri_kernel)
  };
  Cand cands[96];
  int ncand = 0, fallback = 0;
  const bool low = L.prec == LQCD_F32 || L.prec == LQCD_BF16S || L.prec == LQCD_F16S;
  const bool pair = L.prec == LQCD_DF64 && L.recon == 18;
  static const short GM[3] = {0, 4, 8};
  for (int gi = 0; gi < 3; gi++)
    for (int lf = 0; lf < (low ? 2 : 1); lf++) {
      if (pair) {
        for (char pk = 0; pk < 4; pk++) {
          if (nrhs == 1) {
            cands[ncand++] = {64, 1, GM[gi], 1, false, false, pk};
            cands[ncand++] = {128, 1, GM[gi], 1, false, false, pk};
          } else {
            cands[ncand++] = {64, 1, GM[gi], 1, false, false, pk};
            cands[ncand++] = {64, 2, GM[gi], 1, false, false, pk};
          }
        }
      } else if (nrhs == 1) {
        for (short bx : {64, 128, 256}) cands[ncand++] = {bx, 1, GM[gi], 1, lf != 0};
      } else {
        for (short by : {1, 2, 4, 8})
          if (by <= nrhs) cands[ncand++] = {32, by, GM[gi], 1, lf != 0};
      }
    }
  if (low && nrhs > 1)
    for (int gi = 0; gi < 3; gi++)
      for (short rt : {2, 4})
        for (short by : {1, 2, 4})
          if (rt * by <= nrhs) cands[ncand++] = {32, by, GM[gi], rt, false};
  // links staged in shared memory once per site for a group of rg RHS
  // (blocks of 32 or 64 sites; the whole RHS set, half or a quarter of it)
  if (low && nrhs > 1)
    for (short bx : {32, 64})
      for (char mr : {(char)18, (char)12}) {
        if (mr == 12 && L.recon != 12) continue;
        short prev = 0;
        for (int q : {1, 2, 4}) {
          const short rg = (short)((nrhs + q - 1) / q);
          if (rg == prev || rg < 1) continue;
          prev = rg;
          cands[ncand++] = {bx, 1, 0, 1, false, false, 0, mr, rg};
        }
      }
  // F32: the RHS interleaved with the site blocks, blocks of 32 or 64 sites
  if (L.prec == LQCD_F32 && nrhs > 1)
    for (int gi = 0; gi < 3; gi++)
      for (short bx : {32, 64}) cands[ncand++] = {bx, 1, GM[gi], 1, true, false, 0, 0, 0, true};
  // packed two-site kernel: blocks of 64 threads = 128 sites, one RHS per block row
  if (low)
    for (int gi = 0; gi < 3; gi++) cands[ncand++] = {64, 1, GM[gi], 1, false, true};
  // for the 16-bit formats also with its operands staged through shared memory
  if (L.prec == LQCD_BF16S || L.prec == LQCD_F16S)
    for (int gi = 0; gi < 3; gi++) cands[ncand++] = {64, 1, GM[gi], 1, false, true, 1};
  // default without tuning: the full-grid, one-RHS-per-thread candidate with
  // 128-site blocks for one RHS, or with the most RHS per block for several
  for (int c = 0; c < ncand; c++) {
    const Cand &k = cands[c];
    if (k.gm != 0 || k.lf || k.rt != 1 || k.two || k.pk != 0) continue;
    if (nrhs == 1 ? k.bx == 128 : k.by >= cands[fallback].by) fallback = c;
  }
  auto go = [&](int ci, const HopArgs &args) {
    const Cand &k = cands[ci];
    if (k.mr) {
      const dim3 block(k.bx, 1, 1), grid((g.Vh + k.bx - 1) / k.bx, (nrhs + k.rg - 1) / k.rg, 1);
      if (L.prec == LQCD_F32) hop_launch_mrhs_f32(args, L.recon, k.mr, k.rg, grid, block, dag, red, ctx->stream);
      else hop_launch_mrhs_h16(args, L.prec, k.mr, k.rg, grid, block, dag, red, ctx->stream);
      return;
    }
    if (k.ri) {
      // one block per (site block, RHS), RHS fastest; a persistent grid keeps
      // whole groups of nrhs blocks
      unsigned gx = (unsigned)((g.Vh + k.bx - 1) / k.bx) * (unsigned)nrhs;
      if (k.gm > 0) {
        const unsigned cap = (unsigned)(ctx->num_sms * k.gm) / nrhs * nrhs;
        if (cap >= (unsigned)nrhs && gx > cap) gx = cap;
      }
      hop_launch_f32_ri(args, L.recon, dim3(gx, 1, 1), dim3(k.bx, 1, 1), dag, red, ctx->stream);
      return;
    }
    const int rt = k.rt;
    dim3 block(k.bx, k.by, 1), grid;
    const int per_block = pair ? k.bx / 2 : (k.two ? 2 * k.bx : k.bx);  // sites per block row
    const int groups = (nrhs + rt - 1) / rt;                             // RHS groups (of rt) to cover
    grid = dim3((g.Vh + per_block - 1) / per_block, 1, (groups + k.by - 1) / k.by);
    if (k.gm > 0) {
      unsigned cap = (unsigned)(ctx->num_sms * k.gm);
      if (grid.x > cap) grid.x = cap;
    }
    cudaStream_t st = ctx->stream;
    switch (L.prec) {
      case LQCD_F64: hop_launch_f64(args, L.recon, grid, block, dag, red, st); break;
      case LQCD_DF64: hop_launch_df64(args, L.recon, pair, k.pk, grid, block, dag, red, st); break;
      case LQCD_F32: hop_launch_f32(args, L.recon, grid, block, dag, red, k.lf, rt, k.two, st); break;
      default: hop_launch_h16(args, L.prec, grid, block, dag, red, k.lf, rt, k.two, k.pk != 0, st); break;
    }
  };
  char key[160];
  snprintf(key, sizeof(key), "hop7|p%d|r%d|d%d|red%d|aux%d|%dx%dx%dx%d|n%d", L.prec, L.recon, (int)dag, (int)red,
           A.has_aux, g.L[0], g.L[1], g.L[2], g.L[3], nrhs);
  HopArgs At = A;
  At.halt = nullptr;  // timing launches run whatever the solver state
  const int choice = tune_choice(ctx, key, ncand, fallback, [&](int c) { go(c, At); });
  go(choice, A);
  LQCD_CUDA(ctx, cudaGetLastError());
  // algorithmic work: per output site 8 links, the input spinor once, the
  // output (and aux) spinor; 1320 flops for the hop + 48 per epilogue term
  const double sites = (double)g.Vh * nrhs;
  const double link_b = 8.0 * link_bytes_per_site(L.prec, L.recon) * g.Vh;  // shared by all RHS
  const double sb = spinor_site_bytes(L.prec);
  const double bytes = link_b + sites * sb * (2.0 + (L.has_aux ? 1.0 : 0.0));
  const bool trivial_c = L.c_up.re == 1.0 && L.c_up.im == 0.0 && L.c_dn.re == 1.0 && L.c_dn.im == 0.0;
  const double flops = sites * (1320.0 + (trivial_c ? 0.0 : 48.0) + (L.has_aux ? 48.0 : 0.0));
  count_launch(ctx, bytes);
  ctx->cnt.hop_launches += 1;
  ctx->cnt.hop_bytes += bytes;
  ctx->cnt.hop_flops += flops;
  ctx->cnt.hop_sites += sites;
  return LQCD_OK;
}

// Launches the batched hop: descs[nsys] on the device (one per system, each
// with its own geometry, fields and coefficients), tiles[ntiles] = (system,
// first cb) with 128-site tiles.  All systems share precision and recon.
lqcd_status launch_hop_batched(lqcd_ctx *ctx, int prec, int recon, bool dagger, bool reduce,
                               const void *descs, const void *tiles, int ntiles, int grid, const int *halt) {
  const HopArgs *d = (const HopArgs *)descs;
  const int2 *tl = (const int2 *)tiles;
  cudaStream_t st = ctx->stream;
  switch (prec) {
    case LQCD_F64: hop_batched_f64(recon, dagger, reduce, d, tl, ntiles, grid, halt, st); break;
    case LQCD_DF64: hop_batched_df64(recon, dagger, reduce, d, tl, ntiles, grid, halt, st); break;
    case LQCD_F32: hop_batched_f32(recon, dagger, reduce, d, tl, ntiles, grid, halt, st); break;
    case LQCD_BF16S:
    case LQCD_F16S: hop_batched_h16(prec, dagger, reduce, d, tl, ntiles, grid, halt, st); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "batched hop: bad precision");
  }
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

// Host-side HopArgs for a HopLaunch (what launch_hop passes to the kernel).
size_t hop_args_size() { return sizeof(HopArgs); }
void hop_args_fill(const Geom &g, const HopLaunch &L, void *dst) {
  HopArgs &A = *(HopArgs *)dst;
  A.g = g;
  A.U = L.U;
  A.in = (char *)L.in.ptr;
  A.out = (char *)L.out.ptr;
  A.aux = (const char *)L.aux.ptr;
  A.in_scale = L.in.scale;
  A.out_scale = L.out.scale;
  A.aux_scale = L.aux.scale;
  A.in_rs = L.in.rhs_stride;
  A.out_rs = L.out.rhs_stride;
  A.aux_rs = L.aux.rhs_stride;
  A.in_srs = L.in.scale_rhs_stride;
  A.out_srs = L.out.scale_rhs_stride;
  A.aux_srs = L.aux.scale_rhs_stride;
  A.out_parity = L.out_parity;
  A.nrhs = 1;
  A.has_aux = L.has_aux ? 1 : 0;
  A.c_up = L.c_up;
  A.c_dn = L.c_dn;
  A.c_one = L.c_up.re == 1.0 && L.c_up.im == 0.0 && L.c_dn.re == 1.0 && L.c_dn.im == 0.0;
  A.d_up = L.d_up;
  A.d_dn = L.d_dn;
  A.co = make_coef4(L.c_up, L.c_dn, L.d_up, L.d_dn);
  A.partials = L.partials;
  A.halt = nullptr;
}

}  // namespace lqcd
