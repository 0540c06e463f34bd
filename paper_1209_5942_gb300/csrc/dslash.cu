// dslash.cu -- the hopping term of the twisted-mass Wilson matrix (Sec. 2.1,
// eq. "D_tm") on one checkerboard parity, with the site-diagonal factors
// fused into its epilogue.
//
//   out(x) = c_chi * (H in)(x) + d_chi * aux(x),   x of parity p,
//   (H in)(x) = sum_mu (1 - s gamma_mu) U_mu(x) in(x + mu)
//                    + (1 + s gamma_mu) U_mu(x - mu)^+ in(x - mu)
// with s = +1 for H and s = -1 for H^+ (dagger), the fermion boundary factor
// on hops across the time boundary, and chi = upper (spins 0,1) / lower
// (spins 2,3) chirality (gamma_5 = diag(1,1,-1,-1)).  The epilogue gives
//   t_o = A_o^-1 H_oe psi_e            (c = A^-1, no aux)
//   y_e = A_e psi_e - kappa^2 H_eo t_o (c = -kappa^2, d = A, aux = psi_e)
//   y   = A psi - kappa H psi          (full M, one launch for both parities)
//   source preparation and reconstruction of the even-odd solve.
//
// Design (GB300): one thread per output site and right-hand side; all loads
// are 16-byte words of site-ordered SoA planes, so each warp load is fully
// coalesced; neighbour spinors are reused through the 126 MB L2 (a half
// spinor of a 32^3x64 lattice streams through it as a moving t-slab).  For
// nrhs > 1 the block is (32 sites) x (nrhs), so the warps of all right-hand
// sides fetch the same link words back to back and L1 serves all but the
// first: each link is read from HBM once per site for all RHS.  The spin
// projection uses the chiral basis: (1 - s gamma_mu) psi = [h; -s B^+ h] with
// h = psi_up - s B psi_dn, gamma_mu = [[0, B], [B^+, 0]], so only the two
// upper spin components are multiplied by the link.
#include <cstdio>

#include "internal.h"

namespace lqcd {

template <int MU, int S, class R>
LQCD_DEV void project(const Cx<R> ps[12], Cx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const Cx<R> p0 = ps[c], p1 = ps[3 + c], p2 = ps[6 + c], p3 = ps[9 + c];
    if (MU == 0) {  // B = -i sigma_1:  h0 = p0 + s i p3, h1 = p1 + s i p2
      h[c] = S > 0 ? p0 + times_i(p3) : p0 - times_i(p3);
      h[3 + c] = S > 0 ? p1 + times_i(p2) : p1 - times_i(p2);
    } else if (MU == 1) {  // B = -i sigma_2: h0 = p0 + s p3, h1 = p1 - s p2
      h[c] = S > 0 ? p0 + p3 : p0 - p3;
      h[3 + c] = S > 0 ? p1 - p2 : p1 + p2;
    } else if (MU == 2) {  // B = -i sigma_3: h0 = p0 + s i p2, h1 = p1 - s i p3
      h[c] = S > 0 ? p0 + times_i(p2) : p0 - times_i(p2);
      h[3 + c] = S > 0 ? p1 - times_i(p3) : p1 + times_i(p3);
    } else {  // B = 1: h0 = p0 - s p2, h1 = p1 - s p3
      h[c] = S > 0 ? p0 - p2 : p0 + p2;
      h[3 + c] = S > 0 ? p1 - p3 : p1 + p3;
    }
  }
}

// acc += [v; -s B^+ v]
template <int MU, int S, class R>
LQCD_DEV void accumulate(const Cx<R> v[6], Cx<R> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const Cx<R> v0 = v[c], v1 = v[3 + c];
    acc[c] = acc[c] + v0;
    acc[3 + c] = acc[3 + c] + v1;
    if (MU == 0) {  // -s B^+ v = (-s i v1, -s i v0)
      acc[6 + c] = S > 0 ? acc[6 + c] - times_i(v1) : acc[6 + c] + times_i(v1);
      acc[9 + c] = S > 0 ? acc[9 + c] - times_i(v0) : acc[9 + c] + times_i(v0);
    } else if (MU == 1) {  // (-s v1, s v0)
      acc[6 + c] = S > 0 ? acc[6 + c] - v1 : acc[6 + c] + v1;
      acc[9 + c] = S > 0 ? acc[9 + c] + v0 : acc[9 + c] - v0;
    } else if (MU == 2) {  // (-s i v0, s i v1)
      acc[6 + c] = S > 0 ? acc[6 + c] - times_i(v0) : acc[6 + c] + times_i(v0);
      acc[9 + c] = S > 0 ? acc[9 + c] + times_i(v1) : acc[9 + c] - times_i(v1);
    } else {  // (-s v0, -s v1)
      acc[6 + c] = S > 0 ? acc[6 + c] - v0 : acc[6 + c] + v0;
      acc[9 + c] = S > 0 ? acc[9 + c] - v1 : acc[9 + c] + v1;
    }
  }
}

// v = U h (forward) for both upper spin components
template <class R>
LQCD_DEV void mul_link(const Cx<R> u[9], const Cx<R> h[6], Cx<R> v[6]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cx<R> s = u[3 * a] * h[3 * k];
      s = cmadd(u[3 * a + 1], h[3 * k + 1], s);
      s = cmadd(u[3 * a + 2], h[3 * k + 2], s);
      v[3 * k + a] = s;
    }
}
// v = U^+ h (backward)
template <class R>
LQCD_DEV void mul_link_dag(const Cx<R> u[9], const Cx<R> h[6], Cx<R> v[6]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cx<R> s = conj(u[a]) * h[3 * k];
      s = conj_madd(u[3 + a], h[3 * k + 1], s);
      s = conj_madd(u[6 + a], h[3 * k + 2], s);
      v[3 * k + a] = s;
    }
}

// Float-float specialisation of the colour products.  Each real output is a
// sum of six products a*b of double-words; every product contributes its
// exact leading part p = a.hi*b.hi (TwoProduct: the rounding error comes from
// one FMA) plus the first-order cross terms a.hi*b.lo + a.lo*b.hi, and the
// leading parts are summed by a TwoSum chain whose errors join the low-order
// accumulator.  The dropped a.lo*b.lo terms are below 2^-46 of each product.
struct DfAcc {
  float s, e;
};
LQCD_DEV void dfacc_add_prod(DfAcc &A, df a, df b, bool neg) {
  float ah = neg ? -a.hi : a.hi, al = neg ? -a.lo : a.lo;
  float p = __fmul_rn(ah, b.hi);
  float pe = __fmaf_rn(ah, b.hi, -p);
  pe = __fmaf_rn(ah, b.lo, pe);
  pe = __fmaf_rn(al, b.hi, pe);
  df t = two_sum(A.s, p);
  A.s = t.hi;
  A.e = __fadd_rn(A.e, __fadd_rn(t.lo, pe));
}
LQCD_DEV df dfacc_result(const DfAcc &A) { return fast_two_sum(A.s, A.e); }

// sum_j x_j * y_j (conjugating x when CONJ), complex double-words
template <bool CONJ>
LQCD_DEV Cx<df> dfdot3(const Cx<df> x0, const Cx<df> x1, const Cx<df> x2, const Cx<df> y0,
                       const Cx<df> y1, const Cx<df> y2) {
  DfAcc re{0.0f, 0.0f}, im{0.0f, 0.0f};
  const Cx<df> xs[3] = {x0, x1, x2}, ys[3] = {y0, y1, y2};
#pragma unroll
  for (int j = 0; j < 3; j++) {
    // (a + ib)(c + id) = (ac - bd) + i(ad + bc);  conj: (ac + bd) + i(ad - bc)
    dfacc_add_prod(re, xs[j].re, ys[j].re, false);
    dfacc_add_prod(re, xs[j].im, ys[j].im, !CONJ);
    dfacc_add_prod(im, xs[j].re, ys[j].im, false);
    dfacc_add_prod(im, xs[j].im, ys[j].re, CONJ);
  }
  return {dfacc_result(re), dfacc_result(im)};
}

template <>
LQCD_DEV void mul_link<df>(const Cx<df> u[9], const Cx<df> h[6], Cx<df> v[6]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int a = 0; a < 3; a++)
      v[3 * k + a] = dfdot3<false>(u[3 * a], u[3 * a + 1], u[3 * a + 2], h[3 * k], h[3 * k + 1],
                                   h[3 * k + 2]);
}
template <>
LQCD_DEV void mul_link_dag<df>(const Cx<df> u[9], const Cx<df> h[6], Cx<df> v[6]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int a = 0; a < 3; a++)
      v[3 * k + a] = dfdot3<true>(u[a], u[3 + a], u[6 + a], h[3 * k], h[3 * k + 1], h[3 * k + 2]);
}

struct HopArgs {
  Geom g;
  GaugeView U;
  char *in, *out;
  const char *aux;
  float *in_scale, *out_scale;
  const float *aux_scale;
  size_t in_rs, out_rs, aux_rs;       // bytes per rhs
  size_t in_srs, out_srs, aux_srs;    // floats per rhs
  int out_parity, nrhs, has_aux;
  HostC c_up, c_dn, d_up, d_dn;
  double *partials;
  int *halt;
};

template <class R>
LQCD_DEV void negate_if(Cx<R> v[6], bool neg) {
  if (neg) {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = -v[k];
  }
}

template <int PREC, int RECON, int MU, int S>
LQCD_DEV void hop_dir(const HopArgs &A, const Site &s, int p, int cb, const SpinorView &vin,
                      Cx<typename SpinorIO<PREC>::R> acc[12]) {
  using R = typename SpinorIO<PREC>::R;
  Cx<R> ps[12], h[6], v[6], u[9];
  // forward: (1 - S gamma_mu) U_mu(x) in(x + mu)
  {
    int j = neighbour_cb(A.g, s, MU, +1);
    SpinorIO<PREC>::load(vin, j, ps);
    project<MU, S>(ps, h);
    LinkIO<PREC, RECON>::load(A.U, p, MU, cb, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link(u, h, v);
    negate_if(v, MU == 3 && A.g.antiper && s.t == A.g.L[3] - 1);
    accumulate<MU, S>(v, acc);
  }
  // backward: (1 + S gamma_mu) U_mu(x - mu)^+ in(x - mu)
  {
    int j = neighbour_cb(A.g, s, MU, -1);
    SpinorIO<PREC>::load(vin, j, ps);
    project<MU, -S>(ps, h);
    LinkIO<PREC, RECON>::load(A.U, p ^ 1, MU, j, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link_dag(u, h, v);
    negate_if(v, MU == 3 && A.g.antiper && s.t == 0);
    accumulate<MU, -S>(v, acc);
  }
}

template <int PREC, int RECON, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(256) hop_kernel(HopArgs A) {
  using R = typename SpinorIO<PREC>::R;
  if (A.halt && *(volatile int *)A.halt) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.z * blockDim.y + threadIdx.y;
  const int p = A.out_parity;
  const bool active = cb < A.g.Vh && rhs < A.nrhs;
  double nrm = 0.0;
  if (active) {
    const Site s = site_of(A.g, p, cb);
    SpinorView vin{A.in + rhs * A.in_rs, A.in_scale ? A.in_scale + rhs * A.in_srs : nullptr, A.g.Vh};
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = czero<R>();
    constexpr int S = DAG ? -1 : 1;
    hop_dir<PREC, RECON, 0, S>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 1, S>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 2, S>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 3, S>(A, s, p, cb, vin, acc);
    // epilogue: out = c * acc + d * aux
    const Cx<R> cu = cfrom<R>(A.c_up), cd = cfrom<R>(A.c_dn);
    Cx<R> res[12];
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = (k < 6 ? cu : cd) * acc[k];
    if (A.has_aux) {
      SpinorView vaux{(void *)(A.aux + rhs * A.aux_rs),
                      A.aux_scale ? (float *)A.aux_scale + rhs * A.aux_srs : nullptr, A.g.Vh};
      Cx<R> ax[12];
      SpinorIO<PREC>::load(vaux, cb, ax);
      const Cx<R> du = cfrom<R>(A.d_up), dd = cfrom<R>(A.d_dn);
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = cmadd(k < 6 ? du : dd, ax[k], res[k]);
    }
    SpinorView vout{A.out + rhs * A.out_rs, A.out_scale ? A.out_scale + rhs * A.out_srs : nullptr,
                    A.g.Vh};
    SpinorIO<PREC>::store(vout, cb, res);
    if (REDUCE) {
#pragma unroll
      for (int k = 0; k < 12; k++) nrm += norm2_d(res[k]);
    }
  }
  if (REDUCE) {
    // one partial per warp of 32 consecutive sites, whatever the block shape,
    // so single- and multi-RHS launches reduce in the same order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0 && rhs < A.nrhs && cb < A.g.Vh) {
      const int nw = (A.g.Vh + 31) >> 5;
      A.partials[(size_t)rhs * nw + (cb >> 5)] = nrm;
    }
  }
}

// number of reduction partials per right-hand side written by a reducing hop
int hop_blocks(const Geom &g, int nrhs) {
  (void)nrhs;
  return (g.Vh + 31) / 32;
}

template <int PREC, int RECON>
static void launch_t(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) hop_kernel<PREC, RECON, true, true><<<grid, block, 0, st>>>(A);
    else hop_kernel<PREC, RECON, true, false><<<grid, block, 0, st>>>(A);
  } else {
    if (red) hop_kernel<PREC, RECON, false, true><<<grid, block, 0, st>>>(A);
    else hop_kernel<PREC, RECON, false, false><<<grid, block, 0, st>>>(A);
  }
}

lqcd_status launch_hop(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, int *nblocks_out) {
  HopArgs A;
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
  A.nrhs = L.out.nrhs;
  A.has_aux = L.has_aux ? 1 : 0;
  A.c_up = L.c_up;
  A.c_dn = L.c_dn;
  A.d_up = L.d_up;
  A.d_dn = L.d_dn;
  A.partials = L.partials;
  A.halt = L.halt;
  const int nrhs = L.out.nrhs;
  dim3 block, grid;
  if (nrhs == 1) {
    block = dim3(128, 1, 1);
    grid = dim3((g.Vh + 127) / 128, 1, 1);
  } else {
    int by = nrhs < 8 ? nrhs : 8;
    block = dim3(32, by, 1);
    grid = dim3((g.Vh + 31) / 32, 1, (nrhs + by - 1) / by);
  }
  if (nblocks_out) *nblocks_out = hop_blocks(g, nrhs);
  const bool dag = L.dagger != 0, red = L.partials != nullptr;
  cudaStream_t st = ctx->stream;
  switch (L.prec) {
    case LQCD_F64:
      if (L.recon == 12) launch_t<LQCD_F64, 12>(A, grid, block, dag, red, st);
      else launch_t<LQCD_F64, 18>(A, grid, block, dag, red, st);
      break;
    case LQCD_DF64:
      if (L.recon == 12) launch_t<LQCD_DF64, 12>(A, grid, block, dag, red, st);
      else launch_t<LQCD_DF64, 18>(A, grid, block, dag, red, st);
      break;
    case LQCD_F32:
      if (L.recon == 12) launch_t<LQCD_F32, 12>(A, grid, block, dag, red, st);
      else launch_t<LQCD_F32, 18>(A, grid, block, dag, red, st);
      break;
    case LQCD_BF16S: launch_t<LQCD_BF16S, 12>(A, grid, block, dag, red, st); break;
    case LQCD_F16S: launch_t<LQCD_F16S, 12>(A, grid, block, dag, red, st); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "launch_hop: bad precision %d", L.prec);
  }
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

}  // namespace lqcd
