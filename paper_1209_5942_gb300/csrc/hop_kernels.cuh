// hop_kernels.cuh -- device code of the hopping term (included by the
// per-precision translation units dslash_*.cu; see dslash.cu for the design).
#pragma once
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

// acc += f sc w for f = +1, -1, +i, -i (F_P1, F_M1, F_PI, F_MI), in FMAs
enum { F_P1 = 0, F_M1 = 1, F_PI = 2, F_MI = 3 };
template <int F> LQCD_DEV void add_f(Cx<float> &acc, float sc, Cx<float> w) {
  if (F == F_P1) acc = {__fmaf_rn(sc, w.re, acc.re), __fmaf_rn(sc, w.im, acc.im)};
  else if (F == F_M1) acc = {__fmaf_rn(-sc, w.re, acc.re), __fmaf_rn(-sc, w.im, acc.im)};
  else if (F == F_PI) acc = {__fmaf_rn(-sc, w.im, acc.re), __fmaf_rn(sc, w.re, acc.im)};
  else acc = {__fmaf_rn(sc, w.im, acc.re), __fmaf_rn(-sc, w.re, acc.im)};
}

// the same on two lanes (two output sites) with the packed FP32x2 FMA
template <int F> LQCD_DEV void add_f(Cx<float2> &acc, float2 sc, Cx<float2> w) {
  const float2 ms = neg2(sc);
  if (F == F_P1) acc = {__ffma2_rn(sc, w.re, acc.re), __ffma2_rn(sc, w.im, acc.im)};
  else if (F == F_M1) acc = {__ffma2_rn(ms, w.re, acc.re), __ffma2_rn(ms, w.im, acc.im)};
  else if (F == F_PI) acc = {__ffma2_rn(ms, w.im, acc.re), __ffma2_rn(sc, w.re, acc.im)};
  else acc = {__ffma2_rn(sc, w.im, acc.re), __ffma2_rn(ms, w.re, acc.im)};
}

// acc += sc [v; -s B^+ v]: accumulate<MU, S> with the neighbour's 16-bit
// storage scale (and the boundary sign) applied in the accumulation FMAs.
// With sc = +-1 it is accumulate<MU, S> of (+-v) with the same roundings.
template <int MU, int S, class RV, class RS>
LQCD_DEV void accumulate_scaled(const Cx<RV> v[6], RS sc, Cx<RV> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const Cx<RV> v0 = v[c], v1 = v[3 + c];
    add_f<F_P1>(acc[c], sc, v0);
    add_f<F_P1>(acc[3 + c], sc, v1);
    if (MU == 0) {
      add_f<(S > 0 ? F_MI : F_PI)>(acc[6 + c], sc, v1);
      add_f<(S > 0 ? F_MI : F_PI)>(acc[9 + c], sc, v0);
    } else if (MU == 1) {
      add_f<(S > 0 ? F_M1 : F_P1)>(acc[6 + c], sc, v1);
      add_f<(S > 0 ? F_P1 : F_M1)>(acc[9 + c], sc, v0);
    } else if (MU == 2) {
      add_f<(S > 0 ? F_MI : F_PI)>(acc[6 + c], sc, v0);
      add_f<(S > 0 ? F_PI : F_MI)>(acc[9 + c], sc, v1);
    } else {
      add_f<(S > 0 ? F_M1 : F_P1)>(acc[6 + c], sc, v0);
      add_f<(S > 0 ? F_M1 : F_P1)>(acc[9 + c], sc, v1);
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
  int c_one;  // c_up = c_dn = 1: the epilogue skips the multiplication
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

// Neighbour spinor load: 16-bit formats return their values unscaled with
// the site scale, which acc_nb applies; other formats return scale 1.
template <int PREC>
LQCD_DEV float load_nb(const SpinorView &vin, int j, Cx<typename SpinorIO<PREC>::R> ps[12]) {
  if constexpr (kScaled16<PREC>) {
    return SpinorIO<PREC>::load_unscaled(vin, j, ps);
  } else {
    SpinorIO<PREC>::load(vin, j, ps);
    return 1.0f;
  }
}
// acc += (neg ? -1 : 1) sc [v; -s B^+ v]
template <int PREC, int MU, int S>
LQCD_DEV void acc_nb(Cx<typename SpinorIO<PREC>::R> v[6], float sc, bool neg,
                     Cx<typename SpinorIO<PREC>::R> acc[12]) {
  if constexpr (kScaled16<PREC>) {
    accumulate_scaled<MU, S>(v, neg ? -sc : sc, acc);
  } else {
    (void)sc;
    negate_if(v, neg);
    accumulate<MU, S>(v, acc);
  }
}

template <int PREC, int RECON, int MU, int S, bool LF = true>
LQCD_DEV void hop_dir(const HopArgs &A, const Site &s, int p, int cb, const SpinorView &vin,
                      Cx<typename SpinorIO<PREC>::R> acc[12]) {
  using R = typename SpinorIO<PREC>::R;
  Cx<R> ps[12], h[6], v[6], u[9];
  const bool negf = MU == 3 && A.g.antiper && s.t == A.g.L[3] - 1;
  const bool negb = MU == 3 && A.g.antiper && s.t == 0;
  if (LF && (PREC == LQCD_F32 || PREC == LQCD_BF16S || PREC == LQCD_F16S)) {
    // memory-bound formats: issue both neighbours' spinor and link loads
    // before any arithmetic, so one thread has four load groups in flight
    const int jf = neighbour_cb(A.g, s, MU, +1), jb = neighbour_cb(A.g, s, MU, -1);
    Cx<R> pb[12], ub[9];
    const float scf = load_nb<PREC>(vin, jf, ps);
    LinkIO<PREC, RECON>::load(A.U, p, MU, cb, u);
    const float scb = load_nb<PREC>(vin, jb, pb);
    LinkIO<PREC, RECON>::load(A.U, p ^ 1, MU, jb, ub);
    project<MU, S>(ps, h);
    if (RECON == 12) reconstruct_row2(u);
    mul_link(u, h, v);
    acc_nb<PREC, MU, S>(v, scf, negf, acc);
    project<MU, -S>(pb, h);
    if (RECON == 12) reconstruct_row2(ub);
    mul_link_dag(ub, h, v);
    acc_nb<PREC, MU, -S>(v, scb, negb, acc);
    return;
  }
  // forward: (1 - S gamma_mu) U_mu(x) in(x + mu)
  {
    int j = neighbour_cb(A.g, s, MU, +1);
    const float sc = load_nb<PREC>(vin, j, ps);
    project<MU, S>(ps, h);
    LinkIO<PREC, RECON>::load(A.U, p, MU, cb, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link(u, h, v);
    acc_nb<PREC, MU, S>(v, sc, negf, acc);
  }
  // backward: (1 + S gamma_mu) U_mu(x - mu)^+ in(x - mu)
  {
    int j = neighbour_cb(A.g, s, MU, -1);
    const float sc = load_nb<PREC>(vin, j, ps);
    project<MU, -S>(ps, h);
    LinkIO<PREC, RECON>::load(A.U, p ^ 1, MU, j, u);
    if (RECON == 12) reconstruct_row2(u);
    mul_link_dag(u, h, v);
    acc_nb<PREC, MU, -S>(v, sc, negb, acc);
  }
}

// Epilogue of one output site and right-hand side: out = c * acc + d * aux,
// the store, and the site's |out|^2 (the REDUCE partial's summand).
template <int PREC, bool REDUCE>
LQCD_DEV double hop_epilogue(const HopArgs &A, int cb, int rhs, const Cx<typename SpinorIO<PREC>::R> acc[12]) {
  using R = typename SpinorIO<PREC>::R;
  const Cx<R> cu = cfrom<R>(A.c_up), cd = cfrom<R>(A.c_dn);
  Cx<R> res[12];
  if (A.c_one) {
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = acc[k];
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = (k < 6 ? cu : cd) * acc[k];
  }
  if (A.has_aux) {
    SpinorView vaux{(void *)(A.aux + rhs * A.aux_rs),
                    A.aux_scale ? (float *)A.aux_scale + rhs * A.aux_srs : nullptr, A.g.Vh};
    Cx<R> ax[12];
    SpinorIO<PREC>::load(vaux, cb, ax);
    const Cx<R> du = cfrom<R>(A.d_up), dd = cfrom<R>(A.d_dn);
#pragma unroll
    for (int k = 0; k < 12; k++) res[k] = cmadd(k < 6 ? du : dd, ax[k], res[k]);
  }
  SpinorView vout{A.out + rhs * A.out_rs, A.out_scale ? A.out_scale + rhs * A.out_srs : nullptr, A.g.Vh};
  SpinorIO<PREC>::store(vout, cb, res);
  return REDUCE ? site_norm2<R, 12>(res) : 0.0;
}

// One partial per warp of 32 consecutive sites, whatever the block shape or
// the number of right-hand sides per thread, so every launch shape reduces in
// the same order.  All 32 lanes of the warp call it together.
LQCD_DEV void hop_warp_partial(const HopArgs &A, int cb, int rhs, double nrm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0 && rhs < A.nrhs && cb < A.g.Vh) {
    const int nw = (A.g.Vh + 31) >> 5;
    A.partials[(size_t)rhs * nw + (cb >> 5)] = nrm;
  }
}

// Output site cb (of parity A.out_parity) for right-hand side rhs: the hop,
// the epilogue, the store and (REDUCE) the warp's |out|^2 partial.  All 32
// lanes of a warp must call it together (the partial uses a shuffle).
template <int PREC, int RECON, bool DAG, bool REDUCE, bool LF = true>
LQCD_DEV void hop_site(const HopArgs &A, int cb, int rhs) {
  using R = typename SpinorIO<PREC>::R;
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
    hop_dir<PREC, RECON, 0, S, LF>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 1, S, LF>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 2, S, LF>(A, s, p, cb, vin, acc);
    hop_dir<PREC, RECON, 3, S, LF>(A, s, p, cb, vin, acc);
    nrm = hop_epilogue<PREC, REDUCE>(A, cb, rhs, acc);
  }
  if (REDUCE) hop_warp_partial(A, cb, rhs, nrm);
}

// ---------------------------------------------------------------------------
// Register-blocked multi-RHS hop: one thread owns one output site and RT
// consecutive right-hand sides.  Each link is loaded (and its third row
// rebuilt) once per direction and applied to the RT neighbour spinors, which
// cuts the per-RHS load and reconstruction instructions by RT.  Every RHS goes
// through the same arithmetic, in the same order, as in hop_site, so the
// results are bitwise those of single-RHS launches.  Right-hand sides past
// nrhs (a ragged last group) recompute the last valid one and are not stored.
// ---------------------------------------------------------------------------
template <int PREC, int RECON, int MU, int S, int RT>
LQCD_DEV void hop_dir_rt(const HopArgs &A, const Site &s, int p, int cb, const int rhs[RT],
                         Cx<typename SpinorIO<PREC>::R> acc[RT][12]) {
  using R = typename SpinorIO<PREC>::R;
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int j = neighbour_cb(A.g, s, MU, dir == 0 ? +1 : -1);
    Cx<R> u[9];
    LinkIO<PREC, RECON>::load(A.U, dir == 0 ? p : p ^ 1, MU, dir == 0 ? cb : j, u);
    // project each neighbour spinor as soon as it arrives: only the RT
    // half spinors (6 complex each) stay live across the link product
    Cx<R> h[RT][6];
    float sc[RT];
#pragma unroll
    for (int r = 0; r < RT; r++) {
      SpinorView vin{A.in + rhs[r] * A.in_rs, A.in_scale ? A.in_scale + rhs[r] * A.in_srs : nullptr, A.g.Vh};
      Cx<R> ps[12];
      sc[r] = load_nb<PREC>(vin, j, ps);
      if (dir == 0) project<MU, S>(ps, h[r]);
      else project<MU, -S>(ps, h[r]);
    }
    if (RECON == 12) reconstruct_row2(u);
    const bool neg = MU == 3 && A.g.antiper && s.t == (dir == 0 ? A.g.L[3] - 1 : 0);
#pragma unroll
    for (int r = 0; r < RT; r++) {
      Cx<R> v[6];
      if (dir == 0) {
        mul_link(u, h[r], v);
        acc_nb<PREC, MU, S>(v, sc[r], neg, acc[r]);
      } else {
        mul_link_dag(u, h[r], v);
        acc_nb<PREC, MU, -S>(v, sc[r], neg, acc[r]);
      }
    }
  }
}

template <int PREC, int RECON, bool DAG, bool REDUCE, int RT>
LQCD_DEV void hop_site_rt(const HopArgs &A, int cb, int rhs0) {
  using R = typename SpinorIO<PREC>::R;
  const int p = A.out_parity;
  int rhs[RT];
#pragma unroll
  for (int r = 0; r < RT; r++) rhs[r] = min(rhs0 + r, A.nrhs - 1);
  double nrm[RT];
#pragma unroll
  for (int r = 0; r < RT; r++) nrm[r] = 0.0;
  if (cb < A.g.Vh) {
    const Site s = site_of(A.g, p, cb);
    Cx<R> acc[RT][12];
#pragma unroll
    for (int r = 0; r < RT; r++)
#pragma unroll
      for (int k = 0; k < 12; k++) acc[r][k] = czero<R>();
    constexpr int S = DAG ? -1 : 1;
    hop_dir_rt<PREC, RECON, 0, S, RT>(A, s, p, cb, rhs, acc);
    hop_dir_rt<PREC, RECON, 1, S, RT>(A, s, p, cb, rhs, acc);
    hop_dir_rt<PREC, RECON, 2, S, RT>(A, s, p, cb, rhs, acc);
    hop_dir_rt<PREC, RECON, 3, S, RT>(A, s, p, cb, rhs, acc);
#pragma unroll
    for (int r = 0; r < RT; r++)
      if (rhs0 + r < A.nrhs) nrm[r] = hop_epilogue<PREC, REDUCE>(A, cb, rhs0 + r, acc[r]);
  }
  if (REDUCE) {
#pragma unroll
    for (int r = 0; r < RT; r++) hop_warp_partial(A, cb, rhs0 + r, nrm[r]);
  }
}

// Blocks of 32 sites x blockDim.y RHS groups of RT; grid z covers the groups.
template <int PREC, int RECON, bool DAG, bool REDUCE, int RT>
__global__ void __launch_bounds__(128) hop_rt_kernel(HopArgs A) {
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs0 = (blockIdx.z * blockDim.y + threadIdx.y) * RT;
  if (rhs0 >= A.nrhs) return;  // whole warps: blockDim.x is 32
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < A.g.Vh; base += stride)
    hop_site_rt<PREC, RECON, DAG, REDUCE, RT>(A, base + threadIdx.x, rhs0);
}

// Grid-stride over the output sites: a full grid (one site per thread) or a
// smaller persistent grid, whichever the autotuner finds faster.
// LF selects, for the memory-bound formats, whether both neighbours' loads of
// a direction are issued before its arithmetic (the autotuner picks).
template <int PREC, int RECON, bool DAG, bool REDUCE, bool LF>
__global__ void __launch_bounds__(256) hop_kernel(HopArgs A) {
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z * blockDim.y + threadIdx.y;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < A.g.Vh; base += stride)
    hop_site<PREC, RECON, DAG, REDUCE, LF>(A, base + threadIdx.x, rhs);
}

// ---------------------------------------------------------------------------
// Two output sites per thread in packed FP32x2 arithmetic (F32 and 16-bit
// formats): lane x of every float2 belongs to site cb, lane y to site cb + 32,
// so a warp covers 64 consecutive sites as two groups of 32 and writes the
// same per-warp partials as the one-site kernels.  Every packed operation
// rounds as its scalar counterpart, and the F32 format accumulates through
// the scaled form with scale +-1 (the same roundings as negate + add), so the
// results are bitwise those of hop_site.  Half the FP32 instructions per site
// for the same loads.
// ---------------------------------------------------------------------------
template <int PREC, int RECON>
LQCD_DEV void load_link2(const GaugeView &U, int p, int mu, int cbA, int cbB, Cx<float2> u[9]) {
  Cx<float> a[9], b[9];
  LinkIO<PREC, RECON>::load(U, p, mu, cbA, a);
  LinkIO<PREC, RECON>::load(U, p, mu, cbB, b);
#pragma unroll
  for (int k = 0; k < (RECON == 18 ? 9 : 6); k++) u[k] = cpair(a[k], b[k]);
}
template <int PREC>
LQCD_DEV float2 load_nb2(const SpinorView &vin, int jA, int jB, Cx<float2> ps[12]) {
  Cx<float> a[12], b[12];
  const float sa = load_nb<PREC>(vin, jA, a), sb = load_nb<PREC>(vin, jB, b);
#pragma unroll
  for (int k = 0; k < 12; k++) ps[k] = cpair(a[k], b[k]);
  return make_float2(sa, sb);
}

template <int PREC, int RECON, int MU, int S>
LQCD_DEV void hop_dir2(const HopArgs &A, const Site &sA, const Site &sB, int p, int cbA, int cbB,
                       const SpinorView &vin, Cx<float2> acc[12]) {
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int d = dir == 0 ? +1 : -1;
    const int jA = neighbour_cb(A.g, sA, MU, d), jB = neighbour_cb(A.g, sB, MU, d);
    Cx<float2> ps[12], h[6], v[6], u[9];
    float2 sc = load_nb2<PREC>(vin, jA, jB, ps);
    if (dir == 0) load_link2<PREC, RECON>(A.U, p, MU, cbA, cbB, u);
    else load_link2<PREC, RECON>(A.U, p ^ 1, MU, jA, jB, u);
    const int tb = dir == 0 ? A.g.L[3] - 1 : 0;
    if (MU == 3 && A.g.antiper) {
      if (sA.t == tb) sc.x = -sc.x;
      if (sB.t == tb) sc.y = -sc.y;
    }
    if (dir == 0) {
      project<MU, S>(ps, h);
      if (RECON == 12) reconstruct_row2(u);
      mul_link(u, h, v);
      accumulate_scaled<MU, S>(v, sc, acc);
    } else {
      project<MU, -S>(ps, h);
      if (RECON == 12) reconstruct_row2(u);
      mul_link_dag(u, h, v);
      accumulate_scaled<MU, -S>(v, sc, acc);
    }
  }
}

template <int PREC, int RECON, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(64) hop_pair2_kernel(HopArgs A) {
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = A.out_parity;
  const int stride = gridDim.x * 128;
  for (int base = blockIdx.x * 128; base < A.g.Vh; base += stride) {
    const int cbA = base + 64 * w + lane, cbB = cbA + 32;
    const bool okA = cbA < A.g.Vh && rhs < A.nrhs, okB = cbB < A.g.Vh && rhs < A.nrhs;
    // lanes past the end recompute a valid site and store nothing
    const int cA = okA ? cbA : A.g.Vh - 1, cB = okB ? cbB : A.g.Vh - 1;
    const int r = rhs < A.nrhs ? rhs : A.nrhs - 1;
    const Site sA = site_of(A.g, p, cA), sB = site_of(A.g, p, cB);
    SpinorView vin{A.in + r * A.in_rs, A.in_scale ? A.in_scale + r * A.in_srs : nullptr, A.g.Vh};
    Cx<float2> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = czero<float2>();
    constexpr int S = DAG ? -1 : 1;
    hop_dir2<PREC, RECON, 0, S>(A, sA, sB, p, cA, cB, vin, acc);
    hop_dir2<PREC, RECON, 1, S>(A, sA, sB, p, cA, cB, vin, acc);
    hop_dir2<PREC, RECON, 2, S>(A, sA, sB, p, cA, cB, vin, acc);
    hop_dir2<PREC, RECON, 3, S>(A, sA, sB, p, cA, cB, vin, acc);
    double nA = 0.0, nB = 0.0;
    {
      Cx<float> a[12];
#pragma unroll
      for (int k = 0; k < 12; k++) a[k] = lane_x(acc[k]);
      if (okA) nA = hop_epilogue<PREC, REDUCE>(A, cbA, rhs, a);
    }
    {
      Cx<float> b[12];
#pragma unroll
      for (int k = 0; k < 12; k++) b[k] = lane_y(acc[k]);
      if (okB) nB = hop_epilogue<PREC, REDUCE>(A, cbB, rhs, b);
    }
    if (REDUCE) {
      hop_warp_partial(A, cbA, rhs, nA);
      hop_warp_partial(A, cbB, rhs, nB);
    }
  }
}

template <int PREC, int RECON>
inline void launch_pair2(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) hop_pair2_kernel<PREC, RECON, true, true><<<grid, block, 0, st>>>(A);
    else hop_pair2_kernel<PREC, RECON, true, false><<<grid, block, 0, st>>>(A);
  } else {
    if (red) hop_pair2_kernel<PREC, RECON, false, true><<<grid, block, 0, st>>>(A);
    else hop_pair2_kernel<PREC, RECON, false, false><<<grid, block, 0, st>>>(A);
  }
}

// ---------------------------------------------------------------------------
// Float-float hop with two threads per output site.  Thread k (lane parity)
// owns upper spin component k: it projects only h_k, multiplies it by the
// link one row (forward) or column (backward) at a time, and accumulates the
// upper spin k plus two partial lower spins: the one receiving v_k in the x,y
// directions (spin 3-k) and the one receiving it in z,t (spin 2+k).  The
// partner lane's x,y partial completes lower spin 2+k through one shuffle.
// Per thread this halves the dependent float-float chains and the register
// footprint, so twice as many warps hide the FP32 latency.
// ---------------------------------------------------------------------------
template <int MU, int S>
LQCD_DEV void df_pair_dir(const HopArgs &A, const Site &s, int p, int cb, int k, const SpinorView &vin,
                          Cx<df> up[3], Cx<df> lswap[3], Cx<df> lsame[3]) {
  const float4 *pin = (const float4 *)vin.ptr;
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int sgn = dir == 0 ? S : -S;  // projector sign: (1 - S g) forward, (1 + S g) backward
    const int j = neighbour_cb(A.g, s, MU, dir == 0 ? +1 : -1);
    const int lo = (MU < 2) ? 3 - k : 2 + k;  // lower spin paired with upper k in h_k
    Cx<df> h[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float4 a = __ldg(pin + (size_t)(3 * k + c) * vin.Vh + j);
      float4 b = __ldg(pin + (size_t)(3 * lo + c) * vin.Vh + j);
      Cx<df> pa = {{a.x, a.z}, {a.y, a.w}}, pb = {{b.x, b.z}, {b.y, b.w}};
      // h_k = p_k + f * p_lo with f = S*i (x), S*(+-1) (y), S*(+-i) (z), -S (t)
      const bool neg = (MU == 0) ? sgn < 0 : (MU == 1) ? (k == 0 ? sgn < 0 : sgn > 0)
                     : (MU == 2) ? (k == 0 ? sgn < 0 : sgn > 0) : sgn > 0;
      Cx<df> t = (MU == 0 || MU == 2) ? times_i(pb) : pb;
      h[c] = neg ? csub_lazy(pa, t) : cadd_lazy(pa, t);
    }
    const float4 *ub = (const float4 *)((const char *)A.U.ptr + (dir == 0 ? p : p ^ 1) * A.U.parity_stride +
                                        MU * A.U.mu_stride);
    const int lc = dir == 0 ? cb : j;
    Cx<df> v[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cx<df> u3[3];
#pragma unroll
      for (int q = 0; q < 3; q++) {  // forward: row a of U; backward: column a
        float4 w = __ldg(ub + (size_t)(dir == 0 ? 3 * a + q : 3 * q + a) * A.U.Vh + lc);
        u3[q] = {{w.x, w.z}, {w.y, w.w}};
      }
      v[a] = dir == 0 ? dfdot3<false, true>(u3[0], u3[1], u3[2], h[0], h[1], h[2])
                      : dfdot3<true, true>(u3[0], u3[1], u3[2], h[0], h[1], h[2]);
    }
    if (MU == 3 && A.g.antiper && s.t == (dir == 0 ? A.g.L[3] - 1 : 0)) {
#pragma unroll
      for (int a = 0; a < 3; a++) v[a] = -v[a];
    }
    // lower-spin factor of v_k: -sgn*i (x, to 3-k), (k==0 ? +sgn : -sgn) (y, to 3-k),
    // (k==0 ? -sgn*i : +sgn*i) (z, to 2+k), -sgn (t, to 2+k)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      up[a] = cadd_lazy(up[a], v[a]);
      if (MU == 0) lswap[a] = sgn > 0 ? csub_lazy(lswap[a], times_i(v[a])) : cadd_lazy(lswap[a], times_i(v[a]));
      else if (MU == 1) lswap[a] = ((k == 0) == (sgn > 0)) ? cadd_lazy(lswap[a], v[a]) : csub_lazy(lswap[a], v[a]);
      else if (MU == 2)
        lsame[a] = ((k == 0) == (sgn > 0)) ? csub_lazy(lsame[a], times_i(v[a])) : cadd_lazy(lsame[a], times_i(v[a]));
      else lsame[a] = sgn > 0 ? csub_lazy(lsame[a], v[a]) : cadd_lazy(lsame[a], v[a]);
    }
  }
}

template <bool DAG, bool REDUCE>
__global__ void __launch_bounds__(128) hop_df64_pair_kernel(HopArgs A) {
  __shared__ double sh[8][4];
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z * blockDim.y + threadIdx.y;
  const int k = threadIdx.x & 1;
  const int sites_per_block = blockDim.x >> 1;
  const int stride = gridDim.x * sites_per_block;
  for (int base = blockIdx.x * sites_per_block; base < A.g.Vh; base += stride) {
    const int cb = base + (threadIdx.x >> 1);
    const bool active = cb < A.g.Vh && rhs < A.nrhs;
    double nrm = 0.0;
    Cx<df> up[3], lswap[3], lsame[3];
#pragma unroll
    for (int a = 0; a < 3; a++) up[a] = lswap[a] = lsame[a] = czero<df>();
    const int p = A.out_parity;
    Site s{};
    if (active) {
      s = site_of(A.g, p, cb);
      SpinorView vin{A.in + rhs * A.in_rs, nullptr, A.g.Vh};
      constexpr int S = DAG ? -1 : 1;
      df_pair_dir<0, S>(A, s, p, cb, k, vin, up, lswap, lsame);
      df_pair_dir<1, S>(A, s, p, cb, k, vin, up, lswap, lsame);
      df_pair_dir<2, S>(A, s, p, cb, k, vin, up, lswap, lsame);
      df_pair_dir<3, S>(A, s, p, cb, k, vin, up, lswap, lsame);
    }
    // lower spin 2+k = own z,t partial + partner's x,y partial
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cx<df> o;
      o.re.hi = __shfl_xor_sync(0xffffffffu, lswap[a].re.hi, 1);
      o.re.lo = __shfl_xor_sync(0xffffffffu, lswap[a].re.lo, 1);
      o.im.hi = __shfl_xor_sync(0xffffffffu, lswap[a].im.hi, 1);
      o.im.lo = __shfl_xor_sync(0xffffffffu, lswap[a].im.lo, 1);
      lsame[a] = cnormalise(cadd_lazy(lsame[a], o));
      up[a] = cnormalise(up[a]);
    }
    if (active) {
      const Cx<df> cu = cfrom<df>(A.c_up), cd = cfrom<df>(A.c_dn);
      Cx<df> ru[3], rl[3];
#pragma unroll
      for (int a = 0; a < 3; a++) {
        ru[a] = A.c_one ? up[a] : cu * up[a];
        rl[a] = A.c_one ? lsame[a] : cd * lsame[a];
      }
      if (A.has_aux) {
        const float4 *pa = (const float4 *)(A.aux + rhs * A.aux_rs);
        const Cx<df> du = cfrom<df>(A.d_up), dd = cfrom<df>(A.d_dn);
#pragma unroll
        for (int a = 0; a < 3; a++) {
          float4 w1 = __ldg(pa + (size_t)(3 * k + a) * A.g.Vh + cb);
          float4 w2 = __ldg(pa + (size_t)(3 * (2 + k) + a) * A.g.Vh + cb);
          ru[a] = cmadd(du, Cx<df>{{w1.x, w1.z}, {w1.y, w1.w}}, ru[a]);
          rl[a] = cmadd(dd, Cx<df>{{w2.x, w2.z}, {w2.y, w2.w}}, rl[a]);
        }
      }
      float4 *po = (float4 *)(A.out + rhs * A.out_rs);
#pragma unroll
      for (int a = 0; a < 3; a++) {
        po[(size_t)(3 * k + a) * A.g.Vh + cb] = make_float4(ru[a].re.hi, ru[a].im.hi, ru[a].re.lo, ru[a].im.lo);
        po[(size_t)(3 * (2 + k) + a) * A.g.Vh + cb] =
            make_float4(rl[a].re.hi, rl[a].im.hi, rl[a].re.lo, rl[a].im.lo);
        if (REDUCE) nrm += norm2_d(ru[a]) + norm2_d(rl[a]);
      }
    }
    if (REDUCE) {
      // 32 sites = 64 threads = two warps of one block row: warp sums, then
      // the even warp adds its odd neighbour (fixed order)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
      const int w = threadIdx.x >> 5;
      if ((threadIdx.x & 31) == 0) sh[threadIdx.y][w] = nrm;
      __syncthreads();
      const int cb0 = base + ((threadIdx.x >> 6) << 5);  // first site of this 32-site group
      if ((threadIdx.x & 63) == 0 && rhs < A.nrhs && cb0 < A.g.Vh) {
        const int nw = (A.g.Vh + 31) >> 5;
        A.partials[(size_t)rhs * nw + (cb0 >> 5)] = sh[threadIdx.y][w] + sh[threadIdx.y][w + 1];
      }
      __syncthreads();
    }
  }
}

// Persistent batched hop over lattices of different sizes: a fixed grid of
// blocks walks a queue of tiles (system, first site) in round-robin order;
// each tile is 128 output sites of one system, whose HopArgs (geometry,
// links, fields, coefficients, partials) are read from `descs`.  The order of
// tiles per block is fixed, so results and partials are reproducible.
template <int PREC, int RECON, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(128) hop_batched_kernel(const HopArgs *descs, const int2 *tiles,
                                                          int ntiles, const int *halt) {
  if (halt && *(volatile const int *)halt) return;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tile = tiles[t];
    const HopArgs A = descs[tile.x];
    hop_site<PREC, RECON, DAG, REDUCE>(A, tile.y + threadIdx.x, 0);
  }
}

template <int PREC, int RECON, bool LF>
inline void launch_t2(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) hop_kernel<PREC, RECON, true, true, LF><<<grid, block, 0, st>>>(A);
    else hop_kernel<PREC, RECON, true, false, LF><<<grid, block, 0, st>>>(A);
  } else {
    if (red) hop_kernel<PREC, RECON, false, true, LF><<<grid, block, 0, st>>>(A);
    else hop_kernel<PREC, RECON, false, false, LF><<<grid, block, 0, st>>>(A);
  }
}
template <int PREC, int RECON, int RT>
inline void launch_rt2(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) hop_rt_kernel<PREC, RECON, true, true, RT><<<grid, block, 0, st>>>(A);
    else hop_rt_kernel<PREC, RECON, true, false, RT><<<grid, block, 0, st>>>(A);
  } else {
    if (red) hop_rt_kernel<PREC, RECON, false, true, RT><<<grid, block, 0, st>>>(A);
    else hop_rt_kernel<PREC, RECON, false, false, RT><<<grid, block, 0, st>>>(A);
  }
}
// RHS per thread: 2 or 4 (the register-blocked kernel), else the plain one
template <int PREC, int RECON>
inline void launch_rt(const HopArgs &A, int rt, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (rt == 4) launch_rt2<PREC, RECON, 4>(A, grid, block, dag, red, st);
  else launch_rt2<PREC, RECON, 2>(A, grid, block, dag, red, st);
}

// the loads-first variant exists only for the memory-bound formats
template <int PREC, int RECON>
inline void launch_t(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st,
                     bool lf = false) {
  constexpr bool low = PREC == LQCD_F32 || PREC == LQCD_BF16S || PREC == LQCD_F16S;
  if constexpr (low) {
    if (lf) launch_t2<PREC, RECON, true>(A, grid, block, dag, red, st);
    else launch_t2<PREC, RECON, false>(A, grid, block, dag, red, st);
  } else {
    (void)lf;
    launch_t2<PREC, RECON, false>(A, grid, block, dag, red, st);
  }
}

// per-precision launchers (dslash_f64.cu, dslash_df64.cu, dslash_f32.cu, dslash_h16.cu)
void hop_launch_f64(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st);
void hop_launch_df64(const HopArgs &A, int recon, bool pair, dim3 grid, dim3 block, bool dag, bool red,
                     cudaStream_t st);
// rt: right-hand sides per thread (1, 2, 4); two: two sites per thread (packed FP32x2)
void hop_launch_f32(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, cudaStream_t st);
void hop_launch_h16(const HopArgs &A, int prec, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, cudaStream_t st);
void hop_batched_f64(int recon, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st);
void hop_batched_df64(int recon, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                      const int *halt, cudaStream_t st);
void hop_batched_f32(int recon, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st);
void hop_batched_h16(int prec, bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid,
                     const int *halt, cudaStream_t st);

// one batched launch of precision P and link format RC
template <int P, int RC>
inline void batched_t(bool dag, bool red, const HopArgs *d, const int2 *tl, int ntiles, int grid, const int *halt,
                      cudaStream_t st) {
  if (dag) {
    if (red) hop_batched_kernel<P, RC, true, true><<<grid, 128, 0, st>>>(d, tl, ntiles, halt);
    else hop_batched_kernel<P, RC, true, false><<<grid, 128, 0, st>>>(d, tl, ntiles, halt);
  } else {
    if (red) hop_batched_kernel<P, RC, false, true><<<grid, 128, 0, st>>>(d, tl, ntiles, halt);
    else hop_batched_kernel<P, RC, false, false><<<grid, 128, 0, st>>>(d, tl, ntiles, halt);
  }
}

}  // namespace lqcd
