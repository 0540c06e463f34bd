// hop_kernels.cuh -- device code of the hopping term (included by the
// per-precision translation units dslash_*.cu; see dslash.cu for the design).
#pragma once
#include <cstdio>
#include <type_traits>

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
  Coef4 co;  // c_up, c_dn, d_up, d_dn in every arithmetic
  double *partials;
  int *halt;
};

// coefficient i (0 c_up, 1 c_dn, 2 d_up, 3 d_dn) in the arithmetic R
template <class R> LQCD_DEV Cx<R> hop_coef(const HopArgs &A, int i) { return coef_of<R>(A.co, i); }

// Asynchronous global -> shared copies (cp.async, 4, 8 or 16 bytes, both
// addresses aligned to the size) and their group fences.
LQCD_DEV void cp_async16(void *smem, const void *gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
LQCD_DEV void cp_async8(void *smem, const void *gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}
LQCD_DEV void cp_async4(void *smem, const void *gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
LQCD_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> LQCD_DEV void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

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

// acc (FIRST: =, else +=) f w for the unit f = +1, -1, +i, -i (F_P1 .. F_MI)
template <int F, bool FIRST> LQCD_DEV void put_unit(Cx<double> &acc, Cx<double> w) {
  const Cx<double> t = F == F_P1 ? w : F == F_M1 ? Cx<double>{-w.re, -w.im}
                     : F == F_PI ? Cx<double>{-w.im, w.re} : Cx<double>{w.im, -w.re};
  acc = FIRST ? t : acc + t;
}
// -x when flip, by the sign bit (integer work, off the FP64 pipe)
LQCD_DEV double flip_sign(double x, bool flip) {
  return __longlong_as_double(__double_as_longlong(x) ^ (flip ? (long long)0x8000000000000000ull : 0ll));
}
// upper spins (FIRST: =, else +=) sum; lower spins the -S B^+ d of
// accumulate<MU, S> applied to d
template <int MU, int S, bool FIRST>
LQCD_DEV void accumulate_sd(const Cx<double> sum[6], const Cx<double> d[6], Cx<double> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    put_unit<F_P1, FIRST>(acc[c], sum[c]);
    put_unit<F_P1, FIRST>(acc[3 + c], sum[3 + c]);
    const Cx<double> d0 = d[c], d1 = d[3 + c];
    if (MU == 0) {
      put_unit<(S > 0 ? F_MI : F_PI), FIRST>(acc[6 + c], d1);
      put_unit<(S > 0 ? F_MI : F_PI), FIRST>(acc[9 + c], d0);
    } else if (MU == 1) {
      put_unit<(S > 0 ? F_M1 : F_P1), FIRST>(acc[6 + c], d1);
      put_unit<(S > 0 ? F_P1 : F_M1), FIRST>(acc[9 + c], d0);
    } else if (MU == 2) {
      put_unit<(S > 0 ? F_MI : F_PI), FIRST>(acc[6 + c], d0);
      put_unit<(S > 0 ? F_PI : F_MI), FIRST>(acc[9 + c], d1);
    } else {
      put_unit<(S > 0 ? F_M1 : F_P1), FIRST>(acc[6 + c], d0);
      put_unit<(S > 0 ? F_M1 : F_P1), FIRST>(acc[9 + c], d1);
    }
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
  if constexpr (PREC == LQCD_F64) {
    // FP64 (bound by GB300's FP64 pipe): the forward product a = U h_f, then
    // d = a - b with b = U(x - mu)^+ h_b by one multiply-add chain started
    // from a, and sum = a + b = 2a - d.  The upper spins take sum and the
    // lower ones -S B^+ d (the two projectors differ only in the sign of their
    // lower half): 12 fewer FP64 instructions per direction than two
    // products and four sums, and the first direction assigns the
    // accumulators instead of adding to zero.
    Cx<R> a[6], d[6], sum[6];
    {
      const int j = neighbour_cb(A.g, s, MU, +1);
      SpinorIO<PREC>::load(vin, j, ps);
      project<MU, S>(ps, h);
      LinkIO<PREC, RECON>::load(A.U, p, MU, cb, u);
      if (RECON == 12) reconstruct_row2(u);
      mul_link(u, h, a);
      negate_if(a, negf);
    }
    {
      const int j = neighbour_cb(A.g, s, MU, -1);
      SpinorIO<PREC>::load(vin, j, ps);
      project<MU, -S>(ps, h);
      LinkIO<PREC, RECON>::load(A.U, p ^ 1, MU, j, u);
      if (RECON == 12) reconstruct_row2(u);
      // d = a - (negb ? -1 : 1) U^+ h: add conj(u) times h with its sign flipped unless negb
#pragma unroll
      for (int k = 0; k < 6; k++) h[k] = {flip_sign(h[k].re, !negb), flip_sign(h[k].im, !negb)};
#pragma unroll
      for (int k = 0; k < 2; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          Cx<R> t = conj_madd(u[c], h[3 * k], a[3 * k + c]);
          t = conj_madd(u[3 + c], h[3 * k + 1], t);
          d[3 * k + c] = conj_madd(u[6 + c], h[3 * k + 2], t);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; k++) sum[k] = {fma(2.0, a[k].re, -d[k].re), fma(2.0, a[k].im, -d[k].im)};
    accumulate_sd<MU, S, MU == 0>(sum, d, acc);
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
  const Cx<R> cu = hop_coef<R>(A, 0), cd = hop_coef<R>(A, 1);
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
    const Cx<R> du = hop_coef<R>(A, 2), dd = hop_coef<R>(A, 3);
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
  pdl_wait();
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs0 = (blockIdx.z * blockDim.y + threadIdx.y) * RT;
  if (rhs0 >= A.nrhs) return;  // whole warps: blockDim.x is 32
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < A.g.Vh; base += stride)
    hop_site_rt<PREC, RECON, DAG, REDUCE, RT>(A, base + threadIdx.x, rhs0);
}

// ---------------------------------------------------------------------------
// Multi-RHS hop with the links staged in shared memory (F32 and the 16-bit
// formats).  A block owns NT consecutive output sites and a group of RG
// right-hand sides.  Each thread first loads the eight links of its site
// (the four forward ones at the site, the four backward ones at its
// neighbours) once, rebuilds the third row where SREC = 18, and keeps them in
// its own column of shared memory; it then runs the hop for every RHS of the
// group in turn, reading the links back from shared memory, so that L2 serves
// the link words once per site instead of once per RHS-site and only the
// neighbour spinors are fetched per RHS.  SREC = 12 keeps two rows and
// rebuilds the third for every RHS (less shared memory per thread, more
// warps per SM).  The columns are thread-private, so no barrier is needed.
// Every RHS goes through hop_site's operations in hop_site's order (the same
// reconstruct, project, product and accumulation functions), so the results
// are bitwise those of single-RHS launches.
// ---------------------------------------------------------------------------
template <int SREC> struct MrhsLinkCols {
  static constexpr int NW = SREC == 18 ? 4 : 3;  // 16-byte words per link (+ one 8-byte word for 18)
  static constexpr size_t bytes_per_thread = 8 * (NW * 16 + (SREC == 18 ? 8 : 0));
};

template <int PREC, int RECON, int SREC, int MU, int S>
LQCD_DEV void mrhs_dir(const HopArgs &A, const float4 *W, const float2 *T8, int nt, int jf, int jb, bool negf,
                       bool negb, const SpinorView &vin, Cx<float> acc[12]) {
  constexpr int NW = MrhsLinkCols<SREC>::NW;
  Cx<float> ps[12], pb[12], h[6], v[6], u[9];
  // both neighbours' spinor loads in flight before any arithmetic
  const float scf = load_nb<PREC>(vin, jf, ps);
  const float scb = load_nb<PREC>(vin, jb, pb);
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int ds = 2 * MU + dir;
#pragma unroll
    for (int k = 0; k < NW; k++) {
      const float4 w = W[(ds * NW + k) * nt];
      u[2 * k] = {w.x, w.y};
      u[2 * k + 1] = {w.z, w.w};
    }
    if constexpr (SREC == 18) {
      const float2 e = T8[ds * nt];
      u[8] = {e.x, e.y};
    } else {
      reconstruct_row2(u);
    }
    if (dir == 0) {
      project<MU, S>(ps, h);
      mul_link(u, h, v);
      acc_nb<PREC, MU, S>(v, scf, negf, acc);
    } else {
      project<MU, -S>(pb, h);
      mul_link_dag(u, h, v);
      acc_nb<PREC, MU, -S>(v, scb, negb, acc);
    }
  }
}

// Blocks of 32 or 64 threads, bounded to 128 registers: the shared memory
// allows 6 (18-real columns) or 8 (12-real) blocks of 64 sites per SM.
template <int PREC, int RECON, int SREC, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(64, 8) hop_mrhs_kernel(HopArgs A, int rg) {
  static_assert(SREC == 18 || RECON == 12, "12-real link columns need 12-real links");
  constexpr int NW = MrhsLinkCols<SREC>::NW;
  extern __shared__ float4 mrhs_cols[];
  pdl_wait();
  if (A.halt && *(volatile int *)A.halt) return;
  const int nt = blockDim.x;
  const int rhs0 = blockIdx.y * rg;
  const int rhs1 = min(rhs0 + rg, A.nrhs);
  const int p = A.out_parity;
  const int cb = blockIdx.x * nt + threadIdx.x;
  const bool active = cb < A.g.Vh;
  // this thread's column: W[(ds * NW + k) * nt], T8[ds * nt]
  const float4 *W = mrhs_cols + threadIdx.x;
  const float2 *T8 = (const float2 *)(mrhs_cols + 8 * NW * nt) + threadIdx.x;
  int jn[8];
  bool negf = false, negb = false;
  if (active) {
    const Site s = site_of(A.g, p, cb);
    negf = A.g.antiper && s.t == A.g.L[3] - 1;
    negb = A.g.antiper && s.t == 0;
    float4 *Ww = mrhs_cols + threadIdx.x;
    float2 *Tw = (float2 *)(mrhs_cols + 8 * NW * nt) + threadIdx.x;
#pragma unroll
    for (int ds = 0; ds < 8; ds++) {
      const int mu = ds >> 1;
      jn[ds] = neighbour_cb(A.g, s, mu, (ds & 1) ? -1 : +1);
      Cx<float> u[9];
      LinkIO<PREC, RECON>::load(A.U, (ds & 1) ? p ^ 1 : p, mu, (ds & 1) ? jn[ds] : cb, u);
      if (RECON == 12 && SREC == 18) reconstruct_row2(u);
#pragma unroll
      for (int k = 0; k < NW; k++)
        Ww[(ds * NW + k) * nt] = make_float4(u[2 * k].re, u[2 * k].im, u[2 * k + 1].re, u[2 * k + 1].im);
      if (SREC == 18) Tw[ds * nt] = make_float2(u[8].re, u[8].im);
    }
  }
  constexpr int S = DAG ? -1 : 1;
  for (int rhs = rhs0; rhs < rhs1; rhs++) {
    double nrm = 0.0;
    if (active) {
      SpinorView vin{A.in + rhs * A.in_rs, A.in_scale ? A.in_scale + rhs * A.in_srs : nullptr, A.g.Vh};
      Cx<float> acc[12];
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = czero<float>();
      mrhs_dir<PREC, RECON, SREC, 0, S>(A, W, T8, nt, jn[0], jn[1], false, false, vin, acc);
      mrhs_dir<PREC, RECON, SREC, 1, S>(A, W, T8, nt, jn[2], jn[3], false, false, vin, acc);
      mrhs_dir<PREC, RECON, SREC, 2, S>(A, W, T8, nt, jn[4], jn[5], false, false, vin, acc);
      mrhs_dir<PREC, RECON, SREC, 3, S>(A, W, T8, nt, jn[6], jn[7], negf, negb, vin, acc);
      nrm = hop_epilogue<PREC, REDUCE>(A, cb, rhs, acc);
    }
    if (REDUCE) hop_warp_partial(A, cb, rhs, nrm);
  }
}

// shared memory of one hop_mrhs_kernel block of nt threads
inline size_t mrhs_smem_bytes(int srec, int nt) {
  return (size_t)nt * (srec == 18 ? MrhsLinkCols<18>::bytes_per_thread : MrhsLinkCols<12>::bytes_per_thread);
}

// Grid-stride over the output sites: a full grid (one site per thread) or a
// smaller persistent grid, whichever the autotuner finds faster.
// LF selects, for the memory-bound formats, whether both neighbours' loads of
// a direction are issued before its arithmetic (the autotuner picks).
template <int PREC, int RECON, bool DAG, bool REDUCE, bool LF>
__global__ void __launch_bounds__(256, (PREC == LQCD_BF16S || PREC == LQCD_F16S) ? 3 : PREC == LQCD_F32 ? 2 : 1) hop_kernel(HopArgs A) {
  pdl_wait();
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z * blockDim.y + threadIdx.y;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < A.g.Vh; base += stride)
    hop_site<PREC, RECON, DAG, REDUCE, LF>(A, base + threadIdx.x, rhs);
}

// Several right-hand sides with the RHS interleaved with the site blocks:
// block b runs RHS b % nrhs of site block b / nrhs (grid-stride over the site
// blocks; gridDim.x a multiple of nrhs), so the blocks resident at one time
// cover a few site blocks for every RHS, and the links one RHS reads from HBM
// are still in L2 when the others read them.  The same hop_site per (site,
// RHS), so the results are bitwise those of hop_kernel.
template <int PREC, int RECON, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(256, 2) hop_ri_kernel(HopArgs A) {
  pdl_wait();
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.x % A.nrhs;
  const int stride = (gridDim.x / A.nrhs) * blockDim.x;
  for (int base = (blockIdx.x / A.nrhs) * blockDim.x; base < A.g.Vh; base += stride)
    hop_site<PREC, RECON, DAG, REDUCE, true>(A, base + threadIdx.x, rhs);
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

// one (direction, sense) step of the two-site packed hop on loaded operands
template <int RECON, int MU, int S, int DIR>
LQCD_DEV void hop_step2(const HopArgs &A, const Site &sA, const Site &sB, Cx<float2> ps[12], float2 sc,
                        Cx<float2> u[9], Cx<float2> acc[12]) {
  Cx<float2> h[6], v[6];
  const int tb = DIR == 0 ? A.g.L[3] - 1 : 0;
  if (MU == 3 && A.g.antiper) {
    if (sA.t == tb) sc.x = -sc.x;
    if (sB.t == tb) sc.y = -sc.y;
  }
  if (DIR == 0) {
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

template <int PREC, int RECON, int MU, int S>
LQCD_DEV void hop_dir2(const HopArgs &A, const Site &sA, const Site &sB, int p, int cbA, int cbB,
                       const SpinorView &vin, Cx<float2> acc[12]) {
#pragma unroll
  for (int dir = 0; dir < 2; dir++) {
    const int d = dir == 0 ? +1 : -1;
    const int jA = neighbour_cb(A.g, sA, MU, d), jB = neighbour_cb(A.g, sB, MU, d);
    Cx<float2> ps[12], u[9];
    const float2 sc = load_nb2<PREC>(vin, jA, jB, ps);
    if (dir == 0) {
      load_link2<PREC, RECON>(A.U, p, MU, cbA, cbB, u);
      hop_step2<RECON, MU, S, 0>(A, sA, sB, ps, sc, u, acc);
    } else {
      load_link2<PREC, RECON>(A.U, p ^ 1, MU, jA, jB, u);
      hop_step2<RECON, MU, S, 1>(A, sA, sB, ps, sc, u, acc);
    }
  }
}

template <int PREC, int RECON, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(64) hop_pair2_kernel(HopArgs A) {
  pdl_wait();
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
    if (red) launch_pdl(hop_pair2_kernel<PREC, RECON, true, true>, grid, block, 0, st, A);
    else launch_pdl(hop_pair2_kernel<PREC, RECON, true, false>, grid, block, 0, st, A);
  } else {
    if (red) launch_pdl(hop_pair2_kernel<PREC, RECON, false, true>, grid, block, 0, st, A);
    else launch_pdl(hop_pair2_kernel<PREC, RECON, false, false>, grid, block, 0, st, A);
  }
}

// ---------------------------------------------------------------------------
// The two-site packed hop for the 16-bit formats (REC12 links) with its
// operands staged through shared memory: each (direction, sense) step's
// neighbour words, site scales and link words of both sites are copied by
// cp.async one step ahead into the other of two buffers, so their latency
// hides behind the previous step's arithmetic and no registers are held by
// loads in flight.  Every thread stages and reads only its own words.  The
// arithmetic is hop_step2's, so the results are bitwise those of hop_site.
// Per thread and stage: 3 + 3 spinor words and 2 link words of 16 bytes, 2
// link tails of 8 bytes and 2 scales (152 bytes).
// ---------------------------------------------------------------------------
LQCD_HD int h16_staged_bytes(int bx) { return 304 * bx; }

struct H16Stage {
  uint4 *w4;  // [2][8][bx]: spinor A (3), spinor B (3), link A, link B
  uint2 *w2;  // [2][2][bx]: link tails A, B
  float *wf;  // [2][2][bx]: scales A, B
  int bx, tx;
};

template <int MU, int DIR, int ST>
LQCD_DEV void h16_stage_issue(const HopArgs &A, const Site &sA, const Site &sB, int p, int cbA, int cbB,
                              const SpinorView &vin, const H16Stage &B) {
  const int d = DIR == 0 ? +1 : -1;
  const int jA = neighbour_cb(A.g, sA, MU, d), jB = neighbour_cb(A.g, sB, MU, d);
  const uint4 *pin = (const uint4 *)vin.ptr;
  const size_t Vh = vin.Vh;
  uint4 *w4 = B.w4 + ST * 8 * B.bx + B.tx;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    cp_async16(w4 + k * B.bx, pin + k * Vh + jA);
    cp_async16(w4 + (3 + k) * B.bx, pin + k * Vh + jB);
  }
  float *wf = B.wf + ST * 2 * B.bx + B.tx;
  cp_async4(wf, vin.scale + jA);
  cp_async4(wf + B.bx, vin.scale + jB);
  const char *base = (const char *)A.U.ptr + (DIR == 0 ? p : p ^ 1) * A.U.parity_stride + MU * A.U.mu_stride;
  const int lA = DIR == 0 ? cbA : jA, lB = DIR == 0 ? cbB : jB;
  cp_async16(w4 + 6 * B.bx, (const uint4 *)base + lA);
  cp_async16(w4 + 7 * B.bx, (const uint4 *)base + lB);
  const uint2 *tail = (const uint2 *)(base + (size_t)A.U.Vh * 16);
  uint2 *w2 = B.w2 + ST * 2 * B.bx + B.tx;
  cp_async8(w2, tail + lA);
  cp_async8(w2 + B.bx, tail + lB);
}

// N complex values of site A (words wa) and site B (words wb) as packed pairs
template <class H, int N>
LQCD_DEV void h16_unpack2(const uint32_t *wa, const uint32_t *wb, Cx<float2> *out) {
#pragma unroll
  for (int j = 0; j < N; j++) {
    const float2 a = Half16<H>::to_f2(wa[j]), b = Half16<H>::to_f2(wb[j]);
    out[j] = {make_float2(a.x, b.x), make_float2(a.y, b.y)};
  }
}
template <class H> LQCD_DEV void h16_unpack2(uint4 a, uint4 b, Cx<float2> *out) {
  const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
  h16_unpack2<H, 4>(wa, wb, out);
}

template <class H, int STEP, int S>
LQCD_DEV void h16_staged_steps(const HopArgs &A, const Site &sA, const Site &sB, int p, int cbA, int cbB,
                               const SpinorView &vin, const H16Stage &B, Cx<float2> acc[12]) {
  if constexpr (STEP < 8) {
    constexpr int MU = STEP >> 1, DIR = STEP & 1, ST = STEP & 1;
    constexpr int NMU = (STEP + 1) >> 1, NDIR = (STEP + 1) & 1;
    if constexpr (STEP + 1 < 8) {
      h16_stage_issue<NMU, NDIR, NDIR>(A, sA, sB, p, cbA, cbB, vin, B);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    {
      const uint4 *w4 = B.w4 + ST * 8 * B.bx + B.tx;
      const uint2 *w2 = B.w2 + ST * 2 * B.bx + B.tx;
      const float *wf = B.wf + ST * 2 * B.bx + B.tx;
      Cx<float2> ps[12], u[9];
#pragma unroll
      for (int k = 0; k < 3; k++) h16_unpack2<H>(w4[k * B.bx], w4[(3 + k) * B.bx], ps + 4 * k);
      h16_unpack2<H>(w4[6 * B.bx], w4[7 * B.bx], u);
      const uint2 ta = w2[0], tb = w2[B.bx];
      const uint32_t wa[2] = {ta.x, ta.y}, wb[2] = {tb.x, tb.y};
      h16_unpack2<H, 2>(wa, wb, u + 4);
      const float2 sc = make_float2(wf[0], wf[B.bx]);
      hop_step2<12, MU, S, DIR>(A, sA, sB, ps, sc, u, acc);
    }
    __syncwarp();
    h16_staged_steps<H, STEP + 1, S>(A, sA, sB, p, cbA, cbB, vin, B, acc);
  }
}

template <int PREC, bool DAG, bool REDUCE>
__global__ void __launch_bounds__(64, 6) hop_h16_staged_kernel(HopArgs A) {
  pdl_wait();
  using H = typename std::conditional<PREC == LQCD_BF16S, __nv_bfloat16, __half>::type;
  extern __shared__ uint4 h16_words[];
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = A.out_parity;
  H16Stage B;
  B.bx = blockDim.x;
  B.tx = threadIdx.x;
  B.w4 = h16_words;
  B.w2 = (uint2 *)(B.w4 + 16 * B.bx);
  B.wf = (float *)(B.w2 + 4 * B.bx);
  const int stride = gridDim.x * 128;
  for (int base = blockIdx.x * 128; base < A.g.Vh; base += stride) {
    const int cbA = base + 64 * w + lane, cbB = cbA + 32;
    const bool okA = cbA < A.g.Vh && rhs < A.nrhs, okB = cbB < A.g.Vh && rhs < A.nrhs;
    // lanes past the end recompute a valid site and store nothing
    const int cA = okA ? cbA : A.g.Vh - 1, cB = okB ? cbB : A.g.Vh - 1;
    const int r = rhs < A.nrhs ? rhs : A.nrhs - 1;
    const Site sA = site_of(A.g, p, cA), sB = site_of(A.g, p, cB);
    SpinorView vin{A.in + r * A.in_rs, A.in_scale + r * A.in_srs, A.g.Vh};
    Cx<float2> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = czero<float2>();
    constexpr int S = DAG ? -1 : 1;
    h16_stage_issue<0, 0, 0>(A, sA, sB, p, cA, cB, vin, B);
    cp_async_commit();
    h16_staged_steps<H, 0, S>(A, sA, sB, p, cA, cB, vin, B, acc);
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
// One (direction, sense) step of the float-float pair hop.  `sp(q)` yields
// the neighbour's colour q of upper spin k (q < 3) or of the lower spin that
// h_k pairs with it (q >= 3); `lk(e)` yields element e = 3*row + column of
// U_mu(x) (forward) or U_mu(x - mu) (backward).
template <int MU, int S, int DIR, class SP, class LK>
LQCD_DEV void df_pair_step(const HopArgs &A, const Site &s, int k, SP sp, LK lk, Cx<df> up[3], Cx<df> lswap[3],
                           Cx<df> lsame[3]) {
  constexpr int sgn = DIR == 0 ? S : -S;  // projector sign: (1 - S g) forward, (1 + S g) backward
  Cx<df> h[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float4 a = sp(c);
    float4 b = sp(3 + c);
    Cx<df> pa = {{a.x, a.z}, {a.y, a.w}}, pb = {{b.x, b.z}, {b.y, b.w}};
    // h_k = p_k + f * p_lo with f = S*i (x), S*(+-1) (y), S*(+-i) (z), -S (t)
    const bool neg = (MU == 0) ? sgn < 0 : (MU == 1) ? (k == 0 ? sgn < 0 : sgn > 0)
                   : (MU == 2) ? (k == 0 ? sgn < 0 : sgn > 0) : sgn > 0;
    Cx<df> t = (MU == 0 || MU == 2) ? times_i(pb) : pb;
    h[c] = neg ? csub_lazy(pa, t) : cadd_lazy(pa, t);
  }
  Cx<df> v[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    Cx<df> u3[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {  // forward: row a of U; backward: column a
      float4 w = lk(DIR == 0 ? 3 * a + q : 3 * q + a);
      u3[q] = {{w.x, w.z}, {w.y, w.w}};
    }
    v[a] = DIR == 0 ? dfdot3<false, true>(u3[0], u3[1], u3[2], h[0], h[1], h[2])
                    : dfdot3<true, true>(u3[0], u3[1], u3[2], h[0], h[1], h[2]);
  }
  if (MU == 3 && A.g.antiper && s.t == (DIR == 0 ? A.g.L[3] - 1 : 0)) {
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

// global addresses of one step's operands: the neighbour's upper spin k and
// paired lower spin (plane stride Vh), and the link (plane stride U.Vh)
struct DfStepSrc {
  const float4 *pk, *plo, *ub;
};
template <int MU, int DIR>
LQCD_DEV DfStepSrc df_step_src(const HopArgs &A, const Site &s, int p, int cb, int k, const float4 *pin, int Vh) {
  const int j = neighbour_cb(A.g, s, MU, DIR == 0 ? +1 : -1);
  const int lo = (MU < 2) ? 3 - k : 2 + k;  // lower spin paired with upper k in h_k
  const int lc = DIR == 0 ? cb : j;
  const float4 *ub = (const float4 *)((const char *)A.U.ptr + (DIR == 0 ? p : p ^ 1) * A.U.parity_stride +
                                      MU * A.U.mu_stride) + lc;
  return {pin + (size_t)(3 * k) * Vh + j, pin + (size_t)(3 * lo) * Vh + j, ub};
}

template <int DIR>
LQCD_DEV DfStepSrc df_step_src_rt(const HopArgs &A, const Site &s, int p, int cb, int k, int mu,
                                  const float4 *pin, int Vh) {
  const int j = neighbour_cb(A.g, s, mu, DIR == 0 ? +1 : -1);
  const int lo = (mu < 2) ? 3 - k : 2 + k;
  const int lc = DIR == 0 ? cb : j;
  const float4 *ub = (const float4 *)((const char *)A.U.ptr + (DIR == 0 ? p : p ^ 1) * A.U.parity_stride +
                                      mu * A.U.mu_stride) + lc;
  return {pin + (size_t)(3 * k) * Vh + j, pin + (size_t)(3 * lo) * Vh + j, ub};
}

template <int MU, int S>
LQCD_DEV void df_pair_dir(const HopArgs &A, const Site &s, int p, int cb, int k, const SpinorView &vin,
                          Cx<df> up[3], Cx<df> lswap[3], Cx<df> lsame[3]) {
  const float4 *pin = (const float4 *)vin.ptr;
  const size_t Vh = vin.Vh, UVh = A.U.Vh;
  {
    const DfStepSrc f = df_step_src<MU, 0>(A, s, p, cb, k, pin, vin.Vh);
    df_pair_step<MU, S, 0>(
        A, s, k, [&](int q) { return __ldg(q < 3 ? f.pk + q * Vh : f.plo + (q - 3) * Vh); },
        [&](int e) { return __ldg(f.ub + e * UVh); }, up, lswap, lsame);
  }
  {
    const DfStepSrc b = df_step_src<MU, 1>(A, s, p, cb, k, pin, vin.Vh);
    df_pair_step<MU, S, 1>(
        A, s, k, [&](int q) { return __ldg(q < 3 ? b.pk + q * Vh : b.plo + (q - 3) * Vh); },
        [&](int e) { return __ldg(b.ub + e * UVh); }, up, lswap, lsame);
  }
}

template <int MU, int S, int DIR, class SP, class LK>
LQCD_DEV void df_pair_step_p(const HopArgs &A, const Site &s, int k, SP sp, LK lk, df2 up[3], df2 lswap[3],
                             df2 lsame[3]) {
  constexpr int sgn = DIR == 0 ? S : -S;
  df2 y1[3], y2[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const df2 pa = df2_of(sp(c)), pb = df2_of(sp(3 + c));
    const bool neg = (MU == 0) ? sgn < 0 : (MU == 1) ? (k == 0 ? sgn < 0 : sgn > 0)
                   : (MU == 2) ? (k == 0 ? sgn < 0 : sgn > 0) : sgn > 0;
    const df2 t = (MU == 0 || MU == 2) ? times_i_p(pb) : pb;
    y1[c] = add_lazy_p(pa, neg ? neg_p(t) : t);
    y2[c] = DIR == 0 ? times_i_p(y1[c]) : times_mi_p(y1[c]);
  }
  df2 v[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float4 x[3];
#pragma unroll
    for (int q = 0; q < 3; q++) x[q] = lk(DIR == 0 ? 3 * a + q : 3 * q + a);
    v[a] = dfdot3_p(x, y1, y2);
  }
  if (MU == 3 && A.g.antiper && s.t == (DIR == 0 ? A.g.L[3] - 1 : 0)) {
#pragma unroll
    for (int a = 0; a < 3; a++) v[a] = neg_p(v[a]);
  }
  // the lower-spin factors of the scalar step as units: x: -sgn*i, y:
  // (k==0) == (sgn>0) ? +1 : -1, z: (k==0) == (sgn>0) ? -i : +i, t: -sgn
  const bool kp = (k == 0) == (sgn > 0);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    up[a] = add_lazy_p(up[a], v[a]);
    if (MU == 0) lswap[a] = add_lazy_p(lswap[a], sgn > 0 ? unit_p<3>(v[a]) : unit_p<1>(v[a]));
    else if (MU == 1) lswap[a] = add_lazy_p(lswap[a], kp ? v[a] : unit_p<2>(v[a]));
    else if (MU == 2) lsame[a] = add_lazy_p(lsame[a], kp ? unit_p<3>(v[a]) : unit_p<1>(v[a]));
    else lsame[a] = add_lazy_p(lsame[a], sgn > 0 ? unit_p<2>(v[a]) : v[a]);
  }
}

// The packed step for direction mu = 2h + (EV ? 0 : 1) with the pair index
// h a runtime value: EV (x, z) pairs the spins through a factor i, odd
// directions (y, t) through a real one, so one copy of the code serves a
// pair of directions and the direction-dependent signs become exact
// multiplications by +-1 (the bits do not change).  The lower-spin
// contribution goes to `low`, which the caller maps to lswap (h = 0) or
// lsame (h = 1).
LQCD_DEV df2 scale_p(df2 a, float2 f) { return {__fmul2_rn(a.hi, f), __fmul2_rn(a.lo, f)}; }

template <int S, int DIR, bool EV, class SP, class LK>
LQCD_DEV void df_pair_step_h(const HopArgs &A, const Site &s, int k, int h, SP sp, LK lk, df2 up[3],
                             df2 low[3]) {
  constexpr int sgn = DIR == 0 ? S : -S;
  const bool kneg = k == 0 ? sgn < 0 : sgn > 0;
  // projection sign: x sgn<0, y kneg, z kneg, t sgn>0
  const bool neg = EV ? (h == 0 ? sgn < 0 : kneg) : (h == 0 ? kneg : sgn > 0);
  const float2 fp = neg ? make_float2(-1.0f, -1.0f) : make_float2(1.0f, 1.0f);
  df2 y1[3], y2[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const df2 pa = df2_of(sp(c)), pb = df2_of(sp(3 + c));
    y1[c] = add_lazy_p(pa, scale_p(EV ? times_i_p(pb) : pb, fp));
    y2[c] = DIR == 0 ? times_i_p(y1[c]) : times_mi_p(y1[c]);
  }
  df2 v[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float4 x[3];
#pragma unroll
    for (int q = 0; q < 3; q++) x[q] = lk(DIR == 0 ? 3 * a + q : 3 * q + a);
    v[a] = dfdot3_p(x, y1, y2);
  }
  if (!EV && h == 1 && A.g.antiper && s.t == (DIR == 0 ? A.g.L[3] - 1 : 0)) {
#pragma unroll
    for (int a = 0; a < 3; a++) v[a] = neg_p(v[a]);
  }
  // lower-spin unit (EV ? i : 1) times -1 when: x sgn>0, y !kp, z kp, t sgn>0
  const bool kp = (k == 0) == (sgn > 0);
  const bool lneg = EV ? (h == 0 ? sgn > 0 : kp) : (h == 0 ? !kp : sgn > 0);
  const float2 fl = lneg ? make_float2(-1.0f, -1.0f) : make_float2(1.0f, 1.0f);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    up[a] = add_lazy_p(up[a], v[a]);
    low[a] = add_lazy_p(low[a], scale_p(EV ? times_i_p(v[a]) : v[a], fl));
  }
}

template <int MU, int S>
LQCD_DEV void df_pair_dir_p(const HopArgs &A, const Site &s, int p, int cb, int k, const SpinorView &vin,
                            df2 up[3], df2 lswap[3], df2 lsame[3]) {
  const float4 *pin = (const float4 *)vin.ptr;
  const size_t Vh = vin.Vh, UVh = A.U.Vh;
  {
    const DfStepSrc f = df_step_src<MU, 0>(A, s, p, cb, k, pin, vin.Vh);
    df_pair_step_p<MU, S, 0>(
        A, s, k, [&](int q) { return __ldg(q < 3 ? f.pk + q * Vh : f.plo + (q - 3) * Vh); },
        [&](int e) { return __ldg(f.ub + e * UVh); }, up, lswap, lsame);
  }
  {
    const DfStepSrc b = df_step_src<MU, 1>(A, s, p, cb, k, pin, vin.Vh);
    df_pair_step_p<MU, S, 1>(
        A, s, k, [&](int q) { return __ldg(q < 3 ? b.pk + q * Vh : b.plo + (q - 3) * Vh); },
        [&](int e) { return __ldg(b.ub + e * UVh); }, up, lswap, lsame);
  }
}

// End of a float-float pair site: lower spin 2+k = own z,t partial + the
// partner lane's x,y partial, renormalisation, the epilogue coefficients,
// the store and (REDUCE) the fixed-order norm partial of each 32-site group.
template <bool REDUCE>
LQCD_DEV void df_pair_finish(const HopArgs &A, int base, int cb, int rhs, int k, bool active, Cx<df> up[3],
                             Cx<df> lswap[3], Cx<df> lsame[3], double (*sh)[4]) {
  double nrm = 0.0;
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
    const Cx<df> cu = A.co.w[0], cd = A.co.w[1];
    Cx<df> ru[3], rl[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      ru[a] = A.c_one ? up[a] : cu * up[a];
      rl[a] = A.c_one ? lsame[a] : cd * lsame[a];
    }
    if (A.has_aux) {
      const float4 *pa = (const float4 *)(A.aux + rhs * A.aux_rs);
      const Cx<df> du = A.co.w[2], dd = A.co.w[3];
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
      po[(size_t)(3 * (2 + k) + a) * A.g.Vh + cb] = make_float4(rl[a].re.hi, rl[a].im.hi, rl[a].re.lo, rl[a].im.lo);
    }
    if (REDUCE) {
      const Cx<df> w[6] = {ru[0], ru[1], ru[2], rl[0], rl[1], rl[2]};
      nrm = df_site_norm2<6>(w);
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

template <bool DAG, bool REDUCE, bool PK>
__global__ void __launch_bounds__(128, 4) hop_df64_pair_kernel(HopArgs A) {
  pdl_wait();
  __shared__ double sh[8][4];
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z * blockDim.y + threadIdx.y;
  const int k = threadIdx.x & 1;
  const int sites_per_block = blockDim.x >> 1;
  const int stride = gridDim.x * sites_per_block;
  for (int base = blockIdx.x * sites_per_block; base < A.g.Vh; base += stride) {
    const int cb = base + (threadIdx.x >> 1);
    const bool active = cb < A.g.Vh && rhs < A.nrhs;
    Cx<df> up[3], lswap[3], lsame[3];
    constexpr int S = DAG ? -1 : 1;
    if (PK) {
      df2 pu[3], pw[3], pm[3];
#pragma unroll
      for (int a = 0; a < 3; a++) pu[a] = pw[a] = pm[a] = df2_zero();
      if (active) {
        const int p = A.out_parity;
        const Site s = site_of(A.g, p, cb);
        SpinorView vin{A.in + rhs * A.in_rs, nullptr, A.g.Vh};
        df_pair_dir_p<0, S>(A, s, p, cb, k, vin, pu, pw, pm);
        df_pair_dir_p<1, S>(A, s, p, cb, k, vin, pu, pw, pm);
        df_pair_dir_p<2, S>(A, s, p, cb, k, vin, pu, pw, pm);
        df_pair_dir_p<3, S>(A, s, p, cb, k, vin, pu, pw, pm);
      }
#pragma unroll
      for (int a = 0; a < 3; a++) {
        up[a] = cx_of(pu[a]);
        lswap[a] = cx_of(pw[a]);
        lsame[a] = cx_of(pm[a]);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 3; a++) up[a] = lswap[a] = lsame[a] = czero<df>();
      if (active) {
        const int p = A.out_parity;
        const Site s = site_of(A.g, p, cb);
        SpinorView vin{A.in + rhs * A.in_rs, nullptr, A.g.Vh};
        df_pair_dir<0, S>(A, s, p, cb, k, vin, up, lswap, lsame);
        df_pair_dir<1, S>(A, s, p, cb, k, vin, up, lswap, lsame);
        df_pair_dir<2, S>(A, s, p, cb, k, vin, up, lswap, lsame);
        df_pair_dir<3, S>(A, s, p, cb, k, vin, up, lswap, lsame);
      }
    }
    df_pair_finish<REDUCE>(A, base, cb, rhs, k, active, up, lswap, lsame, sh);
  }
}

// ---------------------------------------------------------------------------
// Packed float-float pair hop with its operands staged through shared
// memory, looping over the two pairs of directions (x, y) and (z, t) at run
// time (two copies of the step code, not eight, keep the kernel inside the
// instruction cache).  The eight
// (direction, sense) steps of a site form a two-stage pipeline: while step i is computed from one buffer, 16-byte asynchronous
// copies (cp.async) of step i+1's neighbour words and link words fill the
// other, so the global-load latency is hidden behind a whole step of
// float-float arithmetic without holding registers for loads in flight.
// Per block row of bx threads (bx/2 sites) and stage: the 6 words of each
// thread's spin pair and the 9 link words of each site, which the site's
// two threads copy alternately (even elements: thread 0, odd: thread 1) and
// both read.  Both threads of a site are lanes of one warp, so
// cp.async.wait_group followed by __syncwarp makes the partner's words
// visible, and the __syncwarp after each step keeps a buffer from being
// refilled while it is still read.
// ---------------------------------------------------------------------------

// 16-byte shared-memory words per block row of bx threads: 2 stages x (6 per thread + 9 per site)
LQCD_HD int df_staged_words(int bx) { return 2 * (6 * bx + 9 * (bx / 2)); }

struct DfStage {
  float4 *sp;  // [2][6][bx]: this row's spinor words
  float4 *lk;  // [2][9][bx/2]: this row's link words
  int bx, ns, tx, site;
};

template <int DIR, int ST>
LQCD_DEV void df_stage_issue(const HopArgs &A, const Site &s, int p, int cb, int k, int mu, const float4 *pin,
                             const DfStage &B) {
  const DfStepSrc f = df_step_src_rt<DIR>(A, s, p, cb, k, mu, pin, A.g.Vh);
  const size_t Vh = A.g.Vh, UVh = A.U.Vh;
  float4 *sp = B.sp + ST * 6 * B.bx + B.tx;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cp_async16(sp + c * B.bx, f.pk + c * Vh);
    cp_async16(sp + (3 + c) * B.bx, f.plo + c * Vh);
  }
  float4 *lk = B.lk + ST * 9 * B.ns + B.site;
#pragma unroll
  for (int e = 0; e < 9; e += 2) {
    const int el = e + k;
    if (el < 9) cp_async16(lk + el * B.ns, f.ub + el * UVh);
  }
}

// one step from stage ST: wait for its copies (all but the newest group),
// compute, and release the buffer
template <int S, int DIR, bool EV, int ST>
LQCD_DEV void df_stage_compute(const HopArgs &A, const Site &s, int k, int h, bool active, const DfStage &B,
                               df2 up[3], df2 low[3]) {
  cp_async_wait<1>();
  __syncwarp();
  if (active) {
    const float4 *sp = B.sp + ST * 6 * B.bx + B.tx;
    const float4 *lk = B.lk + ST * 9 * B.ns + B.site;
    df_pair_step_h<S, DIR, EV>(
        A, s, k, h, [&](int q) { return sp[q * B.bx]; }, [&](int e) { return lk[e * B.ns]; }, up, low);
  }
  __syncwarp();
}

// MINB: blocks of 128 threads per SM the register bound allows (4: 128
// registers; 5: 96 registers, more warps for the fixed-latency chains of the
// error-free sums at the cost of a few spilled values; the tuner picks)
template <bool DAG, bool REDUCE, int MINB = 4>
__global__ void __launch_bounds__(128, MINB) hop_df64_staged_kernel(HopArgs A) {
  pdl_wait();
  __shared__ double sh[8][4];
  extern __shared__ float4 stage_words[];
  if (A.halt && *(volatile int *)A.halt) return;
  const int rhs = blockIdx.z * blockDim.y + threadIdx.y;
  const int k = threadIdx.x & 1;
  const int bx = blockDim.x, ns = bx >> 1;
  DfStage B;
  B.sp = stage_words + threadIdx.y * df_staged_words(bx);
  B.lk = B.sp + 12 * bx;
  B.bx = bx;
  B.ns = ns;
  B.tx = threadIdx.x;
  B.site = threadIdx.x >> 1;
  const int stride = gridDim.x * ns;
  constexpr int S = DAG ? -1 : 1;
  for (int base = blockIdx.x * ns; base < A.g.Vh; base += stride) {
    const int cb = base + (threadIdx.x >> 1);
    const bool active = cb < A.g.Vh && rhs < A.nrhs;
    df2 pu[3], low[3], pw[3];
#pragma unroll
    for (int a = 0; a < 3; a++) pu[a] = low[a] = pw[a] = df2_zero();
    const int p = A.out_parity;
    const Site s = active ? site_of(A.g, p, cb) : Site{};
    const float4 *pin = (const float4 *)(A.in + (active ? rhs : 0) * A.in_rs);
    if (active) df_stage_issue<0, 0>(A, s, p, cb, k, 0, pin, B);
    cp_async_commit();
    // per pair h of directions the steps (2h, fwd) (2h, bwd) (2h+1, fwd)
    // (2h+1, bwd) alternate between stage 0 and stage 1; each step first
    // issues the copies of the next one (an empty group after the last)
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
      const int me = 2 * h, mo = 2 * h + 1;
      if (active) df_stage_issue<1, 1>(A, s, p, cb, k, me, pin, B);
      cp_async_commit();
      df_stage_compute<S, 0, true, 0>(A, s, k, h, active, B, pu, low);
      if (active) df_stage_issue<0, 0>(A, s, p, cb, k, mo, pin, B);
      cp_async_commit();
      df_stage_compute<S, 1, true, 1>(A, s, k, h, active, B, pu, low);
      if (active) df_stage_issue<1, 1>(A, s, p, cb, k, mo, pin, B);
      cp_async_commit();
      df_stage_compute<S, 0, false, 0>(A, s, k, h, active, B, pu, low);
      if (active && h == 0) df_stage_issue<0, 0>(A, s, p, cb, k, 2, pin, B);
      cp_async_commit();
      df_stage_compute<S, 1, false, 1>(A, s, k, h, active, B, pu, low);
      if (h == 0) {  // x and y done: their lower partial is lswap
#pragma unroll
        for (int a = 0; a < 3; a++) {
          pw[a] = low[a];
          low[a] = df2_zero();
        }
      }
    }
    Cx<df> up[3], lswap[3], lsame[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      up[a] = cx_of(pu[a]);
      lswap[a] = cx_of(pw[a]);
      lsame[a] = cx_of(low[a]);
    }
    df_pair_finish<REDUCE>(A, base, cb, rhs, k, active, up, lswap, lsame, sh);
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
    if (red) launch_pdl(hop_kernel<PREC, RECON, true, true, LF>, grid, block, 0, st, A);
    else launch_pdl(hop_kernel<PREC, RECON, true, false, LF>, grid, block, 0, st, A);
  } else {
    if (red) launch_pdl(hop_kernel<PREC, RECON, false, true, LF>, grid, block, 0, st, A);
    else launch_pdl(hop_kernel<PREC, RECON, false, false, LF>, grid, block, 0, st, A);
  }
}
template <int PREC, int RECON>
inline void launch_ri(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) launch_pdl(hop_ri_kernel<PREC, RECON, true, true>, grid, block, 0, st, A);
    else launch_pdl(hop_ri_kernel<PREC, RECON, true, false>, grid, block, 0, st, A);
  } else {
    if (red) launch_pdl(hop_ri_kernel<PREC, RECON, false, true>, grid, block, 0, st, A);
    else launch_pdl(hop_ri_kernel<PREC, RECON, false, false>, grid, block, 0, st, A);
  }
}
template <int PREC, int RECON, int RT>
inline void launch_rt2(const HopArgs &A, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (dag) {
    if (red) launch_pdl(hop_rt_kernel<PREC, RECON, true, true, RT>, grid, block, 0, st, A);
    else launch_pdl(hop_rt_kernel<PREC, RECON, true, false, RT>, grid, block, 0, st, A);
  } else {
    if (red) launch_pdl(hop_rt_kernel<PREC, RECON, false, true, RT>, grid, block, 0, st, A);
    else launch_pdl(hop_rt_kernel<PREC, RECON, false, false, RT>, grid, block, 0, st, A);
  }
}
// RHS per thread: 2 or 4 (the register-blocked kernel), else the plain one
template <int PREC, int RECON>
inline void launch_rt(const HopArgs &A, int rt, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  if (rt == 4) launch_rt2<PREC, RECON, 4>(A, grid, block, dag, red, st);
  else launch_rt2<PREC, RECON, 2>(A, grid, block, dag, red, st);
}

// the multi-RHS kernel with links staged in shared memory (srec reals per link)
template <int PREC, int RECON, int SREC>
inline void launch_mrhs2(const HopArgs &A, int rg, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st) {
  const size_t smem = mrhs_smem_bytes(SREC, block.x);
  if (dag) {
    if (red) launch_pdl(hop_mrhs_kernel<PREC, RECON, SREC, true, true>, grid, block, smem, st, A, rg);
    else launch_pdl(hop_mrhs_kernel<PREC, RECON, SREC, true, false>, grid, block, smem, st, A, rg);
  } else {
    if (red) launch_pdl(hop_mrhs_kernel<PREC, RECON, SREC, false, true>, grid, block, smem, st, A, rg);
    else launch_pdl(hop_mrhs_kernel<PREC, RECON, SREC, false, false>, grid, block, smem, st, A, rg);
  }
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
// pair: two threads per site (18-real links); mode 0 scalar, 1 packed FP32x2,
// 2 packed with the operands staged through shared memory, 3 the same bounded
// to 96 registers
void hop_launch_df64(const HopArgs &A, int recon, bool pair, int mode, dim3 grid, dim3 block, bool dag,
                     bool red, cudaStream_t st);
// rt: right-hand sides per thread (1, 2, 4); two: two sites per thread (packed FP32x2)
void hop_launch_f32(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, cudaStream_t st);
// several RHS interleaved with the site blocks (hop_ri_kernel; grid.x a
// multiple of A.nrhs)
void hop_launch_f32_ri(const HopArgs &A, int recon, dim3 grid, dim3 block, bool dag, bool red, cudaStream_t st);
// multi-RHS kernel with the links staged in shared memory: srec reals kept per
// link (18, or 12 for 12-real fields), rg right-hand sides per block, block.x
// sites per block (at most 48 KB of shared memory)
void hop_launch_mrhs_f32(const HopArgs &A, int recon, int srec, int rg, dim3 grid, dim3 block, bool dag, bool red,
                         cudaStream_t st);
void hop_launch_mrhs_h16(const HopArgs &A, int prec, int srec, int rg, dim3 grid, dim3 block, bool dag, bool red,
                         cudaStream_t st);
// staged: the two-site kernel with its operands staged through shared memory
void hop_launch_h16(const HopArgs &A, int prec, dim3 grid, dim3 block, bool dag, bool red, bool lf, int rt,
                    bool two, bool staged, cudaStream_t st);
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
