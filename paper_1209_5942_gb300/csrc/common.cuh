// common.cuh -- device-side building blocks shared by the sm_103a kernels:
// lattice geometry on the even-odd checkerboard, complex arithmetic in
// double / float / float-float ("df64"), and the storage formats of the
// even-odd structure-of-arrays fields (Sec. 4.2 of the paper: SoA on a 16-byte
// base type, gauge field split by the parity of the originating site).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lqcd.h"

#define LQCD_DEV __device__ __forceinline__
#define LQCD_HD __host__ __device__ __forceinline__

namespace lqcd {

// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic-stream-serialization attribute (launch_pdl) may be scheduled
// while its predecessor in the stream is still running, which hides the
// launch latency between the short kernels of a solver iteration;
// griddepcontrol.wait returns once the predecessor grid has completed and its
// writes are visible.  Every kernel launched that way calls pdl_wait() before
// its first global-memory access; launched normally it returns at once.
LQCD_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------

struct Geom {
  int L[4];     // x, y, z, t
  int Lh0;      // Lx / 2
  int Vh;       // sites per parity
  int antiper;  // fermion boundary factor -1 across t
};

// Coordinates of checkerboard site cb of parity p.  The lexicographic index
// is i = x + Lx*r with row r = y + Ly*(z + Lz*t); since Lx is even the pair
// (2k, 2k+1) along x holds one site of each parity and cb = i/2.
struct Site {
  int x, y, z, t, r;
};

LQCD_DEV Site site_of(const Geom& g, int p, int cb) {
  Site s;
  s.r = cb / g.Lh0;
  int xh = cb - s.r * g.Lh0;
  s.y = s.r % g.L[1];
  int zt = s.r / g.L[1];
  s.z = zt % g.L[2];
  s.t = zt / g.L[2];
  s.x = 2 * xh + ((p + s.y + s.z + s.t) & 1);
  return s;
}

// checkerboard index of the neighbour x + dir*mu_hat (dir = +1 / -1); the
// periodic wrap is a compare, and a step along y, z or t moves the row r by
// 1, Ly or Ly*Lz (minus the extent times that across the boundary)
LQCD_DEV int neighbour_cb(const Geom& g, const Site& s, int mu, int dir) {
  if (mu == 0) {
    const int x = dir > 0 ? (s.x + 1 == g.L[0] ? 0 : s.x + 1) : (s.x == 0 ? g.L[0] - 1 : s.x - 1);
    return s.r * g.Lh0 + (x >> 1);
  }
  const int c = mu == 1 ? s.y : mu == 2 ? s.z : s.t;
  const int n = g.L[mu];
  const int stride = mu == 1 ? 1 : mu == 2 ? g.L[1] : g.L[1] * g.L[2];
  const int step = dir > 0 ? (c + 1 == n ? 1 - n : 1) : (c == 0 ? n - 1 : -1);
  return (s.r + step * stride) * g.Lh0 + (s.x >> 1);
}

LQCD_DEV long lexi_index(const Geom& g, const Site& s) {
  return (long)s.x + (long)g.L[0] * s.r;
}

// ---------------------------------------------------------------------------
// float-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2 after
// normalisation).  Error-free transformations: Knuth's TwoSum, Dekker's
// Fast2Sum, and the FMA-based TwoProduct; the double-word add/multiply follow
// Dekker (1971) and the double-double library of Hida, Li and Bailey.
// ---------------------------------------------------------------------------

struct df {
  float hi, lo;
};

LQCD_DEV df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
LQCD_DEV df fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
LQCD_DEV df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
// Double-word addition in the cheaper form (TwoSum of the high parts, the low
// parts added in float, one renormalisation): 11 FP32 operations, absolute
// error below about 2^-46 (|a| + |b|).  The stencil and vector updates only
// need that absolute bound (errors are judged against max |y|), so the
// cancellation-safe 20-operation form is not used.
LQCD_DEV df operator+(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
LQCD_DEV df operator-(df a) { return {-a.hi, -a.lo}; }
LQCD_DEV df operator-(df a, df b) { return a + (-b); }
LQCD_DEV df operator*(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
LQCD_HD df df_from_double(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  return {hi, lo};
}
LQCD_HD double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------------------
// Complex numbers over a real type R (double, float, df)
// ---------------------------------------------------------------------------

template <class R>
struct Cx {
  R re, im;
};

template <class R> LQCD_DEV R rzero();
template <> LQCD_DEV double rzero<double>() { return 0.0; }
template <> LQCD_DEV float rzero<float>() { return 0.0f; }
template <> LQCD_DEV df rzero<df>() { return {0.0f, 0.0f}; }

template <class R> LQCD_DEV Cx<R> czero() { return {rzero<R>(), rzero<R>()}; }
template <class R> LQCD_DEV Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> LQCD_DEV Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> LQCD_DEV Cx<R> operator-(Cx<R> a) { return {-a.re, -a.im}; }
template <class R> LQCD_DEV Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// FP32 / FP64: every rounding step written out with intrinsics, so the compiler
// cannot contract differently in different kernels or launch variants and all
// of them give bit-identical results.
template <> LQCD_DEV Cx<float> operator+(Cx<float> a, Cx<float> b) {
  return {__fadd_rn(a.re, b.re), __fadd_rn(a.im, b.im)};
}
template <> LQCD_DEV Cx<float> operator-(Cx<float> a, Cx<float> b) {
  return {__fsub_rn(a.re, b.re), __fsub_rn(a.im, b.im)};
}
template <> LQCD_DEV Cx<float> operator*(Cx<float> a, Cx<float> b) {
  return {__fmaf_rn(a.re, b.re, -__fmul_rn(a.im, b.im)), __fmaf_rn(a.re, b.im, __fmul_rn(a.im, b.re))};
}
template <> LQCD_DEV Cx<double> operator+(Cx<double> a, Cx<double> b) {
  return {__dadd_rn(a.re, b.re), __dadd_rn(a.im, b.im)};
}
template <> LQCD_DEV Cx<double> operator-(Cx<double> a, Cx<double> b) {
  return {__dsub_rn(a.re, b.re), __dsub_rn(a.im, b.im)};
}
template <> LQCD_DEV Cx<double> operator*(Cx<double> a, Cx<double> b) {
  return {__fma_rn(a.re, b.re, -__dmul_rn(a.im, b.im)), __fma_rn(a.re, b.im, __dmul_rn(a.im, b.re))};
}
// a * b + c for reals with a single rounding where the hardware fuses
LQCD_DEV float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
LQCD_DEV double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
LQCD_DEV df rfma(df a, df b, df c) { return a * b + c; }

// i * a
template <class R> LQCD_DEV Cx<R> times_i(Cx<R> a) { return {-a.im, a.re}; }
template <class R> LQCD_DEV Cx<R> conj(Cx<R> a) { return {a.re, -a.im}; }
// a * b + c
template <class R> LQCD_DEV Cx<R> cmadd(Cx<R> a, Cx<R> b, Cx<R> c) {
  return {c.re + a.re * b.re - a.im * b.im, c.im + a.re * b.im + a.im * b.re};
}
template <> LQCD_DEV Cx<double> cmadd(Cx<double> a, Cx<double> b, Cx<double> c) {
  return {fma(-a.im, b.im, fma(a.re, b.re, c.re)), fma(a.im, b.re, fma(a.re, b.im, c.im))};
}
template <> LQCD_DEV Cx<float> cmadd(Cx<float> a, Cx<float> b, Cx<float> c) {
  return {fmaf(-a.im, b.im, fmaf(a.re, b.re, c.re)), fmaf(a.im, b.re, fmaf(a.re, b.im, c.im))};
}
template <class R> LQCD_DEV Cx<R> conj_madd(Cx<R> a, Cx<R> b, Cx<R> c) {  // conj(a)*b + c
  return {c.re + a.re * b.re + a.im * b.im, c.im + a.re * b.im - a.im * b.re};
}
template <> LQCD_DEV Cx<double> conj_madd(Cx<double> a, Cx<double> b, Cx<double> c) {
  return {fma(a.im, b.im, fma(a.re, b.re, c.re)), fma(-a.im, b.re, fma(a.re, b.im, c.im))};
}
template <> LQCD_DEV Cx<float> conj_madd(Cx<float> a, Cx<float> b, Cx<float> c) {
  return {fmaf(a.im, b.im, fmaf(a.re, b.re, c.re)), fmaf(-a.im, b.re, fmaf(a.re, b.im, c.im))};
}

// ---------------------------------------------------------------------------
// Two lanes of FP32 in one register pair (float2: lane x, lane y), operated on
// with the packed FP32x2 instructions of sm_100+ (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: two IEEE single-precision operations, each rounded as the
// scalar one).  The hop uses Cx<float2> for two output sites at once; every
// packed expression below mirrors the FP32 specialisation above operation by
// operation, so each lane's result is bit-identical to the scalar kernel's.
// ---------------------------------------------------------------------------
LQCD_DEV float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
template <> LQCD_DEV float2 rzero<float2>() { return make_float2(0.0f, 0.0f); }
template <> LQCD_DEV Cx<float2> operator+(Cx<float2> a, Cx<float2> b) {
  return {__fadd2_rn(a.re, b.re), __fadd2_rn(a.im, b.im)};
}
template <> LQCD_DEV Cx<float2> operator-(Cx<float2> a, Cx<float2> b) {
  return {__fadd2_rn(a.re, neg2(b.re)), __fadd2_rn(a.im, neg2(b.im))};
}
template <> LQCD_DEV Cx<float2> operator-(Cx<float2> a) { return {neg2(a.re), neg2(a.im)}; }
template <> LQCD_DEV Cx<float2> operator*(Cx<float2> a, Cx<float2> b) {
  return {__ffma2_rn(a.re, b.re, neg2(__fmul2_rn(a.im, b.im))), __ffma2_rn(a.re, b.im, __fmul2_rn(a.im, b.re))};
}
template <> LQCD_DEV Cx<float2> cmadd(Cx<float2> a, Cx<float2> b, Cx<float2> c) {
  return {__ffma2_rn(neg2(a.im), b.im, __ffma2_rn(a.re, b.re, c.re)),
          __ffma2_rn(a.im, b.re, __ffma2_rn(a.re, b.im, c.im))};
}
template <> LQCD_DEV Cx<float2> conj_madd(Cx<float2> a, Cx<float2> b, Cx<float2> c) {
  return {__ffma2_rn(a.im, b.im, __ffma2_rn(a.re, b.re, c.re)),
          __ffma2_rn(neg2(a.im), b.re, __ffma2_rn(a.re, b.im, c.im))};
}
template <> LQCD_DEV Cx<float2> times_i(Cx<float2> a) { return {neg2(a.im), a.re}; }
template <> LQCD_DEV Cx<float2> conj(Cx<float2> a) { return {a.re, neg2(a.im)}; }
// the pair (a, b) of two scalar complex numbers, and its lanes
LQCD_DEV Cx<float2> cpair(Cx<float> a, Cx<float> b) { return {make_float2(a.re, b.re), make_float2(a.im, b.im)}; }
LQCD_DEV Cx<float> lane_x(Cx<float2> a) { return {a.re.x, a.im.x}; }
LQCD_DEV Cx<float> lane_y(Cx<float2> a) { return {a.re.y, a.im.y}; }

// Host-side complex scalar handed to kernels in the arithmetic of the kernel.
struct HostC {
  double re, im;
};
template <class R> LQCD_DEV R from_double(double v);
template <> LQCD_DEV double from_double<double>(double v) { return v; }
template <> LQCD_DEV float from_double<float>(double v) { return (float)v; }
template <> LQCD_DEV df from_double<df>(double v) { return df_from_double(v); }

// Four complex coefficients prepared on the host in each arithmetic a kernel
// may compute in (the same roundings as from_double), so that no thread
// converts them: the double -> float-float split runs on the FP64 pipe.
struct Coef4 {
  HostC d[4];
  Cx<float> f[4];
  Cx<df> w[4];
};
inline Coef4 make_coef4(HostC a, HostC b, HostC c, HostC e) {
  Coef4 r;
  const HostC in[4] = {a, b, c, e};
  for (int i = 0; i < 4; i++) {
    r.d[i] = in[i];
    r.f[i] = {(float)in[i].re, (float)in[i].im};
    r.w[i] = {df_from_double(in[i].re), df_from_double(in[i].im)};
  }
  return r;
}
template <class R> LQCD_DEV Cx<R> coef_of(const Coef4 &c, int i);
template <> LQCD_DEV Cx<double> coef_of<double>(const Coef4 &c, int i) { return {c.d[i].re, c.d[i].im}; }
template <> LQCD_DEV Cx<float> coef_of<float>(const Coef4 &c, int i) { return c.f[i]; }
template <> LQCD_DEV Cx<df> coef_of<df>(const Coef4 &c, int i) { return c.w[i]; }

LQCD_DEV double to_double(double v) { return v; }
LQCD_DEV double to_double(float v) { return (double)v; }
LQCD_DEV double to_double(df v) { return df_to_double(v); }

// |a|^2 accumulated in double (norms and dot products use FP64 partial sums)
template <class R> LQCD_DEV double norm2_d(Cx<R> a) {
  double re = to_double(a.re), im = to_double(a.im);
  return __fma_rn(re, re, __dmul_rn(im, im));
}
// Float-float complex dot products (the hop's colour products, the gauge
// force's 3x3 products).  Each real output is a
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
// the first product of a sum starts the accumulator (no TwoSum with zero)
LQCD_DEV DfAcc dfacc_first(df a, df b, bool neg) {
  float ah = neg ? -a.hi : a.hi, al = neg ? -a.lo : a.lo;
  float p = __fmul_rn(ah, b.hi);
  float pe = __fmaf_rn(ah, b.hi, -p);
  pe = __fmaf_rn(ah, b.lo, pe);
  pe = __fmaf_rn(al, b.hi, pe);
  return {p, pe};
}
LQCD_DEV df dfacc_result(const DfAcc &A) { return fast_two_sum(A.s, A.e); }

// sum_j x_j * y_j (conjugating x when CONJ), complex double-words.  LAZY
// returns the accumulators unnormalised (value hi + lo exact, |lo| a few
// ulp(hi) at most), for callers that only add the result to other
// double-words before normalising.
template <bool CONJ, bool LAZY = false>
LQCD_DEV Cx<df> dfdot3(const Cx<df> x0, const Cx<df> x1, const Cx<df> x2, const Cx<df> y0,
                       const Cx<df> y1, const Cx<df> y2) {
  const Cx<df> xs[3] = {x0, x1, x2}, ys[3] = {y0, y1, y2};
  // (a + ib)(c + id) = (ac - bd) + i(ad + bc);  conj: (ac + bd) + i(ad - bc)
  DfAcc re = dfacc_first(xs[0].re, ys[0].re, false);
  DfAcc im = dfacc_first(xs[0].re, ys[0].im, false);
  dfacc_add_prod(re, xs[0].im, ys[0].im, !CONJ);
  dfacc_add_prod(im, xs[0].im, ys[0].re, CONJ);
#pragma unroll
  for (int j = 1; j < 3; j++) {
    dfacc_add_prod(re, xs[j].re, ys[j].re, false);
    dfacc_add_prod(re, xs[j].im, ys[j].im, !CONJ);
    dfacc_add_prod(im, xs[j].re, ys[j].im, false);
    dfacc_add_prod(im, xs[j].im, ys[j].re, CONJ);
  }
  if (LAZY) return {{re.s, re.e}, {im.s, im.e}};
  return {dfacc_result(re), dfacc_result(im)};
}

// Double-word sum without the final renormalisation (TwoSum of the high
// parts, low parts added in float: 8 operations).  The value hi + lo is the
// same as with renormalisation; the hop accumulates its sums this way and
// renormalises each accumulator once, before the epilogue.
LQCD_DEV df add_lazy(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return s;
}
LQCD_DEV df neg_df(df a) { return {-a.hi, -a.lo}; }
LQCD_DEV Cx<df> cadd_lazy(Cx<df> a, Cx<df> b) { return {add_lazy(a.re, b.re), add_lazy(a.im, b.im)}; }
LQCD_DEV Cx<df> csub_lazy(Cx<df> a, Cx<df> b) {
  return {add_lazy(a.re, neg_df(b.re)), add_lazy(a.im, neg_df(b.im))};
}
LQCD_DEV Cx<df> cnormalise(Cx<df> a) {
  return {fast_two_sum(a.re.hi, a.re.lo), fast_two_sum(a.im.hi, a.im.lo)};
}

// ---------------------------------------------------------------------------
// Float-float complex arithmetic in packed FP32x2 instructions.  A complex
// double-word is held as df2 {hi = (re.hi, im.hi), lo = (re.lo, im.lo)} --
// the order of its 16-byte word -- and each __fadd2_rn / __fmul2_rn /
// __ffma2_rn does the scalar operation of the real and the imaginary lane at
// once.  Every lane performs exactly the operations of the scalar functions
// above, in the same order (a negated factor is moved to the other operand,
// which rounds identically), so the packed and scalar forms give the same
// bits with about a third fewer instructions.
// ---------------------------------------------------------------------------
struct df2 {
  float2 hi, lo;
};
LQCD_DEV df2 df2_of(float4 w) { return {make_float2(w.x, w.y), make_float2(w.z, w.w)}; }
LQCD_DEV df2 df2_zero() { return {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)}; }
LQCD_DEV Cx<df> cx_of(df2 a) { return {{a.hi.x, a.lo.x}, {a.hi.y, a.lo.y}}; }
LQCD_DEV df2 neg_p(df2 a) { return {neg2(a.hi), neg2(a.lo)}; }
LQCD_DEV df2 times_i_p(df2 a) {  // (-im, re)
  return {make_float2(-a.hi.y, a.hi.x), make_float2(-a.lo.y, a.lo.x)};
}
LQCD_DEV df2 times_mi_p(df2 a) {  // (im, -re)
  return {make_float2(a.hi.y, -a.hi.x), make_float2(a.lo.y, -a.lo.x)};
}
// two_sum on each lane
LQCD_DEV void two_sum_p(float2 a, float2 b, float2 &s, float2 &e) {
  s = __fadd2_rn(a, b);
  const float2 bb = __fadd2_rn(s, neg2(a));
  e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}
// add_lazy on each lane
LQCD_DEV df2 add_lazy_p(df2 a, df2 b) {
  df2 r;
  two_sum_p(a.hi, b.hi, r.hi, r.lo);
  r.lo = __fadd2_rn(r.lo, __fadd2_rn(a.lo, b.lo));
  return r;
}
// product of the broadcast double-word (ah, al) with both lanes of b: the
// leading part p and its first-order error pe, as in dfacc_add_prod
LQCD_DEV void prod_p(float ah, float al, df2 b, float2 &p, float2 &pe) {
  const float2 h2 = make_float2(ah, ah), l2 = make_float2(al, al);
  p = __fmul2_rn(h2, b.hi);
  pe = __ffma2_rn(h2, b.hi, neg2(p));
  pe = __ffma2_rn(h2, b.lo, pe);
  pe = __ffma2_rn(l2, b.hi, pe);
}
LQCD_DEV void acc_p(df2 &A, float ah, float al, df2 b) {
  float2 p, pe, t;
  prod_p(ah, al, b, p, pe);
  two_sum_p(A.hi, p, A.hi, t);
  A.lo = __fadd2_rn(A.lo, __fadd2_rn(t, pe));
}
// dfdot3<CONJ, true> with lanes (re, im): x are the link words, y1 = h and
// y2 = i h (CONJ: -i h), so that lane re takes x.re y.re then -+ x.im y.im
// and lane im takes x.re y.im then +- x.im y.re, as the scalar form does
LQCD_DEV df2 dfdot3_p(const float4 x[3], const df2 y1[3], const df2 y2[3]) {
  df2 A;
  prod_p(x[0].x, x[0].z, y1[0], A.hi, A.lo);
  acc_p(A, x[0].y, x[0].w, y2[0]);
#pragma unroll
  for (int j = 1; j < 3; j++) {
    acc_p(A, x[j].x, x[j].z, y1[j]);
    acc_p(A, x[j].y, x[j].w, y2[j]);
  }
  return A;
}
// v times the unit f: 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
template <int F> LQCD_DEV df2 unit_p(df2 v) {
  return F == 0 ? v : F == 1 ? times_i_p(v) : F == 2 ? neg_p(v) : times_mi_p(v);
}

// |v|^2 of one site's n complex components, returned as a double.  FP64
// values are squared and summed in FP64.  Float-float values are summed in
// float-float: each square (hi + lo)^2 contributes its leading part hi*hi
// exactly (TwoProduct) plus 2 hi lo (lo^2 < 2^-48 hi^2 is dropped), the
// leading parts go through a TwoSum chain, and as all terms are positive
// the relative error stays near 2^-44.  FP32 values (the sloppy formats,
// whose components carry 24-bit mantissas at best) are squared and summed
// in FP32 with FMAs, relative error <= 2n u_32.  Both are converted once:
// per-component FP64 conversions and products would keep GB300's FP64 pipe
// (1/64 of the FP32 rate) busier than the stencil.  Cross-site sums are
// FP64 in every case.
template <class R, int N> LQCD_DEV double site_norm2(const Cx<R> v[N]) {
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < N; k++) t += norm2_d(v[k]);
  return t;
}
template <int N> LQCD_DEV double df_site_norm2(const Cx<df> v[N]) {
  DfAcc A = dfacc_first(v[0].re, v[0].re, false);
  dfacc_add_prod(A, v[0].im, v[0].im, false);
#pragma unroll
  for (int k = 1; k < N; k++) {
    dfacc_add_prod(A, v[k].re, v[k].re, false);
    dfacc_add_prod(A, v[k].im, v[k].im, false);
  }
  return df_to_double(dfacc_result(A));
}
template <> LQCD_DEV double site_norm2<df, 12>(const Cx<df> v[12]) { return df_site_norm2<12>(v); }
template <> LQCD_DEV double site_norm2<float, 12>(const Cx<float> v[12]) {
  float t = 0.0f;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    t = __fmaf_rn(v[k].re, v[k].re, t);
    t = __fmaf_rn(v[k].im, v[k].im, t);
  }
  return (double)t;
}

// Sum of v[0..nb) in a fixed order by one block of FIN_THREADS threads:
// thread t adds v[t], v[t + FIN_THREADS], ... in that order (the loop is
// unrolled, so a thread has several independent loads in flight and the
// whole sum costs a few L2 latencies), then a fixed shuffle tree per warp and
// one over the warps.  The order depends on nb only, so the result is
// reproducible for any launch shape of the kernels that wrote the partials,
// and the single and the batched solver reduce identically.  Call with
// blockDim.x == FIN_THREADS; sh holds 33 doubles.
constexpr int FIN_THREADS = 1024;
LQCD_DEV double block_sum_fixed(const double *v, int nb, double *sh) {
  double t = 0.0;
#pragma unroll 8
  for (int k = threadIdx.x; k < nb; k += FIN_THREADS) t += v[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = t;
  __syncthreads();
  if (w == 0) {
    double r = sh[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (l == 0) sh[32] = r;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Storage formats of even-odd SoA spinor fields.
// A half field is [component 12][Vh] in 16-byte words per the precision.
// ---------------------------------------------------------------------------

struct SpinorView {
  void* ptr;     // start of this half field (one right-hand side)
  float* scale;  // [Vh] for the 16-bit formats
  int Vh;
};

template <int PREC> struct SpinorIO;

template <> struct SpinorIO<LQCD_F64> {
  using R = double;
  static LQCD_DEV void load(const SpinorView& v, int cb, Cx<double> s[12]) {
    const double2* p = (const double2*)v.ptr;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 w = __ldg(p + (size_t)k * v.Vh + cb);
      s[k] = {w.x, w.y};
    }
  }
  static LQCD_DEV void store(const SpinorView& v, int cb, const Cx<double> s[12]) {
    double2* p = (double2*)v.ptr;
#pragma unroll
    for (int k = 0; k < 12; k++) p[(size_t)k * v.Vh + cb] = make_double2(s[k].re, s[k].im);
  }
};

template <> struct SpinorIO<LQCD_DF64> {
  using R = df;
  static LQCD_DEV void load(const SpinorView& v, int cb, Cx<df> s[12]) {
    const float4* p = (const float4*)v.ptr;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      float4 w = __ldg(p + (size_t)k * v.Vh + cb);
      s[k] = {{w.x, w.z}, {w.y, w.w}};
    }
  }
  static LQCD_DEV void store(const SpinorView& v, int cb, const Cx<df> s[12]) {
    float4* p = (float4*)v.ptr;
#pragma unroll
    for (int k = 0; k < 12; k++)
      p[(size_t)k * v.Vh + cb] = make_float4(s[k].re.hi, s[k].im.hi, s[k].re.lo, s[k].im.lo);
  }
};

template <> struct SpinorIO<LQCD_F32> {
  using R = float;
  static LQCD_DEV void load(const SpinorView& v, int cb, Cx<float> s[12]) {
    const float4* p = (const float4*)v.ptr;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 w = __ldg(p + (size_t)k * v.Vh + cb);
      s[2 * k] = {w.x, w.y};
      s[2 * k + 1] = {w.z, w.w};
    }
  }
  static LQCD_DEV void store(const SpinorView& v, int cb, const Cx<float> s[12]) {
    float4* p = (float4*)v.ptr;
#pragma unroll
    for (int k = 0; k < 6; k++)
      p[(size_t)k * v.Vh + cb] = make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
  }
};

// 16-bit reals with one float scale per site: value = stored * scale, the
// scale being the site's largest |real component| (so stored values lie in
// [-1, 1]).  24 reals = three 16-byte words.
template <class H> struct Half16;
template <> struct Half16<__nv_bfloat16> {
  static LQCD_DEV float to_f(uint16_t u) { return __bfloat162float(__ushort_as_bfloat16(u)); }
  // the (low, high) pair of one 32-bit word: a bf16 is the upper half of its
  // float, so each value is one shift or mask (bitwise the same as to_f)
  static LQCD_DEV float2 to_f2(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
  }
  static LQCD_DEV uint16_t from_f(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
  // (lo, hi) rounded to nearest and packed in one conversion
  static LQCD_DEV uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&t);
  }
};
template <> struct Half16<__half> {
  static LQCD_DEV float to_f(uint16_t u) { return __half2float(__ushort_as_half(u)); }
  // the (low, high) pair of one 32-bit word in one conversion (exact, as to_f)
  static LQCD_DEV float2 to_f2(uint32_t w) {
    __half2 h;
    *reinterpret_cast<uint32_t*>(&h) = w;
    return __half22float2(h);
  }
  static LQCD_DEV uint16_t from_f(float f) { return __half_as_ushort(__float2half_rn(f)); }
  static LQCD_DEV uint32_t pack2(float lo, float hi) {
    __half2 t = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&t);
  }
};

template <class H> struct SpinorIO16 {
  using R = float;
  // the stored values without the site scale, which is returned: the hop
  // applies it in its accumulation FMAs instead of to every component
  static LQCD_DEV float load_unscaled(const SpinorView& v, int cb, Cx<float> s[12]) {
    const uint4* p = (const uint4*)v.ptr;
    const float sc = __ldg(v.scale + cb);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 w = __ldg(p + (size_t)k * v.Vh + cb);
      uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 f = Half16<H>::to_f2(ww[j]);
        s[4 * k + j] = {f.x, f.y};
      }
    }
    return sc;
  }
  static LQCD_DEV void load(const SpinorView& v, int cb, Cx<float> s[12]) {
    const uint4* p = (const uint4*)v.ptr;
    float sc = __ldg(v.scale + cb);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 w = __ldg(p + (size_t)k * v.Vh + cb);
      uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 f = Half16<H>::to_f2(ww[j]);
        s[4 * k + j] = {__fmul_rn(f.x, sc), __fmul_rn(f.y, sc)};
      }
    }
  }
  static LQCD_DEV void store(const SpinorView& v, int cb, const Cx<float> s[12]) {
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(s[k].re), fabsf(s[k].im)));
    float inv = m > 0.0f ? 1.0f / m : 0.0f;
    uint4* p = (uint4*)v.ptr;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint32_t ww[4];
#pragma unroll
      for (int j = 0; j < 4; j++)
        ww[j] = Half16<H>::pack2(__fmul_rn(s[4 * k + j].re, inv), __fmul_rn(s[4 * k + j].im, inv));
      p[(size_t)k * v.Vh + cb] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
    }
    v.scale[cb] = m;
  }
};
template <> struct SpinorIO<LQCD_BF16S> : SpinorIO16<__nv_bfloat16> {};
template <> struct SpinorIO<LQCD_F16S> : SpinorIO16<__half> {};
template <int PREC> constexpr bool kScaled16 = PREC == LQCD_BF16S || PREC == LQCD_F16S;

// ---------------------------------------------------------------------------
// Gauge field storage: [parity][mu][entry][Vh] per precision, entry = 3*row +
// col for the 9 (recon 18) or 6 (recon 12) stored complex entries.
//   F64 / DF64 : 16 B per complex entry.
//   F32        : complex entries paired in 16-B words; recon 18 stores
//                entries 0..7 in 4 words and entry 8 in a trailing 8-B word
//                plane; recon 12 uses 3 words.
//   BF16 / F16 : 16-bit reals, recon 12 only: 12 reals = 16-B + 8-B planes.
// ---------------------------------------------------------------------------

struct GaugeView {
  const void* ptr;  // start of the field
  int Vh;
  size_t parity_stride;  // bytes per parity block
  size_t mu_stride;      // bytes per direction block
};

template <int PREC, int RECON> struct LinkIO;

template <int RECON> struct LinkIO<LQCD_F64, RECON> {
  static LQCD_DEV void load(const GaugeView& g, int p, int mu, int cb, Cx<double> u[9]) {
    const double2* b = (const double2*)((const char*)g.ptr + p * g.parity_stride + mu * g.mu_stride);
#pragma unroll
    for (int k = 0; k < (RECON == 18 ? 9 : 6); k++) {
      double2 w = __ldg(b + (size_t)k * g.Vh + cb);
      u[k] = {w.x, w.y};
    }
  }
};
template <int RECON> struct LinkIO<LQCD_DF64, RECON> {
  static LQCD_DEV void load(const GaugeView& g, int p, int mu, int cb, Cx<df> u[9]) {
    const float4* b = (const float4*)((const char*)g.ptr + p * g.parity_stride + mu * g.mu_stride);
#pragma unroll
    for (int k = 0; k < (RECON == 18 ? 9 : 6); k++) {
      float4 w = __ldg(b + (size_t)k * g.Vh + cb);
      u[k] = {{w.x, w.z}, {w.y, w.w}};
    }
  }
};
template <int RECON> struct LinkIO<LQCD_F32, RECON> {
  static LQCD_DEV void load(const GaugeView& g, int p, int mu, int cb, Cx<float> u[9]) {
    const char* base = (const char*)g.ptr + p * g.parity_stride + mu * g.mu_stride;
    const float4* b = (const float4*)base;
    constexpr int NW = RECON == 18 ? 4 : 3;
#pragma unroll
    for (int k = 0; k < NW; k++) {
      float4 w = __ldg(b + (size_t)k * g.Vh + cb);
      u[2 * k] = {w.x, w.y};
      u[2 * k + 1] = {w.z, w.w};
    }
    if (RECON == 18) {
      const float2* t = (const float2*)(base + (size_t)4 * g.Vh * 16);
      float2 w = __ldg(t + cb);
      u[8] = {w.x, w.y};
    }
  }
};
template <class H> struct LinkIO16 {
  static LQCD_DEV void load(const GaugeView& g, int p, int mu, int cb, Cx<float> u[9]) {
    const char* base = (const char*)g.ptr + p * g.parity_stride + mu * g.mu_stride;
    uint4 w = __ldg((const uint4*)base + cb);
    uint2 w2 = __ldg((const uint2*)(base + (size_t)g.Vh * 16) + cb);
    uint32_t ww[6] = {w.x, w.y, w.z, w.w, w2.x, w2.y};
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float2 f = Half16<H>::to_f2(ww[k]);
      u[k] = {f.x, f.y};
    }
  }
};
template <> struct LinkIO<LQCD_BF16S, 12> : LinkIO16<__nv_bfloat16> {};
template <> struct LinkIO<LQCD_F16S, 12> : LinkIO16<__half> {};

// REC12 (Sec. 4.1): row 2 = conj(row0 x row1) for an SU(3) link.
template <class R> LQCD_DEV void reconstruct_row2(Cx<R> u[9]) {
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

// Bytes per link entry block for the sizing of gauge fields (host side).
LQCD_HD size_t link_bytes_per_site(int prec, int recon) {
  switch (prec) {
    case LQCD_F64:
    case LQCD_DF64: return (size_t)16 * (recon == 18 ? 9 : 6);
    case LQCD_F32: return recon == 18 ? 72 : 48;
    default: return 24;  // 16-bit, recon 12
  }
}
LQCD_HD size_t spinor_bytes_per_site(int prec) {
  switch (prec) {
    case LQCD_F64:
    case LQCD_DF64: return 192;
    case LQCD_F32: return 96;
    default: return 48;
  }
}

}  // namespace lqcd
