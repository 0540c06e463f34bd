// gauge.cu -- gauge-field kernels of Sec. 2.1/2.2 in FP64 on the FP64 master
// copy ([parity][mu][9][Vh] complex128):
//   * plaquette and Wilson gauge action  S_g = (beta/3) sum (3 - Re Tr U_munu)
//   * gauge force dS_g/domega^a = -(beta/3) Re Tr[i T^a U_mu(x) A_mu(x)],
//     A = staple sum (Sec. 2.2: the plaquette product without U_mu(x))
//   * Cabibbo-Marinari heatbath (Sec. 2.2, Fig. "heatbath algorithm") with the
//     exact SU(2) update, checkerboarded over (mu, parity) so that every
//     thread owns one link whose staple does not involve another updated link
//   * Gaussian momenta / spinors, U <- exp(i eps P) U, reunitarisation,
//     momentum step and kinetic energy for the HMC of Sec. 2.2.
// Random numbers: Philox4x32-10 (Salmon et al., SC'11) with the counter layout
// documented in lqcd.h, so a run is reproducible for any launch shape.
#include <cmath>

#include "internal.h"

namespace lqcd {

using C = Cx<double>;

// ---------------------------------------------------------------------------
// small SU(3) algebra in FP64 (row-major 3x3)
// ---------------------------------------------------------------------------
struct M3 {
  C m[9];
};
LQCD_DEV M3 mmul(const M3 &a, const M3 &b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C s = a.m[3 * i] * b.m[j];
      s = cmadd(a.m[3 * i + 1], b.m[3 + j], s);
      s = cmadd(a.m[3 * i + 2], b.m[6 + j], s);
      r.m[3 * i + j] = s;
    }
  return r;
}
// a * b^+
LQCD_DEV M3 mmul_nd(const M3 &a, const M3 &b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C s = a.m[3 * i] * conj(b.m[3 * j]);
      s = cmadd(a.m[3 * i + 1], conj(b.m[3 * j + 1]), s);
      s = cmadd(a.m[3 * i + 2], conj(b.m[3 * j + 2]), s);
      r.m[3 * i + j] = s;
    }
  return r;
}
LQCD_DEV double re_trace(const M3 &a) { return a.m[0].re + a.m[4].re + a.m[8].re; }

struct Pos {
  int p, cb;
  long lexi;
};
// position of a site given by coordinates
LQCD_DEV Pos pos_of(const Geom &g, int x, int y, int z, int t) {
  int r = y + g.L[1] * (z + g.L[2] * t);
  long i = (long)x + (long)g.L[0] * r;
  return Pos{(x + y + z + t) & 1, (int)(i >> 1), i};
}
LQCD_DEV void coords_shift(const Geom &g, int c[4], int mu, int d) { c[mu] = (c[mu] + d + g.L[mu]) % g.L[mu]; }

LQCD_DEV M3 load_link(const double2 *master, const Geom &g, const Pos &s, int mu) {
  M3 u;
  const double2 *b = master + ((size_t)(s.p * 4 + mu) * 9) * g.Vh + s.cb;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 w = b[(size_t)k * g.Vh];
    u.m[k] = {w.x, w.y};
  }
  return u;
}
LQCD_DEV void store_link(double2 *master, const Geom &g, const Pos &s, int mu, const M3 &u) {
  double2 *b = master + ((size_t)(s.p * 4 + mu) * 9) * g.Vh + s.cb;
#pragma unroll
  for (int k = 0; k < 9; k++) b[(size_t)k * g.Vh] = make_double2(u.m[k].re, u.m[k].im);
}
LQCD_DEV Pos at(const Geom &g, const int c[4]) { return pos_of(g, c[0], c[1], c[2], c[3]); }

// staple sum A_mu(x) with Re Tr(U_mu(x) A) = sum of the 6 plaquettes through
// U_mu(x); ld(pos, nu) loads the link U_nu at pos
template <class LD>
LQCD_DEV M3 staple_with(LD ld, const Geom &g, const int c[4], int mu) {
  M3 A;
#pragma unroll
  for (int k = 0; k < 9; k++) A.m[k] = czero<double>();
  int cpm[4] = {c[0], c[1], c[2], c[3]};
  coords_shift(g, cpm, mu, +1);
  for (int nu = 0; nu < 4; nu++) {
    if (nu == mu) continue;
    int cpn[4] = {c[0], c[1], c[2], c[3]}, cmn[4] = {c[0], c[1], c[2], c[3]};
    int cpmmn[4] = {cpm[0], cpm[1], cpm[2], cpm[3]};
    coords_shift(g, cpn, nu, +1);
    coords_shift(g, cmn, nu, -1);
    coords_shift(g, cpmmn, nu, -1);
    // upper: U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    M3 t = mmul_nd(ld(at(g, cpm), nu), ld(at(g, cpn), mu));
    t = mmul_nd(t, ld(at(g, c), nu));
#pragma unroll
    for (int k = 0; k < 9; k++) A.m[k] = A.m[k] + t.m[k];
    // lower: U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
    M3 l1 = ld(at(g, cpmmn), nu), l2 = ld(at(g, cmn), mu);
    M3 w = mmul(l2, l1);  // (U_mu(x-nu) U_nu(x+mu-nu))^+ = l1^+ l2^+
    M3 wd;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) wd.m[3 * i + j] = conj(w.m[3 * j + i]);
    t = mmul(wd, ld(at(g, cmn), nu));
#pragma unroll
    for (int k = 0; k < 9; k++) A.m[k] = A.m[k] + t.m[k];
  }
  return A;
}

LQCD_DEV M3 staple(const double2 *U, const Geom &g, const int c[4], int mu) {
  return staple_with([&](const Pos &s, int nu) { return load_link(U, g, s, nu); }, g, c, mu);
}

// ---------------------------------------------------------------------------
// Rectangles of the tree-level Symanzik action (Sec. 2.1, eq. "S_tlsym").
// A step of a path from site c in direction sgn*dir uses U_dir(c) forwards
// or U_dir(c - dir)^+ backwards.
// ---------------------------------------------------------------------------
LQCD_DEV M3 step_link(const double2 *U, const Geom &g, int c[4], int dir, int sgn) {
  if (sgn > 0) {
    M3 u = load_link(U, g, at(g, c), dir);
    coords_shift(g, c, dir, +1);
    return u;
  }
  coords_shift(g, c, dir, -1);
  M3 u = load_link(U, g, at(g, c), dir), d;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) d.m[3 * i + j] = conj(u.m[3 * j + i]);
  return d;
}

// product of the 5 steps (dirs[k], sgns[k]) of a path starting at c
LQCD_DEV M3 path5(const double2 *U, const Geom &g, const int c0[4], const int dirs[5], const int sgns[5]) {
  int c[4] = {c0[0], c0[1], c0[2], c0[3]};
  M3 r = step_link(U, g, c, dirs[0], sgns[0]);
  for (int k = 1; k < 5; k++) r = mmul(r, step_link(U, g, c, dirs[k], sgns[k]));
  return r;
}

// thread -> (parity, cb) over all 2*Vh sites; coordinates
LQCD_DEV bool thread_site(const Geom &g, long tid, int *p, int *cb, int c[4]) {
  if (tid >= 2L * g.Vh) return false;
  *p = (int)(tid / g.Vh);
  *cb = (int)(tid - (long)(*p) * g.Vh);
  Site s = site_of(g, *p, *cb);
  c[0] = s.x;
  c[1] = s.y;
  c[2] = s.z;
  c[3] = s.t;
  return true;
}

// thread -> (direction mu, site): consecutive threads take consecutive sites
// of one direction, so the per-link kernels read and write link-ordered
// planes contiguously and run one thread per link
LQCD_DEV bool thread_link(const Geom &g, long tid, int *mu, int *p, int *cb, int c[4]) {
  const long V = 2L * g.Vh;
  if (tid >= 4 * V) return false;
  *mu = (int)(tid / V);
  return thread_site(g, tid - (long)(*mu) * V, p, cb, c);
}

LQCD_DEV double block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; k++) t += sh[k];
  return t;
}

// sum over sites of sum_{mu<nu} Re Tr U_munu(x): per-block partials
__global__ void __launch_bounds__(128) plaquette_kernel(const double2 *U, Geom g, double *partials) {
  __shared__ double sh[8];
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int p, cb, c[4];
  double acc = 0.0;
  if (thread_site(g, tid, &p, &cb, c)) {
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        int cpm[4] = {c[0], c[1], c[2], c[3]}, cpn[4] = {c[0], c[1], c[2], c[3]};
        coords_shift(g, cpm, mu, +1);
        coords_shift(g, cpn, nu, +1);
        M3 a = mmul(load_link(U, g, Pos{p, cb, 0}, mu), load_link(U, g, at(g, cpm), nu));
        M3 b = mmul(load_link(U, g, Pos{p, cb, 0}, nu), load_link(U, g, at(g, cpn), mu));
        M3 w = mmul_nd(a, b);  // U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^+
        acc += re_trace(w);
      }
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// Rectangle staples from plaquette staples.  With the plaquette staple
//   S(y; mu, nu, s) = U_{s nu}(y + mu) U_mu(y + s nu)^+ U_{s nu}(y)^+
// (s = +-1, U_{-nu}(y) = U_nu(y - nu)^+) and unitary links, the three
// rectangle staples of U_mu(x) in the (mu, s nu) half plane are
//   link first along mu:  U_mu(x + mu) S(x + mu) S(x)
//   link second along mu: S(x) S(x - mu) U_mu(x - mu)
//   long side along nu:   U_{s nu}(x + mu) S(x + s nu) U_{s nu}(x)^+
// (the inner U_{s nu} U_{s nu}^+ pairs cancel), two products each instead of
// four.  A first kernel stores the 6 plaquette staples of every link.
// ---------------------------------------------------------------------------
// staple field layout: [mu][k = 2 * (nu index) + (s < 0)][entry 9][V] complex,
// nu index = nu - (nu > mu), lexicographic V
LQCD_DEV size_t stap_index(long V, int mu, int k, int e, long lexi) {
  return (((size_t)mu * 6 + k) * 9 + e) * (size_t)V + lexi;
}
LQCD_DEV M3 load_stap(const double2 *S, long V, int mu, int k, long lexi) {
  M3 r;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    double2 w = S[stap_index(V, mu, k, e, lexi)];
    r.m[e] = {w.x, w.y};
  }
  return r;
}
LQCD_DEV int stap_k(int mu, int nu, int s) { return 2 * (nu - (nu > mu ? 1 : 0)) + (s < 0 ? 1 : 0); }

// U_{s nu}(y) as a matrix
LQCD_DEV M3 signed_link(const double2 *U, const Geom &g, const int c[4], int nu, int s) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  return step_link(U, g, d, nu, s);
}

__global__ void __launch_bounds__(128) staple6_kernel(const double2 *U, Geom g, double2 *S) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  const long V = 2L * g.Vh;
  const long lexi = at(g, c).lexi;
  {
    int cpm[4] = {c[0], c[1], c[2], c[3]};
    coords_shift(g, cpm, mu, +1);
    for (int nu = 0; nu < 4; nu++) {
      if (nu == mu) continue;
      for (int s = -1; s <= 1; s += 2) {
        int cps[4] = {c[0], c[1], c[2], c[3]};
        coords_shift(g, cps, nu, s);
        // U_{s nu}(x + mu) U_mu(x + s nu)^+ U_{s nu}(x)^+
        M3 t = mmul_nd(signed_link(U, g, cpm, nu, s), load_link(U, g, at(g, cps), mu));
        t = mmul_nd(t, signed_link(U, g, c, nu, s));
        const int k = stap_k(mu, nu, s);
#pragma unroll
        for (int e = 0; e < 9; e++) S[stap_index(V, mu, k, e, lexi)] = make_double2(t.m[e].re, t.m[e].im);
      }
    }
  }
}

LQCD_DEV void add_scaled(M3 &A, double c, const M3 &t) {
#pragma unroll
  for (int e = 0; e < 9; e++) A.m[e] = {fma(c, t.m[e].re, A.m[e].re), fma(c, t.m[e].im, A.m[e].im)};
}

// dS/domega of the tlSym action from the stored plaquette staples: one
// accumulator A = c0 sum S + c1 sum (rectangle staples), the (nu, s) loop
// kept rolled so only a few 3x3 matrices are live at a time.
__global__ void __launch_bounds__(128) gauge_force_sym_kernel(const double2 *U, const double2 *S, Geom g,
                                                              double beta, double c1, double *out) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  const long V = 2L * g.Vh;
  const Pos s0 = at(g, c);
  const double c0 = 1.0 - 8.0 * c1;
  {
    int cpm[4] = {c[0], c[1], c[2], c[3]}, cmm[4] = {c[0], c[1], c[2], c[3]};
    coords_shift(g, cpm, mu, +1);
    coords_shift(g, cmm, mu, -1);
    const Pos spm = at(g, cpm), smm = at(g, cmm);
    M3 A;
#pragma unroll
    for (int e = 0; e < 9; e++) A.m[e] = czero<double>();
#pragma unroll 1
    for (int k = 0; k < 6; k++) {
      const int nu = (k >> 1) + ((k >> 1) >= mu ? 1 : 0), s = (k & 1) ? -1 : 1;
      const M3 Sx = load_stap(S, V, mu, k, s0.lexi);
      add_scaled(A, c0, Sx);
      add_scaled(A, c1, mmul(mmul(load_link(U, g, spm, mu), load_stap(S, V, mu, k, spm.lexi)), Sx));
      add_scaled(A, c1, mmul(mmul(Sx, load_stap(S, V, mu, k, smm.lexi)), load_link(U, g, smm, mu)));
      int cps[4] = {c[0], c[1], c[2], c[3]};
      coords_shift(g, cps, nu, s);
      add_scaled(A, c1, mmul_nd(mmul(signed_link(U, g, cpm, nu, s), load_stap(S, V, mu, k, at(g, cps).lexi)),
                                signed_link(U, g, c, nu, s)));
    }
    const M3 W = mmul(load_link(U, g, s0, mu), A);
    const C *w = W.m;
    double tr[8];
    tr[0] = (w[3] + w[1]).im;
    tr[1] = (times_i(w[1] - w[3])).im;
    tr[2] = (w[0] - w[4]).im;
    tr[3] = (w[6] + w[2]).im;
    tr[4] = (times_i(w[2] - w[6])).im;
    tr[5] = (w[7] + w[5]).im;
    tr[6] = (times_i(w[5] - w[7])).im;
    tr[7] = (w[0] + w[4] - w[8] - w[8]).im * 0.57735026918962576451;
    double *o = out + ((size_t)mu * V + s0.lexi) * 8;
#pragma unroll
    for (int a = 0; a < 8; a++) o[a] = (beta / 3.0) * 0.5 * tr[a];
  }
}

// ---------------------------------------------------------------------------
// The same staple construction in float-float arithmetic (FP64-class
// accuracy on the FP32 pipe, the hop's DF64 format): GB300's FP64 pipe runs at
// 1/64 of the FP32 rate, and the tlSym force is ~10^4 flop per link.  Links
// come from the DF64 copy of the field; 3x3 products use the error-free
// complex dot product of the hop (packed FP32x2); W is converted to FP64 for
// the traces.
// ---------------------------------------------------------------------------
struct M3d {
  Cx<df> m[9];
};
// The 3x3 products run the packed FP32x2 form of the error-free complex dot
// product (the bits of dfdot3, normalised): each column of b (row of a for
// a b^+) and its product with i (or -i) are formed once and reused for the
// three dot products that share it.
LQCD_DEV float4 f4_of(Cx<df> z) { return make_float4(z.re.hi, z.im.hi, z.re.lo, z.im.lo); }
LQCD_DEV df2 p_of(Cx<df> z) { return {make_float2(z.re.hi, z.im.hi), make_float2(z.re.lo, z.im.lo)}; }
LQCD_DEV Cx<df> normalised_of(df2 a) {  // fast_two_sum on each lane
  const float2 s = __fadd2_rn(a.hi, a.lo);
  const float2 e = __fadd2_rn(a.lo, neg2(__fadd2_rn(s, neg2(a.hi))));
  return {{s.x, e.x}, {s.y, e.y}};
}
LQCD_DEV M3d dmul(const M3d &a, const M3d &b) {  // a b
  M3d r;
#pragma unroll
  for (int j = 0; j < 3; j++) {
    df2 y1[3], y2[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      y1[q] = p_of(b.m[3 * q + j]);
      y2[q] = times_i_p(y1[q]);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float4 x[3] = {f4_of(a.m[3 * i]), f4_of(a.m[3 * i + 1]), f4_of(a.m[3 * i + 2])};
      r.m[3 * i + j] = normalised_of(dfdot3_p(x, y1, y2));
    }
  }
  return r;
}
LQCD_DEV M3d dmul_nd(const M3d &a, const M3d &b) {  // a b^+
  M3d r;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    df2 y1[3], y2[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      y1[q] = p_of(a.m[3 * i + q]);
      y2[q] = times_mi_p(y1[q]);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const float4 x[3] = {f4_of(b.m[3 * j]), f4_of(b.m[3 * j + 1]), f4_of(b.m[3 * j + 2])};
      r.m[3 * i + j] = normalised_of(dfdot3_p(x, y1, y2));
    }
  }
  return r;
}
LQCD_DEV M3d load_link_d(const GaugeView &Ud, const Pos &s, int mu) {
  M3d u;
  LinkIO<LQCD_DF64, 18>::load(Ud, s.p, mu, s.cb, u.m);
  return u;
}
LQCD_DEV M3d dagger_d(const M3d &u) {
  M3d d;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) d.m[3 * i + j] = conj(u.m[3 * j + i]);
  return d;
}
// U_{s nu}(c) in float-float
LQCD_DEV M3d signed_link_d(const GaugeView &Ud, const Geom &g, const int c[4], int nu, int s) {
  if (s > 0) return load_link_d(Ud, at(g, c), nu);
  int d[4] = {c[0], c[1], c[2], c[3]};
  coords_shift(g, d, nu, -1);
  return dagger_d(load_link_d(Ud, at(g, d), nu));
}
LQCD_DEV void store_stap_d(float4 *S, long V, int mu, int k, long lexi, const M3d &t) {
#pragma unroll
  for (int e = 0; e < 9; e++)
    S[stap_index(V, mu, k, e, lexi)] = make_float4(t.m[e].re.hi, t.m[e].im.hi, t.m[e].re.lo, t.m[e].im.lo);
}
LQCD_DEV M3d load_stap_d(const float4 *S, long V, int mu, int k, long lexi) {
  M3d r;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const float4 w = S[stap_index(V, mu, k, e, lexi)];
    r.m[e] = {{w.x, w.z}, {w.y, w.w}};
  }
  return r;
}
LQCD_DEV void add_lazy_m(M3d &A, const M3d &t) {  // cadd_lazy on every entry, packed
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const df2 r = add_lazy_p(p_of(A.m[e]), p_of(t.m[e]));
    A.m[e] = {{r.hi.x, r.lo.x}, {r.hi.y, r.lo.y}};
  }
}

__global__ void __launch_bounds__(128) staple6_df_kernel(GaugeView Ud, Geom g, float4 *S) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  const long V = 2L * g.Vh;
  const long lexi = at(g, c).lexi;
  {
    int cpm[4] = {c[0], c[1], c[2], c[3]};
    coords_shift(g, cpm, mu, +1);
#pragma unroll 1
    for (int k = 0; k < 6; k++) {
      const int nu = (k >> 1) + ((k >> 1) >= mu ? 1 : 0), s = (k & 1) ? -1 : 1;
      int cps[4] = {c[0], c[1], c[2], c[3]};
      coords_shift(g, cps, nu, s);
      // U_{s nu}(x + mu) U_mu(x + s nu)^+ U_{s nu}(x)^+
      M3d t = dmul_nd(signed_link_d(Ud, g, cpm, nu, s), load_link_d(Ud, at(g, cps), mu));
      t = dmul_nd(t, signed_link_d(Ud, g, c, nu, s));
      store_stap_d(S, V, mu, k, lexi, t);
    }
  }
}

// dS/domega of c0 (plaquette) + c1 (rectangle) in float-float; c1 = 0 gives
// the Wilson force from the plaquette staples alone
// the force's constants as float-float (c0, c1, 1/sqrt 3) split on the host,
// and the final factor beta/6 in FP64
struct ForceConst {
  df c0, c1, r3;
  double f;
};

__global__ void __launch_bounds__(128, 3) gauge_force_df_kernel(GaugeView Ud, const float4 *S, Geom g, ForceConst cc,
                                                             double c1, double *out) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  const long V = 2L * g.Vh;
  const Pos s0 = at(g, c);
  {
    int cpm[4] = {c[0], c[1], c[2], c[3]}, cmm[4] = {c[0], c[1], c[2], c[3]};
    coords_shift(g, cpm, mu, +1);
    coords_shift(g, cmm, mu, -1);
    const Pos spm = at(g, cpm), smm = at(g, cmm);
    // rectangles first, then the plaquette staples (re-read), so only one
    // 3x3 accumulator is live during the products
    M3d Wr, Wp;
#pragma unroll
    for (int e = 0; e < 9; e++) Wr.m[e] = czero<df>();
    // the three rectangles of each staple k share one copy of the product
    // code: a run-time loop over the terms a b c (c daggered for the third)
    // keeps the kernel inside the instruction cache
#pragma unroll 1
    for (int k = 0; k < 6 && c1 != 0.0; k++) {
      const int nu = (k >> 1) + ((k >> 1) >= mu ? 1 : 0), s = (k & 1) ? -1 : 1;
      int cps[4] = {c[0], c[1], c[2], c[3]};
      coords_shift(g, cps, nu, s);
#pragma unroll 1
      for (int j = 0; j < 3; j++) {
        M3d ab;
        {
          M3d a, b;
          if (j == 0) {  // U_mu(x + mu) S(x + mu) S(x)
            a = load_link_d(Ud, spm, mu);
            b = load_stap_d(S, V, mu, k, spm.lexi);
          } else if (j == 1) {  // S(x) S(x - mu) U_mu(x - mu)
            a = load_stap_d(S, V, mu, k, s0.lexi);
            b = load_stap_d(S, V, mu, k, smm.lexi);
          } else {  // U_{s nu}(x + mu) S(x + s nu) U_{s nu}(x)^+
            a = signed_link_d(Ud, g, cpm, nu, s);
            b = load_stap_d(S, V, mu, k, at(g, cps).lexi);
          }
          ab = dmul(a, b);
        }
        M3d t;
        if (j == 0) t = load_stap_d(S, V, mu, k, s0.lexi);
        else if (j == 1) t = load_link_d(Ud, smm, mu);
        else t = dagger_d(signed_link_d(Ud, g, c, nu, s));
        add_lazy_m(Wr, dmul(ab, t));
      }
    }
#pragma unroll
    for (int e = 0; e < 9; e++) Wp.m[e] = czero<df>();
#pragma unroll 1
    for (int k = 0; k < 6; k++) add_lazy_m(Wp, load_stap_d(S, V, mu, k, s0.lexi));
    // A = c0 Wp + c1 Wr and W = U A in float-float as well (in FP64 this tail
    // kept the FP64 pipe 27 % busy); only the eight traces become doubles
    M3d A;
#pragma unroll
    for (int e = 0; e < 9; e++) {
      const Cx<df> wp = cnormalise(Wp.m[e]), wr = cnormalise(Wr.m[e]);
      A.m[e] = {cc.c0 * wp.re + cc.c1 * wr.re, cc.c0 * wp.im + cc.c1 * wr.im};
    }
    const M3d W = dmul(load_link_d(Ud, s0, mu), A);
    const Cx<df> *w = W.m;
    df tr[8];
    tr[0] = w[3].im + w[1].im;
    tr[1] = w[1].re - w[3].re;  // Im(i (w1 - w3)) = Re(w1 - w3)
    tr[2] = w[0].im - w[4].im;
    tr[3] = w[6].im + w[2].im;
    tr[4] = w[2].re - w[6].re;
    tr[5] = w[7].im + w[5].im;
    tr[6] = w[5].re - w[7].re;
    tr[7] = (w[0].im + w[4].im - (w[8].im + w[8].im)) * cc.r3;
    double *o = out + ((size_t)mu * V + s0.lexi) * 8;
#pragma unroll
    for (int a = 0; a < 8; a++) o[a] = cc.f * df_to_double(tr[a]);
  }
}

// sum over sites of sum_{mu != nu} Re Tr R_munu(x) (R: two links along mu,
// one along nu): per-block partials
__global__ void __launch_bounds__(128) rectangle_kernel(const double2 *U, Geom g, double *partials) {
  __shared__ double sh[8];
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int p, cb, c[4];
  double acc = 0.0;
  if (thread_site(g, tid, &p, &cb, c)) {
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        // U_mu(x) times the path +mu, +nu, -mu, -mu, -nu from x + mu
        const int d[5] = {mu, nu, mu, mu, nu}, sg[5] = {+1, +1, -1, -1, -1};
        int cpm[4] = {c[0], c[1], c[2], c[3]};
        coords_shift(g, cpm, mu, +1);
        M3 w = mmul(load_link(U, g, Pos{p, cb, 0}, mu), path5(U, g, cpm, d, sg));
        acc += re_trace(w);
      }
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// dS_g/domega^a for every link; out [mu][V][8] with lexicographic site index.
// Re Tr(i T^a W) = -Im Tr(lambda^a W) / 2 with the Gell-Mann traces written out.
// Wilson action (c1 = 0); the tlSym force is gauge_force_sym_kernel.
__global__ void __launch_bounds__(128) gauge_force_kernel(const double2 *U, Geom g, double beta, double *out) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  long V = 2L * g.Vh;
  Pos s = at(g, c);
  {
    M3 A = staple(U, g, c, mu);
    M3 W = mmul(load_link(U, g, s, mu), A);
    const C *w = W.m;
    double tr[8];
    tr[0] = (w[3] + w[1]).im;                       // Tr(l1 W) = W10 + W01
    tr[1] = (times_i(w[1] - w[3])).im;              // Tr(l2 W) = i (W01 - W10)
    tr[2] = (w[0] - w[4]).im;                       // Tr(l3 W) = W00 - W11
    tr[3] = (w[6] + w[2]).im;                       // Tr(l4 W) = W20 + W02
    tr[4] = (times_i(w[2] - w[6])).im;              // Tr(l5 W) = i (W02 - W20)
    tr[5] = (w[7] + w[5]).im;                       // Tr(l6 W) = W21 + W12
    tr[6] = (times_i(w[5] - w[7])).im;              // Tr(l7 W) = i (W12 - W21)
    tr[7] = (w[0] + w[4] - w[8] - w[8]).im * 0.57735026918962576451;  // Tr(l8 W)
    double *o = out + ((size_t)mu * V + s.lexi) * 8;
#pragma unroll
    for (int a = 0; a < 8; a++) o[a] = (beta / 3.0) * 0.5 * tr[a];  // -(b/3)(-Im/2)
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 and the uniform / Gaussian conversions
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};
LQCD_DEV U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}
// two uniforms in (0,1): 52-bit integers k -> (k + 1/2) 2^-52
LQCD_DEV void uniform2(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed, double u[2]) {
  U4 w = philox(U4{c0, c1, c2, c3}, (uint32_t)seed, (uint32_t)(seed >> 32));
  unsigned long long ka = ((unsigned long long)w.x << 20) | (w.y >> 12);
  unsigned long long kb = ((unsigned long long)w.z << 20) | (w.w >> 12);
  u[0] = ((double)ka + 0.5) * 0x1p-52;
  u[1] = ((double)kb + 0.5) * 0x1p-52;
}

enum { TAG_HB = 0, TAG_MOM = 1, TAG_ETA = 2, TAG_DIR = 3, TAG_METRO = 4 };

__global__ void philox_test_kernel(const uint32_t *in, uint32_t *out, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  U4 r = philox(U4{in[6 * k], in[6 * k + 1], in[6 * k + 2], in[6 * k + 3]}, in[6 * k + 4], in[6 * k + 5]);
  out[4 * k] = r.x;
  out[4 * k + 1] = r.y;
  out[4 * k + 2] = r.z;
  out[4 * k + 3] = r.w;
}

// ---------------------------------------------------------------------------
// heatbath: one (mu, parity) class per launch
// ---------------------------------------------------------------------------
#define HB_MAX_ATTEMPTS 1024
#define HB_B_SWITCH 1.5

// y0 ~ sqrt(1 - y0^2) exp(b y0): Creutz for b < 1.5, Kennedy-Pendleton above
LQCD_DEV bool sample_y0(double b, uint32_t c0, uint32_t c1, uint32_t c2, uint64_t seed, double *y0) {
  for (int n = 0; n < HB_MAX_ATTEMPTS; n++) {
    double u[2];
    uniform2(c0, c1, c2, (uint32_t)(2 * n), seed, u);
    if (b < HB_B_SWITCH) {
      // b -> 0 (beta = 0): the inversion's limit is y0 uniform on [-1, 1]
      double y = b > 1e-300 ? 1.0 + log1p(expm1(-2.0 * b) * (1.0 - u[0])) / b : 2.0 * u[0] - 1.0;
      if (u[1] * u[1] <= 1.0 - y * y) {
        *y0 = y;
        return true;
      }
      continue;
    }
    double v[2];
    uniform2(c0, c1, c2, (uint32_t)(2 * n + 1), seed, v);
    double cs = cos(2.0 * M_PI * u[1]);
    double lam2 = -(log(u[0]) + cs * cs * log(v[0])) / (2.0 * b);
    if (v[1] * v[1] <= 1.0 - lam2) {
      *y0 = 1.0 - 2.0 * lam2;
      return true;
    }
  }
  return false;
}

// FP64 links of the heatbath: the master (18 reals) or, for a field imported
// with recon = 12, its FP64 REC12 copy with the third row rebuilt on load
// (Sec. 4.1; Sec. 6 suggests REC12 for the heatbath kernels as well)
template <int RECON>
LQCD_DEV M3 hb_load(const GaugeView &Uv, const Pos &s, int mu) {
  M3 u;
  LinkIO<LQCD_F64, RECON>::load(Uv, s.p, mu, s.cb, u.m);
  if (RECON == 12) reconstruct_row2(u.m);
  return u;
}
template <int RECON>
LQCD_DEV void hb_store(const GaugeView &Uv, const Pos &s, int mu, const M3 &u) {
  double2 *b = (double2 *)((char *)Uv.ptr + s.p * Uv.parity_stride + mu * Uv.mu_stride);
#pragma unroll
  for (int k = 0; k < (RECON == 18 ? 9 : 6); k++) b[(size_t)k * Uv.Vh + s.cb] = make_double2(u.m[k].re, u.m[k].im);
}

// The Cabibbo-Marinari update of one link u with staple sum A: for each of
// the three SU(2) subgroups a Kennedy-Pendleton heatbath draw (or, with
// overrelax, the reflection v = (w_hat^+)^2) left-multiplied onto u.  Returns
// the number of subgroup updates skipped (degenerate staple or sampler
// failure).
LQCD_DEV unsigned hb_update_link(M3 &u, const M3 &A, double beta, const Pos &s, int mu, uint32_t sweep,
                                 uint64_t seed, int overrelax) {
  unsigned fails = 0;
  const int SG[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  // unrolled: the subgroup's rows i, j are then compile-time indices and u,
  // W stay in registers instead of local memory
#pragma unroll
  for (int sg = 0; sg < 3; sg++) {
    const int i = SG[sg][0], j = SG[sg][1];
    M3 W = mmul(u, A);
    C wa = W.m[3 * i + i], wb = W.m[3 * i + j], wc = W.m[3 * j + i], wd = W.m[3 * j + j];
    // quaternion part of the 2x2 block: [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
    double q0 = 0.5 * (wa.re + wd.re), q3 = 0.5 * (wa.im - wd.im);
    double q1 = 0.5 * (wb.im + wc.im), q2 = 0.5 * (wb.re - wc.re);
    double k = sqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    if (!(k > 1e-300)) {
      fails++;
      continue;
    }
    double h0 = q0 / k, h1 = q1 / k, h2 = q2 / k, h3 = q3 / k;
    // w_hat^+ = [[h0 - i h3, -h2 - i h1], [h2 - i h1, h0 + i h3]]
    C whd[2][2] = {{{h0, -h3}, {-h2, -h1}}, {{h2, -h1}, {h0, h3}}};
    C v[2][2];
    if (overrelax) {  // v = (w_hat^+)^2 keeps Re Tr(v w) fixed
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 2; q++) v[r][q] = whd[r][0] * whd[0][q] + whd[r][1] * whd[1][q];
    } else {
      double b = 2.0 * beta * k / 3.0;
      uint32_t c2 = (uint32_t)mu | ((uint32_t)sg << 2) | (TAG_HB << 8);
      double y0;
      if (!sample_y0(b, (uint32_t)s.lexi, sweep, c2, seed, &y0)) {
        fails++;
        continue;
      }
      double ud[2];
      uniform2((uint32_t)s.lexi, sweep, (uint32_t)mu | ((uint32_t)sg << 2) | (TAG_DIR << 8), 0u, seed, ud);
      double ct = 2.0 * ud[0] - 1.0, stt = sqrt(1.0 - ct * ct), ph = 2.0 * M_PI * ud[1];
      double rr = sqrt(fmax(1.0 - y0 * y0, 0.0));
      double y1 = rr * stt * cos(ph), y2 = rr * stt * sin(ph), y3 = rr * ct;
      C Y[2][2] = {{{y0, y3}, {y2, y1}}, {{-y2, y1}, {y0, -y3}}};
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 2; q++) v[r][q] = Y[r][0] * whd[0][q] + Y[r][1] * whd[1][q];
    }
    // U <- V U with V = v embedded at rows/cols (i, j)
    C ri[3], rj[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      ri[q] = v[0][0] * u.m[3 * i + q] + v[0][1] * u.m[3 * j + q];
      rj[q] = v[1][0] * u.m[3 * i + q] + v[1][1] * u.m[3 * j + q];
    }
#pragma unroll
    for (int q = 0; q < 3; q++) {
      u.m[3 * i + q] = ri[q];
      u.m[3 * j + q] = rj[q];
    }
  }
  return fails;
}

template <int RECON>
__global__ void __launch_bounds__(128) heatbath_kernel(GaugeView Uv, Geom g, int mu, int par, double beta,
                                                       uint64_t seed, uint32_t sweep, int overrelax,
                                                       unsigned int *fail_count) {
  int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  Site st = site_of(g, par, cb);
  int c[4] = {st.x, st.y, st.z, st.t};
  Pos s = at(g, c);
  M3 A = staple_with([&](const Pos &q, int nu) { return hb_load<RECON>(Uv, q, nu); }, g, c, mu);
  M3 u = hb_load<RECON>(Uv, s, mu);
  const unsigned fails = hb_update_link(u, A, beta, s, mu, sweep, seed, overrelax);
  hb_store<RECON>(Uv, s, mu, u);
  if (fails) atomicAdd(fail_count, fails);
}

// FP64 REC12 copy -> FP64 master, the third row rebuilt
__global__ void rec12_to_master_kernel(GaugeView Uv, double2 *m, int Vh) {
  const size_t nl = (size_t)2 * 4 * Vh;
  const size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int blk = (int)(l / Vh), cb = (int)(l % Vh);  // blk = parity * 4 + mu
  Cx<double> u[9];
  LinkIO<LQCD_F64, 12>::load(Uv, blk >> 2, blk & 3, cb, u);
  reconstruct_row2(u);
#pragma unroll
  for (int k = 0; k < 9; k++) m[((size_t)blk * 9 + k) * Vh + cb] = make_double2(u[k].re, u[k].im);
}

// ---------------------------------------------------------------------------
// The heatbath and overrelaxation in single precision (the paper's main
// heatbath measurements are FP32): the same update on the FP32 copy of the
// links (18 reals), with FP32 staples, SU(2) projection and sampling, and
// FP32 uniforms (24 bits) from the same Philox counters.  The caller writes the copy back into the FP64
// field and reunitarises it in FP64.
// ---------------------------------------------------------------------------
struct M3s {
  Cx<float> m[9];
};
LQCD_DEV M3s smul(const M3s &a, const M3s &b) {
  M3s r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      Cx<float> t = a.m[3 * i] * b.m[j];
      t = cmadd(a.m[3 * i + 1], b.m[3 + j], t);
      t = cmadd(a.m[3 * i + 2], b.m[6 + j], t);
      r.m[3 * i + j] = t;
    }
  return r;
}
LQCD_DEV M3s sdag(const M3s &u) {
  M3s d;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) d.m[3 * i + j] = conj(u.m[3 * j + i]);
  return d;
}
// FP32 links with 18 reals, or 12 (REC12, Sec. 4.1: the paper suggests it for
// the heatbath too) with the third row rebuilt on load and not stored
template <int RECON>
LQCD_DEV M3s load_link_s(const GaugeView &Uf, const Pos &s, int mu) {
  M3s u;
  LinkIO<LQCD_F32, RECON>::load(Uf, s.p, mu, s.cb, u.m);
  if (RECON == 12) reconstruct_row2(u.m);
  return u;
}
template <int RECON>
LQCD_DEV void store_link_s(const GaugeView &Uf, const Pos &s, int mu, const M3s &u) {
  char *base = (char *)Uf.ptr + s.p * Uf.parity_stride + mu * Uf.mu_stride;
  float4 *b = (float4 *)base;
#pragma unroll
  for (int k = 0; k < (RECON == 18 ? 4 : 3); k++)
    b[(size_t)k * Uf.Vh + s.cb] = make_float4(u.m[2 * k].re, u.m[2 * k].im, u.m[2 * k + 1].re, u.m[2 * k + 1].im);
  if (RECON == 18) ((float2 *)(base + (size_t)4 * Uf.Vh * 16))[s.cb] = make_float2(u.m[8].re, u.m[8].im);
}
// staple sum as staple(), in FP32
template <int RECON>
LQCD_DEV M3s staple_s(const GaugeView &Uf, const Geom &g, const int c[4], int mu) {
  M3s A;
#pragma unroll
  for (int k = 0; k < 9; k++) A.m[k] = czero<float>();
  int cpm[4] = {c[0], c[1], c[2], c[3]};
  coords_shift(g, cpm, mu, +1);
  for (int nu = 0; nu < 4; nu++) {
    if (nu == mu) continue;
    int cpn[4] = {c[0], c[1], c[2], c[3]}, cmn[4] = {c[0], c[1], c[2], c[3]};
    int cpmmn[4] = {cpm[0], cpm[1], cpm[2], cpm[3]};
    coords_shift(g, cpn, nu, +1);
    coords_shift(g, cmn, nu, -1);
    coords_shift(g, cpmmn, nu, -1);
    // upper: U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    M3s t = smul(smul(load_link_s<RECON>(Uf, at(g, cpm), nu), sdag(load_link_s<RECON>(Uf, at(g, cpn), mu))),
                 sdag(load_link_s<RECON>(Uf, at(g, c), nu)));
#pragma unroll
    for (int k = 0; k < 9; k++) A.m[k] = A.m[k] + t.m[k];
    // lower: U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
    t = smul(sdag(smul(load_link_s<RECON>(Uf, at(g, cmn), mu), load_link_s<RECON>(Uf, at(g, cpmmn), nu))),
             load_link_s<RECON>(Uf, at(g, cmn), nu));
#pragma unroll
    for (int k = 0; k < 9; k++) A.m[k] = A.m[k] + t.m[k];
  }
  return A;
}

// four uniforms in (0, 1) with 24 random bits each from one Philox block:
// (k + 1/2) 2^-24, k the top 24 bits of each word (no FP64 arithmetic)
LQCD_DEV void uniform4f(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed, float u[4]) {
  const U4 w = philox(U4{c0, c1, c2, c3}, (uint32_t)seed, (uint32_t)(seed >> 32));
  u[0] = __fmaf_rn((float)(w.x >> 8), 0x1p-24f, 0x1p-25f);
  u[1] = __fmaf_rn((float)(w.y >> 8), 0x1p-24f, 0x1p-25f);
  u[2] = __fmaf_rn((float)(w.z >> 8), 0x1p-24f, 0x1p-25f);
  u[3] = __fmaf_rn((float)(w.w >> 8), 0x1p-24f, 0x1p-25f);
}

// the exact SU(2) update in FP32: the same method as sample_y0, with the
// uniforms of one Philox block (counter word 3 = attempt) per attempt
LQCD_DEV bool sample_y0_f(float b, uint32_t c0, uint32_t c1, uint32_t c2, uint64_t seed, float *y0) {
  for (int n = 0; n < HB_MAX_ATTEMPTS; n++) {
    float r[4];
    uniform4f(c0, c1, c2, (uint32_t)n, seed, r);
    const float u0 = r[0], u1 = r[1];
    if (b < (float)HB_B_SWITCH) {
      float y = b > 1e-30f ? 1.0f + log1pf(expm1f(-2.0f * b) * (1.0f - u0)) / b : 2.0f * u0 - 1.0f;
      if (u1 * u1 <= 1.0f - y * y) {
        *y0 = y;
        return true;
      }
      continue;
    }
    const float cs = cospif(2.0f * u1);
    const float lam2 = -(logf(u0) + cs * cs * logf(r[2])) / (2.0f * b);
    if (r[3] * r[3] <= 1.0f - lam2) {
      *y0 = 1.0f - 2.0f * lam2;
      return true;
    }
  }
  return false;
}

template <int RECON>
__global__ void __launch_bounds__(128, 5) heatbath_f32_kernel(GaugeView Uf, Geom g, int mu, int par, float beta,
                                                           uint64_t seed, uint32_t sweep, int overrelax,
                                                           unsigned int *fail_count) {
  int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  Site st = site_of(g, par, cb);
  int c[4] = {st.x, st.y, st.z, st.t};
  Pos s = at(g, c);
  const M3s A = staple_s<RECON>(Uf, g, c, mu);
  M3s u = load_link_s<RECON>(Uf, s, mu);
  const int SG[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  unsigned fails = 0;
  // unrolled: compile-time rows i, j keep u and W in registers
#pragma unroll
  for (int sg = 0; sg < 3; sg++) {
    const int i = SG[sg][0], j = SG[sg][1];
    const M3s W = smul(u, A);
    const Cx<float> wa = W.m[3 * i + i], wb = W.m[3 * i + j], wc = W.m[3 * j + i], wd = W.m[3 * j + j];
    const float q0 = 0.5f * (wa.re + wd.re), q3 = 0.5f * (wa.im - wd.im);
    const float q1 = 0.5f * (wb.im + wc.im), q2 = 0.5f * (wb.re - wc.re);
    const float k = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    if (!(k > 1e-30f)) {
      fails++;
      continue;
    }
    const float ik = 1.0f / k;  // one division for the four components
    const float h0 = q0 * ik, h1 = q1 * ik, h2 = q2 * ik, h3 = q3 * ik;
    const Cx<float> whd[2][2] = {{{h0, -h3}, {-h2, -h1}}, {{h2, -h1}, {h0, h3}}};
    Cx<float> v[2][2];
    if (overrelax) {
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 2; q++) v[r][q] = whd[r][0] * whd[0][q] + whd[r][1] * whd[1][q];
    } else {
      const float b = 2.0f * beta * k / 3.0f;
      const uint32_t c2 = (uint32_t)mu | ((uint32_t)sg << 2) | (TAG_HB << 8);
      float y0;
      if (!sample_y0_f(b, (uint32_t)s.lexi, sweep, c2, seed, &y0)) {
        fails++;
        continue;
      }
      float ud[4];
      uniform4f((uint32_t)s.lexi, sweep, (uint32_t)mu | ((uint32_t)sg << 2) | (TAG_DIR << 8), 0u, seed, ud);
      const float ct = 2.0f * ud[0] - 1.0f, stt = sqrtf(fmaxf(1.0f - ct * ct, 0.0f));
      float sp, cp;
      sincospif(2.0f * ud[1], &sp, &cp);
      const float rr = sqrtf(fmaxf(1.0f - y0 * y0, 0.0f));
      const float y1 = rr * stt * cp, y2 = rr * stt * sp, y3 = rr * ct;
      const Cx<float> Y[2][2] = {{{y0, y3}, {y2, y1}}, {{-y2, y1}, {y0, -y3}}};
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 2; q++) v[r][q] = Y[r][0] * whd[0][q] + Y[r][1] * whd[1][q];
    }
    Cx<float> ri[3], rj[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      ri[q] = v[0][0] * u.m[3 * i + q] + v[0][1] * u.m[3 * j + q];
      rj[q] = v[1][0] * u.m[3 * i + q] + v[1][1] * u.m[3 * j + q];
    }
#pragma unroll
    for (int q = 0; q < 3; q++) {
      u.m[3 * i + q] = ri[q];
      u.m[3 * j + q] = rj[q];
    }
  }
  store_link_s<RECON>(Uf, s, mu, u);
  if (fails) atomicAdd(fail_count, fails);
}

// The end of an FP32 sweep in one pass per link: the FP32 link into the FP64
// field, reunitarised (Gram-Schmidt on the first two rows, the third rebuilt
// as the conjugate cross product), and the FP32 copy rewritten from the new
// FP64 link with the rounding of the master -> FP32 copy conversion, so that
// the copy stays current for the next sweep.  GB300's FP64 pipe runs at 1/64
// of the FP32 rate, and an FP64 Gram-Schmidt with its conversions (about 150
// FP64 operations per link) took 1.97 ms on 32^3 x 64, more than the eight
// heatbath launches of the sweep; here the Gram-Schmidt runs in float-float
// arithmetic on the FP32 pipe (the inputs are exact FP32 values, every
// product is error-free, sums carry about 2^-48 of their magnitude), the
// conversions between float and double are bit operations on the integer
// pipe, and one FP64 addition per real (hi + lo) forms each double.  A row
// norm is n = 1 + e with |e| of order 1e-7 (the links leave the heatbath
// unitary to FP32 rounding), so 1 / sqrt(n) = 1 - e/2 + 3e^2/8 + O(e^3) with
// e^3 below 1e-19; a row with |e| > 2^-20 takes the FP64 rsqrt instead.
// Unitarity of the written links: |U U^+ - 1| of order 1e-15.

// float -> double by its bits on the integer pipe: exact for normal floats,
// zeros, infinities and NaNs; a subnormal float (below 2^-126, never a link
// entry or the low word of one at this precision) becomes a signed zero
LQCD_DEV double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xFFu, sg = u & 0x80000000u;
  const unsigned ed = e == 0xFFu ? 0x7FFu : e + 896u;
  const unsigned hi = e == 0u ? sg : (sg | (ed << 20) | ((u >> 3) & 0xFFFFFu));
  const unsigned lo = e == 0u ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}
// double -> float rounded to nearest even by its bits on the integer pipe:
// the bits of __double2float_rn for results in the normal float range and
// for zeros; magnitudes below 2^-126 become signed zeros and above the float
// range infinities (neither is met by link entries)
LQCD_DEV float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu, sg = hi & 0x80000000u;
  unsigned f = ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1FFFFFFFu;
  if (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) f += 1u;  // a carry moves into the exponent
  f = e < 897u ? 0u : (e > 1150u ? 0x7F800000u : f);
  return __uint_as_float(f | sg);
}
LQCD_DEV double df_to_double_bits(df v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }

// the FP64 fallback of inv_sqrt_near1_df, kept out of line so that the
// common path carries no FP64 instructions
__device__ __noinline__ df inv_sqrt_df_slow(df n) { return df_from_double(rsqrt((double)n.hi + (double)n.lo)); }

// 1 / sqrt(n) for n = 1 + e, |e| small (see above)
LQCD_DEV df inv_sqrt_near1_df(df n) {
  const df e = n - df{1.0f, 0.0f};
  if (fabsf(e.hi) > 0x1p-20f) return inv_sqrt_df_slow(n);
  const df half = {-0.5f * e.hi, -0.5f * e.lo};
  return (df{1.0f, 0.0f} + half) + df{0.375f * e.hi * e.hi, 0.0f};
}
LQCD_DEV df row_norm2_df(const Cx<df> r[3]) { return dfdot3<true>(r[0], r[1], r[2], r[0], r[1], r[2]).re; }

template <int RECON>
__global__ void f32_to_master_unitary_kernel(GaugeView Uf, double2 *m, int Vh) {
  const size_t nl = (size_t)2 * 4 * Vh;
  const size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int blk = (int)(l / Vh), cb = (int)(l % Vh);  // blk = parity * 4 + mu
  Cx<float> f[9];
  LinkIO<LQCD_F32, RECON>::load(Uf, blk >> 2, blk & 3, cb, f);
  Cx<df> u[9];
#pragma unroll
  for (int k = 0; k < 6; k++) u[k] = {{f[k].re, 0.0f}, {f[k].im, 0.0f}};
  const df r0 = inv_sqrt_near1_df(row_norm2_df(u));
#pragma unroll
  for (int k = 0; k < 3; k++) u[k] = {u[k].re * r0, u[k].im * r0};
  const Cx<df> d = dfdot3<true>(u[0], u[1], u[2], u[3], u[4], u[5]);  // (row 0)^+ row 1
#pragma unroll
  for (int k = 0; k < 3; k++) u[3 + k] = u[3 + k] - d * u[k];
  const df r1 = inv_sqrt_near1_df(row_norm2_df(u + 3));
#pragma unroll
  for (int k = 0; k < 3; k++) u[3 + k] = {u[3 + k].re * r1, u[3 + k].im * r1};
  reconstruct_row2(u);
  double2 w[9];
#pragma unroll
  for (int k = 0; k < 9; k++) {
    w[k] = make_double2(df_to_double_bits(u[k].re), df_to_double_bits(u[k].im));
    m[((size_t)blk * 9 + k) * Vh + cb] = w[k];
  }
  // the FP32 copy as gauge_copy_kernel makes it from the master
  char *base = (char *)Uf.ptr + (blk >> 2) * Uf.parity_stride + (blk & 3) * Uf.mu_stride;
  float4 *b = (float4 *)base;
  constexpr int NW = RECON == 18 ? 4 : 3;
#pragma unroll
  for (int k = 0; k < NW; k++)
    b[(size_t)k * Vh + cb] = make_float4(d2f_bits(w[2 * k].x), d2f_bits(w[2 * k].y), d2f_bits(w[2 * k + 1].x),
                                         d2f_bits(w[2 * k + 1].y));
  if (RECON == 18) ((float2 *)(base + (size_t)4 * Vh * 16))[cb] = make_float2(d2f_bits(w[8].x), d2f_bits(w[8].y));
}

// The FP64-class heatbath with its staple sum in float-float: the twelve
// 3x3 products of the six staples (about half the FP64 work of a link update)
// run as error-free complex dot products on the FP32 pipe from the field's
// float-float copy, and the sum is handed to the FP64 update (the SU(2)
// samplers, the subgroup products and the link itself stay in IEEE FP64).
// The staple differs from the FP64 one by rounding of order 2^-46 relative;
// the link is written into the FP64 field and, as df_from_double would split
// it, into the float-float copy, which the next class of the sweep reads.
LQCD_DEV M3 staple_df(const GaugeView &Ud, const Geom &g, const int c[4], int mu) {
  M3d A;
#pragma unroll
  for (int e = 0; e < 9; e++) A.m[e] = czero<df>();
  int cpm[4] = {c[0], c[1], c[2], c[3]};
  coords_shift(g, cpm, mu, +1);
#pragma unroll 1
  for (int k = 0; k < 6; k++) {
    const int nu = (k >> 1) + ((k >> 1) >= mu ? 1 : 0), sg = (k & 1) ? -1 : 1;
    int cps[4] = {c[0], c[1], c[2], c[3]};
    coords_shift(g, cps, nu, sg);
    // U_{s nu}(x + mu) U_mu(x + s nu)^+ U_{s nu}(x)^+
    M3d t = dmul_nd(signed_link_d(Ud, g, cpm, nu, sg), load_link_d(Ud, at(g, cps), mu));
    t = dmul_nd(t, signed_link_d(Ud, g, c, nu, sg));
    add_lazy_m(A, t);
  }
  M3 r;
#pragma unroll
  for (int e = 0; e < 9; e++) r.m[e] = {df_to_double_bits(A.m[e].re), df_to_double_bits(A.m[e].im)};
  return r;
}
// df_from_double on the integer pipe: the high word rounded to nearest, the
// low word the rounded remainder (one FP64 subtraction)
LQCD_DEV float4 df_word_of(C z) {
  const float rh = d2f_bits(z.re), ih = d2f_bits(z.im);
  return make_float4(rh, ih, d2f_bits(z.re - f2d_bits(rh)), d2f_bits(z.im - f2d_bits(ih)));
}

__global__ void __launch_bounds__(128) heatbath_df_kernel(GaugeView Um, GaugeView Ud, Geom g, int mu, int par,
                                                          double beta, uint64_t seed, uint32_t sweep,
                                                          int overrelax, unsigned int *fail_count) {
  int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  Site st = site_of(g, par, cb);
  int c[4] = {st.x, st.y, st.z, st.t};
  Pos s = at(g, c);
  const M3 A = staple_df(Ud, g, c, mu);
  M3 u = hb_load<18>(Um, s, mu);
  const unsigned fails = hb_update_link(u, A, beta, s, mu, sweep, seed, overrelax);
  hb_store<18>(Um, s, mu, u);
  float4 *w = (float4 *)((char *)Ud.ptr + s.p * Ud.parity_stride + mu * Ud.mu_stride);
#pragma unroll
  for (int e = 0; e < 9; e++) w[(size_t)e * Ud.Vh + s.cb] = df_word_of(u.m[e]);
  if (fails) atomicAdd(fail_count, fails);
}

// ---------------------------------------------------------------------------
// momenta, Gaussian spinors, link update, reunitarisation
// ---------------------------------------------------------------------------

// P[mu][i][8], p^a ~ N(0,1): block k of (i, traj, mu | TAG_MOM<<8, k) -> (p_2k, p_2k+1)
__global__ void momenta_kernel(double *P, long V, uint64_t seed, uint32_t traj) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= 4 * V) return;
  int mu = (int)(t / V);
  long i = t - mu * V;
  double *o = P + t * 8;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    double u[2];
    uniform2((uint32_t)i, traj, (uint32_t)mu | (TAG_MOM << 8), (uint32_t)k, seed, u);
    double r = sqrt(-2.0 * log(u[0]));
    double sn, cs;
    sincos(2.0 * M_PI * u[1], &sn, &cs);
    o[2 * k] = r * cs;
    o[2 * k + 1] = r * sn;
  }
}

// eta on the sites of `parity` (0 even, 1 odd, 2 both), component k from block
// (i, traj, TAG_ETA<<8, k); written to an EO full F64 field (other sites zeroed)
__global__ void gaussian_spinor_kernel(double2 *eo, Geom g, int parity, uint64_t seed, uint32_t traj) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int p, cb, c[4];
  if (!thread_site(g, tid, &p, &cb, c)) return;
  Pos s = at(g, c);
  double2 *base = eo + (size_t)p * 12 * g.Vh;
  bool on = parity == 2 || parity == p;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 v = make_double2(0.0, 0.0);
    if (on) {
      double u[2];
      uniform2((uint32_t)s.lexi, traj, (uint32_t)(TAG_ETA << 8), (uint32_t)k, seed, u);
      double r = sqrt(-2.0 * log(u[0])) * 0.70710678118654752440;
      double sn, cs;
      sincos(2.0 * M_PI * u[1], &sn, &cs);
      v = make_double2(r * cs, r * sn);
    }
    base[(size_t)k * g.Vh + cb] = v;
  }
}

LQCD_DEV void reunitarize(M3 &u) {
  double n0 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; k++) n0 += norm2_d(u.m[k]);
  n0 = rsqrt(n0);
#pragma unroll
  for (int k = 0; k < 3; k++) u.m[k] = {u.m[k].re * n0, u.m[k].im * n0};
  C d = czero<double>();
#pragma unroll
  for (int k = 0; k < 3; k++) d = conj_madd(u.m[k], u.m[3 + k], d);
#pragma unroll
  for (int k = 0; k < 3; k++) u.m[3 + k] = u.m[3 + k] - d * u.m[k];
  double n1 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; k++) n1 += norm2_d(u.m[3 + k]);
  n1 = rsqrt(n1);
#pragma unroll
  for (int k = 0; k < 3; k++) u.m[3 + k] = {u.m[3 + k].re * n1, u.m[3 + k].im * n1};
  reconstruct_row2(u.m);
}

// exp(i h) for a traceless Hermitian 3x3 h (the molecular-dynamics step
// h = eps sum_a p^a lambda^a / 2).  h is scaled by 2^-s until its Frobenius
// norm r is at most 1/2 (the result is squared s times).  By Cayley-Hamilton
// h^3 = c1 h + c0 with c1 = tr(h^2)/2 and c0 = det h, so every power is
// h^k = p_k + q_k h + r_k h^2 with the scalar recurrence
//   (p, q, r)_{k+1} = (c0 r_k, p_k + c1 r_k, q_k),
// and exp(i h) = a0 + a1 h + a2 h^2 with a_j = sum_k i^k / k! (p, q, r)_k.
// The series is summed up to the smallest degree whose first omitted term
// r^(n+1)/(n+1)! is below 2^-60 (the remainder is below twice that): one
// 3x3 product (h^2) instead of one per Taylor degree.
LQCD_DEV M3 expi_herm(const M3 &h0) {
  double nrm = 0.0;
#pragma unroll
  for (int k = 0; k < 9; k++) nrm += norm2_d(h0.m[k]);
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.5 && s < 60) {
    nrm *= 0.5;
    s++;
  }
  int deg = 1;
  for (double t = nrm * nrm * 0.5; deg < 30 && t >= 0x1p-60; t *= nrm / (deg + 1)) deg++;
  const double sc = ldexp(1.0, -s);
  M3 h;
#pragma unroll
  for (int k = 0; k < 9; k++) h.m[k] = {h0.m[k].re * sc, h0.m[k].im * sc};
  const M3 h2 = mmul(h, h);
  const double c1 = 0.5 * (h2.m[0].re + h2.m[4].re + h2.m[8].re);
  const C dt = h.m[0] * (h.m[4] * h.m[8] - h.m[5] * h.m[7]) - h.m[1] * (h.m[3] * h.m[8] - h.m[5] * h.m[6]) +
               h.m[2] * (h.m[3] * h.m[7] - h.m[4] * h.m[6]);
  const double c0 = dt.re;  // det of a Hermitian matrix is real
  // k = 0: h^0 = 1; the terms i^k / k! alternate between the real part
  // (k even, sign (-1)^(k/2)) and the imaginary part (k odd)
  double p = 1.0, q = 0.0, r = 0.0, w = 1.0;
  double a0r = 1.0, a0i = 0.0, a1r = 0.0, a1i = 0.0, a2r = 0.0, a2i = 0.0;
  for (int k = 1; k <= deg; k++) {
    const double pn = c0 * r, qn = fma(c1, r, p), rn = q;
    p = pn;
    q = qn;
    r = rn;
    w /= k;
    const double f = (k & 2) ? -w : w;  // i^k = f-sign times 1 (k even) or i (k odd)
    if (k & 1) {
      a0i = fma(f, p, a0i);
      a1i = fma(f, q, a1i);
      a2i = fma(f, r, a2i);
    } else {
      a0r = fma(f, p, a0r);
      a1r = fma(f, q, a1r);
      a2r = fma(f, r, a2r);
    }
  }
  const C a1 = {a1r, a1i}, a2 = {a2r, a2i};
  M3 E;
#pragma unroll
  for (int k = 0; k < 9; k++) E.m[k] = a1 * h.m[k] + a2 * h2.m[k];
  E.m[0] = E.m[0] + C{a0r, a0i};
  E.m[4] = E.m[4] + C{a0r, a0i};
  E.m[8] = E.m[8] + C{a0r, a0i};
  for (int t = 0; t < s; t++) E = mmul(E, E);
  return E;
}

// eps sum_a p^a lambda^a / 2 (Hermitian, traceless)
LQCD_DEV M3 algebra_herm(const double *p, double eps) {
  const double e = 0.5 * eps, r3 = 0.57735026918962576451;
  M3 H;
  H.m[0] = {e * (p[2] + p[7] * r3), 0.0};
  H.m[4] = {e * (-p[2] + p[7] * r3), 0.0};
  H.m[8] = {e * (-2.0 * p[7] * r3), 0.0};
  H.m[1] = {e * p[0], -e * p[1]};
  H.m[3] = {e * p[0], e * p[1]};
  H.m[2] = {e * p[3], -e * p[4]};
  H.m[6] = {e * p[3], e * p[4]};
  H.m[5] = {e * p[5], -e * p[6]};
  H.m[7] = {e * p[5], e * p[6]};
  return H;
}

__global__ void __launch_bounds__(128) gauge_update_kernel(double2 *U, Geom g, const double *P, double eps) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  long V = 2L * g.Vh;
  Pos s = at(g, c);
  {
    M3 E = expi_herm(algebra_herm(P + ((size_t)mu * V + s.lexi) * 8, eps));
    M3 u = mmul(E, load_link(U, g, s, mu));
    reunitarize(u);
    store_link(U, g, s, mu, u);
  }
}

// ---------------------------------------------------------------------------
// The same link update in float-float arithmetic on the FP32 pipe (GB300's
// FP64 pipe runs at 1/64 of the FP32 rate, and the FP64 update above costs
// ~450 FP64 operations per link): the algebra element, the Cayley-Hamilton
// exponential (same recurrence and scaling as expi_herm, the series summed
// until its first omitted term is below 2^-52), the product E U and the
// reunitarisation are double-word (value hi + lo, ~2^-46 relative); P and U
// are read from, and U written back to, the FP64 field, whose values hold
// every double-word exactly.  Only those conversions use the FP64 pipe.
// ---------------------------------------------------------------------------
LQCD_DEV df df_of_d(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(__dsub_rn(x, (double)hi))};
}
LQCD_DEV double d_of_df(df v) { return __dadd_rn((double)v.hi, (double)v.lo); }
LQCD_DEV Cx<df> cxd(double re, double im) { return {df_of_d(re), df_of_d(im)}; }
LQCD_DEV Cx<df> cscale(Cx<df> a, df f) { return {a.re * f, a.im * f}; }
LQCD_DEV df dsq(Cx<df> a) { return a.re * a.re + a.im * a.im; }

// row *= 1/sqrt(|row|^2): a float rsqrt of the high part refined by one
// Newton step in double-word arithmetic (relative error ~2^-46)
LQCD_DEV void normalise_row(Cx<df> *r) {
  const df n = dsq(r[0]) + dsq(r[1]) + dsq(r[2]);
  const float y0 = rsqrtf(n.hi);
  const df y = {y0, 0.0f};
  // y1 = y (3 - n y^2) / 2
  const df f = y * (df{1.5f, 0.0f} - (df{0.5f, 0.0f} * n) * (y * y));
#pragma unroll
  for (int k = 0; k < 3; k++) r[k] = cscale(r[k], f);
}

// exp(i h) for traceless Hermitian h in double-words (see expi_herm)
LQCD_DEV M3d expi_herm_df(const M3d &h0) {
  float nrm = 0.0f;
#pragma unroll
  for (int k = 0; k < 9; k++) nrm = fmaf(h0.m[k].re.hi, h0.m[k].re.hi, fmaf(h0.m[k].im.hi, h0.m[k].im.hi, nrm));
  nrm = sqrtf(nrm);
  int s = 0;
  while (nrm > 0.5f && s < 60) {
    nrm *= 0.5f;
    s++;
  }
  int deg = 1;
  for (float t = nrm * nrm * 0.5f; deg < 30 && t >= 0x1p-52f; t *= nrm / (deg + 1)) deg++;
  const float sc = ldexpf(1.0f, -s);  // exact power of two
  M3d h;
#pragma unroll
  for (int k = 0; k < 9; k++) h.m[k] = {{h0.m[k].re.hi * sc, h0.m[k].re.lo * sc}, {h0.m[k].im.hi * sc, h0.m[k].im.lo * sc}};
  const M3d h2 = dmul(h, h);
  const df c1 = df{0.5f, 0.0f} * (h2.m[0].re + h2.m[4].re + h2.m[8].re);
  const Cx<df> dt = h.m[0] * (h.m[4] * h.m[8] - h.m[5] * h.m[7]) - h.m[1] * (h.m[3] * h.m[8] - h.m[5] * h.m[6]) +
                    h.m[2] * (h.m[3] * h.m[7] - h.m[4] * h.m[6]);
  const df c0 = dt.re;
  df p = {1.0f, 0.0f}, q = {0.0f, 0.0f}, r = {0.0f, 0.0f}, w = {1.0f, 0.0f};
  df a0r = {1.0f, 0.0f}, a0i = {0.0f, 0.0f}, a1r = {0.0f, 0.0f}, a1i = {0.0f, 0.0f}, a2r = {0.0f, 0.0f},
     a2i = {0.0f, 0.0f};
  for (int k = 1; k <= deg; k++) {
    const df pn = c0 * r, qn = c1 * r + p, rn = q;
    p = pn;
    q = qn;
    r = rn;
    // w = 1/k! as a double-word: w /= k by one float-division estimate and a correction
    const float kf = (float)k;
    const float qh = w.hi / kf;
    const df rem = w - df{qh, 0.0f} * df{kf, 0.0f};
    w = fast_two_sum(qh, (rem.hi + rem.lo) / kf);
    const df f = (k & 2) ? -w : w;
    if (k & 1) {
      a0i = f * p + a0i;
      a1i = f * q + a1i;
      a2i = f * r + a2i;
    } else {
      a0r = f * p + a0r;
      a1r = f * q + a1r;
      a2r = f * r + a2r;
    }
  }
  const Cx<df> a0 = {a0r, a0i}, a1 = {a1r, a1i}, a2 = {a2r, a2i};
  M3d E;
#pragma unroll
  for (int k = 0; k < 9; k++) E.m[k] = a1 * h.m[k] + a2 * h2.m[k];
  E.m[0] = E.m[0] + a0;
  E.m[4] = E.m[4] + a0;
  E.m[8] = E.m[8] + a0;
  for (int t = 0; t < s; t++) E = dmul(E, E);
  return E;
}

// U is read from the field's float-float copy (no FP64 conversions) and the
// result is written to both the FP64 master and that copy, which therefore
// stays current (each FP64 <-> FP32 conversion and FP64 add runs on the FP64
// pipe: read from the master and with the copy rebuilt afterwards they kept
// it 69 % busy)
__global__ void __launch_bounds__(128) gauge_update_df_kernel(double2 *U, GaugeView Ud, Geom g, const double *P,
                                                              double eps) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int mu, p, cb, c[4];
  if (!thread_link(g, tid, &mu, &p, &cb, c)) return;
  const long V = 2L * g.Vh;
  const Pos s = at(g, c);
  const double *pp = P + ((size_t)mu * V + s.lexi) * 8;
  df pa[8];
#pragma unroll
  for (int a = 0; a < 8; a++) pa[a] = df_of_d(pp[a]);
  // eps sum_a p^a lambda^a / 2, as algebra_herm
  const df e = df_of_d(0.5 * eps), r3 = df_of_d(0.57735026918962576451);
  const df z = {0.0f, 0.0f};
  const df d8 = pa[7] * r3;
  M3d H;
  H.m[0] = {e * (pa[2] + d8), z};
  H.m[4] = {e * (d8 - pa[2]), z};
  H.m[8] = {-(e * (d8 + d8)), z};
  H.m[1] = {e * pa[0], -(e * pa[1])};
  H.m[3] = {e * pa[0], e * pa[1]};
  H.m[2] = {e * pa[3], -(e * pa[4])};
  H.m[6] = {e * pa[3], e * pa[4]};
  H.m[5] = {e * pa[5], -(e * pa[6])};
  H.m[7] = {e * pa[5], e * pa[6]};
  const M3d E = expi_herm_df(H);
  M3d v = dmul(E, load_link_d(Ud, s, mu));
  // reunitarise: row 0 normalised, row 1 orthogonalised and normalised,
  // row 2 = conj(row0 x row1) (REC12, Sec. 4.1)
  normalise_row(v.m);
  Cx<df> d = {z, z};
#pragma unroll
  for (int k = 0; k < 3; k++) d = d + conj(v.m[k]) * v.m[3 + k];
#pragma unroll
  for (int k = 0; k < 3; k++) v.m[3 + k] = v.m[3 + k] - d * v.m[k];
  normalise_row(v.m + 3);
  reconstruct_row2(v.m);
  M3 u64;
#pragma unroll
  for (int k = 0; k < 9; k++) u64.m[k] = {d_of_df(v.m[k].re), d_of_df(v.m[k].im)};
  store_link(U, g, s, mu, u64);
  float4 *w = (float4 *)((char *)Ud.ptr + s.p * Ud.parity_stride + mu * Ud.mu_stride);
#pragma unroll
  for (int k = 0; k < 9; k++) w[(size_t)k * Ud.Vh + s.cb] = f4_of(v.m[k]);
}

__global__ void momenta_update_kernel(double *P, const double *F, double eps, size_t n) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) P[k] = fma(-eps, F[k], P[k]);
}

__global__ void __launch_bounds__(128) sumsq_kernel(const double *P, size_t n, double *partials) {
  __shared__ double sh[8];
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  double v = k < n ? P[k] * P[k] : 0.0;
  double t = block_sum(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static unsigned nblk(long n, int b = 128) { return (unsigned)((n + b - 1) / b); }

// sum of nb partials on the host (fixed order), synchronous
static lqcd_status sum_partials(lqcd_ctx *ctx, int nb, double *out) {
  LQCD_TRY(ensure_pinned(ctx, nb));
  LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, ctx->partials, nb * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double s = 0.0;
  for (int k = 0; k < nb; k++) s += ctx->pinned[k];
  *out = s;
  return LQCD_OK;
}

lqcd_status plaquette_sum(lqcd_ctx *ctx, const lqcd_gauge *U, double *sum_retr) {
  long V = 2L * U->g.Vh;
  unsigned nb = nblk(V);
  LQCD_TRY(ensure_partials(ctx, nb));
  plaquette_kernel<<<nb, 128, 0, ctx->stream>>>((const double2 *)U->master, U->g, ctx->partials);
  LQCD_CUDA(ctx, cudaGetLastError());
  return sum_partials(ctx, nb, sum_retr);
}

lqcd_status rectangle_sum(lqcd_ctx *ctx, const lqcd_gauge *U, double *sum_retr) {
  long V = 2L * U->g.Vh;
  int nb = (int)nblk(V);
  LQCD_TRY(ensure_partials(ctx, nb));
  rectangle_kernel<<<nb, 128, 0, ctx->stream>>>((const double2 *)U->master, U->g, ctx->partials);
  LQCD_CUDA(ctx, cudaGetLastError());
  return sum_partials(ctx, nb, sum_retr);
}

// dS_g/dw into dSdw; prec LQCD_F64 (IEEE FP64 throughout) or LQCD_DF64
// (staples and products in float-float from the DF64 copy of the links)
lqcd_status gauge_force_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, double c1, int prec, double *dSdw) {
  long V = 2L * U->g.Vh;
  if (c1 != 0.0 || prec == LQCD_DF64) {
    // plaquette staples of every link (6 x 144 B per link), then the force
    const size_t need = (size_t)4 * 6 * 9 * V * sizeof(double2);
    if (ctx->staple_cap < need) {
      dfree(ctx, ctx->staples);
      ctx->staples = nullptr;
      ctx->staple_cap = 0;
      LQCD_TRY(dalloc(ctx, &ctx->staples, need));
      ctx->staple_cap = need;
    }
    if (prec == LQCD_DF64) {
      GaugeView Ud;
      LQCD_TRY(gauge_view(ctx, U, LQCD_DF64, 18, &Ud));
      staple6_df_kernel<<<nblk(4 * V), 128, 0, ctx->stream>>>(Ud, U->g, (float4 *)ctx->staples);
      ForceConst cc;
      cc.c0 = df_from_double(1.0 - 8.0 * c1);
      cc.c1 = df_from_double(c1);
      cc.r3 = df_from_double(0.57735026918962576451);
      cc.f = beta / 6.0;
      gauge_force_df_kernel<<<nblk(4 * V), 128, 0, ctx->stream>>>(Ud, (const float4 *)ctx->staples, U->g, cc, c1,
                                                              dSdw);
      LQCD_CUDA(ctx, cudaGetLastError());
      return LQCD_OK;
    }
    staple6_kernel<<<nblk(4 * V), 128, 0, ctx->stream>>>((const double2 *)U->master, U->g,
                                                     (double2 *)ctx->staples);
    gauge_force_sym_kernel<<<nblk(4 * V), 128, 0, ctx->stream>>>((const double2 *)U->master,
                                                             (const double2 *)ctx->staples, U->g, beta, c1,
                                                             dSdw);
    LQCD_CUDA(ctx, cudaGetLastError());
    return LQCD_OK;
  }
  gauge_force_kernel<<<nblk(4 * V), 128, 0, ctx->stream>>>((const double2 *)U->master, U->g, beta, dSdw);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

// FP32 sweep: on the FP32 copy, then back into the FP64 field, reunitarised.
// Passes: one heatbath pass if hb, then n_or overrelaxation passes.
lqcd_status heatbath_f32_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep, int hb,
                             int n_or, unsigned int *fail_dev) {
  // the link format follows the field's (18 reals, or REC12 if imported so)
  const bool r12 = U->recon == 12;
  GaugeView Uf;
  LQCD_TRY(gauge_view(ctx, U, LQCD_F32, r12 ? 12 : 18, &Uf));
  for (int pass = hb ? 0 : 1; pass <= n_or; pass++)
    for (int mu = 0; mu < 4; mu++)
      for (int par = 0; par < 2; par++) {
        if (r12)
          heatbath_f32_kernel<12><<<nblk(U->g.Vh), 128, 0, ctx->stream>>>(
              Uf, U->g, mu, par, (float)beta, seed, (uint32_t)sweep, pass > 0 ? 1 : 0, fail_dev);
        else
          heatbath_f32_kernel<18><<<nblk(U->g.Vh), 128, 0, ctx->stream>>>(
              Uf, U->g, mu, par, (float)beta, seed, (uint32_t)sweep, pass > 0 ? 1 : 0, fail_dev);
        LQCD_CUDA(ctx, cudaGetLastError());
      }
  if (r12)
    f32_to_master_unitary_kernel<12><<<nblk(8L * U->g.Vh), 128, 0, ctx->stream>>>(Uf, (double2 *)U->master,
                                                                                    U->g.Vh);
  else
    f32_to_master_unitary_kernel<18><<<nblk(8L * U->g.Vh), 128, 0, ctx->stream>>>(Uf, (double2 *)U->master,
                                                                                    U->g.Vh);
  LQCD_CUDA(ctx, cudaGetLastError());
  U->version++;
  // the FP32 copy was rewritten from the new master: still current
  for (auto &k : U->copies)
    if (k.prec == LQCD_F32 && k.recon == (r12 ? 12 : 18)) k.version = U->version;
  return LQCD_OK;
}

// FP64-class sweep with float-float staples (heatbath_df_kernel) on the
// master and the float-float copy, which stays current.  Passes as
// heatbath_f32_raw.
lqcd_status heatbath_df_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep, int hb,
                            int n_or, unsigned int *fail_dev) {
  GaugeView Um, Ud;
  LQCD_TRY(gauge_view(ctx, U, LQCD_F64, 18, &Um));
  LQCD_TRY(gauge_view(ctx, U, LQCD_DF64, 18, &Ud));
  for (int pass = hb ? 0 : 1; pass <= n_or; pass++)
    for (int mu = 0; mu < 4; mu++)
      for (int par = 0; par < 2; par++) {
        heatbath_df_kernel<<<nblk(U->g.Vh), 128, 0, ctx->stream>>>(Um, Ud, U->g, mu, par, beta, seed,
                                                                  (uint32_t)sweep, pass > 0 ? 1 : 0, fail_dev);
        LQCD_CUDA(ctx, cudaGetLastError());
      }
  U->version++;
  for (auto &k : U->copies)
    if (k.prec == LQCD_DF64 && k.recon == 18) k.version = U->version;
  return LQCD_OK;
}

// FP64 sweep in place: on the master (18 reals), or for a field imported with
// recon = 12 on its FP64 REC12 copy, whose first two rows are then written
// back into the master with the third rebuilt.  Passes as heatbath_f32_raw.
lqcd_status heatbath_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep, int hb,
                         int n_or, unsigned int *fail_dev) {
  const bool r12 = U->recon == 12;
  GaugeView Uv;
  LQCD_TRY(gauge_view(ctx, U, LQCD_F64, r12 ? 12 : 18, &Uv));
  for (int pass = hb ? 0 : 1; pass <= n_or; pass++)
    for (int mu = 0; mu < 4; mu++)
      for (int par = 0; par < 2; par++) {
        if (r12)
          heatbath_kernel<12><<<nblk(U->g.Vh), 128, 0, ctx->stream>>>(Uv, U->g, mu, par, beta, seed,
                                                                      (uint32_t)sweep, pass > 0 ? 1 : 0, fail_dev);
        else
          heatbath_kernel<18><<<nblk(U->g.Vh), 128, 0, ctx->stream>>>(Uv, U->g, mu, par, beta, seed,
                                                                      (uint32_t)sweep, pass > 0 ? 1 : 0, fail_dev);
        LQCD_CUDA(ctx, cudaGetLastError());
      }
  if (r12) {
    rec12_to_master_kernel<<<nblk(8L * U->g.Vh), 128, 0, ctx->stream>>>(Uv, (double2 *)U->master, U->g.Vh);
    LQCD_CUDA(ctx, cudaGetLastError());
  }
  U->version++;
  if (r12)  // the REC12 copy holds the master's first two rows: still current
    for (auto &k : U->copies)
      if (k.prec == LQCD_F64 && k.recon == 12) k.version = U->version;
  return LQCD_OK;
}

lqcd_status momenta_raw(lqcd_ctx *ctx, long V, double *P, uint64_t seed, uint32_t traj) {
  momenta_kernel<<<nblk(4 * V), 128, 0, ctx->stream>>>(P, V, seed, traj);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status gaussian_spinor_raw(lqcd_ctx *ctx, const Geom &g, void *eo_full, int parity, uint64_t seed,
                                uint32_t traj) {
  gaussian_spinor_kernel<<<nblk(2L * g.Vh), 128, 0, ctx->stream>>>((double2 *)eo_full, g, parity, seed, traj);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status gauge_update_raw(lqcd_ctx *ctx, lqcd_gauge *U, const double *P, double eps, int prec) {
  if (prec == LQCD_DF64) {
    GaugeView Ud;
    LQCD_TRY(gauge_view(ctx, U, LQCD_DF64, 18, &Ud));
    gauge_update_df_kernel<<<nblk(8L * U->g.Vh), 128, 0, ctx->stream>>>((double2 *)U->master, Ud, U->g, P, eps);
    LQCD_CUDA(ctx, cudaGetLastError());
    U->version++;
    for (auto &k : U->copies)  // written alongside the master: still current
      if (k.prec == LQCD_DF64 && k.recon == 18) k.version = U->version;
    return LQCD_OK;
  }
  gauge_update_kernel<<<nblk(8L * U->g.Vh), 128, 0, ctx->stream>>>((double2 *)U->master, U->g, P, eps);
  LQCD_CUDA(ctx, cudaGetLastError());
  U->version++;
  return LQCD_OK;
}

lqcd_status momenta_update_raw(lqcd_ctx *ctx, long V, double *P, const double *F, double eps) {
  size_t n = (size_t)32 * V;
  momenta_update_kernel<<<nblk((long)n, 256), 256, 0, ctx->stream>>>(P, F, eps, n);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status sumsq_raw(lqcd_ctx *ctx, const double *P, size_t n, double *out) {
  unsigned nb = nblk((long)n);
  LQCD_TRY(ensure_partials(ctx, nb));
  sumsq_kernel<<<nb, 128, 0, ctx->stream>>>(P, n, ctx->partials);
  LQCD_CUDA(ctx, cudaGetLastError());
  return sum_partials(ctx, nb, out);
}

lqcd_status philox_test_raw(lqcd_ctx *ctx, const uint32_t *in_dev, uint32_t *out_dev, int n) {
  philox_test_kernel<<<nblk(n), 128, 0, ctx->stream>>>(in_dev, out_dev, n);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

// Metropolis uniform for trajectory traj: block (0, traj, TAG_METRO << 8, 0)
__global__ void metro_uniform_kernel(uint64_t seed, uint32_t traj, double *out) {
  double u[2];
  uniform2(0u, traj, (uint32_t)(TAG_METRO << 8), 0u, seed, u);
  *out = u[0];
}
lqcd_status metro_uniform(lqcd_ctx *ctx, uint64_t seed, uint32_t traj, double *u) {
  metro_uniform_kernel<<<1, 1, 0, ctx->stream>>>(seed, traj, ctx->partials);
  LQCD_CUDA(ctx, cudaGetLastError());
  return sum_partials(ctx, 1, u);
}

}  // namespace lqcd
