// hmc.cu -- ABI entry points for the molecular-dynamics side of Sec. 2.2:
// gauge force and action, plaquette, heatbath, momenta, link update, the
// fermion force (through (Mhat^+ Mhat)^-1 solved by the even-odd CG) and one
// complete HMC trajectory:
//   H = 1/2 sum p^2 + S_g + phi^+ (Mhat^+ Mhat)^-1 phi,  phi = Mhat^+ eta,
//   leapfrog: p <- p - eps/2 dS/dw; (U <- exp(i eps P) U; p <- p - eps dS/dw) ...
//   accept with probability min(1, exp(-dH)) (the printed exponent's sign is
//   read as exp(-(H' - H))).
// H, dH and every action are accumulated in FP64 on the device.
#include <chrono>
#include <functional>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

lqcd_status check_geom(lqcd_ctx *ctx, const lqcd_geom *g);
lqcd_status check_field(lqcd_ctx *ctx, const lqcd_field &f, const char *name, bool allow_lexi);
lqcd_status plaquette_sum(lqcd_ctx *ctx, const lqcd_gauge *U, double *sum_retr);
lqcd_status gauge_force_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, double c1, int prec, double *dSdw);
lqcd_status rectangle_sum(lqcd_ctx *ctx, const lqcd_gauge *U, double *sum_retr);
lqcd_status heatbath_f32_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep, int hb, int n_or,
                             unsigned int *fail_dev);
lqcd_status heatbath_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep, int hb, int n_or,
                         unsigned int *fail_dev);
lqcd_status heatbath_df_raw(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep, int hb, int n_or,
                         unsigned int *fail_dev);
lqcd_status momenta_raw(lqcd_ctx *ctx, long V, double *P, uint64_t seed, uint32_t traj);
lqcd_status gaussian_spinor_raw(lqcd_ctx *ctx, const Geom &g, void *eo_full, int parity, uint64_t seed,
                                uint32_t traj);
lqcd_status gauge_update_raw(lqcd_ctx *ctx, lqcd_gauge *U, const double *P, double eps, int prec);
lqcd_status momenta_update_raw(lqcd_ctx *ctx, long V, double *P, const double *F, double eps);
lqcd_status sumsq_raw(lqcd_ctx *ctx, const double *P, size_t n, double *out);
lqcd_status metro_uniform(lqcd_ctx *ctx, uint64_t seed, uint32_t traj, double *u);
lqcd_status fermion_force_raw(lqcd_ctx *ctx, const lqcd_gauge *U, const GaugeView &Uv, int recon, const void *Lf,
                              const void *Rf, double kappa, double *out);
lqcd_status cgls_even(lqcd_ctx *ctx, lqcd_gauge *U, const Geom &g, double kappa, double mu,
                      const lqcd_cg_params &prm, const HalfField &bhat, const HalfField &xo,
                      const std::vector<double> &b2, lqcd_cg_stats *st, int nrhs, int *iters_used,
                      bool normal);

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static HalfField f64_half(void *ptr, int Vh) {
  HalfField h;
  h.ptr = ptr;
  h.prec = LQCD_F64;
  h.nrhs = 1;
  h.rhs_stride = spinor_half_bytes(LQCD_F64, Vh);
  return h;
}

// |f|^2 of one F64 half field (synchronous)
static lqcd_status half_norm2(lqcd_ctx *ctx, int Vh, const HalfField &f, double *out) {
  DBuf tmp(ctx);
  LQCD_TRY(tmp.alloc(f.rhs_stride));
  HalfField t = f;
  t.ptr = tmp.p;
  int nb = 0;
  LQCD_TRY(lincomb(ctx, Vh, t, f, nullptr, {1, 0}, {1, 0}, {0, 0}, {0, 0}, ctx->partials, &nb));
  LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, ctx->partials, nb * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double s = 0.0;
  for (int k = 0; k < nb; k++) s += ctx->pinned[k];
  *out = s;
  return LQCD_OK;
}

// Re <a, b> of two F64 half fields (synchronous): via |a+b|^2 - |a-b|^2 = 4 Re<a,b>
static lqcd_status half_redot(lqcd_ctx *ctx, int Vh, const HalfField &a, const HalfField &b, double *out) {
  DBuf tmp(ctx);
  LQCD_TRY(tmp.alloc(a.rhs_stride));
  HalfField t = a;
  t.ptr = tmp.p;
  double np, nm;
  LQCD_TRY(lincomb(ctx, Vh, t, a, &b, {1, 0}, {1, 0}, {1, 0}, {1, 0}, nullptr, nullptr));
  LQCD_TRY(half_norm2(ctx, Vh, t, &np));
  LQCD_TRY(lincomb(ctx, Vh, t, a, &b, {1, 0}, {1, 0}, {-1, 0}, {-1, 0}, nullptr, nullptr));
  LQCD_TRY(half_norm2(ctx, Vh, t, &nm));
  *out = 0.25 * (np - nm);
  return LQCD_OK;
}

// X_e = (Mhat^+ Mhat)^-1 phi_e (F64 half fields); solver statistics added to st.
// guess: X holds a starting vector X0 (the HMC passes the solution of the
// previous force evaluation of the same pseudofermion, a chronological
// guess); the solve then runs on A d = phi - A X0 (A = Mhat^+ Mhat, residual
// formed in the outer format) with the stopping test still relative to
// |phi|, and returns X = X0 + d.
lqcd_status solve_normal(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField &phi, const HalfField &X, double kappa,
                         double mu, const lqcd_cg_params &prm_in, lqcd_cg_stats *st, bool guess) {
  const Geom &g = U->g;
  const int Vh = g.Vh;
  lqcd_cg_params prm = prm_in;
  if (prm.sloppy_recon == 0) prm.sloppy_recon = U->recon;
  if (prm.check_every <= 0) prm.check_every = 10;
  double phi2;
  LQCD_TRY(half_norm2(ctx, Vh, phi, &phi2));
  if (!std::isfinite(phi2)) return fail(ctx, LQCD_ERR_NONFINITE, "pseudofermion field is not finite");
  std::vector<double> b2(1, phi2);
  const int outer = prm.outer_prec;
  const size_t hb = spinor_half_bytes(outer, Vh);
  DBuf phio(ctx), xo(ctx), t1(ctx), t2(ctx);
  HalfField ph = phi, xx = X;
  auto outer_half = [&](DBuf &b) -> HalfField {
    HalfField h = phi;
    h.ptr = b.p;
    h.prec = outer;
    h.rhs_stride = hb;
    return h;
  };
  if (outer != LQCD_F64 || guess) {
    LQCD_TRY(phio.alloc(hb));
    LQCD_TRY(xo.alloc(hb));
    LQCD_TRY(spinor_convert_raw(ctx, Vh, 1, phi.ptr, nullptr, LQCD_F64, phio.p, nullptr, outer));
    ph = outer_half(phio);
    xx = outer_half(xo);
  }
  if (phi2 == 0.0) {
    LQCD_CUDA(ctx, cudaMemsetAsync(X.ptr, 0, X.rhs_stride, ctx->stream));
    return LQCD_OK;
  }
  if (guess) {  // ph <- phi - Mhat^+ Mhat X0 in the outer format
    LQCD_TRY(t1.alloc(hb));
    LQCD_TRY(t2.alloc(hb));
    Op op{ctx, g, {}, outer, U->recon, kappa, mu};
    LQCD_TRY(gauge_view(ctx, U, outer, U->recon, &op.U));
    const HalfField T1 = outer_half(t1), T2 = outer_half(t2);
    LQCD_TRY(spinor_convert_raw(ctx, Vh, 1, X.ptr, nullptr, LQCD_F64, xo.p, nullptr, outer));
    LQCD_TRY(apply_schur(op, xx, T1, T2, 0, false, nullptr, nullptr, nullptr));
    LQCD_TRY(apply_schur(op, T1, xx, T2, 0, true, nullptr, nullptr, nullptr));
    LQCD_TRY(lincomb(ctx, Vh, ph, ph, &xx, {1, 0}, {1, 0}, {-1, 0}, {-1, 0}, nullptr, nullptr));
  }
  LQCD_CUDA(ctx, cudaMemsetAsync(xx.ptr, 0, xx.rhs_stride, ctx->stream));
  lqcd_cg_stats s1;
  std::memset(&s1, 0, sizeof(s1));
  lqcd_status s = cgls_even(ctx, U, g, kappa, mu, prm, ph, xx, b2, &s1, 1, nullptr, true);
  if (st) {
    st->iters += s1.iters;
    st->reliable_updates += s1.reliable_updates;
  }
  if (s != LQCD_OK) return s;
  if (guess) {  // X = X0 + d (in FP64)
    DBuf d64(ctx);
    LQCD_TRY(d64.alloc(X.rhs_stride));
    const HalfField D = f64_half(d64.p, Vh);
    LQCD_TRY(spinor_convert_raw(ctx, Vh, 1, xx.ptr, nullptr, outer, d64.p, nullptr, LQCD_F64));
    return lincomb(ctx, Vh, X, X, &D, {1, 0}, {1, 0}, {1, 0}, {1, 0}, nullptr, nullptr);
  }
  if (outer != LQCD_F64) LQCD_TRY(spinor_convert_raw(ctx, Vh, 1, xx.ptr, nullptr, outer, X.ptr, nullptr, LQCD_F64));
  return LQCD_OK;
}

// dS/dw of S = phi^+ (Mhat^+ Mhat)^-1 phi given X (F64 half fields) -> out [4][V][8]
// -2 Re[Y^+ dMhat(mu) X] / domega into out; Y = NULL: Y = Mhat X (the force of
// phi^+ (Mhat^+ Mhat)^-1 phi)
lqcd_status fermion_force_lr(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField *Y, const HalfField &X, double kappa,
                             double mu, double *out) {
  const Geom &g = U->g;
  const int Vh = g.Vh;
  size_t hb = spinor_half_bytes(LQCD_F64, Vh);
  DBuf Lf(ctx), Rf(ctx), tmp(ctx);
  LQCD_TRY(Lf.alloc(2 * hb));
  LQCD_TRY(Rf.alloc(2 * hb));
  LQCD_TRY(tmp.alloc(hb));
  HalfField Le = f64_half(Lf.p, Vh), Lo = f64_half((char *)Lf.p + hb, Vh);
  HalfField Re = f64_half(Rf.p, Vh), Ro = f64_half((char *)Rf.p + hb, Vh);
  HalfField T = f64_half(tmp.p, Vh);
  Op op{ctx, g, {}, LQCD_F64, U->recon, kappa, mu};
  LQCD_TRY(gauge_view(ctx, U, LQCD_F64, U->recon, &op.U));
  // Re = X_e;  Le = Y_e (= Mhat X_e unless given)
  LQCD_CUDA(ctx, cudaMemcpyAsync(Re.ptr, X.ptr, hb, cudaMemcpyDeviceToDevice, ctx->stream));
  if (Y) LQCD_CUDA(ctx, cudaMemcpyAsync(Le.ptr, Y->ptr, hb, cudaMemcpyDeviceToDevice, ctx->stream));
  else LQCD_TRY(apply_schur(op, X, Le, T, 0, false, nullptr, nullptr, nullptr));
  double a = 2.0 * kappa * mu, n = 1.0 / (1.0 + a * a);
  // Ro = Z_o = A_o^-1 H_oe X_e
  HopLaunch L;
  L.prec = LQCD_F64;
  L.recon = U->recon;
  L.U = op.U;
  L.in = Re;
  L.out = Ro;
  L.out_parity = 1;
  L.c_up = {n, -a * n};
  L.c_dn = {n, a * n};
  LQCD_TRY(launch_hop(ctx, g, L, nullptr));
  // Lo = W_o = A_o^-+ (H^+)_oe Y_e,  A^-+ = (1 + i a g5)/(1 + a^2)
  HopLaunch L2 = L;
  L2.in = Le;
  L2.out = Lo;
  L2.dagger = 1;
  L2.c_up = {n, a * n};
  L2.c_dn = {n, -a * n};
  LQCD_TRY(launch_hop(ctx, g, L2, nullptr));
  return fermion_force_raw(ctx, U, op.U, U->recon, Lf.p, Rf.p, kappa, out);
}

}  // namespace lqcd

using namespace lqcd;

static lqcd_status check_u(lqcd_ctx *ctx, const lqcd_gauge *U) {
  if (!U) return fail(ctx, LQCD_ERR_INVALID, "gauge field is NULL");
  return LQCD_OK;
}

extern "C" int lqcd_plaquette(lqcd_ctx *ctx, const lqcd_gauge *U, double *plaq_out) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (!plaq_out) return fail(ctx, LQCD_ERR_INVALID, "plaq_out is NULL");
  double s;
  LQCD_TRY(plaquette_sum(ctx, U, &s));
  *plaq_out = s / (3.0 * 6.0 * 2.0 * U->g.Vh);
  return LQCD_OK;
}

// S_g = (beta/3) [c0 (18 V - sum Re Tr P) + c1 (36 V - sum Re Tr R)]
static lqcd_status gauge_action_sym(lqcd_ctx *ctx, const lqcd_gauge *U, double beta, double c1, double *S) {
  const double V = 2.0 * U->g.Vh;
  double sp, sr = 36.0 * V;
  LQCD_TRY(plaquette_sum(ctx, U, &sp));
  if (c1 != 0.0) LQCD_TRY(rectangle_sum(ctx, U, &sr));
  *S = beta / 3.0 * ((1.0 - 8.0 * c1) * (18.0 * V - sp) + c1 * (36.0 * V - sr));
  return LQCD_OK;
}

extern "C" int lqcd_gauge_force(lqcd_ctx *ctx, const lqcd_gauge *U, double beta, double c1, int prec,
                                double *dSdw, double *S_out) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (!dSdw || !aligned16(dSdw)) return fail(ctx, LQCD_ERR_INVALID, "dSdw: NULL or misaligned");
  if (!std::isfinite(beta) || !std::isfinite(c1)) return fail(ctx, LQCD_ERR_NONFINITE, "beta or c1 not finite");
  if (prec != LQCD_F64 && prec != LQCD_DF64) return fail(ctx, LQCD_ERR_INVALID, "prec must be LQCD_F64 or LQCD_DF64");
  // the DF64 copy of the links is a cache of the field: it does not change U
  LQCD_TRY(gauge_force_raw(ctx, const_cast<lqcd_gauge *>(U), beta, c1, prec, dSdw));
  if (S_out) LQCD_TRY(gauge_action_sym(ctx, U, beta, c1, S_out));
  return LQCD_OK;
}

extern "C" int lqcd_heatbath_sweep(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed, uint64_t sweep_idx,
                                   int n_or, int prec) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(ctx, LQCD_ERR_INVALID, "beta must be finite, >= 0");
  if (n_or < 0 || n_or > 64) return fail(ctx, LQCD_ERR_INVALID, "n_or out of [0, 64]");
  if (prec != LQCD_F64 && prec != LQCD_F32 && prec != LQCD_DF64)
    return fail(ctx, LQCD_ERR_INVALID, "prec must be LQCD_F64, LQCD_DF64 or LQCD_F32");
  unsigned int *fails = (unsigned int *)ctx->partials;  // scratch word; not read by anyone else
  LQCD_CUDA(ctx, cudaMemsetAsync(fails, 0, sizeof(unsigned int), ctx->stream));
  if (prec == LQCD_F32) return heatbath_f32_raw(ctx, U, beta, seed, sweep_idx, 1, n_or, fails);
  if (prec == LQCD_DF64) return heatbath_df_raw(ctx, U, beta, seed, sweep_idx, 1, n_or, fails);
  return heatbath_raw(ctx, U, beta, seed, sweep_idx, 1, n_or, fails);
}

extern "C" int lqcd_overrelax_sweep(lqcd_ctx *ctx, lqcd_gauge *U, int n_or, int prec) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (n_or < 1 || n_or > 64) return fail(ctx, LQCD_ERR_INVALID, "n_or out of [1, 64]");
  if (prec != LQCD_F64 && prec != LQCD_F32 && prec != LQCD_DF64)
    return fail(ctx, LQCD_ERR_INVALID, "prec must be LQCD_F64, LQCD_DF64 or LQCD_F32");
  unsigned int *fails = (unsigned int *)ctx->partials;  // scratch word; not read by anyone else
  LQCD_CUDA(ctx, cudaMemsetAsync(fails, 0, sizeof(unsigned int), ctx->stream));
  if (prec == LQCD_F32) return heatbath_f32_raw(ctx, U, 0.0, 0, 0, 0, n_or, fails);
  if (prec == LQCD_DF64) return heatbath_df_raw(ctx, U, 0.0, 0, 0, 0, n_or, fails);
  return heatbath_raw(ctx, U, 0.0, 0, 0, 0, n_or, fails);
}

extern "C" int lqcd_momenta_gaussian(lqcd_ctx *ctx, const lqcd_geom *geom, double *P, uint64_t seed,
                                     uint32_t traj) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  if (!P || !aligned16(P)) return fail(ctx, LQCD_ERR_INVALID, "P: NULL or misaligned");
  Geom g = make_geom(*geom);
  return momenta_raw(ctx, 2L * g.Vh, P, seed, traj);
}

extern "C" int lqcd_spinor_gaussian(lqcd_ctx *ctx, const lqcd_geom *geom, lqcd_field eta, int parity,
                                    uint64_t seed, uint32_t traj) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  LQCD_TRY(check_field(ctx, eta, "eta", false));
  if (eta.prec != LQCD_F64 || eta.nrhs != 1) return fail(ctx, LQCD_ERR_INVALID, "eta must be one F64 EO full field");
  if (parity != LQCD_FULL && parity != LQCD_EVEN && parity != LQCD_ODD)
    return fail(ctx, LQCD_ERR_INVALID, "bad parity");
  Geom g = make_geom(*geom);
  int p = parity == LQCD_FULL ? 2 : (parity == LQCD_EVEN ? 0 : 1);
  return gaussian_spinor_raw(ctx, g, eta.ptr, p, seed, traj);
}

extern "C" int lqcd_gauge_update(lqcd_ctx *ctx, lqcd_gauge *U, const double *P, double eps) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (!P || !aligned16(P)) return fail(ctx, LQCD_ERR_INVALID, "P: NULL or misaligned");
  if (!std::isfinite(eps)) return fail(ctx, LQCD_ERR_NONFINITE, "eps not finite");
  return gauge_update_raw(ctx, U, P, eps, LQCD_F64);
}

extern "C" int lqcd_gauge_update_prec(lqcd_ctx *ctx, lqcd_gauge *U, const double *P, double eps, int prec) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (!P || !aligned16(P)) return fail(ctx, LQCD_ERR_INVALID, "P: NULL or misaligned");
  if (!std::isfinite(eps)) return fail(ctx, LQCD_ERR_NONFINITE, "eps not finite");
  if (prec != LQCD_F64 && prec != LQCD_DF64) return fail(ctx, LQCD_ERR_INVALID, "prec must be LQCD_F64 or LQCD_DF64");
  return gauge_update_raw(ctx, U, P, eps, prec);
}

extern "C" int lqcd_momenta_update(lqcd_ctx *ctx, const lqcd_geom *geom, double *P, const double *dSdw,
                                   double eps) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  if (!P || !dSdw) return fail(ctx, LQCD_ERR_INVALID, "NULL argument");
  Geom g = make_geom(*geom);
  return momenta_update_raw(ctx, 2L * g.Vh, P, dSdw, eps);
}

extern "C" int lqcd_momenta_kinetic(lqcd_ctx *ctx, const lqcd_geom *geom, const double *P, double *K_out) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  if (!P || !K_out) return fail(ctx, LQCD_ERR_INVALID, "NULL argument");
  Geom g = make_geom(*geom);
  double s;
  LQCD_TRY(sumsq_raw(ctx, P, (size_t)32 * 2 * g.Vh, &s));
  *K_out = 0.5 * s;
  return LQCD_OK;
}

extern "C" int lqcd_gauge_copy(lqcd_ctx *ctx, const lqcd_gauge *src, lqcd_gauge *dst) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (!src || !dst) return fail(ctx, LQCD_ERR_INVALID, "NULL gauge field");
  if (!geom_equal(src->geom, dst->geom)) return fail(ctx, LQCD_ERR_INVALID, "geometry mismatch");
  size_t bytes = (size_t)2 * 4 * 9 * src->g.Vh * 16;
  LQCD_CUDA(ctx, cudaMemcpyAsync(dst->master, src->master, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  dst->version++;
  return LQCD_OK;
}

lqcd_status fermion_force_from_X(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField &X, double kappa, double mu,
                                 double *out) {
  return fermion_force_lr(ctx, U, nullptr, X, kappa, mu, out);
}

// Mass preconditioning with a heavier twisted mass mu2 (Sec. 2.2: det D =
// det A det(D / A)): the ratio action S2 = phi2^+ W (Mhat^+ Mhat)^-1 W^+ phi2,
// W = Mhat(mu2), and its derivative
//   dS2 = -2 Re[Y^+ dMhat(mu) X] + 2 Re[phi2^+ dW X],
//   X = (Mhat^+ Mhat)^-1 psi, psi = W^+ phi2, Y = Mhat X.
// psi and X (F64 half fields) are outputs; S2 (host) = Re psi^+ X.
lqcd_status ratio_solve(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField &phi2, const HalfField &psi,
                        const HalfField &X, double kappa, double mu, double mu2, const lqcd_cg_params &prm,
                        lqcd_cg_stats *st, double *S2, bool guess) {
  const int Vh = U->g.Vh;
  DBuf tmp(ctx);
  LQCD_TRY(tmp.alloc(spinor_half_bytes(LQCD_F64, Vh)));
  Op op{ctx, U->g, {}, LQCD_F64, U->recon, kappa, mu2};
  LQCD_TRY(gauge_view(ctx, U, LQCD_F64, U->recon, &op.U));
  LQCD_TRY(apply_schur(op, phi2, psi, f64_half(tmp.p, Vh), 0, true, nullptr, nullptr, nullptr));
  LQCD_TRY(solve_normal(ctx, U, psi, X, kappa, mu, prm, st, guess));
  if (S2) LQCD_TRY(half_redot(ctx, Vh, psi, X, S2));
  return LQCD_OK;
}
lqcd_status ratio_force(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField &phi2, const HalfField &X, double kappa,
                        double mu, double mu2, double *out) {
  const long V = 2L * U->g.Vh;
  DBuf f2(ctx);
  LQCD_TRY(f2.alloc((size_t)32 * V * sizeof(double)));
  LQCD_TRY(fermion_force_lr(ctx, U, nullptr, X, kappa, mu, out));
  LQCD_TRY(fermion_force_lr(ctx, U, &phi2, X, kappa, mu2, (double *)f2.p));
  return momenta_update_raw(ctx, V, out, (const double *)f2.p, 1.0);  // out -= G(phi2, X; mu2)
}

extern "C" int lqcd_fermion_force_ratio(lqcd_ctx *ctx, const lqcd_gauge *Uc, lqcd_field phi2, double *dSdw,
                                        const lqcd_geom *geom, double kappa, double mu, double mu2,
                                        const lqcd_cg_params *params, lqcd_cg_stats *stats, double *S_out) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, Uc));
  LQCD_TRY(check_geom(ctx, geom));
  if (!geom_equal(Uc->geom, *geom)) return fail(ctx, LQCD_ERR_INVALID, "geometry mismatch");
  LQCD_TRY(check_field(ctx, phi2, "phi2", false));
  if (phi2.prec != LQCD_F64 || phi2.nrhs != 1) return fail(ctx, LQCD_ERR_INVALID, "phi2 must be one F64 EO half field");
  if (!dSdw || !aligned16(dSdw)) return fail(ctx, LQCD_ERR_INVALID, "dSdw: NULL or misaligned");
  if (!params) return fail(ctx, LQCD_ERR_INVALID, "params is NULL");
  if (params->outer_prec != LQCD_F64 && params->outer_prec != LQCD_DF64)
    return fail(ctx, LQCD_ERR_INVALID, "outer_prec must be F64 or DF64");
  if (!std::isfinite(kappa) || !std::isfinite(mu) || !std::isfinite(mu2))
    return fail(ctx, LQCD_ERR_NONFINITE, "kappa/mu/mu2 not finite");
  lqcd_gauge *U = const_cast<lqcd_gauge *>(Uc);
  const int Vh = U->g.Vh;
  DBuf pbuf(ctx), xbuf(ctx);
  LQCD_TRY(pbuf.alloc(spinor_half_bytes(LQCD_F64, Vh)));
  LQCD_TRY(xbuf.alloc(spinor_half_bytes(LQCD_F64, Vh)));
  HalfField ph = f64_half(phi2.ptr, Vh), psi = f64_half(pbuf.p, Vh), X = f64_half(xbuf.p, Vh);
  lqcd_cg_stats st;
  std::memset(&st, 0, sizeof(st));
  lqcd_status s = ratio_solve(ctx, U, ph, psi, X, kappa, mu, mu2, *params, &st, S_out, false);
  if (stats) *stats = st;
  if (s != LQCD_OK) return s;
  return ratio_force(ctx, U, ph, X, kappa, mu, mu2, dSdw);
}

extern "C" int lqcd_fermion_force(lqcd_ctx *ctx, const lqcd_gauge *Uc, lqcd_field phi, double *dSdw,
                                  lqcd_field *X_cache, const lqcd_geom *geom, double kappa, double mu,
                                  const lqcd_cg_params *params, lqcd_cg_stats *stats, double *S_out) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, Uc));
  LQCD_TRY(check_geom(ctx, geom));
  if (!geom_equal(Uc->geom, *geom)) return fail(ctx, LQCD_ERR_INVALID, "geometry mismatch");
  LQCD_TRY(check_field(ctx, phi, "phi", false));
  if (phi.prec != LQCD_F64 || phi.nrhs != 1) return fail(ctx, LQCD_ERR_INVALID, "phi must be one F64 EO half field");
  if (!dSdw && !S_out) return fail(ctx, LQCD_ERR_INVALID, "dSdw and S_out are both NULL");
  if (dSdw && !aligned16(dSdw)) return fail(ctx, LQCD_ERR_INVALID, "dSdw misaligned");
  if (!params) return fail(ctx, LQCD_ERR_INVALID, "params is NULL");
  if (params->outer_prec != LQCD_F64 && params->outer_prec != LQCD_DF64)
    return fail(ctx, LQCD_ERR_INVALID, "outer_prec must be F64 or DF64");
  if (!std::isfinite(kappa) || !std::isfinite(mu)) return fail(ctx, LQCD_ERR_NONFINITE, "kappa/mu not finite");
  lqcd_gauge *U = const_cast<lqcd_gauge *>(Uc);
  const int Vh = U->g.Vh;
  HalfField ph = f64_half(phi.ptr, Vh);
  DBuf xbuf(ctx);
  HalfField X;
  if (X_cache) {
    LQCD_TRY(check_field(ctx, *X_cache, "X_cache", false));
    X = f64_half(X_cache->ptr, Vh);
  } else {
    LQCD_TRY(xbuf.alloc(spinor_half_bytes(LQCD_F64, Vh)));
    X = f64_half(xbuf.p, Vh);
  }
  lqcd_cg_stats st;
  std::memset(&st, 0, sizeof(st));
  if (!X_cache || X_cache->reserved != 1) {
    lqcd_status s = solve_normal(ctx, U, ph, X, kappa, mu, *params, &st, false);
    if (stats) *stats = st;
    if (s != LQCD_OK) return s;
    if (X_cache) X_cache->reserved = 1;
  } else if (stats) {
    *stats = st;
  }
  if (S_out) LQCD_TRY(half_redot(ctx, Vh, ph, X, S_out));
  if (!dSdw) return LQCD_OK;  // the action alone
  return fermion_force_from_X(ctx, U, X, kappa, mu, dSdw);
}

// ---------------------------------------------------------------------------
// HMC trajectory
// ---------------------------------------------------------------------------

extern "C" int lqcd_hmc_trajectory(lqcd_ctx *ctx, lqcd_gauge *U, const lqcd_hmc_params *prm,
                                   lqcd_hmc_stats *stats) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_u(ctx, U));
  if (!prm || !stats) return fail(ctx, LQCD_ERR_INVALID, "NULL params or stats");
  if (prm->nsteps < 1 || !(prm->tau > 0.0)) return fail(ctx, LQCD_ERR_INVALID, "nsteps >= 1 and tau > 0 required");
  if (prm->integrator != LQCD_LEAPFROG && prm->integrator != LQCD_2MN)
    return fail(ctx, LQCD_ERR_INVALID, "integrator must be LQCD_LEAPFROG or LQCD_2MN");
  if (prm->integrator == LQCD_2MN && prm->nsteps_gauge < 1)
    return fail(ctx, LQCD_ERR_INVALID, "2MN needs nsteps_gauge >= 1");
  if (!std::isfinite(prm->c1) || !std::isfinite(prm->lambda) || prm->lambda < 0.0 || prm->lambda >= 0.5)
    return fail(ctx, LQCD_ERR_INVALID, "c1 must be finite and lambda in [0, 0.5)");
  if (prm->force_prec != LQCD_F64 && prm->force_prec != LQCD_DF64)
    return fail(ctx, LQCD_ERR_INVALID, "force_prec must be LQCD_F64 or LQCD_DF64");
  if (!std::isfinite(prm->mu2)) return fail(ctx, LQCD_ERR_NONFINITE, "mu2 not finite");
  if (prm->mu2 != 0.0 && prm->integrator == LQCD_2MN && prm->nsteps_mid < 1)
    return fail(ctx, LQCD_ERR_INVALID, "mass preconditioning with 2MN needs nsteps_mid >= 1");
  auto t0 = std::chrono::steady_clock::now();
  std::memset(stats, 0, sizeof(*stats));
  const Geom &g = U->g;
  const int Vh = g.Vh;
  const long V = 2L * Vh;
  const size_t nP = (size_t)32 * V;
  const bool fermions = prm->nf != 0;
  const bool hasen = fermions && prm->mu2 != 0.0;  // mass preconditioning
  const bool two_mn = prm->integrator == LQCD_2MN;
  const double lam = prm->lambda != 0.0 ? prm->lambda : 0.1931833275037836;
  const double mu1 = hasen ? prm->mu2 : prm->mu;  // twisted mass of the first pseudofermion
  size_t hb = spinor_half_bytes(LQCD_F64, Vh);
  DBuf P(ctx), F(ctx), eta(ctx), phi(ctx), X(ctx), tmp(ctx), save(ctx), phi2(ctx), psi2(ctx), X2(ctx);
  LQCD_TRY(P.alloc(nP * sizeof(double)));
  LQCD_TRY(F.alloc(nP * sizeof(double)));
  LQCD_TRY(save.alloc((size_t)2 * 4 * 9 * Vh * 16));
  if (fermions) {
    LQCD_TRY(eta.alloc(2 * hb));
    LQCD_TRY(phi.alloc(hb));
    LQCD_TRY(X.alloc(hb));
    LQCD_TRY(tmp.alloc(hb));
  }
  if (hasen) {
    LQCD_TRY(phi2.alloc(hb));
    LQCD_TRY(psi2.alloc(hb));
    LQCD_TRY(X2.alloc(hb));
  }
  LQCD_CUDA(ctx, cudaMemcpyAsync(save.p, U->master, (size_t)2 * 4 * 9 * Vh * 16, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
  const uint64_t seed = prm->seed;
  const uint32_t traj = prm->traj;
  LQCD_TRY(momenta_raw(ctx, V, (double *)P.p, seed, traj));
  HalfField Phi = f64_half(phi.p, Vh), Xh = f64_half(X.p, Vh);
  HalfField Phi2 = f64_half(phi2.p, Vh), Psi2 = f64_half(psi2.p, Vh), X2h = f64_half(X2.p, Vh);
  int cg_iters = 0;
  // X = (W^+ W)^-1 phi (W = Mhat(mu1)) at the current links, once per field
  uint64_t x_version = 0, x2_version = 0;
  double S2_cur = 0.0;
  auto solve_x = [&]() -> lqcd_status {
    if (x_version == U->version) return LQCD_OK;
    lqcd_cg_stats st;
    std::memset(&st, 0, sizeof(st));
    // from the second solve on, the previous field's X is the starting vector
    LQCD_TRY(solve_normal(ctx, U, Phi, Xh, prm->kappa, mu1, prm->cg, &st, x_version != 0));
    cg_iters += st.iters;
    x_version = U->version;
    return LQCD_OK;
  };
  // the ratio pseudofermion: psi2 = W^+ phi2, X2 = (Mhat^+ Mhat)^-1 psi2
  auto solve_x2 = [&]() -> lqcd_status {
    if (x2_version == U->version) return LQCD_OK;
    lqcd_cg_stats st;
    std::memset(&st, 0, sizeof(st));
    LQCD_TRY(ratio_solve(ctx, U, Phi2, Psi2, X2h, prm->kappa, prm->mu, prm->mu2, prm->cg, &st, &S2_cur,
                         x2_version != 0));
    cg_iters += st.iters;
    x2_version = U->version;
    return LQCD_OK;
  };
  // Momentum kicks are collected and applied when the links are about to
  // change (or at the end): P -= w[k] dS_k/dw for the gauge force (k = 0),
  // the first pseudofermion (k = 1) and the ratio (k = 2); one evaluation
  // per field and kind.
  double w[3] = {0.0, 0.0, 0.0};
  auto flush = [&]() -> lqcd_status {
    if (w[0] != 0.0) {
      LQCD_TRY(gauge_force_raw(ctx, U, prm->beta, prm->c1, prm->force_prec, (double *)F.p));
      LQCD_TRY(momenta_update_raw(ctx, V, (double *)P.p, (const double *)F.p, w[0]));
    }
    if (w[1] != 0.0 && fermions) {
      LQCD_TRY(solve_x());
      LQCD_TRY(fermion_force_from_X(ctx, U, Xh, prm->kappa, mu1, (double *)F.p));
      LQCD_TRY(momenta_update_raw(ctx, V, (double *)P.p, (const double *)F.p, w[1]));
    }
    if (w[2] != 0.0 && hasen) {
      LQCD_TRY(solve_x2());
      LQCD_TRY(ratio_force(ctx, U, Phi2, X2h, prm->kappa, prm->mu, prm->mu2, (double *)F.p));
      LQCD_TRY(momenta_update_raw(ctx, V, (double *)P.p, (const double *)F.p, w[2]));
    }
    w[0] = w[1] = w[2] = 0.0;
    return LQCD_OK;
  };
  auto drift = [&](double h) -> lqcd_status {
    LQCD_TRY(flush());
    return gauge_update_raw(ctx, U, (const double *)P.p, h, prm->force_prec);
  };
  // 2MN on nested time scales: level 0 is the outermost force; each of its
  // position updates over time h is the 2MN integration of the next level
  // over h, down to the gauge force, whose position update is the link update
  int kinds[3], steps[3], nlev = 0;
  if (hasen) {
    kinds[nlev] = 2;
    steps[nlev++] = prm->nsteps;
    kinds[nlev] = 1;
    steps[nlev++] = prm->nsteps_mid > 0 ? prm->nsteps_mid : 1;
  } else if (fermions) {
    kinds[nlev] = 1;
    steps[nlev++] = prm->nsteps;
  }
  kinds[nlev] = 0;
  steps[nlev++] = (fermions || two_mn) ? prm->nsteps_gauge : prm->nsteps;
  // pure gauge: the gauge scale alone, with the step size it has under an
  // outer scale of nsteps steps (two position updates of e/2 each)
  if (!fermions) steps[0] = two_mn ? 2 * prm->nsteps * prm->nsteps_gauge : prm->nsteps;
  std::function<lqcd_status(int, double)> integrate = [&](int lev, double h) -> lqcd_status {
    const double d = h / steps[lev];
    auto sub = [&](double t) -> lqcd_status { return lev + 1 < nlev ? integrate(lev + 1, t) : drift(t); };
    for (int j = 0; j < steps[lev]; j++) {
      w[kinds[lev]] += lam * d;
      LQCD_TRY(sub(0.5 * d));
      w[kinds[lev]] += (1.0 - 2.0 * lam) * d;
      LQCD_TRY(sub(0.5 * d));
      w[kinds[lev]] += lam * d;
    }
    return LQCD_OK;
  };
  auto fermion_action = [&](double *S) -> lqcd_status {
    *S = 0.0;
    if (!fermions) return LQCD_OK;
    LQCD_TRY(solve_x());
    LQCD_TRY(half_redot(ctx, Vh, Phi, Xh, S));
    if (hasen) {
      LQCD_TRY(solve_x2());
      *S += S2_cur;
    }
    return LQCD_OK;
  };
  double Sf0 = 0.0, Sf1 = 0.0, Sg0, Sg1, K0, K1;
  if (fermions) {
    // phi = W^+ eta with W = Mhat(mu1)
    Op op1{ctx, g, {}, LQCD_F64, U->recon, prm->kappa, mu1};
    LQCD_TRY(gauge_view(ctx, U, LQCD_F64, U->recon, &op1.U));
    LQCD_TRY(gaussian_spinor_raw(ctx, g, eta.p, 0, seed, traj));
    LQCD_TRY(apply_schur(op1, f64_half(eta.p, Vh), Phi, f64_half(tmp.p, Vh), 0, true, nullptr, nullptr,
                         nullptr));
    if (hasen) {
      // phi2 = W^-+ Mhat^+ eta2 = W (W^+ W)^-1 Mhat^+ eta2, eta2 from the stream of seed ^ 0x9E3779B97F4A7C15
      Op op{ctx, g, {}, LQCD_F64, U->recon, prm->kappa, prm->mu};
      op.U = op1.U;
      LQCD_TRY(gaussian_spinor_raw(ctx, g, eta.p, 0, seed ^ 0x9E3779B97F4A7C15ull, traj));
      LQCD_TRY(apply_schur(op, f64_half(eta.p, Vh), Psi2, f64_half(tmp.p, Vh), 0, true, nullptr, nullptr,
                           nullptr));
      lqcd_cg_stats st;
      std::memset(&st, 0, sizeof(st));
      LQCD_TRY(solve_normal(ctx, U, Psi2, X2h, prm->kappa, prm->mu2, prm->cg, &st, false));
      cg_iters += st.iters;
      LQCD_TRY(apply_schur(op1, X2h, Phi2, f64_half(tmp.p, Vh), 0, false, nullptr, nullptr, nullptr));
    }
  }
  LQCD_TRY(sumsq_raw(ctx, (const double *)P.p, nP, &K0));
  K0 *= 0.5;
  LQCD_TRY(gauge_action_sym(ctx, U, prm->beta, prm->c1, &Sg0));
  LQCD_TRY(fermion_action(&Sf0));
  const double H0 = K0 + Sg0 + Sf0;
  const double e = prm->tau / prm->nsteps;
  if (two_mn) {
    LQCD_TRY(integrate(0, prm->tau));
  } else {
    for (int step = 0; step < prm->nsteps; step++) {
      w[0] += 0.5 * e;
      w[1] += 0.5 * e;
      w[2] += 0.5 * e;
      LQCD_TRY(drift(e));
      w[0] += 0.5 * e;
      w[1] += 0.5 * e;
      w[2] += 0.5 * e;
    }
  }
  LQCD_TRY(flush());
  LQCD_TRY(sumsq_raw(ctx, (const double *)P.p, nP, &K1));
  K1 *= 0.5;
  LQCD_TRY(gauge_action_sym(ctx, U, prm->beta, prm->c1, &Sg1));
  LQCD_TRY(fermion_action(&Sf1));
  const double H1 = K1 + Sg1 + Sf1;
  const double dH = H1 - H0;
  if (!std::isfinite(dH)) return fail(ctx, LQCD_ERR_NONFINITE, "dH is not finite");
  double u;
  LQCD_TRY(metro_uniform(ctx, seed, traj, &u));
  const bool accept = dH <= 0.0 || u < std::exp(-dH);
  if (!accept) {
    LQCD_CUDA(ctx, cudaMemcpyAsync(U->master, save.p, (size_t)2 * 4 * 9 * Vh * 16, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    U->version++;
  }
  double plaq_sum;
  LQCD_TRY(plaquette_sum(ctx, U, &plaq_sum));
  stats->dH = dH;
  stats->H0 = H0;
  stats->H1 = H1;
  stats->plaquette = plaq_sum / (18.0 * V);
  stats->accepted = accept ? 1 : 0;
  stats->cg_iters = cg_iters;
  stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return LQCD_OK;
}
