// dd_cg.cu -- the even-odd CG (CGLS on Mhat^+ Mhat, Sec. 2.1) on a lattice
// split into a grid of domains along t and z (the paper's Sec. 6 outlook: the
// solver over several GPUs).  Each half hop of the operator is the
// domain-decomposed hop of dd.cu: pack the faces of every held domain, move
// the faces, run the domain hops with the operator's diagonal epilogue.  Every norm is a
// fixed-order sum on each domain, summed over the held domains in order on
// the host, then over processes by the caller's allreduce hook.  The solver
// arithmetic, the source preparation bhat_e = b_e + kappa H_eo A_o^-1 b_o, the
// reconstruction x_o = A_o^-1 (b_o + kappa H_oe x_e) and the FP64 true
// residual with outer refinement follow the single-domain solver in cg.cu
// (one right-hand side), with host-side scalars: a decomposed solve
// synchronises on every norm anyway, to sum it over processes.  Mixed
// precision (Sec. 3: the bulk of the work in a cheaper format, the accuracy
// restored in FP64) takes the form of defect correction: each refinement
// cycle runs the CGLS in the inner format (F32 or float-float) on its cycle's
// prepared residual until that residual has dropped by inner_tol, and the
// correction, the reconstruction and the true residual are formed in FP64.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

// sum of partials[0..n) in a fixed order (one block of 256 threads)
__global__ void __launch_bounds__(256) dd_sum_kernel(const double *partials, int n, double *out) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) t += partials[i];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

namespace {

struct Tm {  // per-chirality factors of A = 1 + i a gamma_5 (a = 2 kappa mu) and A^-1
  HostC A_up, A_dn, Ai_up, Ai_dn;
};
Tm tm_of(double kappa, double mu, bool dagger) {
  double a = 2.0 * kappa * mu;
  if (dagger) a = -a;
  const double n = 1.0 / (1.0 + a * a);
  return {{1.0, a}, {1.0, -a}, {n, -a * n}, {n, a * n}};
}
HostC scaled(HostC c, double f) { return {f * c.re, f * c.im}; }

// one half field per held domain (FP64 unless alloc() is given another
// format); alloc() makes it own its memory, a view of the caller's fields (f
// filled directly) frees nothing
struct DVec {
  lqcd_ctx *ctx = nullptr;
  std::vector<HalfField> f;
  DVec() = default;
  DVec(const DVec &) = delete;
  DVec &operator=(const DVec &) = delete;
  ~DVec() {
    if (ctx)
      for (auto &h : f) dfree(ctx, h.ptr);
  }
  lqcd_status alloc(lqcd_ctx *c, int nd, int Vh, int prec = LQCD_F64) {
    ctx = c;
    f.resize(nd);
    for (auto &h : f) {
      h.prec = prec;
      h.nrhs = 1;
      h.rhs_stride = spinor_half_bytes(prec, Vh);
      LQCD_TRY(dalloc(c, &h.ptr, h.rhs_stride));
      LQCD_CUDA(c, cudaMemsetAsync(h.ptr, 0, h.rhs_stride, c->stream));
    }
    return LQCD_OK;
  }
};

struct Dd {
  lqcd_ctx *ctx;
  int nd, first, nz, nt, antiper;  // held domains first.. of the nz x nt grid (domain dz + nz dt)
  Geom g;  // local geometry; the global boundary sign travels in the faces
  int recon, recon_i;
  std::vector<GaugeView> U, Ui;  // FP64 links; links of the inner format
  // per held domain: to_prev, to_next, from_next, from_prev along t, then
  // (nz > 1) along z
  std::vector<void *> faces;
  const lqcd_dd_comm *comm;
  double kappa, mu;
  double *dsum;  // device [nd]

  int nf() const { return nz > 1 ? 8 : 4; }
  void *face(int d, int k) const { return faces[(size_t)nf() * d + k]; }
  // neighbours of global domain gd along t (mu = 3) or z (mu = 2)
  int next(int gd, int mu) const {
    const int dz = gd % nz, dt = gd / nz;
    return mu == 3 ? dz + nz * ((dt + 1) % nt) : (dz + 1) % nz + nz * dt;
  }
  int prev(int gd, int mu) const {
    const int dz = gd % nz, dt = gd / nz;
    return mu == 3 ? dz + nz * ((dt + nt - 1) % nt) : (dz + nz - 1) % nz + nz * dt;
  }
  // bytes of one face along mu in the format prec
  size_t face_bytes(int mu, int prec) const {
    return (size_t)dd_face_sites(g, mu) * 6 * dd_face_word_bytes(prec);
  }

  // per-domain sums in dsum[0..nd) -> the total over all domains of all processes
  lqcd_status total(double *out) {
    LQCD_TRY(ensure_pinned(ctx, nd));
    LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, dsum, nd * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double t = 0.0;
    for (int d = 0; d < nd; d++) t += ctx->pinned[d];
    if (comm && comm->allreduce) {
      if (comm->allreduce(comm->user, &t, 1) != 0)
        return fail(ctx, LQCD_ERR_COMM, "domain-decomposed CG: the allreduce hook failed");
    }
    *out = t;
    return LQCD_OK;
  }

  // the faces written by the packs (in the format prec) reach their
  // neighbours; without hooks every domain is held here (global = local index)
  lqcd_status exchange(int prec) {
    const size_t nb_t = face_bytes(3, prec), nb_z = nz > 1 ? face_bytes(2, prec) : 0;
    if (comm) {
      LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (comm->exchange(comm->user, nb_t, nb_z) != 0)
        return fail(ctx, LQCD_ERR_COMM, "domain-decomposed CG: the exchange hook failed");
      return LQCD_OK;
    }
    for (int d = 0; d < nd; d++)
      for (int mu = 3; mu >= (nz > 1 ? 2 : 3); mu--) {
        const int o = mu == 3 ? 0 : 4;
        const size_t nb = mu == 3 ? nb_t : nb_z;
        LQCD_CUDA(ctx, cudaMemcpyAsync(face(d, o + 2), face(next(d, mu), o + 0), nb, cudaMemcpyDeviceToDevice,
                                       ctx->stream));
        LQCD_CUDA(ctx, cudaMemcpyAsync(face(d, o + 3), face(prev(d, mu), o + 1), nb, cudaMemcpyDeviceToDevice,
                                       ctx->stream));
      }
    return LQCD_OK;
  }

  // out_p = c * H in + d * aux on every held domain (aux optional), in the
  // format of the fields (FP64 or the inner one); norm: |out|^2 over the whole
  // lattice
  lqcd_status hop(const DVec &in, const DVec &out, const DVec *aux, int p, bool dagger, HostC c_up, HostC c_dn,
                  HostC d_up, HostC d_dn, double *norm) {
    const int prec = in.f[0].prec;
    const bool f64 = prec == LQCD_F64;
    for (int d = 0; d < nd; d++) {
      HopLaunch L;
      L.prec = prec;
      L.recon = f64 ? recon : recon_i;
      L.U = f64 ? U[d] : Ui[d];
      L.in = in.f[d];
      L.out_parity = p;
      L.dagger = dagger ? 1 : 0;
      const int dt = (first + d) / nz;
      LQCD_TRY(dd_pack(ctx, g, L, 3, face(d, 0), face(d, 1), antiper && dt == 0, antiper && dt == nt - 1));
      if (nz > 1) LQCD_TRY(dd_pack(ctx, g, L, 2, face(d, 4), face(d, 5), 0, 0));
    }
    LQCD_TRY(exchange(prec));
    const int nw = (g.Vh + 31) / 32;
    for (int d = 0; d < nd; d++) {
      HopLaunch L;
      L.prec = prec;
      L.recon = f64 ? recon : recon_i;
      L.U = f64 ? U[d] : Ui[d];
      L.in = in.f[d];
      L.out = out.f[d];
      L.out_parity = p;
      L.dagger = dagger ? 1 : 0;
      L.c_up = c_up;
      L.c_dn = c_dn;
      if (aux) {
        L.aux = aux->f[d];
        L.has_aux = true;
        L.d_up = d_up;
        L.d_dn = d_dn;
      }
      L.partials = norm ? ctx->partials : nullptr;
      LQCD_TRY(dd_hop(ctx, g, L, face(d, 2), face(d, 3), nz > 1 ? face(d, 6) : nullptr,
                      nz > 1 ? face(d, 7) : nullptr));
      if (norm) dd_sum_kernel<<<1, 256, 0, ctx->stream>>>(ctx->partials, nw, dsum + d);
    }
    LQCD_CUDA(ctx, cudaGetLastError());
    return norm ? total(norm) : LQCD_OK;
  }

  // out = ca x + cb y on every held domain (y optional); norm: |out|^2 overall
  lqcd_status lin(const DVec &out, const DVec &x, const DVec *y, HostC ca_up, HostC ca_dn, HostC cb_up,
                  HostC cb_dn, double *norm) {
    for (int d = 0; d < nd; d++) {
      int nb = 0;
      LQCD_TRY(lincomb(ctx, g.Vh, out.f[d], x.f[d], y ? &y->f[d] : nullptr, ca_up, ca_dn, cb_up, cb_dn,
                       norm ? ctx->partials : nullptr, &nb));
      if (norm) dd_sum_kernel<<<1, 256, 0, ctx->stream>>>(ctx->partials, nb, dsum + d);
    }
    LQCD_CUDA(ctx, cudaGetLastError());
    return norm ? total(norm) : LQCD_OK;
  }

  // out = in converted to out's format on every held domain
  lqcd_status convert(const DVec &in, const DVec &out) {
    for (int d = 0; d < nd; d++)
      LQCD_TRY(spinor_convert_raw(ctx, g.Vh, 1, in.f[d].ptr, in.f[d].scale, in.f[d].prec, out.f[d].ptr,
                                  out.f[d].scale, out.f[d].prec));
    return LQCD_OK;
  }

  // out_e = Mhat in_e (dagger: Mhat^+), as apply_schur: -kappa^2 folded into
  // the first hop, the second adds A in_e
  lqcd_status mhat(const DVec &in, const DVec &out, const DVec &tmp_o, bool dagger, double *norm) {
    const Tm c = tm_of(kappa, mu, dagger);
    const double k2 = kappa * kappa;
    const HostC one{1.0, 0.0}, zero{0.0, 0.0};
    LQCD_TRY(hop(in, tmp_o, nullptr, 1, dagger, scaled(c.Ai_up, -k2), scaled(c.Ai_dn, -k2), zero, zero, nullptr));
    return hop(tmp_o, out, &in, 0, dagger, one, one, c.A_up, c.A_dn, norm);
  }
};

}  // namespace

lqcd_status dd_cg_solve(lqcd_ctx *ctx, int nd, int first, int nz, int nt, int antiper, const Geom &g, int recon,
                        const std::vector<GaugeView> &U, int recon_i, const std::vector<GaugeView> &Ui,
                        const std::vector<HalfField> &b_full, const std::vector<HalfField> &x_full,
                        const std::vector<void *> &faces, const lqcd_dd_comm *comm, double kappa, double mu,
                        const lqcd_cg_params &prm, lqcd_cg_stats *st) {
  const auto t0 = std::chrono::steady_clock::now();
  std::memset(st, 0, sizeof(*st));
  const int Vh = g.Vh;
  DBuf dsum(ctx);
  LQCD_TRY(dsum.alloc(sizeof(double) * nd));
  const int nb = (Vh + 127) / 128 > (Vh + 31) / 32 ? (Vh + 127) / 128 : (Vh + 31) / 32;
  LQCD_TRY(ensure_partials(ctx, (size_t)nb));
  Dd S{ctx, nd, first, nz, nt, antiper, g, recon, recon_i, U, Ui, faces, comm, kappa, mu, (double *)dsum.p};
  const int inner = prm.inner_prec;
  const bool mixed = inner != LQCD_F64;
  // a mixed cycle stops once its residual has dropped by itol (F32; a
  // float-float recursion runs to the tolerance itself)
  const double itol = !mixed || inner == LQCD_DF64 ? 0.0 : prm.inner_tol > 0.0 ? prm.inner_tol : 1e-5;
  // views of the caller's even and odd halves
  DVec be, bo, xe, xo;
  be.f.resize(nd);
  bo.f.resize(nd);
  xe.f.resize(nd);
  xo.f.resize(nd);
  const size_t hb = spinor_half_bytes(LQCD_F64, Vh);
  for (int d = 0; d < nd; d++) {
    HalfField h;
    h.prec = LQCD_F64;
    h.nrhs = 1;
    h.rhs_stride = hb;
    h.ptr = b_full[d].ptr;
    be.f[d] = h;
    h.ptr = (char *)b_full[d].ptr + hb;
    bo.f[d] = h;
    h.ptr = x_full[d].ptr;
    xe.f[d] = h;
    h.ptr = (char *)x_full[d].ptr + hb;
    xo.f[d] = h;
  }
  // FP64: the prepared source, reconstruction and true residual; the CGLS
  // vectors in the inner format (xs64, ti: separate only when mixed)
  DVec rhs_e, rhs_o, t_o, bhat, corr_o, res_e, res_o, xs, s, p, q, z, xs64_, ti_;
  for (DVec *v : {&rhs_e, &rhs_o, &t_o, &bhat, &corr_o, &res_e, &res_o}) LQCD_TRY(v->alloc(ctx, nd, Vh));
  for (DVec *v : {&xs, &s, &p, &q, &z}) LQCD_TRY(v->alloc(ctx, nd, Vh, inner));
  if (mixed) {
    LQCD_TRY(xs64_.alloc(ctx, nd, Vh));
    LQCD_TRY(ti_.alloc(ctx, nd, Vh, inner));
  }
  const DVec &xs64 = mixed ? xs64_ : xs, &ti = mixed ? ti_ : t_o;
  const size_t hbi = spinor_half_bytes(inner, Vh);
  const HostC one{1.0, 0.0}, zero{0.0, 0.0}, mone{-1.0, 0.0};
  lqcd_status result = LQCD_OK;
  for (int d = 0; d < nd; d++) {
    LQCD_CUDA(ctx, cudaMemsetAsync(xe.f[d].ptr, 0, hb, ctx->stream));
    LQCD_CUDA(ctx, cudaMemsetAsync(xo.f[d].ptr, 0, hb, ctx->stream));
  }
  // |b|^2 over the whole lattice; rhs = b
  double e2 = 0.0, o2 = 0.0;
  LQCD_TRY(S.lin(rhs_e, be, nullptr, one, one, zero, zero, &e2));
  LQCD_TRY(S.lin(rhs_o, bo, nullptr, one, one, zero, zero, &o2));
  const double b2 = e2 + o2;
  if (!std::isfinite(b2)) return fail(ctx, LQCD_ERR_NONFINITE, "right-hand side is not finite");
  const Tm c = tm_of(kappa, mu, false);
  const double stop2 = 0.25 * prm.tol * prm.tol * b2;
  for (int cycle = 0;; cycle++) {
    // bhat_e = rhs_e + kappa H_eo A_o^-1 rhs_o
    lqcd_status e = S.lin(t_o, rhs_o, nullptr, c.Ai_up, c.Ai_dn, zero, zero, nullptr);
    if (e == LQCD_OK)
      e = S.hop(t_o, bhat, &rhs_e, 0, false, {kappa, 0.0}, {kappa, 0.0}, one, one, nullptr);
    // CGLS on Mhat^+ Mhat in the inner format: xs = 0, s = bhat, z = p = Mhat^+ s
    double ss = 0.0, zz = 0.0, qq = 0.0;
    for (int d = 0; d < nd && e == LQCD_OK; d++)
      if (cudaMemsetAsync(xs.f[d].ptr, 0, hbi, ctx->stream) != cudaSuccess)
        e = cuda_check(ctx, cudaGetLastError(), "cudaMemsetAsync");
    if (e == LQCD_OK && mixed) e = S.convert(bhat, s);
    if (e == LQCD_OK) e = S.lin(s, mixed ? s : bhat, nullptr, one, one, zero, zero, &ss);
    const double istop2 = std::fmax(stop2, itol * itol * ss);
    if (e == LQCD_OK && ss > istop2) e = S.mhat(s, z, ti, true, &zz);
    if (e == LQCD_OK && ss > istop2) e = S.lin(p, z, nullptr, one, one, zero, zero, nullptr);
    while (e == LQCD_OK && ss > istop2 && st->iters < prm.max_iter) {
      e = S.mhat(p, q, ti, false, &qq);
      if (e != LQCD_OK) break;
      if (!(qq > 0.0) || !std::isfinite(qq)) {
        if (!std::isfinite(qq)) e = fail(ctx, LQCD_ERR_NONFINITE, "domain-decomposed CG: |Mhat p|^2 not finite");
        break;
      }
      const double alpha = zz / qq;
      e = S.lin(xs, xs, &p, one, one, {alpha, 0.0}, {alpha, 0.0}, nullptr);
      if (e == LQCD_OK) e = S.lin(s, s, &q, one, one, {-alpha, 0.0}, {-alpha, 0.0}, &ss);
      if (e != LQCD_OK) break;
      st->iters++;
      if (ss <= istop2) break;
      double zz1 = 0.0;
      e = S.mhat(s, z, ti, true, &zz1);
      if (e != LQCD_OK) break;
      const double beta = zz1 / zz;
      zz = zz1;
      e = S.lin(p, z, &p, one, one, {beta, 0.0}, {beta, 0.0}, nullptr);
    }
    // corr_o = A_o^-1 (rhs_o + kappa H_oe xs) in FP64; x += corr
    if (e == LQCD_OK && mixed) e = S.convert(xs, xs64);
    if (e == LQCD_OK)
      e = S.hop(xs64, corr_o, &rhs_o, 1, false, scaled(c.Ai_up, kappa), scaled(c.Ai_dn, kappa), c.Ai_up, c.Ai_dn,
                nullptr);
    if (e == LQCD_OK) e = S.lin(xe, xe, &xs64, one, one, one, one, nullptr);
    if (e == LQCD_OK) e = S.lin(xo, xo, &corr_o, one, one, one, one, nullptr);
    // true residual: rhs = b - M x, M x = A x - kappa H x on both parities
    if (e == LQCD_OK) e = S.hop(xo, res_e, &xe, 0, false, {-kappa, 0.0}, {-kappa, 0.0}, c.A_up, c.A_dn, nullptr);
    if (e == LQCD_OK) e = S.hop(xe, res_o, &xo, 1, false, {-kappa, 0.0}, {-kappa, 0.0}, c.A_up, c.A_dn, nullptr);
    if (e == LQCD_OK) e = S.lin(rhs_e, be, &res_e, one, one, mone, mone, &e2);
    if (e == LQCD_OK) e = S.lin(rhs_o, bo, &res_o, one, one, mone, mone, &o2);
    if (e != LQCD_OK) return e;
    const double tr = b2 > 0.0 ? std::sqrt((e2 + o2) / b2) : std::sqrt(e2 + o2);
    if (!std::isfinite(tr)) return fail(ctx, LQCD_ERR_NONFINITE, "domain-decomposed CG: true residual is not finite");
    st->true_resid = tr;
    st->converged = tr <= prm.tol;
    if (st->converged) break;
    if (cycle >= prm.max_restarts || st->iters >= prm.max_iter) {
      result = LQCD_ERR_NOCONV;
      break;
    }
    st->restarts++;  // the next cycle solves M d = b - M x (rhs holds the residual)
  }
  st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (result == LQCD_ERR_NOCONV)
    fail(ctx, LQCD_ERR_NOCONV, "domain-decomposed CG stopped with true residual %.3e > tol %.3e", st->true_resid,
         prm.tol);
  return result;
}

}  // namespace lqcd
