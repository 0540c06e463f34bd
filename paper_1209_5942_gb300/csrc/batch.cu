// batch.cu -- one CG solve over a batch of independent lattices of different
// sizes (e.g. 8 each of 8^4, 12^3x24, 16^3x32, 20^3x40).
//
// Each system k solves M_k x_k = b_k with the even-odd CGLS of cg.cu (source
// preparation, Mhat^+ Mhat recursion with reliable updates, reconstruction,
// FP64 true residual, outer refinement).  What is batched is the inner
// iteration: every stage (the four half hops of Mhat p and Mhat^+ s, the x/s
// update, the p update and the scalar steps) is ONE persistent launch whose
// fixed grid walks a queue of 128-site tiles spanning all systems, reading
// each system's geometry, links, fields and coefficients from a descriptor
// table in device memory.  Small lattices therefore share launches with large
// ones instead of each leaving the GPU mostly idle, and the whole inner
// iteration is replayed from one CUDA graph.  The scalar step is one block
// per system (fixed-order sums) with the last block deciding convergence and
// reliable-update triggers for the batch.
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

// solver state of one system (same meaning as in cg.cu)
struct BState {
  double zz, qq, ss, alpha, beta, stop2, rel2, rmax2;
  int done, iters, need_rel;
  int since, gap;  // iterations since the last reliable update, and its cap
};
struct BHdr {
  int halt, all_done, need_rel, nonfinite;
  int iters, nsys, mixed;
  unsigned int ticket;
  int loops, pad;  // pass counter of the graph's device-side loop
};
LQCD_DEV BState *bstate(BHdr *h) { return (BState *)(h + 1); }

enum { BF_ALPHA = 0, BF_SS = 1, BF_BETA = 2, BF_INIT_ZZ = 3 };

// One block per system: fixed-order sum of that system's partials and the CG
// scalar step; the last block to finish sets the batch-wide flags.
__global__ void __launch_bounds__(FIN_THREADS) bfinalize_kernel(BHdr *h, const double *partials, const long *poff, const int *pnb, int op) {
  __shared__ double sh[33];
  __shared__ int last;
  if (op != BF_INIT_ZZ && *(volatile int *)&h->halt) return;
  const int k = blockIdx.x;
  // the same fixed-order sum as the single-system solver's finalize
  const double x = block_sum_fixed(partials + poff[k], pnb[k], sh);
  if (threadIdx.x == 0) {
    BState &R = bstate(h)[k];
    int bad = !isfinite(x);
    switch (op) {
      case BF_ALPHA:
        R.qq = x;
        if (R.done) R.alpha = 0.0;
        else if (x > 0.0) R.alpha = R.zz / x;
        else { R.alpha = 0.0; if (R.zz > 0.0) bad = 1; }
        break;
      case BF_SS:
        R.ss = x;
        if (!R.done) {
          R.iters += 1;
          if (x <= R.stop2) R.done = 1;
          if (h->mixed && !R.done) {
            if (x > R.rmax2) R.rmax2 = x;
            R.since += 1;
            if (x < R.rel2 * R.rmax2 || R.since >= R.gap) R.need_rel = 1;
          }
        }
        break;
      case BF_BETA:
        R.beta = R.done ? 0.0 : (R.zz > 0.0 ? x / R.zz : 0.0);
        R.zz = x;
        break;
      default:
        R.zz = x;
        break;
    }
    if (bad) atomicOr(&h->nonfinite, 1);
    __threadfence();
    last = atomicAdd(&h->ticket, 1u) == (unsigned)(gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    int all = 1, rel = 0, maxit = 0;
    for (int j = 0; j < h->nsys; j++) {
      const volatile BState &R = bstate(h)[j];
      all &= R.done;
      rel |= R.need_rel;
      maxit = R.iters > maxit ? R.iters : maxit;
    }
    h->all_done = all;
    h->need_rel = rel;
    h->iters = maxit;
    if ((op == BF_SS && (all || rel)) || h->nonfinite) h->halt = 1;
    h->ticket = 0u;
  }
}

// per-system vector descriptors for the batched updates
struct VecDesc {
  int Vh;
  char *x, *p, *s, *q, *z;
  float *xs, *ps, *ss, *qs, *zs;
  double *partials;  // one per warp of 32 sites
};

// x += alpha p; s -= alpha q; per-warp |s|^2 partials
template <int P>
__global__ void __launch_bounds__(128) bxs_kernel(BHdr *h, const VecDesc *d, const int2 *tiles, int ntiles) {
  using R = typename SpinorIO<P>::R;
  if (*(volatile int *)&h->halt) return;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tile = tiles[t];
    const VecDesc D = d[tile.x];
    const int cb = tile.y + threadIdx.x;
    double nrm = 0.0;
    if (cb < D.Vh) {
      const R al = from_double<R>(bstate(h)[tile.x].alpha);
      Cx<R> X[12], Pp[12], S[12], Q[12];
      SpinorIO<P>::load({D.x, D.xs, D.Vh}, cb, X);
      SpinorIO<P>::load({D.p, D.ps, D.Vh}, cb, Pp);
      SpinorIO<P>::load({D.s, D.ss, D.Vh}, cb, S);
      SpinorIO<P>::load({D.q, D.qs, D.Vh}, cb, Q);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        X[k] = {rfma(al, Pp[k].re, X[k].re), rfma(al, Pp[k].im, X[k].im)};
        S[k] = {rfma(-al, Q[k].re, S[k].re), rfma(-al, Q[k].im, S[k].im)};
      }
      nrm = site_norm2<R, 12>(S);
      SpinorIO<P>::store({D.x, D.xs, D.Vh}, cb, X);
      SpinorIO<P>::store({D.s, D.ss, D.Vh}, cb, S);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0 && cb < D.Vh) D.partials[cb >> 5] = nrm;
  }
}

// p = z + beta p
template <int P>
__global__ void __launch_bounds__(128) bp_kernel(BHdr *h, const VecDesc *d, const int2 *tiles, int ntiles) {
  using R = typename SpinorIO<P>::R;
  if (*(volatile int *)&h->halt) return;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tile = tiles[t];
    const VecDesc D = d[tile.x];
    const int cb = tile.y + threadIdx.x;
    if (cb >= D.Vh) continue;
    const R be = from_double<R>(bstate(h)[tile.x].beta);
    Cx<R> Pp[12], Z[12];
    SpinorIO<P>::load({D.p, D.ps, D.Vh}, cb, Pp);
    SpinorIO<P>::load({D.z, D.zs, D.Vh}, cb, Z);
#pragma unroll
    for (int k = 0; k < 12; k++) Pp[k] = {rfma(be, Pp[k].re, Z[k].re), rfma(be, Pp[k].im, Z[k].im)};
    SpinorIO<P>::store({D.p, D.ps, D.Vh}, cb, Pp);
  }
}

__global__ void bstate_init_kernel(BHdr *h, int nsys, int mixed, const double *stop2, double rel, int gap) {
  for (int k = threadIdx.x; k < nsys; k += blockDim.x) {
    BState &R = bstate(h)[k];
    R.zz = R.qq = R.ss = R.alpha = R.beta = 0.0;
    R.stop2 = stop2[k];
    R.rel2 = rel * rel;
    R.rmax2 = 0.0;
    R.done = 0;
    R.iters = 0;
    R.need_rel = 0;
    R.since = 0;
    R.gap = gap;
  }
  if (threadIdx.x == 0) {
    h->halt = h->all_done = h->need_rel = h->nonfinite = 0;
    h->iters = 0;
    h->nsys = nsys;
    h->mixed = mixed;
    h->ticket = 0u;
    h->loops = 0;
  }
}

// after a host-driven reliable update: new residual norms ss2[k]
__global__ void bstate_after_reliable_kernel(BHdr *h, const double *ss2) {
  for (int k = threadIdx.x; k < h->nsys; k += blockDim.x) {
    BState &R = bstate(h)[k];
    R.need_rel = 0;
    R.rmax2 = ss2[k];
    R.since = 0;
    R.ss = ss2[k];
    if (ss2[k] > R.stop2) R.done = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int k = 0; k < h->nsys; k++) all &= bstate(h)[k].done;
    h->need_rel = 0;
    h->all_done = all;
    h->halt = all;
  }
}

template <int PO, int PI>
__global__ void accum_kernel(int Vh, void *outer, const void *inner, const float *iscale) {
  int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= Vh) return;
  using RO = typename SpinorIO<PO>::R;
  Cx<RO> O[12];
  Cx<typename SpinorIO<PI>::R> I[12];
  SpinorIO<PO>::load({outer, nullptr, Vh}, cb, O);
  SpinorIO<PI>::load({(void *)inner, (float *)iscale, Vh}, cb, I);
#pragma unroll
  for (int k = 0; k < 12; k++)
    O[k] = O[k] + Cx<RO>{from_double<RO>(to_double(I[k].re)), from_double<RO>(to_double(I[k].im))};
  SpinorIO<PO>::store({outer, nullptr, Vh}, cb, O);
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

namespace {

struct HostTm {
  HostC A_up, A_dn, Ai_up, Ai_dn;
};
HostTm host_tm(double kappa, double mu, bool dag) {
  double a = 2.0 * kappa * mu;
  if (dag) a = -a;
  double n = 1.0 / (1.0 + a * a);
  return {{1.0, a}, {1.0, -a}, {n, -a * n}, {n, a * n}};
}

struct Buf {
  lqcd_ctx *ctx;
  void *p = nullptr;
  explicit Buf(lqcd_ctx *c) : ctx(c) {}
  Buf(const Buf &) = delete;
  ~Buf() { dfree(ctx, p); }
};

HalfField mk_half(void *ptr, float *scale, int prec, int Vh) {
  HalfField h;
  h.ptr = ptr;
  h.scale = scale;
  h.prec = prec;
  h.nrhs = 1;
  h.rhs_stride = spinor_half_bytes(prec, Vh);
  h.scale_rhs_stride = spinor_scale_half_bytes(prec, Vh) / sizeof(float);
  return h;
}

template <class F>
lqcd_status dispatch(lqcd_ctx *ctx, int prec, F &&f) {
  switch (prec) {
    case LQCD_F64: f(std::integral_constant<int, LQCD_F64>()); break;
    case LQCD_DF64: f(std::integral_constant<int, LQCD_DF64>()); break;
    case LQCD_F32: f(std::integral_constant<int, LQCD_F32>()); break;
    case LQCD_BF16S: f(std::integral_constant<int, LQCD_BF16S>()); break;
    case LQCD_F16S: f(std::integral_constant<int, LQCD_F16S>()); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "bad precision");
  }
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

}  // namespace

lqcd_status check_field(lqcd_ctx *ctx, const lqcd_field &f, const char *name, bool allow_lexi);

lqcd_status cg_solve_batch_impl(lqcd_ctx *ctx, int n, lqcd_gauge *const *U, const lqcd_field *b,
                                const lqcd_field *x, const double *kappa, const double *mu,
                                const lqcd_cg_params &prm, lqcd_cg_stats *st) {
  auto t0 = std::chrono::steady_clock::now();
  const int outer = prm.outer_prec, inner = prm.inner_prec;
  const bool mixed = inner != outer;
  const int irecon = (inner == LQCD_BF16S || inner == LQCD_F16S) ? 12 : prm.sloppy_recon;
  const HostC one{1, 0}, zero{0, 0}, mone{-1, 0};
  for (int k = 0; k < n; k++) std::memset(&st[k], 0, sizeof(lqcd_cg_stats));

  // --- per-system views and workspace -------------------------------------
  struct Sys {
    Geom g;
    int Vh;
    GaugeView U64, Uo, Ui;
    HalfField be, bo, xe, xo;                 // user fields (F64, full-field halves)
    HalfField rhs_e, rhs_o, t64, bhat64, corr_e, corr_o, res_e, res_o;  // F64
    HalfField bhat_o, xout, r_o, tmp_o;       // outer precision
    HalfField s, p, q, z, t, xs;              // inner precision
    double b2;
    long poff;
    int nb;
  };
  std::vector<Sys> S(n);
  std::vector<void *> allocs;
  struct Freer {
    lqcd_ctx *c;
    std::vector<void *> &a;
    ~Freer() {
      for (void *p : a) dfree(c, p);
    }
  } freer{ctx, allocs};
  auto alloc_half = [&](int prec, int Vh, HalfField *h) -> lqcd_status {
    void *p = nullptr;
    float *sc = nullptr;
    LQCD_TRY(dalloc(ctx, &p, spinor_half_bytes(prec, Vh)));
    allocs.push_back(p);
    LQCD_CUDA(ctx, cudaMemsetAsync(p, 0, spinor_half_bytes(prec, Vh), ctx->stream));
    size_t sb = spinor_scale_half_bytes(prec, Vh);
    if (sb) {
      LQCD_TRY(dalloc(ctx, (void **)&sc, sb));
      allocs.push_back(sc);
      LQCD_CUDA(ctx, cudaMemsetAsync(sc, 0, sb, ctx->stream));
    }
    *h = mk_half(p, sc, prec, Vh);
    return LQCD_OK;
  };
  long ptotal = 0;
  int ntiles = 0;
  std::vector<int2> tiles;
  for (int k = 0; k < n; k++) {
    Sys &s = S[k];
    s.g = U[k]->g;
    s.Vh = s.g.Vh;
    LQCD_TRY(gauge_view(ctx, U[k], LQCD_F64, U[k]->recon, &s.U64));
    LQCD_TRY(gauge_view(ctx, U[k], outer, U[k]->recon, &s.Uo));
    LQCD_TRY(gauge_view(ctx, U[k], inner, mixed ? irecon : U[k]->recon, &s.Ui));
    size_t hb = spinor_half_bytes(LQCD_F64, s.Vh);
    s.be = mk_half(b[k].ptr, nullptr, LQCD_F64, s.Vh);
    s.bo = mk_half((char *)b[k].ptr + hb, nullptr, LQCD_F64, s.Vh);
    s.xe = mk_half(x[k].ptr, nullptr, LQCD_F64, s.Vh);
    s.xo = mk_half((char *)x[k].ptr + hb, nullptr, LQCD_F64, s.Vh);
    HalfField *f64s[] = {&s.rhs_e, &s.rhs_o, &s.t64, &s.bhat64, &s.corr_e, &s.corr_o, &s.res_e, &s.res_o};
    for (HalfField *h : f64s) LQCD_TRY(alloc_half(LQCD_F64, s.Vh, h));
    HalfField *outs[] = {&s.bhat_o, &s.xout, &s.r_o, &s.tmp_o};
    for (HalfField *h : outs) LQCD_TRY(alloc_half(outer, s.Vh, h));
    HalfField *ins[] = {&s.s, &s.p, &s.q, &s.z, &s.t};
    for (HalfField *h : ins) LQCD_TRY(alloc_half(inner, s.Vh, h));
    if (mixed) LQCD_TRY(alloc_half(inner, s.Vh, &s.xs));
    else s.xs = s.xout;
    s.nb = (s.Vh + 31) / 32;
    s.poff = ptotal;
    ptotal += s.nb;
    for (int c = 0; c < s.Vh; c += 128) tiles.push_back(make_int2(k, c));
  }
  ntiles = (int)tiles.size();
  LQCD_TRY(ensure_partials(ctx, (size_t)ptotal + 1024));

  // --- device tables ---------------------------------------------------------
  const size_t ha = hop_args_size();
  std::vector<char> hdesc((size_t)4 * n * ha);
  std::vector<VecDesc> vdesc(n);
  std::vector<long> poffs(n);
  std::vector<int> pnbs(n);
  for (int k = 0; k < n; k++) {
    Sys &s = S[k];
    double *part = ctx->partials + s.poff;
    HostTm c = host_tm(kappa[k], mu[k], false), cd = host_tm(kappa[k], mu[k], true);
    double k2 = kappa[k] * kappa[k];
    HopLaunch L;
    L.prec = inner;
    L.recon = mixed ? irecon : U[k]->recon;
    L.U = s.Ui;
    // stage 0: t = -k^2 A^-1 H p     stage 1: q = A p + H t   (partials)
    L.in = s.p; L.out = s.t; L.out_parity = 1; L.dagger = 0;
    L.c_up = {-k2 * c.Ai_up.re, -k2 * c.Ai_up.im};
    L.c_dn = {-k2 * c.Ai_dn.re, -k2 * c.Ai_dn.im};
    L.has_aux = false; L.partials = nullptr;
    hop_args_fill(s.g, L, &hdesc[(0 * n + k) * ha]);
    L.in = s.t; L.out = s.q; L.aux = s.p; L.has_aux = true; L.out_parity = 0;
    L.c_up = L.c_dn = {1.0, 0.0}; L.d_up = c.A_up; L.d_dn = c.A_dn; L.partials = part;
    hop_args_fill(s.g, L, &hdesc[(1 * n + k) * ha]);
    // stage 2: t = -k^2 A^-+ H^+ s   stage 3: z = A^+ s + H^+ t (partials)
    L.in = s.s; L.out = s.t; L.has_aux = false; L.out_parity = 1; L.dagger = 1;
    L.c_up = {-k2 * cd.Ai_up.re, -k2 * cd.Ai_up.im};
    L.c_dn = {-k2 * cd.Ai_dn.re, -k2 * cd.Ai_dn.im};
    L.partials = nullptr;
    hop_args_fill(s.g, L, &hdesc[(2 * n + k) * ha]);
    L.in = s.t; L.out = s.z; L.aux = s.s; L.has_aux = true; L.out_parity = 0;
    L.c_up = L.c_dn = {1.0, 0.0}; L.d_up = cd.A_up; L.d_dn = cd.A_dn; L.partials = part;
    hop_args_fill(s.g, L, &hdesc[(3 * n + k) * ha]);
    VecDesc &v = vdesc[k];
    v.Vh = s.Vh;
    v.x = (char *)s.xs.ptr; v.xs = s.xs.scale;
    v.p = (char *)s.p.ptr; v.ps = s.p.scale;
    v.s = (char *)s.s.ptr; v.ss = s.s.scale;
    v.q = (char *)s.q.ptr; v.qs = s.q.scale;
    v.z = (char *)s.z.ptr; v.zs = s.z.scale;
    v.partials = part;
    poffs[k] = s.poff;
    pnbs[k] = s.nb;
  }
  size_t hdr_bytes = sizeof(BHdr) + sizeof(BState) * n;
  size_t tbl_bytes = hdesc.size() + sizeof(VecDesc) * n + sizeof(int2) * ntiles + sizeof(long) * n +
                     sizeof(int) * n + sizeof(double) * 2 * n + 256 * 6;
  Buf tbl(ctx);
  LQCD_TRY(dalloc(ctx, &tbl.p, hdr_bytes + tbl_bytes));
  char *base = (char *)tbl.p;
  auto carve = [&](size_t bytes) {
    char *p = base;
    base += (bytes + 255) & ~(size_t)255;
    return (void *)p;
  };
  BHdr *h = (BHdr *)carve(hdr_bytes);
  void *d_hdesc = carve(hdesc.size());
  VecDesc *d_vdesc = (VecDesc *)carve(sizeof(VecDesc) * n);
  int2 *d_tiles = (int2 *)carve(sizeof(int2) * ntiles);
  long *d_poff = (long *)carve(sizeof(long) * n);
  int *d_pnb = (int *)carve(sizeof(int) * n);
  double *d_scal = (double *)carve(sizeof(double) * 2 * n);
  LQCD_CUDA(ctx, cudaMemcpyAsync(d_hdesc, hdesc.data(), hdesc.size(), cudaMemcpyHostToDevice, ctx->stream));
  LQCD_CUDA(ctx, cudaMemcpyAsync(d_vdesc, vdesc.data(), sizeof(VecDesc) * n, cudaMemcpyHostToDevice, ctx->stream));
  LQCD_CUDA(ctx, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * ntiles, cudaMemcpyHostToDevice, ctx->stream));
  LQCD_CUDA(ctx, cudaMemcpyAsync(d_poff, poffs.data(), sizeof(long) * n, cudaMemcpyHostToDevice, ctx->stream));
  LQCD_CUDA(ctx, cudaMemcpyAsync(d_pnb, pnbs.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  // host tables must outlive the async copies
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));

  const int grid = std::min(ntiles, ctx->num_sms * 8);
  const char *hd = (const char *)d_hdesc;
  auto stage = [&](int sidx, bool dag, bool red, const int *halt) {
    return launch_hop_batched(ctx, inner, mixed ? irecon : U[0]->recon, dag, red, hd + (size_t)sidx * n * ha,
                              d_tiles, ntiles, grid, halt);
  };
  // counted work of one batched stage
  double sites_total = 0.0, link_total = 0.0;
  for (int k = 0; k < n; k++) {
    sites_total += S[k].Vh;
    link_total += 8.0 * link_bytes_per_site(inner, mixed ? irecon : U[k]->recon) * S[k].Vh;
  }
  const double sbi = spinor_site_bytes(inner);
  auto count_hop = [&](bool aux, bool trivial) {
    double by = link_total + sites_total * sbi * (aux ? 3.0 : 2.0);
    count_launch(ctx, by);
    ctx->cnt.hop_launches++;
    ctx->cnt.hop_bytes += by;
    ctx->cnt.hop_flops += sites_total * (1320.0 + (trivial ? 0.0 : 48.0) + (aux ? 48.0 : 0.0));
    ctx->cnt.hop_sites += sites_total;
  };
  auto fin = [&](int op) {
    bfinalize_kernel<<<n, FIN_THREADS, 0, ctx->stream>>>(h, ctx->partials, d_poff, d_pnb, op);
    count_launch(ctx, 8.0 * ptotal);
  };

  // --- outer refinement cycles -------------------------------------------
  std::vector<double> stop2(n), ss2(n);
  lqcd_status result = LQCD_OK;
  for (int k = 0; k < n; k++) {
    Sys &s = S[k];
    LQCD_CUDA(ctx, cudaMemsetAsync(x[k].ptr, 0, 2 * spinor_half_bytes(LQCD_F64, s.Vh), ctx->stream));
    LQCD_TRY(lincomb(ctx, s.Vh, s.rhs_e, s.be, nullptr, one, one, zero, zero, nullptr, nullptr));
    LQCD_TRY(lincomb(ctx, s.Vh, s.rhs_o, s.bo, nullptr, one, one, zero, zero, nullptr, nullptr));
  }
  // |b_k|^2 (F64, both parities)
  auto norm2_full = [&](int k, const HalfField &e, const HalfField &o, double *out) -> lqcd_status {
    double sum = 0.0;
    for (const HalfField *f : {&e, &o}) {
      int nbv = 0;
      LQCD_TRY(lincomb(ctx, S[k].Vh, S[k].t64, *f, nullptr, one, one, zero, zero, ctx->partials, &nbv));
      LQCD_TRY(ensure_pinned(ctx, nbv));
      LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, ctx->partials, nbv * sizeof(double), cudaMemcpyDeviceToHost,
                                     ctx->stream));
      LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (int i = 0; i < nbv; i++) sum += ctx->pinned[i];
    }
    *out = sum;
    return LQCD_OK;
  };
  for (int k = 0; k < n; k++) {
    LQCD_TRY(norm2_full(k, S[k].be, S[k].bo, &S[k].b2));
    if (!std::isfinite(S[k].b2)) return fail(ctx, LQCD_ERR_NONFINITE, "right-hand side %d is not finite", k);
    stop2[k] = 0.25 * prm.tol * prm.tol * S[k].b2;
  }
  Buf stopd(ctx);
  LQCD_TRY(dalloc(ctx, &stopd.p, sizeof(double) * n));

  for (int cycle = 0;; cycle++) {
    // source preparation per system (F64), then the outer-precision bhat
    for (int k = 0; k < n; k++) {
      Sys &s = S[k];
      HostTm c = host_tm(kappa[k], mu[k], false);
      LQCD_TRY(lincomb(ctx, s.Vh, s.t64, s.rhs_o, nullptr, c.Ai_up, c.Ai_dn, zero, zero, nullptr, nullptr));
      HopLaunch L;
      L.prec = LQCD_F64;
      L.recon = U[k]->recon;
      L.U = s.U64;
      L.in = s.t64;
      L.out = s.bhat64;
      L.aux = s.rhs_e;
      L.has_aux = true;
      L.out_parity = 0;
      L.c_up = L.c_dn = {kappa[k], 0.0};
      L.d_up = L.d_dn = one;
      LQCD_TRY(launch_hop(ctx, s.g, L, nullptr));
      LQCD_TRY(spinor_convert_raw(ctx, s.Vh, 1, s.bhat64.ptr, nullptr, LQCD_F64, s.bhat_o.ptr, nullptr, outer));
      LQCD_CUDA(ctx, cudaMemsetAsync(s.xout.ptr, 0, s.xout.rhs_stride, ctx->stream));
      if (mixed) {
        LQCD_CUDA(ctx, cudaMemsetAsync(s.xs.ptr, 0, s.xs.rhs_stride, ctx->stream));
        LQCD_TRY(spinor_convert_raw(ctx, s.Vh, 1, s.bhat_o.ptr, nullptr, outer, s.s.ptr, s.s.scale, inner));
      } else {
        LQCD_TRY(lincomb(ctx, s.Vh, s.s, s.bhat_o, nullptr, one, one, zero, zero, nullptr, nullptr));
      }
    }
    for (int k = 0; k < n; k++) ctx->pinned[k] = stop2[k];
    LQCD_CUDA(ctx, cudaMemcpyAsync(stopd.p, ctx->pinned, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    bstate_init_kernel<<<1, 256, 0, ctx->stream>>>(h, n, mixed ? 1 : 0, (const double *)stopd.p,
                                                   prm.delta > 0 ? prm.delta : default_delta(inner),
                                                   mixed && inner == LQCD_BF16S ? kBf16Gap : INT_MAX);
    count_launch(ctx, 0.0);
    // z = Mhat^+ s; zz; p = z
    LQCD_TRY(stage(2, true, false, nullptr));
    count_hop(false, false);
    LQCD_TRY(stage(3, true, true, nullptr));
    count_hop(true, true);
    fin(BF_INIT_ZZ);
    for (int k = 0; k < n; k++)
      LQCD_TRY(lincomb(ctx, S[k].Vh, S[k].p, S[k].z, nullptr, one, one, zero, zero, nullptr, nullptr));

    IterWork work;
    auto iteration = [&]() -> lqcd_status {
      const lqcd_counters c0 = ctx->cnt;
      LQCD_TRY(stage(0, false, false, &h->halt));
      count_hop(false, false);
      LQCD_TRY(stage(1, false, true, &h->halt));
      count_hop(true, true);
      fin(BF_ALPHA);
      LQCD_TRY(dispatch(ctx, inner, [&](auto P) {
        bxs_kernel<decltype(P)::value><<<grid, 128, 0, ctx->stream>>>(h, d_vdesc, d_tiles, ntiles);
      }));
      count_launch(ctx, sites_total * sbi * 6.0);
      fin(BF_SS);
      const lqcd_counters cmid = ctx->cnt;  // a halted iteration stops here
      LQCD_TRY(stage(2, true, false, &h->halt));
      count_hop(false, false);
      LQCD_TRY(stage(3, true, true, &h->halt));
      count_hop(true, true);
      fin(BF_BETA);
      LQCD_TRY(dispatch(ctx, inner, [&](auto P) {
        bp_kernel<decltype(P)::value><<<grid, 128, 0, ctx->stream>>>(h, d_vdesc, d_tiles, ntiles);
      }));
      count_launch(ctx, sites_total * sbi * 3.0);
      if (!work.known) {
        work.full = cnt_sub(ctx->cnt, c0);
        work.first = cnt_sub(cmid, c0);
        work.known = true;
      }
      return LQCD_OK;
    };

    const int chunk = prm.check_every > 0 ? prm.check_every : 10;
    SolverGraph graph;
    if (prm.use_graph) LQCD_TRY(build_solver_graph(ctx, chunk, &h->halt, &h->loops, iteration, &graph));

    BHdr hh;
    int reliable = 0, last_rel_iter = 0;
    std::vector<BState> bs(n);
    int iters_seen = 0;  // h->iters at the last poll
    for (;;) {
      lqcd_counters chunk_launches{};
      if (graph.exec) {
        LQCD_CUDA(ctx, cudaGraphLaunch(graph.exec, ctx->stream));
      } else {
        const lqcd_counters c0 = ctx->cnt;
        for (int i = 0; i < chunk; i++) LQCD_TRY(iteration());
        chunk_launches = cnt_sub(ctx->cnt, c0);
        ctx->cnt = c0;
      }
      LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, h, sizeof(BHdr), cudaMemcpyDeviceToHost, ctx->stream));
      LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      std::memcpy(&hh, ctx->pinned, sizeof(hh));
      if (graph.exec) chunk_launches = graph.launches(hh.iters - iters_seen);
      count_chunk(ctx, work, chunk_launches, hh.iters - iters_seen, hh.halt != 0);
      iters_seen = hh.iters;
      if (hh.nonfinite) return fail(ctx, LQCD_ERR_NONFINITE, "batched CG: non-finite scalar");
      const bool finished = hh.all_done != 0;
      // stalled low-precision recursion: force a reliable update and restart p
      const bool stalled = mixed && !finished && !hh.need_rel && hh.iters - last_rel_iter >= 200;
      if (mixed && (hh.need_rel || finished || stalled)) {
        reliable++;
        last_rel_iter = hh.iters;
        bool all_ok = true;
        for (int k = 0; k < n; k++) {
          Sys &s = S[k];
          LQCD_TRY(dispatch(ctx, outer, [&](auto PO) {
            dispatch(ctx, inner, [&](auto PI) {
              accum_kernel<decltype(PO)::value, decltype(PI)::value><<<(s.Vh + 127) / 128, 128, 0, ctx->stream>>>(
                  s.Vh, s.xout.ptr, s.xs.ptr, s.xs.scale);
            });
          }));
          count_launch(ctx, (double)s.Vh * (2.0 * spinor_site_bytes(outer) + sbi));
          LQCD_CUDA(ctx, cudaMemsetAsync(s.xs.ptr, 0, s.xs.rhs_stride, ctx->stream));
          Op oo{ctx, s.g, s.Uo, outer, U[k]->recon, kappa[k], mu[k]};
          LQCD_TRY(apply_schur(oo, s.xout, s.r_o, s.tmp_o, 0, false, nullptr, nullptr, nullptr));
          int nbl = 0;
          LQCD_TRY(lincomb(ctx, s.Vh, s.r_o, s.bhat_o, &s.r_o, one, one, mone, mone, ctx->partials, &nbl));
          LQCD_TRY(ensure_pinned(ctx, nbl + n));
          LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, ctx->partials, nbl * sizeof(double), cudaMemcpyDeviceToHost,
                                         ctx->stream));
          LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
          double sum = 0.0;
          for (int i = 0; i < nbl; i++) sum += ctx->pinned[i];
          ss2[k] = sum;
          if (!(sum <= stop2[k])) all_ok = false;
          LQCD_TRY(spinor_convert_raw(ctx, s.Vh, 1, s.r_o.ptr, nullptr, outer, s.s.ptr, s.s.scale, inner));
        }
        if (finished && all_ok) break;
        for (int k = 0; k < n; k++) ctx->pinned[k] = ss2[k];
        LQCD_CUDA(ctx, cudaMemcpyAsync(d_scal, ctx->pinned, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
        bstate_after_reliable_kernel<<<1, 256, 0, ctx->stream>>>(h, d_scal);
        LQCD_TRY(stage(2, true, false, nullptr));
        count_hop(false, false);
        LQCD_TRY(stage(3, true, true, nullptr));
        count_hop(true, true);
        if (stalled) {  // beta = 0: p = z
          fin(BF_INIT_ZZ);
          for (int k = 0; k < n; k++)
            LQCD_TRY(lincomb(ctx, S[k].Vh, S[k].p, S[k].z, nullptr, one, one, zero, zero, nullptr, nullptr));
        } else {
          fin(BF_BETA);
          LQCD_TRY(dispatch(ctx, inner, [&](auto P) {
            bp_kernel<decltype(P)::value><<<grid, 128, 0, ctx->stream>>>(h, d_vdesc, d_tiles, ntiles);
          }));
        }
        if (hh.iters >= prm.max_iter) {
          result = LQCD_ERR_NOCONV;
          break;
        }
        continue;
      }
      if (finished) break;
      if (hh.iters >= prm.max_iter) {
        result = LQCD_ERR_NOCONV;
        break;
      }
    }
    // per-system statistics, reconstruction and FP64 true residual
    LQCD_CUDA(ctx, cudaMemcpyAsync(bs.data(), (char *)h + sizeof(BHdr), sizeof(BState) * n, cudaMemcpyDeviceToHost,
                                   ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    bool all = true;
    int total_iters = 0;
    for (int k = 0; k < n; k++) {
      Sys &s = S[k];
      st[k].iters += bs[k].iters;
      st[k].reliable_updates += reliable;
      total_iters = std::max(total_iters, st[k].iters);
      if (mixed && result != LQCD_OK) {
        LQCD_TRY(dispatch(ctx, outer, [&](auto PO) {
          dispatch(ctx, inner, [&](auto PI) {
            accum_kernel<decltype(PO)::value, decltype(PI)::value><<<(s.Vh + 127) / 128, 128, 0, ctx->stream>>>(
                s.Vh, s.xout.ptr, s.xs.ptr, s.xs.scale);
          });
        }));
      }
      LQCD_TRY(spinor_convert_raw(ctx, s.Vh, 1, s.xout.ptr, nullptr, outer, s.corr_e.ptr, nullptr, LQCD_F64));
      HostTm c = host_tm(kappa[k], mu[k], false);
      HopLaunch L;
      L.prec = LQCD_F64;
      L.recon = U[k]->recon;
      L.U = s.U64;
      L.in = s.corr_e;
      L.out = s.corr_o;
      L.aux = s.rhs_o;
      L.has_aux = true;
      L.out_parity = 1;
      L.c_up = {kappa[k] * c.Ai_up.re, kappa[k] * c.Ai_up.im};
      L.c_dn = {kappa[k] * c.Ai_dn.re, kappa[k] * c.Ai_dn.im};
      L.d_up = c.Ai_up;
      L.d_dn = c.Ai_dn;
      LQCD_TRY(launch_hop(ctx, s.g, L, nullptr));
      LQCD_TRY(lincomb(ctx, s.Vh, s.xe, s.xe, &s.corr_e, one, one, one, one, nullptr, nullptr));
      LQCD_TRY(lincomb(ctx, s.Vh, s.xo, s.xo, &s.corr_o, one, one, one, one, nullptr, nullptr));
      Op o64{ctx, s.g, s.U64, LQCD_F64, U[k]->recon, kappa[k], mu[k]};
      LQCD_TRY(apply_full(o64, s.xe, s.xo, s.res_e, s.res_o, false, nullptr, nullptr, nullptr));
      LQCD_TRY(lincomb(ctx, s.Vh, s.rhs_e, s.be, &s.res_e, one, one, mone, mone, nullptr, nullptr));
      LQCD_TRY(lincomb(ctx, s.Vh, s.rhs_o, s.bo, &s.res_o, one, one, mone, mone, nullptr, nullptr));
      double r2;
      LQCD_TRY(norm2_full(k, s.rhs_e, s.rhs_o, &r2));
      st[k].true_resid = s.b2 > 0.0 ? std::sqrt(r2 / s.b2) : std::sqrt(r2);  // b = 0: x = 0
      st[k].converged = st[k].true_resid <= prm.tol;
      if (!std::isfinite(st[k].true_resid)) return fail(ctx, LQCD_ERR_NONFINITE, "true residual not finite");
      all = all && st[k].converged;
    }
    if (all) {
      result = LQCD_OK;
      break;
    }
    if (cycle >= prm.max_restarts || total_iters >= prm.max_iter) {
      result = LQCD_ERR_NOCONV;
      break;
    }
    result = LQCD_OK;
    for (int k = 0; k < n; k++) {
      if (st[k].converged) {  // zero correction for converged systems
        LQCD_CUDA(ctx, cudaMemsetAsync(S[k].rhs_e.ptr, 0, S[k].rhs_e.rhs_stride, ctx->stream));
        LQCD_CUDA(ctx, cudaMemsetAsync(S[k].rhs_o.ptr, 0, S[k].rhs_o.rhs_stride, ctx->stream));
      } else {
        st[k].restarts++;
      }
    }
  }
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int k = 0; k < n; k++) st[k].seconds = secs;
  if (result == LQCD_ERR_NOCONV) fail(ctx, LQCD_ERR_NOCONV, "batched CG did not reach tol");
  return result;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_cg_solve_batch(lqcd_ctx *ctx, int n, const lqcd_gauge *const *U, const lqcd_field *b,
                                   const lqcd_field *x, const double *kappa, const double *mu,
                                   const lqcd_cg_params *params, lqcd_cg_stats *stats) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (n < 1 || n > 4096) return fail(ctx, LQCD_ERR_INVALID, "n out of [1, 4096]");
  if (!U || !b || !x || !kappa || !mu || !params || !stats) return fail(ctx, LQCD_ERR_INVALID, "NULL array");
  const lqcd_cg_params &p = *params;
  if (!(p.tol > 0.0) || p.max_iter < 1 || p.max_restarts < 0) return fail(ctx, LQCD_ERR_INVALID, "bad params");
  if (p.solver != LQCD_SOLVER_CG) return fail(ctx, LQCD_ERR_UNSUPPORTED, "the batched solver is CG only");
  if (p.outer_prec != LQCD_F64 && p.outer_prec != LQCD_DF64) return fail(ctx, LQCD_ERR_INVALID, "bad outer_prec");
  if (p.inner_prec < LQCD_F64 || p.inner_prec > LQCD_F16S) return fail(ctx, LQCD_ERR_INVALID, "bad inner_prec");
  if (p.inner_prec == LQCD_F64 && p.outer_prec != LQCD_F64) return fail(ctx, LQCD_ERR_INVALID, "inner F64 needs outer F64");
  std::vector<lqcd_gauge *> Us(n);
  for (int k = 0; k < n; k++) {
    if (!U[k]) return fail(ctx, LQCD_ERR_INVALID, "U[%d] is NULL", k);
    LQCD_TRY(check_field(ctx, b[k], "b", false));
    LQCD_TRY(check_field(ctx, x[k], "x", false));
    if (b[k].prec != LQCD_F64 || x[k].prec != LQCD_F64 || b[k].nrhs != 1 || x[k].nrhs != 1)
      return fail(ctx, LQCD_ERR_INVALID, "batched fields must be single F64 EO full fields");
    if (!std::isfinite(kappa[k]) || !std::isfinite(mu[k])) return fail(ctx, LQCD_ERR_NONFINITE, "kappa/mu");
    if (U[k]->recon != U[0]->recon) return fail(ctx, LQCD_ERR_INVALID, "all gauge fields need the same recon");
    Us[k] = const_cast<lqcd_gauge *>(U[k]);
  }
  lqcd_cg_params prm = p;
  if (prm.sloppy_recon == 0) prm.sloppy_recon = U[0]->recon;
  if (prm.check_every <= 0) prm.check_every = 10;
  return cg_solve_batch_impl(ctx, n, Us.data(), b, x, kappa, mu, prm, stats);
}
