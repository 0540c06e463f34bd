// cg.cu -- even-odd preconditioned CG (Sec. 2.1: "D phi = psi", "the most
// common solvers used are CG and BiCGStab", "even-odd-preconditioning").
//
// The system M x = b is reduced to the even sites (Schur complement
//   Mhat = A_e - kappa^2 H_eo A_o^-1 H_oe,   A = 1 + i a gamma_5, a = 2 kappa mu)
// with bhat_e = b_e + kappa H_eo A_o^-1 b_o and x_o = A_o^-1 (b_o + kappa H_oe x_e),
// and Mhat x_e = bhat_e is solved by CG on the normal equations in CGLS form,
// which keeps the residual s = bhat - Mhat x of the unsquared system:
//   q = Mhat p;  alpha = |z|^2/|q|^2;  x += alpha p;  s -= alpha q;
//   z = Mhat^+ s;  beta = |z_new|^2/|z|^2;  p = z + beta p.
// It stops when |s| <= tol |b| (|b| of the full system: the full residual is
// (s, 0) exactly), then the true residual |b - M x| / |b| is recomputed with
// the full FP64 operator.
//
// Mixed precision (the paper's outlook, Sec. 5 and 6): the recursion runs in
// a sloppy format (F32, or BF16/F16 with per-site scale) while x and the
// residual are kept in the outer FP64-class format (F64 or DF64).  A reliable
// update (Sleijpen & van der Vorst) folds the sloppy x into the outer x and
// replaces s by the outer-precision residual whenever |s| has dropped below
// delta times its largest value since the last update; p is kept.  Outer
// iterative refinement restarts the whole solve on the true residual.
//
// GB300 execution: every scalar (alpha, beta, norms, convergence flags) lives
// in device memory, so an iteration is six kernel launches with no host
// round trip; check_every iterations are captured once in a CUDA graph and
// replayed; the host reads a status word after each replay.  Reductions are
// FP64 partial sums per block finished by one block in a fixed order, so the
// iteration count is reproducible run to run.
#include <chrono>
#include <climits>
#include <complex>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "internal.h"

namespace lqcd {


// ---------------------------------------------------------------------------
// device solver state
// ---------------------------------------------------------------------------

struct RhsState {
  double zz, qq, ss, alpha, beta, stop2, rel2, rmax2;
  int done, iters, need_rel;
  int since, gap;  // iterations since the last reliable update, and its cap
};
struct SolverHdr {
  int halt, all_done, need_rel, nonfinite;
  int iters, nrhs, mixed;
  unsigned ticket;  // blocks of the current finalize that have finished
  int loops, pad;   // pass counter of the graph's device-side loop
};
// layout in device memory: SolverHdr, then RhsState[nrhs]
LQCD_DEV RhsState *rhs_state(SolverHdr *h) { return (RhsState *)(h + 1); }

// FIN_SS_BETA: FIN_SS, then (by the last block, for every right-hand side,
// unless the step halted the solve) FIN_BETA on the same sums -- the
// normal-equation iteration reduces one vector for both
enum { FIN_ALPHA = 0, FIN_SS = 1, FIN_BETA = 2, FIN_INIT_ZZ = 3, FIN_STORE = 4, FIN_SS_BETA = 5 };

// One block per right-hand side finishes its reduction and applies the CG
// scalar step `op`; the last block to finish (ticket) sets the flags over all
// right-hand sides.  FIN_STORE only writes the plain sums to out[r] and does
// not touch the solver state.
__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel(SolverHdr *h, int nrhs, const double *partials,
                                                              int nb, int op, double *out) {
  pdl_wait();
  __shared__ double sh[33];
  __shared__ int last;
  const int r = blockIdx.x;  // one block per right-hand side
  const double v = (op == FIN_STORE || op == FIN_INIT_ZZ || !*(volatile int *)&h->halt)
                       ? block_sum_fixed(partials + (size_t)r * nb, nb, sh)
                       : 0.0;
  if (op == FIN_STORE) {
    if (threadIdx.x == 0) out[r] = v;
    return;
  }
  if (op != FIN_INIT_ZZ && *(volatile int *)&h->halt) return;
  RhsState *rs = rhs_state(h);
  if (threadIdx.x == 0) {
    RhsState &R = rs[r];
    int bad = !isfinite(v);
    switch (op) {
      case FIN_ALPHA:
        R.qq = v;
        if (R.done) R.alpha = 0.0;
        else if (v > 0.0) R.alpha = R.zz / v;
        else { R.alpha = 0.0; if (R.zz > 0.0) bad = 1; }
        break;
      case FIN_SS:
      case FIN_SS_BETA:
        R.ss = v;
        if (!R.done) {
          R.iters += 1;
          if (v <= R.stop2) R.done = 1;
          if (h->mixed && !R.done) {
            if (v > R.rmax2) R.rmax2 = v;
            R.since += 1;
            if (v < R.rel2 * R.rmax2 || R.since >= R.gap) R.need_rel = 1;
          }
        }
        break;
      case FIN_BETA:
        if (R.done) R.beta = 0.0;
        else R.beta = R.zz > 0.0 ? v / R.zz : 0.0;
        R.zz = v;
        break;
      default:  // FIN_INIT_ZZ
        R.zz = v;
        break;
    }
    if (bad) atomicOr(&h->nonfinite, 1);
    __threadfence();
    last = atomicAdd(&h->ticket, 1u) == (unsigned)(nrhs - 1);
  }
  __syncthreads();
  // the last block to finish sets the flags over all right-hand sides
  if (last && threadIdx.x == 0) {
    __threadfence();
    int all_done = 1, any_rel = 0, maxit = 0;
    for (int k = 0; k < nrhs; k++) {
      const volatile RhsState &R = rs[k];
      all_done &= R.done;
      any_rel |= R.need_rel;
      if (R.iters > maxit) maxit = R.iters;
    }
    h->iters = maxit;
    h->all_done = all_done;
    h->need_rel = any_rel;
    if ((op == FIN_SS || op == FIN_SS_BETA) && (all_done || any_rel)) h->halt = 1;
    if (*(volatile int *)&h->nonfinite) h->halt = 1;
    if (op == FIN_SS_BETA && !h->halt)
      for (int k = 0; k < nrhs; k++) {  // FIN_BETA with v = |z|^2 = ss
        volatile RhsState &R = rs[k];
        const double ss = R.ss, zz = R.zz;
        R.beta = R.done ? 0.0 : (zz > 0.0 ? ss / zz : 0.0);
        R.zz = ss;
      }
    h->ticket = 0u;
  }
}


static void launch_finalize(lqcd_ctx *ctx, SolverHdr *h, int nrhs, int nb, int op, double *out) {
  launch_pdl(finalize_kernel, dim3(nrhs), dim3(FIN_THREADS), 0, ctx->stream, h, nrhs, (const double *)ctx->partials,
             nb, op, out);
  count_launch(ctx, 8.0 * nb * nrhs);
}

// Last kernel of a loop pass: ends the while loop once the solver halted or
// after `cap` passes (the pass counter goes back to zero for the next launch).
__global__ void loop_ctl_kernel(const int *halt, int *loops, cudaGraphConditionalHandle cond, int cap) {
  const int n = *loops + 1;
  if (*(volatile const int *)halt || n >= cap) {
    *loops = 0;
    cudaGraphSetConditional(cond, 0);
  } else {
    *loops = n;
  }
}

// The device-side loop: a graph with one conditional while node (condition
// 1 at every launch) whose body is captured from one iteration and the
// control kernel.  Returns false (and leaves nothing behind) if the driver
// rejects any step; *cs receives a failure of the iteration itself.
static bool build_loop_graph(lqcd_ctx *ctx, cudaStream_t cap, int chunk, const int *halt, int *loops,
                             const std::function<lqcd_status()> &iteration, SolverGraph *G, lqcd_status *cs) {
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle cond;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  // zero-filled storage: the parameter union has no default constructor and
  // its unused bytes must be zero
  alignas(cudaGraphNodeParams) unsigned char np_bytes[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_bytes);
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      cudaStream_t saved = ctx->stream;
      ctx->stream = cap;
      *cs = iteration();
      if (*cs == LQCD_OK) {
        loop_ctl_kernel<<<1, 1, 0, cap>>>(halt, loops, cond, chunk);
        count_launch(ctx, 0.0);
      }
      ctx->stream = saved;
      cudaGraph_t out = body;
      ok = cudaStreamEndCapture(cap, &out) == cudaSuccess && *cs == LQCD_OK;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&G->exec, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    G->exec = nullptr;
    if (g) cudaGraphDestroy(g);
    return false;
  }
  G->graph = g;
  G->loop = true;
  return true;
}

lqcd_status build_solver_graph(lqcd_ctx *ctx, int chunk, const int *halt, int *loops,
                               const std::function<lqcd_status()> &iteration, SolverGraph *G) {
  cudaStream_t cap;
  LQCD_CUDA(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const lqcd_counters before = ctx->cnt;
  lqcd_status cs = LQCD_OK;
  bool ok = build_loop_graph(ctx, cap, chunk, halt, loops, iteration, G, &cs);
  if (!ok) {
    // unrolled chunk of iterations
    ctx->cnt = before;
    cs = LQCD_OK;
    cudaGraph_t g = nullptr;
    cudaStream_t saved = ctx->stream;
    ctx->stream = cap;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k = 0; k < chunk && cs == LQCD_OK; k++) cs = iteration();
      e = cudaStreamEndCapture(cap, &g);
    }
    ctx->stream = saved;
    if (e == cudaSuccess && cs == LQCD_OK) e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess || cs != LQCD_OK) {
      G->exec = nullptr;
      if (g) cudaGraphDestroy(g);
      ctx->cnt = before;
      cudaStreamDestroy(cap);
      if (cs != LQCD_OK) return cs;
      return cuda_check(ctx, e, "solver graph capture");
    }
    G->graph = g;
  }
  // the capture executed nothing: its launch counts are the per-pass increment
  G->per_pass = cnt_sub(ctx->cnt, before);
  ctx->cnt = before;
  cudaStreamDestroy(cap);
  return LQCD_OK;
}

// ---------------------------------------------------------------------------
// BLAS-1 kernels on half fields with nrhs right-hand sides (grid.y = rhs)
// ---------------------------------------------------------------------------

struct VecArgs {
  int Vh;
  size_t rs, srs;  // bytes / scale floats per rhs (same precision for all operands)
};

LQCD_DEV SpinorView sv(const VecArgs &a, const void *p, const float *s, int r) {
  return SpinorView{(char *)p + r * a.rs, s ? (float *)s + r * a.srs : nullptr, a.Vh};
}

LQCD_DEV double warp_block_sum(double v, double *sh) {
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

// x += alpha p;  s -= alpha q;  partial |s|^2
template <int P>
__global__ void __launch_bounds__(128) cg_xs_kernel(VecArgs a, SolverHdr *h, void *x, float *xs,
                                                    const void *p, const float *ps, void *s,
                                                    float *ss, const void *q, const float *qs,
                                                    double *partials) {
  pdl_wait();
  using R = typename SpinorIO<P>::R;
  __shared__ double sh[8];
  if (*(volatile int *)&h->halt) return;
  int cb = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  double nrm = 0.0;
  if (cb < a.Vh) {
    const R al = from_double<R>(rhs_state(h)[r].alpha);
    Cx<R> X[12], Pp[12], S[12], Q[12];
    SpinorIO<P>::load(sv(a, x, xs, r), cb, X);
    SpinorIO<P>::load(sv(a, p, ps, r), cb, Pp);
    SpinorIO<P>::load(sv(a, s, ss, r), cb, S);
    SpinorIO<P>::load(sv(a, q, qs, r), cb, Q);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      X[k] = {rfma(al, Pp[k].re, X[k].re), rfma(al, Pp[k].im, X[k].im)};
      S[k] = {rfma(-al, Q[k].re, S[k].re), rfma(-al, Q[k].im, S[k].im)};
    }
    nrm = site_norm2<R, 12>(S);
    SpinorIO<P>::store(sv(a, x, xs, r), cb, X);
    SpinorIO<P>::store(sv(a, s, ss, r), cb, S);
  }
  // one partial per warp of 32 sites (the grouping of the hop kernels and of
  // the batched solver, so all of them reduce in the same order)
  (void)sh;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0 && cb < a.Vh) partials[(size_t)r * ((a.Vh + 31) >> 5) + (cb >> 5)] = nrm;
}

// p = z + beta p
template <int P>
__global__ void __launch_bounds__(128) cg_p_kernel(VecArgs a, SolverHdr *h, void *p, float *ps,
                                                   const void *z, const float *zs) {
  pdl_wait();
  using R = typename SpinorIO<P>::R;
  if (*(volatile int *)&h->halt) return;
  int cb = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (cb >= a.Vh) return;
  const R be = from_double<R>(rhs_state(h)[r].beta);
  Cx<R> Pp[12], Z[12];
  SpinorIO<P>::load(sv(a, p, ps, r), cb, Pp);
  SpinorIO<P>::load(sv(a, z, zs, r), cb, Z);
#pragma unroll
  for (int k = 0; k < 12; k++) Pp[k] = {rfma(be, Pp[k].re, Z[k].re), rfma(be, Pp[k].im, Z[k].im)};
  SpinorIO<P>::store(sv(a, p, ps, r), cb, Pp);
}

// out = ca x + cb y (host scalars, per chirality complex), optional |out|^2 partials
template <int P>
// (each operand has its own right-hand-side stride: a for out, ax for x, ay for y)
__global__ void __launch_bounds__(128) lincomb_kernel(VecArgs a, VecArgs ax, VecArgs ay, void *out,
                                                      float *os, const void *x, const float *xsc,
                                                      const void *y, const float *ysc, Coef4 co, int unit,
                                                      double *partials) {
  using R = typename SpinorIO<P>::R;
  __shared__ double sh[8];
  int cb = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  double nrm = 0.0;
  if (cb < a.Vh) {
    Cx<R> X[12], Y[12];
    SpinorIO<P>::load(sv(ax, x, xsc, r), cb, X);
    if (y) SpinorIO<P>::load(sv(ay, y, ysc, r), cb, Y);
    if (unit) {
      // ca = 1 and cb = +-1 (copies, residuals b - q): no multiplications
      if (y) {
#pragma unroll
        for (int k = 0; k < 12; k++) X[k] = unit > 0 ? X[k] + Y[k] : X[k] - Y[k];
      }
    } else {
      const Cx<R> au = coef_of<R>(co, 0), ad = coef_of<R>(co, 1), bu = coef_of<R>(co, 2), bd = coef_of<R>(co, 3);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        Cx<R> o = (k < 6 ? au : ad) * X[k];
        if (y) o = cmadd(k < 6 ? bu : bd, Y[k], o);
        X[k] = o;
      }
    }
    nrm = site_norm2<R, 12>(X);
    SpinorIO<P>::store(sv(a, out, os, r), cb, X);
  }
  if (partials) {
    double t = warp_block_sum(nrm, sh);
    if (threadIdx.x == 0) partials[(size_t)r * gridDim.x + blockIdx.x] = t;
  }
}

// outer += convert(inner) (F64/DF64 outer, any inner precision)
template <int PO, int PI>
__global__ void __launch_bounds__(128) accum_convert_kernel(int Vh, size_t ors, size_t irs,
                                                            size_t isrs, void *outer, const void *inner,
                                                            const float *iscale) {
  using RO = typename SpinorIO<PO>::R;
  int cb = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (cb >= Vh) return;
  Cx<RO> O[12];
  Cx<typename SpinorIO<PI>::R> I[12];
  SpinorView vo{(char *)outer + r * ors, nullptr, Vh};
  SpinorView vi{(char *)inner + r * irs, iscale ? (float *)iscale + r * isrs : nullptr, Vh};
  SpinorIO<PO>::load(vo, cb, O);
  SpinorIO<PI>::load(vi, cb, I);
#pragma unroll
  for (int k = 0; k < 12; k++)
    O[k] = O[k] + Cx<RO>{from_double<RO>(to_double(I[k].re)), from_double<RO>(to_double(I[k].im))};
  SpinorIO<PO>::store(vo, cb, O);
}

__global__ void state_init_kernel(SolverHdr *h, int nrhs, int mixed, const double *b2, double tol,
                                  double rel, int gap) {
  int r = threadIdx.x;
  if (r == 0) {
    h->halt = 0;
    h->all_done = 0;
    h->need_rel = 0;
    h->nonfinite = 0;
    h->iters = 0;
    h->nrhs = nrhs;
    h->mixed = mixed;
    h->ticket = 0u;
    h->loops = 0;
  }
  if (r < nrhs) {
    RhsState &R = rhs_state(h)[r];
    R.zz = R.qq = R.ss = R.alpha = R.beta = 0.0;
    R.stop2 = tol * tol * b2[r];
    R.rel2 = rel * rel;
    R.rmax2 = 0.0;
    R.done = 0;
    R.iters = 0;
    R.need_rel = 0;
    R.since = 0;
    R.gap = gap;
  }
}

// After a reliable update: new residual norms, reset triggers, beta from the
// new z.  ss2[r] = |s|^2 of the recomputed residual.
__global__ void state_after_reliable_kernel(SolverHdr *h, const double *ss2) {
  int r = threadIdx.x;
  if (r < h->nrhs) {
    RhsState &R = rhs_state(h)[r];
    R.need_rel = 0;
    R.rmax2 = ss2[r];
    R.since = 0;
    R.ss = ss2[r];
    if (ss2[r] > R.stop2) R.done = 0;
  }
  __syncthreads();
  if (r == 0) {
    h->need_rel = 0;
    h->halt = 0;
    int ad = 1;
    for (int k = 0; k < h->nrhs; k++) ad &= rhs_state(h)[k].done;
    h->all_done = ad;
    if (ad) h->halt = 1;
  }
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------


struct TmCoef {  // per-chirality coefficients of A = 1 + i a g5 and friends
  HostC A_up, A_dn, Ai_up, Ai_dn;
};
static TmCoef tm_coef(double kappa, double mu, bool dagger) {
  double a = 2.0 * kappa * mu;
  if (dagger) a = -a;  // A^+ = 1 - i a g5, A^-+ = (1 + i a g5)/(1 + a^2)
  double n = 1.0 / (1.0 + a * a);
  return {{1.0, a}, {1.0, -a}, {n, -a * n}, {n, a * n}};
}

// Spinor workspace vector of nrhs half fields in precision prec.
struct Vec {
  HalfField f;
  lqcd_ctx *ctx = nullptr;
  Vec() = default;
  Vec(const Vec &) = delete;
  Vec &operator=(const Vec &) = delete;
  ~Vec() {
    if (ctx) {
      dfree(ctx, f.ptr);
      dfree(ctx, f.scale);
    }
  }
  lqcd_status alloc(lqcd_ctx *c, int prec, int Vh, int nrhs) {
    ctx = c;
    f.prec = prec;
    f.nrhs = nrhs;
    f.rhs_stride = spinor_half_bytes(prec, Vh);
    f.scale_rhs_stride = spinor_scale_half_bytes(prec, Vh) / sizeof(float);
    LQCD_TRY(dalloc(c, &f.ptr, f.rhs_stride * nrhs));
    if (f.scale_rhs_stride) LQCD_TRY(dalloc(c, (void **)&f.scale, f.scale_rhs_stride * sizeof(float) * nrhs));
    LQCD_CUDA(c, cudaMemsetAsync(f.ptr, 0, f.rhs_stride * nrhs, c->stream));
    if (f.scale)
      LQCD_CUDA(c, cudaMemsetAsync(f.scale, 0, f.scale_rhs_stride * sizeof(float) * nrhs, c->stream));
    return LQCD_OK;
  }
};

static VecArgs vargs(const HalfField &f, int Vh) { return VecArgs{Vh, f.rhs_stride, f.scale_rhs_stride}; }

template <class F>
static lqcd_status dispatch_prec(lqcd_ctx *ctx, int prec, F &&f) {
  switch (prec) {
    case LQCD_F64: f(std::integral_constant<int, LQCD_F64>()); break;
    case LQCD_DF64: f(std::integral_constant<int, LQCD_DF64>()); break;
    case LQCD_F32: f(std::integral_constant<int, LQCD_F32>()); break;
    case LQCD_BF16S: f(std::integral_constant<int, LQCD_BF16S>()); break;
    case LQCD_F16S: f(std::integral_constant<int, LQCD_F16S>()); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "bad precision %d", prec);
  }
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lincomb(lqcd_ctx *ctx, int Vh, const HalfField &out, const HalfField &x, const HalfField *y,
                    HostC ca_up, HostC ca_dn, HostC cb_up, HostC cb_dn, double *partials,
                    int *nb_out) {
  dim3 grid((Vh + 127) / 128, out.nrhs);
  if (nb_out) *nb_out = grid.x;
  if (x.prec != out.prec || (y && y->prec != out.prec) || x.nrhs != out.nrhs || (y && y->nrhs != out.nrhs))
    return fail(ctx, LQCD_ERR_INVALID, "lincomb: operand precision or nrhs mismatch");
  VecArgs a = vargs(out, Vh), ax = vargs(x, Vh), ay = y ? vargs(*y, Vh) : a;
  count_launch(ctx, (double)Vh * out.nrhs * spinor_site_bytes(out.prec) * (y ? 3.0 : 2.0));
  auto is = [](HostC c, double v) { return c.re == v && c.im == 0.0; };
  int unit = 0;  // +1: x + y (or x alone), -1: x - y
  if (is(ca_up, 1.0) && is(ca_dn, 1.0)) {
    if (!y) unit = 1;
    else if (is(cb_up, 1.0) && is(cb_dn, 1.0)) unit = 1;
    else if (is(cb_up, -1.0) && is(cb_dn, -1.0)) unit = -1;
  }
  return dispatch_prec(ctx, out.prec, [&](auto P) {
    lincomb_kernel<decltype(P)::value><<<grid, 128, 0, ctx->stream>>>(
        a, ax, ay, out.ptr, out.scale, x.ptr, x.scale, y ? y->ptr : nullptr, y ? y->scale : nullptr,
        make_coef4(ca_up, ca_dn, cb_up, cb_dn), unit, partials);
  });
}

// sums partials[r][0..nb) into the pinned host array (synchronous)
static lqcd_status host_sums(lqcd_ctx *ctx, SolverHdr *h, int nb, int nrhs, double *dst_dev,
                             std::vector<double> *host) {
  launch_finalize(ctx, h, nrhs, nb, FIN_STORE, dst_dev);
  LQCD_CUDA(ctx, cudaGetLastError());
  if (host) {
    LQCD_TRY(ensure_pinned(ctx, nrhs));
    LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, dst_dev, nrhs * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    host->assign(ctx->pinned, ctx->pinned + nrhs);
  }
  return LQCD_OK;
}

// ---------------------------------------------------------------------------
// Schur-complement operator in one precision: out_e = Mhat (or Mhat^+) in_e
// (parity p = 0 even, 1 odd), tmp: half field of the other parity.
// ---------------------------------------------------------------------------


lqcd_status apply_schur(const Op &op, const HalfField &in, const HalfField &out, const HalfField &tmp,
                        int p, bool dagger, double *partials, int *nb, int *halt) {
  TmCoef c = tm_coef(op.kappa, op.mu, dagger);
  HopLaunch L1;
  L1.prec = op.prec;
  L1.recon = op.recon;
  L1.U = op.U;
  L1.in = in;
  L1.out = tmp;
  L1.out_parity = p ^ 1;
  L1.dagger = dagger;
  // -kappa^2 is folded into the first hop's factor, so the second hop's
  // epilogue is out = H tmp + A in with no multiplication of the hop sum
  const double k2 = op.kappa * op.kappa;
  L1.c_up = {-k2 * c.Ai_up.re, -k2 * c.Ai_up.im};
  L1.c_dn = {-k2 * c.Ai_dn.re, -k2 * c.Ai_dn.im};
  L1.halt = halt;
  LQCD_TRY(launch_hop(op.ctx, op.g, L1, nullptr));
  HopLaunch L2 = L1;
  L2.in = tmp;
  L2.out = out;
  L2.aux = in;
  L2.has_aux = true;
  L2.out_parity = p;
  L2.c_up = {1.0, 0.0};
  L2.c_dn = {1.0, 0.0};
  L2.d_up = c.A_up;
  L2.d_dn = c.A_dn;
  L2.partials = partials;
  return launch_hop(op.ctx, op.g, L2, nb);
}

// full M (or M^+) on an EO full field: both parities, out_p = A in_p - kappa H in_{1-p}
lqcd_status apply_full(const Op &op, const HalfField &in_e, const HalfField &in_o, const HalfField &out_e,
                       const HalfField &out_o, bool dagger, double *partials_e, double *partials_o,
                       int *nb) {
  TmCoef c = tm_coef(op.kappa, op.mu, dagger);
  for (int p = 0; p < 2; p++) {
    HopLaunch L;
    L.prec = op.prec;
    L.recon = op.recon;
    L.U = op.U;
    L.in = p == 0 ? in_o : in_e;
    L.out = p == 0 ? out_e : out_o;
    L.aux = p == 0 ? in_e : in_o;
    L.has_aux = true;
    L.out_parity = p;
    L.dagger = dagger;
    L.c_up = {-op.kappa, 0.0};
    L.c_dn = {-op.kappa, 0.0};
    L.d_up = c.A_up;
    L.d_dn = c.A_dn;
    L.partials = p == 0 ? partials_e : partials_o;
    LQCD_TRY(launch_hop(op.ctx, op.g, L, nb));
  }
  return LQCD_OK;
}

static HalfField half_of(const HalfField &full, int p, int Vh) {
  // full field [nrhs][2][..]: parity p half with rhs stride of the full field
  HalfField h = full;
  size_t hb = spinor_half_bytes(full.prec, Vh);
  h.ptr = (char *)full.ptr + p * hb;
  if (full.scale) h.scale = full.scale + (size_t)p * Vh;
  return h;
}

// ---------------------------------------------------------------------------
// The solver
// ---------------------------------------------------------------------------

struct CgWork {
  // outer-precision even vectors
  Vec bhat, xo, r, tmpo, yo;
  // sloppy vectors
  Vec xs, s, p, q, z, t;
};

static lqcd_status ensure_state(lqcd_ctx *ctx, int nrhs, SolverHdr **h) {
  size_t need = sizeof(SolverHdr) + sizeof(RhsState) * nrhs + sizeof(double) * 4 * nrhs;
  if (ctx->solver_state_cap < need) {
    if (ctx->solver_state) {
      cudaStreamSynchronize(ctx->stream);
      dfree(ctx, ctx->solver_state);
    }
    ctx->solver_state = nullptr;
    ctx->solver_state_cap = 0;
    LQCD_TRY(dalloc(ctx, &ctx->solver_state, need));
    ctx->solver_state_cap = need;
  }
  *h = (SolverHdr *)ctx->solver_state;
  return LQCD_OK;
}
static double *state_scratch(SolverHdr *h, int nrhs, int k) {  // 4 double arrays [nrhs]
  return (double *)((char *)h + sizeof(SolverHdr) + sizeof(RhsState) * nrhs) + (size_t)k * nrhs;
}

// Solves Mhat x_e = bhat_e for all right-hand sides; x_e (outer precision)
// must be zero on entry.  b2[r] = |b_r|^2 of the full system (stop criterion).
lqcd_status cgls_even(lqcd_ctx *ctx, lqcd_gauge *U, const Geom &g, double kappa, double mu,
                             const lqcd_cg_params &prm, const HalfField &bhat, const HalfField &xo,
                             const std::vector<double> &b2, lqcd_cg_stats *st, int nrhs,
                             int *iters_used, bool normal) {
  const int Vh = g.Vh;
  const int outer = prm.outer_prec, inner = prm.inner_prec;
  const bool mixed = inner != outer;
  Op Oo{ctx, g, {}, outer, U->recon, kappa, mu};
  LQCD_TRY(gauge_view(ctx, U, outer, U->recon, &Oo.U));
  Op Oi = Oo;
  if (mixed) {
    Oi.prec = inner;
    Oi.recon = (inner == LQCD_BF16S || inner == LQCD_F16S) ? 12 : prm.sloppy_recon;
    LQCD_TRY(gauge_view(ctx, U, inner, Oi.recon, &Oi.U));
  }
  Vec s, p, q, z, t, xs, r_o, tmp_o, y_o;
  LQCD_TRY(s.alloc(ctx, inner, Vh, nrhs));
  LQCD_TRY(p.alloc(ctx, inner, Vh, nrhs));
  LQCD_TRY(q.alloc(ctx, inner, Vh, nrhs));
  LQCD_TRY(z.alloc(ctx, inner, Vh, nrhs));
  LQCD_TRY(t.alloc(ctx, inner, Vh, nrhs));
  HalfField X = xo;  // sloppy x: the outer x itself when not mixed
  if (mixed) {
    LQCD_TRY(xs.alloc(ctx, inner, Vh, nrhs));
    LQCD_TRY(r_o.alloc(ctx, outer, Vh, nrhs));
    LQCD_TRY(tmp_o.alloc(ctx, outer, Vh, nrhs));
    if (normal) LQCD_TRY(y_o.alloc(ctx, outer, Vh, nrhs));
    X = xs.f;
  }
  int nb = hop_blocks(g, nrhs);
  int nbv = (Vh + 127) / 128;
  const int nbw = (Vh + 31) / 32;  // per-warp partials of cg_xs_kernel
  LQCD_TRY(ensure_partials(ctx, (size_t)nrhs * (nb > nbv ? nb : nbv)));
  SolverHdr *h;
  LQCD_TRY(ensure_state(ctx, nrhs, &h));
  double *b2d = state_scratch(h, nrhs, 0), *tmpd = state_scratch(h, nrhs, 1);
  LQCD_TRY(ensure_pinned(ctx, 64 + 4 * nrhs));
  for (int r = 0; r < nrhs; r++) ctx->pinned[r] = b2[r];
  LQCD_CUDA(ctx, cudaMemcpyAsync(b2d, ctx->pinned, nrhs * sizeof(double), cudaMemcpyHostToDevice,
                                 ctx->stream));
  state_init_kernel<<<1, 64, 0, ctx->stream>>>(h, nrhs, mixed ? 1 : 0, b2d, prm.tol * 0.5,
                                               prm.delta > 0 ? prm.delta : default_delta(inner),
                                               mixed && inner == LQCD_BF16S ? kBf16Gap : INT_MAX);
  LQCD_CUDA(ctx, cudaGetLastError());
  const HostC one{1, 0}, zero{0, 0}, mone{-1, 0};
  if (!normal) {
    // s = bhat (converted to the sloppy format); z = Mhat^+ s, p = z, zz = |z|^2
    if (mixed) LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, bhat.ptr, bhat.scale, outer, s.f.ptr, s.f.scale, inner));
    else LQCD_TRY(lincomb(ctx, Vh, s.f, bhat, nullptr, one, one, zero, zero, nullptr, nullptr));
    LQCD_TRY(apply_schur(Oi, s.f, z.f, t.f, 0, true, ctx->partials, &nb, nullptr));
    launch_finalize(ctx, h, nrhs, nb, FIN_INIT_ZZ, nullptr);
  } else {
    // normal equations Mhat^+ Mhat x = phi: the normal residual z = phi, p = z
    if (mixed) LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, bhat.ptr, bhat.scale, outer, z.f.ptr, z.f.scale, inner));
    else LQCD_TRY(lincomb(ctx, Vh, z.f, bhat, nullptr, one, one, zero, zero, nullptr, nullptr));
    int nbl = 0;
    LQCD_TRY(lincomb(ctx, Vh, z.f, z.f, nullptr, one, one, zero, zero, ctx->partials, &nbl));
    launch_finalize(ctx, h, nrhs, nbl, FIN_INIT_ZZ, nullptr);
  }
  LQCD_TRY(lincomb(ctx, Vh, p.f, z.f, nullptr, one, one, zero, zero, nullptr, nullptr));

  VecArgs va = vargs(s.f, Vh);
  dim3 vgrid(nbv, nrhs);
  IterWork work;
  auto iteration = [&]() -> lqcd_status {
    const lqcd_counters c0 = ctx->cnt;
    lqcd_counters cmid{};
    LQCD_TRY(apply_schur(Oi, p.f, q.f, t.f, 0, false, ctx->partials, &nb, &h->halt));
    launch_finalize(ctx, h, nrhs, nb, FIN_ALPHA, nullptr);
    if (!normal) {
      // CGLS: x += alpha p; s -= alpha q; z = Mhat^+ s
      count_launch(ctx, (double)Vh * nrhs * spinor_site_bytes(inner) * 6.0);
      LQCD_TRY(dispatch_prec(ctx, inner, [&](auto P) {
        launch_pdl(cg_xs_kernel<decltype(P)::value>, vgrid, dim3(128), 0, ctx->stream,
            va, h, X.ptr, X.scale, p.f.ptr, p.f.scale, s.f.ptr, s.f.scale, q.f.ptr, q.f.scale,
            ctx->partials);
      }));
      launch_finalize(ctx, h, nrhs, nbw, FIN_SS, nullptr);
      cmid = ctx->cnt;  // a halted iteration stops here
      LQCD_TRY(apply_schur(Oi, s.f, z.f, t.f, 0, true, ctx->partials, &nb, &h->halt));
      launch_finalize(ctx, h, nrhs, nb, FIN_BETA, nullptr);
    } else {
      // CGNR: w = Mhat^+ q (held in s); x += alpha p; z -= alpha w
      LQCD_TRY(apply_schur(Oi, q.f, s.f, t.f, 0, true, nullptr, nullptr, &h->halt));
      count_launch(ctx, (double)Vh * nrhs * spinor_site_bytes(inner) * 6.0);
      LQCD_TRY(dispatch_prec(ctx, inner, [&](auto P) {
        launch_pdl(cg_xs_kernel<decltype(P)::value>, vgrid, dim3(128), 0, ctx->stream,
            va, h, X.ptr, X.scale, p.f.ptr, p.f.scale, z.f.ptr, z.f.scale, s.f.ptr, s.f.scale,
            ctx->partials);
      }));
      launch_finalize(ctx, h, nrhs, nbw, FIN_SS_BETA, nullptr);
      cmid = ctx->cnt;  // a halted iteration stops here
    }
    count_launch(ctx, (double)Vh * nrhs * spinor_site_bytes(inner) * 3.0);
    LQCD_TRY(dispatch_prec(ctx, inner, [&](auto P) {
      launch_pdl(cg_p_kernel<decltype(P)::value>, vgrid, dim3(128), 0, ctx->stream, va, h, p.f.ptr, p.f.scale,
                 z.f.ptr, z.f.scale);
    }));
    LQCD_CUDA(ctx, cudaGetLastError());
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

  SolverHdr hh;
  int reliable = 0;
  int last_rel_iter = 0;
  const int kStallIters = 200;
  lqcd_status result = LQCD_OK;
  std::vector<double> ss2;
  int iters_seen = 0;  // h->iters at the last poll
  for (;;) {
    lqcd_counters chunk_launches{};
    if (graph.exec) {
      LQCD_CUDA(ctx, cudaGraphLaunch(graph.exec, ctx->stream));
    } else {
      const lqcd_counters c0 = ctx->cnt;
      for (int k = 0; k < chunk; k++) LQCD_TRY(iteration());
      chunk_launches = cnt_sub(ctx->cnt, c0);
      ctx->cnt = c0;
    }
    LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, h, sizeof(SolverHdr), cudaMemcpyDeviceToHost, ctx->stream));
    LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memcpy(&hh, ctx->pinned, sizeof(hh));
    if (graph.exec) chunk_launches = graph.launches(hh.iters - iters_seen);
    count_chunk(ctx, work, chunk_launches, hh.iters - iters_seen, hh.halt != 0);
    iters_seen = hh.iters;
    if (hh.nonfinite) {
      result = fail(ctx, LQCD_ERR_NONFINITE, "CG: non-finite or breakdown scalar after %d iterations", hh.iters);
      break;
    }
    bool finished = hh.all_done != 0;
    // A low-precision recursion can stall before its residual drops by delta
    // (16-bit links perturb the operator by ~1e-3): after kStallIters
    // iterations without a reliable update, force one and restart p = z.
    const bool stalled = mixed && !finished && !hh.need_rel && hh.iters - last_rel_iter >= kStallIters;
    if (mixed && (hh.need_rel || finished || stalled)) {
      // reliable update: xo += X; X = 0; r = bhat - Mhat xo (outer); s = r
      reliable++;
      last_rel_iter = hh.iters;
      dim3 g2(nbv, nrhs);
      count_launch(ctx, (double)Vh * nrhs * (2.0 * spinor_site_bytes(outer) + spinor_site_bytes(inner)));
      LQCD_TRY(dispatch_prec(ctx, outer, [&](auto PO) {
        dispatch_prec(ctx, inner, [&](auto PI) {
          accum_convert_kernel<decltype(PO)::value, decltype(PI)::value><<<g2, 128, 0, ctx->stream>>>(
              Vh, xo.rhs_stride, X.rhs_stride, X.scale_rhs_stride, xo.ptr, X.ptr, X.scale);
        });
      }));
      LQCD_CUDA(ctx, cudaMemsetAsync(X.ptr, 0, X.rhs_stride * nrhs, ctx->stream));
      int nbo = 0;
      LQCD_TRY(apply_schur(Oo, xo, r_o.f, tmp_o.f, 0, false, nullptr, &nbo, nullptr));
      if (normal) {  // r = phi - Mhat^+ Mhat xo
        LQCD_TRY(apply_schur(Oo, r_o.f, y_o.f, tmp_o.f, 0, true, nullptr, &nbo, nullptr));
        std::swap(r_o.f.ptr, y_o.f.ptr);
      }
      int nbl = 0;
      LQCD_TRY(lincomb(ctx, Vh, r_o.f, bhat, &r_o.f, one, one, mone, mone, ctx->partials, &nbl));
      LQCD_TRY(host_sums(ctx, h, nbl, nrhs, tmpd, &ss2));
      HalfField &res_s = normal ? z.f : s.f;
      LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, r_o.f.ptr, r_o.f.scale, outer, res_s.ptr, res_s.scale, inner));
      bool all_ok = true;
      for (int r = 0; r < nrhs; r++)
        if (!(ss2[r] <= prm.tol * prm.tol * b2[r] * 0.25)) all_ok = false;
      if (finished && all_ok) break;
      // z = Mhat^+ s; beta = |z|^2 / zz_old; p = z + beta p
      state_after_reliable_kernel<<<1, 64, 0, ctx->stream>>>(h, tmpd);
      // keep p (beta from the new z) -- or, after a stall, restart with beta = 0
      const int zop = stalled ? FIN_INIT_ZZ : FIN_BETA;
      if (!normal) {
        LQCD_TRY(apply_schur(Oi, s.f, z.f, t.f, 0, true, ctx->partials, &nb, nullptr));
        launch_finalize(ctx, h, nrhs, nb, zop, nullptr);
      } else {
        LQCD_TRY(lincomb(ctx, Vh, z.f, z.f, nullptr, one, one, zero, zero, ctx->partials, &nbl));
        launch_finalize(ctx, h, nrhs, nbl, zop, nullptr);
      }
      if (stalled) LQCD_TRY(lincomb(ctx, Vh, p.f, z.f, nullptr, one, one, zero, zero, nullptr, nullptr));
      if (stalled) {
        if (hh.iters >= prm.max_iter) {
          result = LQCD_ERR_NOCONV;
          break;
        }
        continue;
      }
      // FIN_BETA skips when halted: state_after_reliable clears halt unless all done
      count_launch(ctx, (double)Vh * nrhs * spinor_site_bytes(inner) * 3.0);
      LQCD_TRY(dispatch_prec(ctx, inner, [&](auto P) {
        launch_pdl(cg_p_kernel<decltype(P)::value>, dim3(nbv, nrhs), dim3(128), 0, ctx->stream,
            va, h, p.f.ptr, p.f.scale, z.f.ptr, z.f.scale);
      }));
      LQCD_CUDA(ctx, cudaGetLastError());
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
  if (mixed && result != LQCD_OK) {
    // fold the sloppy iterate into x before returning
    dim3 g2(nbv, nrhs);
    LQCD_TRY(dispatch_prec(ctx, outer, [&](auto PO) {
      dispatch_prec(ctx, inner, [&](auto PI) {
        accum_convert_kernel<decltype(PO)::value, decltype(PI)::value><<<g2, 128, 0, ctx->stream>>>(
            Vh, xo.rhs_stride, X.rhs_stride, X.scale_rhs_stride, xo.ptr, X.ptr, X.scale);
      });
    }));
  }
  // per-rhs iteration counts
  std::vector<RhsState> rsh(nrhs);
  LQCD_CUDA(ctx, cudaMemcpyAsync(rsh.data(), (char *)h + sizeof(SolverHdr), sizeof(RhsState) * nrhs,
                                 cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int itmax = 0;
  for (int r = 0; r < nrhs; r++) {
    st[r].iters += rsh[r].iters;
    st[r].reliable_updates += reliable;
    if (rsh[r].iters > itmax) itmax = rsh[r].iters;
  }
  if (iters_used) *iters_used = itmax;
  if (result == LQCD_ERR_NOCONV) return LQCD_ERR_NOCONV;
  return result;
}

// ---------------------------------------------------------------------------
// BiCGStab on Mhat x = bhat (Sec. 2.1 names CG and BiCGStab as the common
// solvers; van der Vorst 1992), one right-hand side, in precision P of the
// vectors r, r0, p, v, s, t, x:
//   r = bhat - Mhat x;  r0 = r;  rho = alpha = omega = 1;  v = p = 0
//   repeat:  rho' = (r0, r);  beta = (rho'/rho)(alpha/omega)
//            p = r + beta (p - omega v);  v = Mhat p;  alpha = rho' / (r0, v)
//            s = r - alpha v;  t = Mhat s;  omega = (t, s) / (t, t)
//            x += alpha p + omega s;  r = s - omega t
// until |r| <= tol |b|.  The scalars are complex and stay on the device; the
// dot products are FP64 partial sums per block finished in a fixed order.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// BiCGStab with every scalar on the device.  The complex scalars live in a
// device BiState; each reduction (cdot_kernel: per-block partials of
// conj(x) y and |y|^2) is finished by bicg_fin_kernel, one block that sums
// the partials in a fixed order and applies the scalar step; the vector
// kernels read the scalars they need.  check_every iterations are captured
// once in a CUDA graph and replayed; the host reads the state after each
// replay.  Every kernel returns at once when the state says halt.
// ---------------------------------------------------------------------------
struct Zd {
  double re, im;
};
LQCD_HD Zd zmul(Zd a, Zd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
LQCD_HD Zd zdiv(Zd a, Zd b) {  // a / b, scaled by the larger component of b
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
LQCD_HD double zabs2(Zd a) { return a.re * a.re + a.im * a.im; }

struct BiState {
  Zd rho, rho_new, alpha, omega, beta;
  double rr, rr0, stop2;
  int it, first, halt, done, nonconv, bad, max_iter;
  int loops;  // pass counter of the graph's device-side loop
};
enum { BI_RV = 0, BI_OMEGA = 1, BI_RHO = 2 };

// one block: fixed-order sums of the three partial columns, then the step
__global__ void __launch_bounds__(FIN_THREADS) bicg_fin_kernel(BiState *S, const double *partials, int nb, int op) {
  pdl_wait();
  __shared__ double sh[33];
  if (*(volatile int *)&S->halt) return;
  double v[3];
  for (int k = 0; k < 3; k++) {
    double t = 0.0;
#pragma unroll 4
    for (int j = threadIdx.x; j < nb; j += FIN_THREADS) t += partials[3 * j + k];
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
    v[k] = sh[32];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const Zd xy = {v[0], v[1]};
  if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
    S->bad = 1;
    S->halt = 1;
    return;
  }
  if (op == BI_RV) {  // alpha = rho / (r0, v);  rho <- rho_new
    S->rho = S->rho_new;
    if (zabs2(xy) == 0.0) {  // breakdown: the outer refinement restarts
      S->halt = 1;
      return;
    }
    S->alpha = zdiv(S->rho, xy);
  } else if (op == BI_OMEGA) {  // omega = (t, s) / |t|^2 = conj((s, t)) / |t|^2
    S->omega = v[2] > 0.0 ? Zd{xy.re / v[2], -xy.im / v[2]} : Zd{0.0, 0.0};
  } else {  // rho_new = (r0, r), rr = |r|^2; stop, growth and breakdown tests; next beta
    S->rho_new = xy;
    S->rr = v[2];
    S->it += 1;
    S->first = 0;
    if (v[2] <= S->stop2) {
      S->done = 1;
      S->halt = 1;
    } else if (v[2] > 1e12 * S->rr0) {  // spectrum around the origin: diverging
      S->nonconv = 1;
      S->halt = 1;
    } else if (zabs2(S->omega) == 0.0 || zabs2(xy) == 0.0) {
      S->halt = 1;  // breakdown: the outer refinement restarts
    } else if (S->it >= S->max_iter) {
      S->nonconv = 1;
      S->halt = 1;
    } else {
      S->beta = zmul(zdiv(xy, S->rho), zdiv(S->alpha, S->omega));
    }
  }
}

// per block: Re, Im of sum conj(x) y and sum |y|^2 -> partials[3 * block + k]
template <int P>
__global__ void __launch_bounds__(128) bicg_dot_kernel(int Vh, const BiState *S, const void *x, const float *xs,
                                                       const void *y, const float *ys, double *partials) {
  pdl_wait();
  if (S && *(volatile const int *)&S->halt) return;
  using R = typename SpinorIO<P>::R;
  __shared__ double sh[3][8];
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  double re = 0.0, im = 0.0, yy = 0.0;
  if (cb < Vh) {
    Cx<R> X[12], Y[12];
    SpinorIO<P>::load(SpinorView{(void *)x, (float *)xs, Vh}, cb, X);
    SpinorIO<P>::load(SpinorView{(void *)y, (float *)ys, Vh}, cb, Y);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double xr = to_double(X[k].re), xi = to_double(X[k].im);
      const double yr = to_double(Y[k].re), yi = to_double(Y[k].im);
      re = __fma_rn(xr, yr, __fma_rn(xi, yi, re));
      im = __fma_rn(xr, yi, __fma_rn(-xi, yr, im));
      yy = __fma_rn(yr, yr, __fma_rn(yi, yi, yy));
    }
  }
  const double a = warp_block_sum(re, sh[0]);
  const double b = warp_block_sum(im, sh[1]);
  const double c = warp_block_sum(yy, sh[2]);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = a;
    partials[3 * blockIdx.x + 1] = b;
    partials[3 * blockIdx.x + 2] = c;
  }
}

template <class R> LQCD_DEV Cx<R> zc(Zd z) { return {from_double<R>(z.re), from_double<R>(z.im)}; }

// MODE 0: p = r (first iteration) or p = r + beta (p - omega v)
// MODE 1: s = r - alpha v
// MODE 2: x += alpha p + omega s;  r = s - omega t
template <int P, int MODE>
__global__ void __launch_bounds__(128) bicg_vec_kernel(int Vh, const BiState *S, void *a0, float *a0s, void *a1,
                                                       float *a1s, const void *b0, const float *b0s,
                                                       const void *b1, const float *b1s, const void *b2,
                                                       const float *b2s) {
  pdl_wait();
  if (*(volatile const int *)&S->halt) return;
  using R = typename SpinorIO<P>::R;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= Vh) return;
  Cx<R> A[12], B[12], C[12];
  if (MODE == 0) {  // a0 = p, b0 = r, b1 = v
    SpinorIO<P>::load(SpinorView{(void *)b0, (float *)b0s, Vh}, cb, B);
    if (!S->first) {
      const Cx<R> be = zc<R>(S->beta), bo = zc<R>(zmul(S->beta, S->omega));
      SpinorIO<P>::load(SpinorView{a0, a0s, Vh}, cb, A);
      SpinorIO<P>::load(SpinorView{(void *)b1, (float *)b1s, Vh}, cb, C);
#pragma unroll
      for (int k = 0; k < 12; k++) B[k] = B[k] + (be * A[k] - bo * C[k]);
    }
    SpinorIO<P>::store(SpinorView{a0, a0s, Vh}, cb, B);
  } else if (MODE == 1) {  // a0 = s, b0 = r, b1 = v
    const Cx<R> al = zc<R>(S->alpha);
    SpinorIO<P>::load(SpinorView{(void *)b0, (float *)b0s, Vh}, cb, B);
    SpinorIO<P>::load(SpinorView{(void *)b1, (float *)b1s, Vh}, cb, C);
#pragma unroll
    for (int k = 0; k < 12; k++) B[k] = B[k] - al * C[k];
    SpinorIO<P>::store(SpinorView{a0, a0s, Vh}, cb, B);
  } else {  // a0 = x, a1 = r, b0 = p, b1 = s, b2 = t
    const Cx<R> al = zc<R>(S->alpha), om = zc<R>(S->omega);
    Cx<R> X[12];
    SpinorIO<P>::load(SpinorView{a0, a0s, Vh}, cb, X);
    SpinorIO<P>::load(SpinorView{(void *)b0, (float *)b0s, Vh}, cb, A);
    SpinorIO<P>::load(SpinorView{(void *)b1, (float *)b1s, Vh}, cb, B);
#pragma unroll
    for (int k = 0; k < 12; k++) X[k] = X[k] + (al * A[k] + om * B[k]);
    SpinorIO<P>::store(SpinorView{a0, a0s, Vh}, cb, X);
    SpinorIO<P>::load(SpinorView{(void *)b2, (float *)b2s, Vh}, cb, C);
#pragma unroll
    for (int k = 0; k < 12; k++) B[k] = B[k] - om * C[k];
    SpinorIO<P>::store(SpinorView{a1, a1s, Vh}, cb, B);
  }
}

// Solves Mhat xo = bhat (outer-format fields, one RHS) with BiCGStab in the
// inner format to the relative residual tol_rel * |b| / |bhat| of the
// current cycle; xo receives the solution.  st->iters counts iterations.
lqcd_status bicgstab_even(lqcd_ctx *ctx, lqcd_gauge *U, const Geom &g, double kappa, double mu,
                          const lqcd_cg_params &prm, const HalfField &bhat, const HalfField &xo, double b2,
                          lqcd_cg_stats *st, int *iters_used) {
  const int Vh = g.Vh;
  const int outer = prm.outer_prec, P = prm.inner_prec;
  const bool mixed = P != outer;
  Op Oi{ctx, g, {}, P, U->recon, kappa, mu};
  if (mixed) Oi.recon = (P == LQCD_BF16S || P == LQCD_F16S) ? 12 : (prm.sloppy_recon ? prm.sloppy_recon : 18);
  LQCD_TRY(gauge_view(ctx, U, P, Oi.recon, &Oi.U));
  Vec r, r0, p, v, sv_, t, tmp, xs;
  for (Vec *w : {&r, &r0, &p, &v, &sv_, &t, &tmp}) LQCD_TRY(w->alloc(ctx, P, Vh, 1));
  HalfField X = xo;
  if (mixed) {
    LQCD_TRY(xs.alloc(ctx, P, Vh, 1));
    X = xs.f;
  }
  const HostC one{1, 0}, zero{0, 0};
  // x = 0, r = bhat, r0 = r
  if (mixed) LQCD_TRY(spinor_convert_raw(ctx, Vh, 1, bhat.ptr, bhat.scale, outer, r.f.ptr, r.f.scale, P));
  else LQCD_TRY(lincomb(ctx, Vh, r.f, bhat, nullptr, one, one, zero, zero, nullptr, nullptr));
  LQCD_TRY(lincomb(ctx, Vh, r0.f, r.f, nullptr, one, one, zero, zero, nullptr, nullptr));
  const int nb = (Vh + 127) / 128;
  LQCD_TRY(ensure_partials(ctx, (size_t)3 * nb));
  DBuf sbuf(ctx);
  LQCD_TRY(sbuf.alloc(sizeof(BiState)));
  BiState *S = (BiState *)sbuf.p;
  const dim3 vgrid(nb);
  cudaStream_t cst = ctx->stream;
  auto dot = [&](const HalfField &a, const HalfField &b, const BiState *state) -> lqcd_status {
    count_launch(ctx, (double)Vh * 2.0 * spinor_site_bytes(P));
    return dispatch_prec(ctx, P, [&](auto PP) {
      launch_pdl(bicg_dot_kernel<decltype(PP)::value>, vgrid, dim3(128), 0, ctx->stream, Vh, state,
                 (const void *)a.ptr, (const float *)a.scale, (const void *)b.ptr, (const float *)b.scale,
                 ctx->partials);
    });
  };
  auto fin = [&](int op) -> lqcd_status {
    launch_pdl(bicg_fin_kernel, dim3(1), dim3(FIN_THREADS), 0, ctx->stream, S, (const double *)ctx->partials, nb,
               op);
    count_launch(ctx, 24.0 * nb);
    LQCD_CUDA(ctx, cudaGetLastError());
    return LQCD_OK;
  };
  // rho_new = (r0, r), rr = |r|^2 on the host once: the stop criterion
  LQCD_TRY(dot(r0.f, r.f, nullptr));
  LQCD_TRY(ensure_pinned(ctx, (size_t)3 * nb));
  LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, ctx->partials, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, cst));
  LQCD_CUDA(ctx, cudaStreamSynchronize(cst));
  double a = 0.0, b = 0.0, rr = 0.0;
  for (int k = 0; k < nb; k++) {
    a += ctx->pinned[3 * k];
    b += ctx->pinned[3 * k + 1];
    rr += ctx->pinned[3 * k + 2];
  }
  // stop on |r|^2 <= (tol/2)^2 |b|^2 (|b| of the full system, as the CG does);
  // a mixed solve stops earlier, once |r| <= inner_tol times this cycle's |bhat|
  double stop2 = 0.25 * prm.tol * prm.tol * b2;
  if (mixed) {
    const double itol = prm.inner_tol > 0.0 ? prm.inner_tol : 1e-5;
    stop2 = std::fmax(stop2, itol * itol * rr);
  }
  BiState hs{};
  hs.rho = {1.0, 0.0};
  hs.rho_new = {a, b};
  hs.alpha = hs.omega = {1.0, 0.0};
  hs.rr = hs.rr0 = rr;
  hs.stop2 = stop2;
  hs.first = 1;
  hs.max_iter = prm.max_iter;
  hs.halt = rr <= stop2 ? 1 : 0;
  hs.done = hs.halt;
  std::memcpy(ctx->pinned, &hs, sizeof(hs));
  LQCD_CUDA(ctx, cudaMemcpyAsync(S, ctx->pinned, sizeof(hs), cudaMemcpyHostToDevice, cst));
  IterWork work;  // BiCGStab halts at the end of an iteration (or on a breakdown)
  auto iteration = [&]() -> lqcd_status {
    const lqcd_counters c0 = ctx->cnt;
    LQCD_TRY(dispatch_prec(ctx, P, [&](auto PP) {  // p = r (+ beta (p - omega v))
      launch_pdl(bicg_vec_kernel<decltype(PP)::value, 0>, vgrid, dim3(128), 0, ctx->stream, Vh, (const BiState *)S,
                 p.f.ptr, p.f.scale, (void *)nullptr, (float *)nullptr, (const void *)r.f.ptr,
                 (const float *)r.f.scale, (const void *)v.f.ptr, (const float *)v.f.scale, (const void *)nullptr,
                 (const float *)nullptr);
    }));
    count_launch(ctx, (double)Vh * 4.0 * spinor_site_bytes(P));
    LQCD_TRY(apply_schur(Oi, p.f, v.f, tmp.f, 0, false, nullptr, nullptr, &S->halt));
    LQCD_TRY(dot(r0.f, v.f, S));
    LQCD_TRY(fin(BI_RV));
    LQCD_TRY(dispatch_prec(ctx, P, [&](auto PP) {  // s = r - alpha v
      launch_pdl(bicg_vec_kernel<decltype(PP)::value, 1>, vgrid, dim3(128), 0, ctx->stream, Vh, (const BiState *)S,
                 sv_.f.ptr, sv_.f.scale, (void *)nullptr, (float *)nullptr, (const void *)r.f.ptr,
                 (const float *)r.f.scale, (const void *)v.f.ptr, (const float *)v.f.scale, (const void *)nullptr,
                 (const float *)nullptr);
    }));
    count_launch(ctx, (double)Vh * 3.0 * spinor_site_bytes(P));
    LQCD_TRY(apply_schur(Oi, sv_.f, t.f, tmp.f, 0, false, nullptr, nullptr, &S->halt));
    LQCD_TRY(dot(sv_.f, t.f, S));
    LQCD_TRY(fin(BI_OMEGA));
    LQCD_TRY(dispatch_prec(ctx, P, [&](auto PP) {  // x += alpha p + omega s; r = s - omega t
      launch_pdl(bicg_vec_kernel<decltype(PP)::value, 2>, vgrid, dim3(128), 0, ctx->stream, Vh, (const BiState *)S,
                 X.ptr, X.scale, r.f.ptr, r.f.scale, (const void *)p.f.ptr, (const float *)p.f.scale,
                 (const void *)sv_.f.ptr, (const float *)sv_.f.scale, (const void *)t.f.ptr,
                 (const float *)t.f.scale);
    }));
    count_launch(ctx, (double)Vh * 6.0 * spinor_site_bytes(P));
    LQCD_TRY(dot(r0.f, r.f, S));
    LQCD_TRY(fin(BI_RHO));
    if (!work.known) {
      work.full = work.first = cnt_sub(ctx->cnt, c0);
      work.known = true;
    }
    return LQCD_OK;
  };
  const int chunk = prm.check_every > 0 ? prm.check_every : 10;
  SolverGraph graph;
  if (prm.use_graph) {
    // one operator application outside the capture, so the autotuner times
    // the hop configurations the captured iterations launch (v is
    // overwritten before it is read)
    LQCD_TRY(apply_schur(Oi, r.f, v.f, tmp.f, 0, false, nullptr, nullptr, nullptr));
    LQCD_TRY(build_solver_graph(ctx, chunk, &S->halt, &S->loops, iteration, &graph));
  }
  lqcd_status result = LQCD_OK;
  while (!hs.halt) {
    const int it_seen = hs.it;
    lqcd_counters chunk_launches{};
    if (graph.exec) {
      LQCD_CUDA(ctx, cudaGraphLaunch(graph.exec, cst));
    } else {
      const lqcd_counters c0 = ctx->cnt;
      for (int k = 0; k < chunk; k++) LQCD_TRY(iteration());
      chunk_launches = cnt_sub(ctx->cnt, c0);
      ctx->cnt = c0;
    }
    LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, S, sizeof(hs), cudaMemcpyDeviceToHost, cst));
    LQCD_CUDA(ctx, cudaStreamSynchronize(cst));
    std::memcpy(&hs, ctx->pinned, sizeof(hs));
    if (graph.exec) chunk_launches = graph.launches(hs.it - it_seen);
    // iterations that ran to their end (a breakdown's partial one is not counted)
    count_chunk(ctx, work, chunk_launches, hs.it - it_seen, false);
  }
  if (hs.bad) result = fail(ctx, LQCD_ERR_NONFINITE, "BiCGStab: non-finite scalar after %d iterations", hs.it);
  else if (hs.nonconv) result = LQCD_ERR_NOCONV;
  if (mixed) {
    dim3 g2((Vh + 127) / 128, 1);
    LQCD_TRY(dispatch_prec(ctx, outer, [&](auto PO) {
      dispatch_prec(ctx, P, [&](auto PI) {
        accum_convert_kernel<decltype(PO)::value, decltype(PI)::value><<<g2, 128, 0, ctx->stream>>>(
            Vh, xo.rhs_stride, X.rhs_stride, X.scale_rhs_stride, xo.ptr, X.ptr, X.scale);
      });
    }));
    LQCD_CUDA(ctx, cudaGetLastError());
  }
  st->iters += hs.it;
  if (iters_used) *iters_used = hs.it;
  return result;
}

// Full solve on EO full fields (outer F64 user fields b, x).
lqcd_status cg_solve_eo(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField &b_full, const HalfField &x_full,
                        double kappa, double mu, const lqcd_cg_params &prm, lqcd_cg_stats *st) {
  auto t0 = std::chrono::steady_clock::now();
  const Geom &g = U->g;
  const int Vh = g.Vh, nrhs = b_full.nrhs;
  const int outer = prm.outer_prec;
  for (int r = 0; r < nrhs; r++) std::memset(&st[r], 0, sizeof(lqcd_cg_stats));
  Op O64{ctx, g, {}, LQCD_F64, U->recon, kappa, mu};
  LQCD_TRY(gauge_view(ctx, U, LQCD_F64, U->recon, &O64.U));
  HalfField be = half_of(b_full, 0, Vh), bo = half_of(b_full, 1, Vh);
  HalfField xe = half_of(x_full, 0, Vh), xodd = half_of(x_full, 1, Vh);
  const HostC one{1, 0}, zero{0, 0}, mone{-1, 0};
  int nbv = (Vh + 127) / 128;
  int nb = hop_blocks(g, nrhs);
  LQCD_TRY(ensure_partials(ctx, (size_t)nrhs * 2 * (nb > nbv ? nb : nbv)));
  SolverHdr *h;
  LQCD_TRY(ensure_state(ctx, nrhs, &h));
  // |b|^2
  std::vector<double> b2(nrhs), e2;
  {
    Vec tmp;
    LQCD_TRY(tmp.alloc(ctx, LQCD_F64, Vh, nrhs));
    int n1 = 0;
    LQCD_TRY(lincomb(ctx, Vh, tmp.f, be, nullptr, one, one, zero, zero, ctx->partials, &n1));
    LQCD_TRY(host_sums(ctx, h, n1, nrhs, state_scratch(h, nrhs, 2), &e2));
    LQCD_TRY(lincomb(ctx, Vh, tmp.f, bo, nullptr, one, one, zero, zero, ctx->partials, &n1));
    std::vector<double> o2;
    LQCD_TRY(host_sums(ctx, h, n1, nrhs, state_scratch(h, nrhs, 2), &o2));
    for (int r = 0; r < nrhs; r++) b2[r] = e2[r] + o2[r];
  }
  for (int r = 0; r < nrhs; r++)
    if (!std::isfinite(b2[r])) return fail(ctx, LQCD_ERR_NONFINITE, "right-hand side %d is not finite", r);
  LQCD_CUDA(ctx, cudaMemsetAsync(x_full.ptr, 0, x_full.rhs_stride * nrhs, ctx->stream));
  // working copies of the current right-hand side (b, later the true residual)
  Vec rhs_e, rhs_o, t_o, bhat64, corr_e, corr_o, res_e, res_o, xo_outer, bhat_outer;
  LQCD_TRY(rhs_e.alloc(ctx, LQCD_F64, Vh, nrhs));
  LQCD_TRY(rhs_o.alloc(ctx, LQCD_F64, Vh, nrhs));
  if (outer == LQCD_F64) {
    LQCD_TRY(t_o.alloc(ctx, LQCD_F64, Vh, nrhs));
    LQCD_TRY(bhat64.alloc(ctx, LQCD_F64, Vh, nrhs));
  }
  LQCD_TRY(corr_e.alloc(ctx, LQCD_F64, Vh, nrhs));
  LQCD_TRY(corr_o.alloc(ctx, LQCD_F64, Vh, nrhs));
  LQCD_TRY(res_e.alloc(ctx, LQCD_F64, Vh, nrhs));
  LQCD_TRY(res_o.alloc(ctx, LQCD_F64, Vh, nrhs));
  LQCD_TRY(xo_outer.alloc(ctx, outer, Vh, nrhs));
  // With a float-float outer format the source preparation and the
  // reconstruction run in float-float too (the CG works on bhat in that format,
  // and x_o enters the IEEE-FP64 true residual, whose check decides); their
  // half hops then cost a quarter of the FP64 ones on GB300.
  const bool prep_outer = outer != LQCD_F64;
  Vec rhs_e_w, rhs_o_w, t_o_w, corr_o_w;
  GaugeView Uw{};
  if (prep_outer) {
    LQCD_TRY(bhat_outer.alloc(ctx, outer, Vh, nrhs));
    LQCD_TRY(rhs_e_w.alloc(ctx, outer, Vh, nrhs));
    LQCD_TRY(rhs_o_w.alloc(ctx, outer, Vh, nrhs));
    LQCD_TRY(t_o_w.alloc(ctx, outer, Vh, nrhs));
    LQCD_TRY(corr_o_w.alloc(ctx, outer, Vh, nrhs));
    LQCD_TRY(gauge_view(ctx, U, outer, U->recon, &Uw));
  }
  LQCD_TRY(lincomb(ctx, Vh, rhs_e.f, be, nullptr, one, one, zero, zero, nullptr, nullptr));
  LQCD_TRY(lincomb(ctx, Vh, rhs_o.f, bo, nullptr, one, one, zero, zero, nullptr, nullptr));
  TmCoef c = tm_coef(kappa, mu, false);
  lqcd_status result = LQCD_OK;
  double worst = 0.0;
  for (int cycle = 0;; cycle++) {
    // bhat_e = rhs_e + kappa H_eo A_o^-1 rhs_o
    HopLaunch Ls;
    Ls.recon = U->recon;
    Ls.has_aux = true;
    Ls.out_parity = 0;
    Ls.c_up = Ls.c_dn = {kappa, 0.0};
    Ls.d_up = Ls.d_dn = one;
    HalfField bh;
    if (prep_outer) {
      LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, rhs_e.f.ptr, nullptr, LQCD_F64, rhs_e_w.f.ptr, nullptr, outer));
      LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, rhs_o.f.ptr, nullptr, LQCD_F64, rhs_o_w.f.ptr, nullptr, outer));
      LQCD_TRY(lincomb(ctx, Vh, t_o_w.f, rhs_o_w.f, nullptr, c.Ai_up, c.Ai_dn, zero, zero, nullptr, nullptr));
      Ls.prec = outer;
      Ls.U = Uw;
      Ls.in = t_o_w.f;
      Ls.out = bhat_outer.f;
      Ls.aux = rhs_e_w.f;
      bh = bhat_outer.f;
    } else {
      LQCD_TRY(lincomb(ctx, Vh, t_o.f, rhs_o.f, nullptr, c.Ai_up, c.Ai_dn, zero, zero, nullptr, nullptr));
      Ls.prec = LQCD_F64;
      Ls.U = O64.U;
      Ls.in = t_o.f;
      Ls.out = bhat64.f;
      Ls.aux = rhs_e.f;
      bh = bhat64.f;
    }
    LQCD_TRY(launch_hop(ctx, g, Ls, nullptr));
    LQCD_CUDA(ctx, cudaMemsetAsync(xo_outer.f.ptr, 0, xo_outer.f.rhs_stride * nrhs, ctx->stream));
    int used = 0;
    lqcd_status s = prm.solver == LQCD_SOLVER_BICGSTAB
                        ? bicgstab_even(ctx, U, g, kappa, mu, prm, bh, xo_outer.f, b2[0], st, &used)
                        : cgls_even(ctx, U, g, kappa, mu, prm, bh, xo_outer.f, b2, st, nrhs, &used, false);
    if (s != LQCD_OK && s != LQCD_ERR_NOCONV) return s;
    // corr_e = x_e (F64); corr_o = A_o^-1 (rhs_o + kappa H_oe corr_e)
    if (prep_outer)
      LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, xo_outer.f.ptr, nullptr, outer, corr_e.f.ptr, nullptr,
                                  LQCD_F64));
    else
      LQCD_TRY(lincomb(ctx, Vh, corr_e.f, xo_outer.f, nullptr, one, one, zero, zero, nullptr, nullptr));
    HopLaunch Lr;
    Lr.prec = prep_outer ? outer : LQCD_F64;
    Lr.recon = U->recon;
    Lr.U = prep_outer ? Uw : O64.U;
    Lr.in = prep_outer ? xo_outer.f : corr_e.f;
    Lr.out = prep_outer ? corr_o_w.f : corr_o.f;
    Lr.aux = prep_outer ? rhs_o_w.f : rhs_o.f;
    Lr.has_aux = true;
    Lr.out_parity = 1;
    Lr.c_up = {kappa * c.Ai_up.re, kappa * c.Ai_up.im};
    Lr.c_dn = {kappa * c.Ai_dn.re, kappa * c.Ai_dn.im};
    Lr.d_up = c.Ai_up;
    Lr.d_dn = c.Ai_dn;
    LQCD_TRY(launch_hop(ctx, g, Lr, nullptr));
    if (prep_outer)
      LQCD_TRY(spinor_convert_raw(ctx, Vh, nrhs, corr_o_w.f.ptr, nullptr, outer, corr_o.f.ptr, nullptr, LQCD_F64));
    // x += corr
    LQCD_TRY(lincomb(ctx, Vh, xe, xe, &corr_e.f, one, one, one, one, nullptr, nullptr));
    LQCD_TRY(lincomb(ctx, Vh, xodd, xodd, &corr_o.f, one, one, one, one, nullptr, nullptr));
    // true residual: res = b - M x (FP64, both parities)
    int nbh = 0;
    LQCD_TRY(apply_full(O64, xe, xodd, res_e.f, res_o.f, false, nullptr, nullptr, &nbh));
    int n1 = 0;
    LQCD_TRY(lincomb(ctx, Vh, rhs_e.f, be, &res_e.f, one, one, mone, mone, ctx->partials, &n1));
    LQCD_TRY(host_sums(ctx, h, n1, nrhs, state_scratch(h, nrhs, 2), &e2));
    std::vector<double> o2;
    LQCD_TRY(lincomb(ctx, Vh, rhs_o.f, bo, &res_o.f, one, one, mone, mone, ctx->partials, &n1));
    LQCD_TRY(host_sums(ctx, h, n1, nrhs, state_scratch(h, nrhs, 2), &o2));
    worst = 0.0;
    bool all = true;
    int total_iters = 0;
    for (int r = 0; r < nrhs; r++) {
      // a zero right-hand side has the solution x = 0 and an absolute residual
      double tr = b2[r] > 0.0 ? std::sqrt((e2[r] + o2[r]) / b2[r]) : std::sqrt(e2[r] + o2[r]);
      st[r].true_resid = tr;
      st[r].converged = tr <= prm.tol;
      all = all && st[r].converged;
      worst = std::fmax(worst, tr);
      total_iters = st[r].iters > total_iters ? st[r].iters : total_iters;
      if (!std::isfinite(tr)) return fail(ctx, LQCD_ERR_NONFINITE, "true residual is not finite");
    }
    if (all) break;
    if (cycle >= prm.max_restarts || total_iters >= prm.max_iter || (s == LQCD_ERR_NOCONV && worst > 1.0)) {
      result = LQCD_ERR_NOCONV;
      break;
    }
    for (int r = 0; r < nrhs; r++) {
      if (st[r].converged) {  // converged right-hand sides get a zero correction
        LQCD_CUDA(ctx, cudaMemsetAsync((char *)rhs_e.f.ptr + r * rhs_e.f.rhs_stride, 0,
                                       rhs_e.f.rhs_stride, ctx->stream));
        LQCD_CUDA(ctx, cudaMemsetAsync((char *)rhs_o.f.ptr + r * rhs_o.f.rhs_stride, 0,
                                       rhs_o.f.rhs_stride, ctx->stream));
      } else {
        st[r].restarts++;
      }
    }
    // next cycle solves M d = (b - M x): rhs_e, rhs_o already hold the residual
  }
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int r = 0; r < nrhs; r++) st[r].seconds = secs;
  if (result == LQCD_ERR_NOCONV)
    fail(ctx, LQCD_ERR_NOCONV, "%s stopped with true residual %.3e > tol %.3e",
         prm.solver == LQCD_SOLVER_BICGSTAB ? "BiCGStab" : "CG", worst, prm.tol);
  return result;
}

}  // namespace lqcd
