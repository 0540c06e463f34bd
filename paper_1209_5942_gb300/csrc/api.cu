// api.cu -- the extern "C" entry points of lqcd.h: argument validation,
// layout handling and dispatch to the kernels.  Validation happens before any
// launch; failures return a status and leave a message in the context.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <new>
#include <string>

#include "internal.h"

namespace lqcd {

lqcd_status gauge_import_raw(lqcd_ctx *ctx, const lqcd_gauge *U, const void *src);
lqcd_status gauge_export_raw(lqcd_ctx *ctx, const lqcd_gauge *U, void *dst);
lqcd_status gauge_su3_deviation(lqcd_ctx *ctx, const lqcd_gauge *U, double *dev);
lqcd_status cg_solve_eo(lqcd_ctx *ctx, lqcd_gauge *U, const HalfField &b_full, const HalfField &x_full,
                        double kappa, double mu, const lqcd_cg_params &prm, lqcd_cg_stats *st);


lqcd_status fail(lqcd_ctx *ctx, lqcd_status s, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

lqcd_status cuda_check(lqcd_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return LQCD_OK;
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation)
    return fail(ctx, LQCD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(ctx, LQCD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

Geom make_geom(const lqcd_geom &g) {
  Geom d;
  for (int k = 0; k < 4; k++) d.L[k] = g.L[k];
  d.Lh0 = g.L[0] / 2;
  d.Vh = (int)((long)g.L[0] * g.L[1] * g.L[2] * g.L[3] / 2);
  d.antiper = g.antiperiodic_t ? 1 : 0;
  return d;
}

bool geom_equal(const lqcd_geom &a, const lqcd_geom &b) {
  return a.L[0] == b.L[0] && a.L[1] == b.L[1] && a.L[2] == b.L[2] && a.L[3] == b.L[3] &&
         (a.antiperiodic_t != 0) == (b.antiperiodic_t != 0);
}

size_t spinor_half_bytes(int prec, int Vh) { return spinor_bytes_per_site(prec) * (size_t)Vh; }
size_t spinor_scale_half_bytes(int prec, int Vh) {
  return (prec == LQCD_BF16S || prec == LQCD_F16S) ? sizeof(float) * (size_t)Vh : 0;
}

lqcd_status raw_alloc(lqcd_ctx *ctx, const DevAllocator &A, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LQCD_OK;
  if (A.alloc) {
    *p = A.alloc(bytes, A.user);
    if (!*p) return fail(ctx, LQCD_ERR_OOM, "caller allocator returned NULL for %zu bytes", bytes);
    if ((uintptr_t)*p % 256 != 0) {
      A.free(*p, A.user);
      *p = nullptr;
      return fail(ctx, LQCD_ERR_INVALID, "caller allocator returned memory not aligned to 256 bytes");
    }
    return LQCD_OK;
  }
  cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream)
                            : cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, LQCD_ERR_OOM, "device allocation of %zu bytes failed", bytes);
  }
  return LQCD_OK;
}
void raw_free(lqcd_ctx *ctx, const DevAllocator &A, void *p) {
  if (!p) return;
  if (A.free) A.free(p, A.user);
  else cudaFreeAsync(p, ctx->stream);
}
lqcd_status dalloc(lqcd_ctx *ctx, void **p, size_t bytes) { return raw_alloc(ctx, ctx->A, p, bytes); }
void dfree(lqcd_ctx *ctx, void *p) { raw_free(ctx, ctx->A, p); }

lqcd_status ensure_partials(lqcd_ctx *ctx, size_t doubles) {
  if (ctx->partials_cap >= doubles) return LQCD_OK;
  if (ctx->partials) {
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx, ctx->partials);
  }
  ctx->partials = nullptr;
  ctx->partials_cap = 0;
  size_t n = doubles < 4096 ? 4096 : doubles;
  LQCD_TRY(dalloc(ctx, (void **)&ctx->partials, n * sizeof(double)));
  ctx->partials_cap = n;
  return LQCD_OK;
}

lqcd_status ensure_pinned(lqcd_ctx *ctx, size_t doubles) {
  if (ctx->pinned_cap >= doubles) return LQCD_OK;
  if (ctx->pinned) {
    cudaStreamSynchronize(ctx->stream);
    cudaFreeHost(ctx->pinned);
  }
  ctx->pinned = nullptr;
  ctx->pinned_cap = 0;
  size_t n = doubles < 4096 ? 4096 : doubles;
  if (cudaMallocHost(&ctx->pinned, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, LQCD_ERR_OOM, "pinned allocation failed");
  }
  ctx->pinned_cap = n;
  return LQCD_OK;
}

// ---------------------------------------------------------------------------
// validation helpers
// ---------------------------------------------------------------------------

lqcd_status check_geom(lqcd_ctx *ctx, const lqcd_geom *g) {
  if (!g) return fail(ctx, LQCD_ERR_INVALID, "geometry is NULL");
  long V = 1;
  for (int k = 0; k < 4; k++) {
    if (g->L[k] < 2 || (g->L[k] & 1))
      return fail(ctx, LQCD_ERR_INVALID, "extent L[%d] = %d must be even and >= 2", k, g->L[k]);
    V *= g->L[k];
  }
  if (V / 2 > (1L << 30)) return fail(ctx, LQCD_ERR_INVALID, "lattice too large");
  return LQCD_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

lqcd_status check_field(lqcd_ctx *ctx, const lqcd_field &f, const char *name, bool allow_lexi) {
  if (!f.ptr) return fail(ctx, LQCD_ERR_INVALID, "%s: NULL pointer", name);
  if (!aligned16(f.ptr)) return fail(ctx, LQCD_ERR_INVALID, "%s: pointer not 16-byte aligned", name);
  if (f.nrhs < 1 || f.nrhs > 64) return fail(ctx, LQCD_ERR_INVALID, "%s: nrhs %d out of [1, 64]", name, f.nrhs);
  if (f.prec < LQCD_F64 || f.prec > LQCD_F16S) return fail(ctx, LQCD_ERR_INVALID, "%s: bad precision", name);
  if (f.layout == LQCD_LAYOUT_LEXI) {
    if (!allow_lexi) return fail(ctx, LQCD_ERR_INVALID, "%s: lexicographic layout not accepted here", name);
    if (f.prec != LQCD_F64) return fail(ctx, LQCD_ERR_INVALID, "%s: lexicographic fields are complex128", name);
  } else if (f.layout != LQCD_LAYOUT_EO) {
    return fail(ctx, LQCD_ERR_INVALID, "%s: bad layout", name);
  }
  bool scaled = f.prec == LQCD_BF16S || f.prec == LQCD_F16S;
  if (scaled && !f.scale) return fail(ctx, LQCD_ERR_INVALID, "%s: scaled precision needs a scale array", name);
  return LQCD_OK;
}

static HalfField to_half(const lqcd_field &f, const Geom &g, bool full) {
  HalfField h;
  h.ptr = f.ptr;
  h.scale = (float *)f.scale;
  h.prec = f.prec;
  h.nrhs = f.nrhs;
  size_t hb = spinor_half_bytes(f.prec, g.Vh);
  size_t hs = spinor_scale_half_bytes(f.prec, g.Vh) / sizeof(float);
  h.rhs_stride = full ? 2 * hb : hb;
  h.scale_rhs_stride = full ? 2 * hs : hs;
  return h;
}
static HalfField half_of_full(const HalfField &full, int p, int Vh) {
  HalfField h = full;
  h.ptr = (char *)full.ptr + p * spinor_half_bytes(full.prec, Vh);
  if (full.scale) h.scale = full.scale + (size_t)p * Vh;
  return h;
}

static bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
  uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

}  // namespace lqcd

using namespace lqcd;

// ===========================================================================
// Context
// ===========================================================================

extern "C" int lqcd_abi_version(void) { return LQCD_ABI_VERSION; }

extern "C" int lqcd_create(lqcd_ctx **out, int device, void *stream) {
  if (!out) return LQCD_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return LQCD_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return LQCD_ERR_CUDA;
  lqcd_ctx *c = new (std::nothrow) lqcd_ctx();
  if (!c) return LQCD_ERR_OOM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess)
    c->gpu_name = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount);
  if (const char *tp = std::getenv("LQCD_TUNE_CACHE")) {
    c->tune_path = tp;
    tune_load(c);
  }
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      c->pool = nullptr;
      lqcd_destroy(c);
      return LQCD_ERR_CUDA;
    }
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      lqcd_destroy(c);
      return LQCD_ERR_CUDA;
    }
  }
  if (ensure_partials(c, 1 << 16) != LQCD_OK || ensure_pinned(c, 4096) != LQCD_OK) {
    lqcd_destroy(c);
    return LQCD_ERR_OOM;
  }
  *out = c;
  return LQCD_OK;
}

// releases the context's device workspace (through its current allocator)
static void release_workspace(lqcd_ctx *ctx) {
  cudaStreamSynchronize(ctx->stream);
  dfree(ctx, ctx->partials);
  dfree(ctx, ctx->solver_state);
  dfree(ctx, ctx->staples);
  cudaStreamSynchronize(ctx->stream);
  ctx->partials = nullptr;
  ctx->partials_cap = 0;
  ctx->solver_state = nullptr;
  ctx->solver_state_cap = 0;
  ctx->staples = nullptr;
  ctx->staple_cap = 0;
}

extern "C" int lqcd_destroy(lqcd_ctx *ctx) {
  if (!ctx) return LQCD_ERR_INVALID;
  release_workspace(ctx);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  // allocations still outstanding (gauge fields not yet freed) keep the
  // pool's memory alive until they are freed
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return LQCD_OK;
}

extern "C" int lqcd_trim_memory(lqcd_ctx *ctx) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (!ctx->pool) return LQCD_OK;
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  LQCD_CUDA(ctx, cudaMemPoolTrimTo(ctx->pool, 0));
  return LQCD_OK;
}

extern "C" int lqcd_memory_stats(lqcd_ctx *ctx, uint64_t *reserved, uint64_t *used) {
  if (!ctx || !reserved || !used) return LQCD_ERR_INVALID;
  *reserved = *used = 0;
  if (!ctx->pool) return LQCD_OK;
  LQCD_CUDA(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrReservedMemCurrent, reserved));
  LQCD_CUDA(ctx, cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, used));
  return LQCD_OK;
}

extern "C" int lqcd_set_allocator(lqcd_ctx *ctx, lqcd_alloc_fn alloc, lqcd_free_fn free_fn, void *user) {
  if (!ctx) return LQCD_ERR_INVALID;
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(ctx, LQCD_ERR_INVALID, "alloc and free must both be set or both be NULL");
  release_workspace(ctx);
  ctx->A.alloc = alloc;
  ctx->A.free = free_fn;
  ctx->A.user = user;
  return ensure_partials(ctx, 1 << 16);
}

extern "C" int lqcd_set_stream(lqcd_ctx *ctx, void *stream) {
  if (!ctx) return LQCD_ERR_INVALID;
  ctx->stream = (cudaStream_t)stream;
  return LQCD_OK;
}

extern "C" const char *lqcd_last_error(const lqcd_ctx *ctx) {
  if (!ctx) return "context is NULL";
  return ctx->err.c_str();
}

extern "C" int lqcd_get_counters(const lqcd_ctx *ctx, lqcd_counters *out) {
  if (!ctx || !out) return LQCD_ERR_INVALID;
  *out = ctx->cnt;
  return LQCD_OK;
}

extern "C" int lqcd_reset_counters(lqcd_ctx *ctx) {
  if (!ctx) return LQCD_ERR_INVALID;
  ctx->cnt = lqcd_counters{};
  return LQCD_OK;
}

extern "C" size_t lqcd_field_bytes(const lqcd_geom *geom, int parity, int prec, int nrhs,
                                   size_t *scale_bytes) {
  if (scale_bytes) *scale_bytes = 0;
  if (!geom || nrhs < 1 || prec < LQCD_F64 || prec > LQCD_F16S) return 0;
  for (int k = 0; k < 4; k++)
    if (geom->L[k] < 2 || (geom->L[k] & 1)) return 0;
  Geom g = make_geom(*geom);
  size_t np = parity == LQCD_FULL ? 2 : 1;
  if (scale_bytes) *scale_bytes = spinor_scale_half_bytes(prec, g.Vh) * np * nrhs;
  return spinor_half_bytes(prec, g.Vh) * np * nrhs;
}

// ===========================================================================
// Gauge fields
// ===========================================================================

extern "C" int lqcd_gauge_import(lqcd_ctx *ctx, const void *U_lexi, const lqcd_geom *geom, int recon,
                                 lqcd_gauge **out) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (!out) return fail(ctx, LQCD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  LQCD_TRY(check_geom(ctx, geom));
  if (!U_lexi || !aligned16(U_lexi)) return fail(ctx, LQCD_ERR_INVALID, "U: NULL or misaligned pointer");
  if (recon != 18 && recon != 12) return fail(ctx, LQCD_ERR_INVALID, "recon must be 18 or 12");
  lqcd_gauge *U = new (std::nothrow) lqcd_gauge();
  if (!U) return fail(ctx, LQCD_ERR_OOM, "host allocation failed");
  U->geom = *geom;
  U->g = make_geom(*geom);
  U->recon = recon;
  size_t bytes = (size_t)2 * 4 * 9 * U->g.Vh * 16;
  U->A = ctx->A;
  if (raw_alloc(ctx, U->A, &U->master, bytes) != LQCD_OK) {
    delete U;
    return fail(ctx, LQCD_ERR_OOM, "gauge allocation of %zu bytes failed", bytes);
  }
  lqcd_status s = gauge_import_raw(ctx, U, U_lexi);
  double dev = 0.0;
  if (s == LQCD_OK && recon == 12) {
    s = gauge_su3_deviation(ctx, U, &dev);
    if (s == LQCD_OK && !(dev <= 1e-12))
      s = fail(ctx, LQCD_ERR_INVALID, "REC12 needs SU(3) links: max deviation %.3e", dev);
  }
  if (s == LQCD_OK) s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "gauge import");
  if (s != LQCD_OK) {
    cudaStreamSynchronize(ctx->stream);
    raw_free(ctx, U->A, U->master);
    delete U;
    return s;
  }
  *out = U;
  return LQCD_OK;
}

extern "C" int lqcd_gauge_export(lqcd_ctx *ctx, const lqcd_gauge *U, void *U_lexi) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (!U || !U_lexi || !aligned16(U_lexi)) return fail(ctx, LQCD_ERR_INVALID, "NULL or misaligned argument");
  return gauge_export_raw(ctx, U, U_lexi);
}

extern "C" int lqcd_gauge_free(lqcd_ctx *ctx, lqcd_gauge *U) {
  if (!U) return ctx ? fail(ctx, LQCD_ERR_INVALID, "U is NULL") : LQCD_ERR_INVALID;
  if (!ctx) return LQCD_ERR_INVALID;
  cudaStreamSynchronize(ctx->stream);
  raw_free(ctx, U->A, U->master);
  for (auto &c : U->copies) raw_free(ctx, U->A, c.ptr);
  cudaStreamSynchronize(ctx->stream);
  delete U;
  return LQCD_OK;
}

// ===========================================================================
// Spinor layout / precision
// ===========================================================================

extern "C" int lqcd_spinor_pack(lqcd_ctx *ctx, const lqcd_geom *geom, const void *lexi, lqcd_field eo) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  LQCD_TRY(check_field(ctx, eo, "eo", false));
  if (!lexi || !aligned16(lexi)) return fail(ctx, LQCD_ERR_INVALID, "lexi: NULL or misaligned");
  Geom g = make_geom(*geom);
  return spinor_pack_raw(ctx, g, lexi, to_half(eo, g, true));
}

extern "C" int lqcd_spinor_unpack(lqcd_ctx *ctx, const lqcd_geom *geom, lqcd_field eo, void *lexi) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  LQCD_TRY(check_field(ctx, eo, "eo", false));
  if (!lexi || !aligned16(lexi)) return fail(ctx, LQCD_ERR_INVALID, "lexi: NULL or misaligned");
  Geom g = make_geom(*geom);
  return spinor_unpack_raw(ctx, g, to_half(eo, g, true), lexi);
}

extern "C" int lqcd_spinor_convert(lqcd_ctx *ctx, const lqcd_geom *geom, int parity, lqcd_field in,
                                   lqcd_field out) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_geom(ctx, geom));
  LQCD_TRY(check_field(ctx, in, "in", false));
  LQCD_TRY(check_field(ctx, out, "out", false));
  if (in.nrhs != out.nrhs) return fail(ctx, LQCD_ERR_INVALID, "nrhs mismatch");
  Geom g = make_geom(*geom);
  int nh = in.nrhs * (parity == LQCD_FULL ? 2 : 1);
  return spinor_convert_raw(ctx, g.Vh, nh, in.ptr, (const float *)in.scale, in.prec, out.ptr,
                            (float *)out.scale, out.prec);
}

// ===========================================================================
// Operators
// ===========================================================================

static lqcd_status check_gauge(lqcd_ctx *ctx, const lqcd_gauge *U, const lqcd_geom *geom) {
  if (!U) return fail(ctx, LQCD_ERR_INVALID, "gauge field is NULL");
  LQCD_TRY(check_geom(ctx, geom));
  if (!geom_equal(U->geom, *geom)) return fail(ctx, LQCD_ERR_INVALID, "geometry does not match the gauge field");
  return LQCD_OK;
}

static int link_recon_for(const lqcd_gauge *U, int prec) {
  return (prec == LQCD_BF16S || prec == LQCD_F16S) ? 12 : U->recon;
}

extern "C" int lqcd_dslash(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                           const lqcd_geom *geom, int out_parity, int dagger) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_gauge(ctx, U, geom));
  LQCD_TRY(check_field(ctx, in, "in", false));
  LQCD_TRY(check_field(ctx, out, "out", false));
  if (in.prec != out.prec || in.nrhs != out.nrhs)
    return fail(ctx, LQCD_ERR_INVALID, "in/out precision or nrhs differ");
  if (out_parity != LQCD_EVEN && out_parity != LQCD_ODD)
    return fail(ctx, LQCD_ERR_INVALID, "out_parity must be LQCD_EVEN or LQCD_ODD");
  Geom g = make_geom(*geom);
  size_t bytes = spinor_half_bytes(in.prec, g.Vh) * in.nrhs;
  if (ranges_overlap(in.ptr, bytes, out.ptr, bytes)) return fail(ctx, LQCD_ERR_INVALID, "in and out alias");
  HopLaunch L;
  L.prec = in.prec;
  L.recon = link_recon_for(U, in.prec);
  LQCD_TRY(gauge_view(ctx, const_cast<lqcd_gauge *>(U), in.prec, L.recon, &L.U));
  L.in = to_half(in, g, false);
  L.out = to_half(out, g, false);
  L.out_parity = out_parity == LQCD_EVEN ? 0 : 1;
  L.dagger = dagger ? 1 : 0;
  return launch_hop(ctx, g, L, nullptr);
}

// ===========================================================================
// Domain decomposition along t and z
// ===========================================================================

extern "C" size_t lqcd_dd_face_bytes_dir(const lqcd_geom *local, int mu, int prec) {
  if (!local || (prec != LQCD_F64 && prec != LQCD_DF64 && prec != LQCD_F32) || (mu != 2 && mu != 3)) return 0;
  for (int k = 0; k < 4; k++)
    if (local->L[k] < 2 || (local->L[k] & 1)) return 0;
  return (size_t)(local->L[0] / 2) * local->L[1] * local->L[mu == 3 ? 2 : 3] * 6 * dd_face_word_bytes(prec);
}

extern "C" size_t lqcd_dd_face_bytes(const lqcd_geom *local, int prec) {
  return lqcd_dd_face_bytes_dir(local, 3, prec);
}

static bool bad_face(const void *f) { return !f || ((uintptr_t)f & 15u); }

static lqcd_status dd_common(lqcd_ctx *ctx, const lqcd_gauge *U, const lqcd_field &in, const lqcd_geom *local,
                             int out_parity, int dagger, HopLaunch *L, Geom *g) {
  LQCD_TRY(check_gauge(ctx, U, local));
  LQCD_TRY(check_field(ctx, in, "in", false));
  if (in.nrhs != 1) return fail(ctx, LQCD_ERR_UNSUPPORTED, "domain-decomposed hop: nrhs must be 1");
  if (in.prec != LQCD_F64 && in.prec != LQCD_DF64 && in.prec != LQCD_F32)
    return fail(ctx, LQCD_ERR_UNSUPPORTED, "domain-decomposed hop: precision must be F64, DF64 or F32");
  if (out_parity != LQCD_EVEN && out_parity != LQCD_ODD)
    return fail(ctx, LQCD_ERR_INVALID, "out_parity must be LQCD_EVEN or LQCD_ODD");
  lqcd_geom lg = *local;
  lg.antiperiodic_t = 0;  // the global boundary sign travels in the faces
  *g = make_geom(lg);
  L->prec = in.prec;
  L->recon = link_recon_for(U, in.prec);
  LQCD_TRY(gauge_view(ctx, const_cast<lqcd_gauge *>(U), in.prec, L->recon, &L->U));
  L->in = to_half(in, *g, false);
  L->out_parity = out_parity == LQCD_EVEN ? 0 : 1;
  L->dagger = dagger ? 1 : 0;
  return LQCD_OK;
}

extern "C" int lqcd_dd_pack_dir(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, int mu, void *face_to_prev,
                                void *face_to_next, const lqcd_geom *local, int out_parity, int dagger,
                                int negate_to_prev, int negate_to_next) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (mu != 2 && mu != 3) return fail(ctx, LQCD_ERR_INVALID, "faces along mu = 2 (z) or 3 (t)");
  if (bad_face(face_to_prev) || bad_face(face_to_next))
    return fail(ctx, LQCD_ERR_INVALID, "faces: NULL or not 16-byte aligned");
  HopLaunch L;
  Geom g;
  LQCD_TRY(dd_common(ctx, U, in, local, out_parity, dagger, &L, &g));
  const size_t fb = lqcd_dd_face_bytes_dir(local, mu, in.prec);
  if (ranges_overlap(face_to_prev, fb, face_to_next, fb)) return fail(ctx, LQCD_ERR_INVALID, "faces alias");
  return dd_pack(ctx, g, L, mu, face_to_prev, face_to_next, negate_to_prev ? 1 : 0, negate_to_next ? 1 : 0);
}

extern "C" int lqcd_dd_pack(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, void *face_to_prev,
                            void *face_to_next, const lqcd_geom *local, int out_parity, int dagger,
                            int negate_to_prev, int negate_to_next) {
  return lqcd_dd_pack_dir(ctx, U, in, 3, face_to_prev, face_to_next, local, out_parity, dagger, negate_to_prev,
                          negate_to_next);
}

extern "C" int lqcd_dd_dslash_zt(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                                 const void *t_from_next, const void *t_from_prev, const void *z_from_next,
                                 const void *z_from_prev, const lqcd_geom *local, int out_parity, int dagger) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (bad_face(t_from_next) || bad_face(t_from_prev))
    return fail(ctx, LQCD_ERR_INVALID, "faces: NULL or not 16-byte aligned");
  if ((z_from_next == nullptr) != (z_from_prev == nullptr) ||
      (z_from_next && (bad_face(z_from_next) || bad_face(z_from_prev))))
    return fail(ctx, LQCD_ERR_INVALID, "z faces: both NULL, or both 16-byte aligned");
  HopLaunch L;
  Geom g;
  LQCD_TRY(dd_common(ctx, U, in, local, out_parity, dagger, &L, &g));
  LQCD_TRY(check_field(ctx, out, "out", false));
  if (out.prec != in.prec || out.nrhs != 1) return fail(ctx, LQCD_ERR_INVALID, "in/out precision or nrhs differ");
  const size_t bytes = spinor_half_bytes(in.prec, g.Vh);
  if (ranges_overlap(in.ptr, bytes, out.ptr, bytes)) return fail(ctx, LQCD_ERR_INVALID, "in and out alias");
  L.out = to_half(out, g, false);
  return dd_hop(ctx, g, L, t_from_next, t_from_prev, z_from_next, z_from_prev);
}

extern "C" int lqcd_dd_dslash(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                              const void *face_from_next, const void *face_from_prev, const lqcd_geom *local,
                              int out_parity, int dagger) {
  return lqcd_dd_dslash_zt(ctx, U, in, out, face_from_next, face_from_prev, nullptr, nullptr, local, out_parity,
                           dagger);
}

static lqcd_status check_cg_params(lqcd_ctx *ctx, const lqcd_cg_params *p);

extern "C" int lqcd_dd_cg_solve(lqcd_ctx *ctx, int nd, const lqcd_gauge *const *U, const lqcd_field *b,
                                const lqcd_field *x, void *const *faces, const lqcd_geom *local, int first_domain,
                                int nz, int nt, int antiperiodic_t, double kappa, double mu,
                                const lqcd_cg_params *params, const lqcd_dd_comm *comm, lqcd_cg_stats *stats) {
  if (!ctx) return LQCD_ERR_INVALID;
  if (!U || !b || !x || !faces || !local || !params || !stats)
    return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: NULL argument");
  if (nz < 1 || nt < 1 || nd < 1 || first_domain < 0 || first_domain + nd > nz * nt)
    return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: domains %d..%d of %d x %d", first_domain,
                first_domain + nd - 1, nz, nt);
  if (!comm && (nd != nz * nt || first_domain != 0))
    return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG without comm hooks must hold every domain");
  if (comm && !comm->exchange) return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: no exchange hook");
  LQCD_TRY(check_cg_params(ctx, params));
  const int inner = params->inner_prec;
  if (params->outer_prec != LQCD_F64 || params->solver != LQCD_SOLVER_CG ||
      (inner != LQCD_F64 && inner != LQCD_DF64 && inner != LQCD_F32))
    return fail(ctx, LQCD_ERR_UNSUPPORTED,
                "domain-decomposed CG: CG with outer_prec F64 and inner_prec F64, DF64 or F32");
  if (!std::isfinite(kappa) || !std::isfinite(mu)) return fail(ctx, LQCD_ERR_NONFINITE, "kappa/mu not finite");
  const size_t fb_t = lqcd_dd_face_bytes_dir(local, 3, LQCD_F64), fb_z = lqcd_dd_face_bytes_dir(local, 2, LQCD_F64);
  if (fb_t == 0) return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: bad local geometry");
  lqcd_geom lg = *local;
  lg.antiperiodic_t = 0;  // the global boundary sign travels in the faces
  const Geom g = make_geom(lg);
  const size_t full_bytes = 2 * spinor_half_bytes(LQCD_F64, g.Vh);
  const int nf = nz > 1 ? 8 : 4;  // faces per held domain: t, then z
  std::vector<GaugeView> views(nd), views_i(inner == LQCD_F64 ? 0 : nd);
  std::vector<HalfField> bf(nd), xf(nd);
  std::vector<void *> fv((size_t)nf * nd);
  auto fsize = [&](int i) { return i % nf < 4 ? fb_t : fb_z; };
  int recon = 0, recon_i = 0;
  for (int d = 0; d < nd; d++) {
    LQCD_TRY(check_gauge(ctx, U[d], local));
    if (d == 0) {
      recon = U[0]->recon;
      recon_i = params->sloppy_recon ? params->sloppy_recon : recon;
    }
    if (U[d]->recon != recon) return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: mixed link formats");
    LQCD_TRY(gauge_view(ctx, const_cast<lqcd_gauge *>(U[d]), LQCD_F64, recon, &views[d]));
    if (inner != LQCD_F64) LQCD_TRY(gauge_view(ctx, const_cast<lqcd_gauge *>(U[d]), inner, recon_i, &views_i[d]));
    LQCD_TRY(check_field(ctx, b[d], "b", false));
    LQCD_TRY(check_field(ctx, x[d], "x", false));
    if (b[d].prec != LQCD_F64 || x[d].prec != LQCD_F64 || b[d].nrhs != 1 || x[d].nrhs != 1)
      return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: b and x must be LQCD_F64 with nrhs = 1");
    if (ranges_overlap(b[d].ptr, full_bytes, x[d].ptr, full_bytes))
      return fail(ctx, LQCD_ERR_INVALID, "domain-decomposed CG: b and x alias");
    bf[d] = to_half(b[d], g, true);
    xf[d] = to_half(x[d], g, true);
    for (int k = 0; k < nf; k++) {
      const int i = nf * d + k;
      void *f = faces[i];
      if (bad_face(f)) return fail(ctx, LQCD_ERR_INVALID, "faces: NULL or not 16-byte aligned");
      for (int j = 0; j < i; j++)
        if (ranges_overlap(f, fsize(i), faces[j], fsize(j)))
          return fail(ctx, LQCD_ERR_INVALID, "face buffers alias");
      fv[i] = f;
    }
  }
  return dd_cg_solve(ctx, nd, first_domain, nz, nt, antiperiodic_t ? 1 : 0, g, recon, views, recon_i, views_i, bf,
                     xf, fv, comm, kappa, mu, *params, stats);
}

static int apply_impl(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                      const lqcd_geom *geom, double kappa, double mu, int parity, bool dagger) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_gauge(ctx, U, geom));
  LQCD_TRY(check_field(ctx, in, "in", true));
  LQCD_TRY(check_field(ctx, out, "out", true));
  if (in.prec != out.prec || in.nrhs != out.nrhs || in.layout != out.layout)
    return fail(ctx, LQCD_ERR_INVALID, "in/out precision, layout or nrhs differ");
  if (!std::isfinite(kappa) || !std::isfinite(mu)) return fail(ctx, LQCD_ERR_NONFINITE, "kappa/mu not finite");
  if (in.prec != LQCD_F64 && in.prec != LQCD_DF64 && in.prec != LQCD_F32)
    return fail(ctx, LQCD_ERR_UNSUPPORTED, "apply_M: precision must be F64, DF64 or F32");
  Geom g = make_geom(*geom);
  const bool full = parity == LQCD_FULL;
  if (!full && parity != LQCD_EVEN && parity != LQCD_ODD) return fail(ctx, LQCD_ERR_INVALID, "bad parity");
  if (!full && in.layout != LQCD_LAYOUT_EO)
    return fail(ctx, LQCD_ERR_INVALID, "Schur complement operates on EO half fields");
  size_t bytes = spinor_half_bytes(in.prec, g.Vh) * in.nrhs * (full ? 2 : 1);
  if (ranges_overlap(in.ptr, bytes, out.ptr, bytes)) return fail(ctx, LQCD_ERR_INVALID, "in and out alias");
  Op op{ctx, g, {}, in.prec, link_recon_for(U, in.prec), kappa, mu};
  LQCD_TRY(gauge_view(ctx, const_cast<lqcd_gauge *>(U), op.prec, op.recon, &op.U));
  if (!full) {
    HalfField hi = to_half(in, g, false), ho = to_half(out, g, false);
    HalfField tmp;
    tmp.prec = in.prec;
    tmp.nrhs = in.nrhs;
    tmp.rhs_stride = hi.rhs_stride;
    LQCD_TRY(dalloc(ctx, &tmp.ptr, tmp.rhs_stride * in.nrhs));
    lqcd_status s = apply_schur(op, hi, ho, tmp, parity == LQCD_EVEN ? 0 : 1, dagger, nullptr, nullptr, nullptr);
    dfree(ctx, tmp.ptr);
    return s;
  }
  if (in.layout == LQCD_LAYOUT_EO) {
    HalfField fi = to_half(in, g, true), fo = to_half(out, g, true);
    return apply_full(op, half_of_full(fi, 0, g.Vh), half_of_full(fi, 1, g.Vh), half_of_full(fo, 0, g.Vh),
                      half_of_full(fo, 1, g.Vh), dagger, nullptr, nullptr, nullptr);
  }
  // lexicographic complex128: pack, apply, unpack
  HalfField wi, wo;
  wi.prec = wo.prec = LQCD_F64;
  wi.nrhs = wo.nrhs = in.nrhs;
  wi.rhs_stride = wo.rhs_stride = 2 * spinor_half_bytes(LQCD_F64, g.Vh);
  LQCD_TRY(dalloc(ctx, &wi.ptr, wi.rhs_stride * in.nrhs));
  lqcd_status s = dalloc(ctx, &wo.ptr, wo.rhs_stride * in.nrhs);
  if (s == LQCD_OK) s = spinor_pack_raw(ctx, g, in.ptr, wi);
  if (s == LQCD_OK)
    s = apply_full(op, half_of_full(wi, 0, g.Vh), half_of_full(wi, 1, g.Vh), half_of_full(wo, 0, g.Vh),
                   half_of_full(wo, 1, g.Vh), dagger, nullptr, nullptr, nullptr);
  if (s == LQCD_OK) s = spinor_unpack_raw(ctx, g, wo, out.ptr);
  dfree(ctx, wi.ptr);
  dfree(ctx, wo.ptr);
  return s;
}

extern "C" int lqcd_apply_M(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                            const lqcd_geom *geom, double kappa, double mu, int parity) {
  return apply_impl(ctx, U, in, out, geom, kappa, mu, parity, false);
}

extern "C" int lqcd_apply_Mdag(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                               const lqcd_geom *geom, double kappa, double mu, int parity) {
  return apply_impl(ctx, U, in, out, geom, kappa, mu, parity, true);
}

// ===========================================================================
// Solver
// ===========================================================================

static lqcd_status check_cg_params(lqcd_ctx *ctx, const lqcd_cg_params *p) {
  if (!p) return fail(ctx, LQCD_ERR_INVALID, "params is NULL");
  if (!(p->tol > 0.0) || !std::isfinite(p->tol)) return fail(ctx, LQCD_ERR_INVALID, "tol must be > 0");
  if (p->max_iter < 1) return fail(ctx, LQCD_ERR_INVALID, "max_iter must be >= 1");
  if (p->outer_prec != LQCD_F64 && p->outer_prec != LQCD_DF64)
    return fail(ctx, LQCD_ERR_INVALID, "outer_prec must be LQCD_F64 or LQCD_DF64");
  if (p->inner_prec < LQCD_F64 || p->inner_prec > LQCD_F16S)
    return fail(ctx, LQCD_ERR_INVALID, "bad inner_prec");
  if (p->inner_prec == LQCD_F64 && p->outer_prec != LQCD_F64)
    return fail(ctx, LQCD_ERR_INVALID, "inner F64 needs outer F64");
  if (p->sloppy_recon != 18 && p->sloppy_recon != 12 && p->sloppy_recon != 0)
    return fail(ctx, LQCD_ERR_INVALID, "sloppy_recon must be 18 or 12");
  if (p->max_restarts < 0) return fail(ctx, LQCD_ERR_INVALID, "max_restarts must be >= 0");
  if (p->solver != LQCD_SOLVER_CG && p->solver != LQCD_SOLVER_BICGSTAB)
    return fail(ctx, LQCD_ERR_INVALID, "solver must be LQCD_SOLVER_CG or LQCD_SOLVER_BICGSTAB");
  if (!std::isfinite(p->inner_tol) || p->inner_tol < 0.0 || p->inner_tol >= 1.0)
    return fail(ctx, LQCD_ERR_INVALID, "inner_tol must be in [0, 1)");
  return LQCD_OK;
}

extern "C" int lqcd_cg_solve(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field b, lqcd_field x,
                             const lqcd_geom *geom, double kappa, double mu, const lqcd_cg_params *params,
                             lqcd_cg_stats *stats) {
  if (!ctx) return LQCD_ERR_INVALID;
  LQCD_TRY(check_gauge(ctx, U, geom));
  LQCD_TRY(check_field(ctx, b, "b", true));
  LQCD_TRY(check_field(ctx, x, "x", true));
  LQCD_TRY(check_cg_params(ctx, params));
  if (!stats) return fail(ctx, LQCD_ERR_INVALID, "stats is NULL");
  if (b.prec != LQCD_F64 || x.prec != LQCD_F64) return fail(ctx, LQCD_ERR_INVALID, "b and x must be LQCD_F64");
  if (b.layout != x.layout || b.nrhs != x.nrhs) return fail(ctx, LQCD_ERR_INVALID, "b/x layout or nrhs differ");
  if (params->solver == LQCD_SOLVER_BICGSTAB && b.nrhs != 1)
    return fail(ctx, LQCD_ERR_UNSUPPORTED, "BiCGStab solves one right-hand side at a time");
  if (!std::isfinite(kappa) || !std::isfinite(mu)) return fail(ctx, LQCD_ERR_NONFINITE, "kappa/mu not finite");
  Geom g = make_geom(*geom);
  size_t bytes = 2 * spinor_half_bytes(LQCD_F64, g.Vh) * b.nrhs;
  if (ranges_overlap(b.ptr, bytes, x.ptr, bytes)) return fail(ctx, LQCD_ERR_INVALID, "b and x alias");
  lqcd_cg_params prm = *params;
  if (prm.sloppy_recon == 0) prm.sloppy_recon = U->recon;
  if (prm.check_every <= 0) prm.check_every = 10;
  lqcd_gauge *Um = const_cast<lqcd_gauge *>(U);
  if (b.layout == LQCD_LAYOUT_EO)
    return cg_solve_eo(ctx, Um, to_half(b, g, true), to_half(x, g, true), kappa, mu, prm, stats);
  HalfField wb, wx;
  wb.prec = wx.prec = LQCD_F64;
  wb.nrhs = wx.nrhs = b.nrhs;
  wb.rhs_stride = wx.rhs_stride = 2 * spinor_half_bytes(LQCD_F64, g.Vh);
  LQCD_TRY(dalloc(ctx, &wb.ptr, wb.rhs_stride * b.nrhs));
  lqcd_status s = dalloc(ctx, &wx.ptr, wx.rhs_stride * b.nrhs);
  if (s == LQCD_OK) s = spinor_pack_raw(ctx, g, b.ptr, wb);
  if (s == LQCD_OK) s = cg_solve_eo(ctx, Um, wb, wx, kappa, mu, prm, stats);
  if (s == LQCD_OK || s == LQCD_ERR_NOCONV) {
    lqcd_status s2 = spinor_unpack_raw(ctx, g, wx, x.ptr);
    if (s2 != LQCD_OK) s = s2;
  }
  dfree(ctx, wb.ptr);
  dfree(ctx, wx.ptr);
  cudaStreamSynchronize(ctx->stream);
  return s;
}
