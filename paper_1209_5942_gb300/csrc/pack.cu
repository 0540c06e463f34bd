// pack.cu -- layout and precision conversion at the library boundary.
//
// The paper converts transparently between the CPU's array-of-structures and
// the GPU's structure-of-arrays when data moves to the device (Sec. 4.3) and
// splits the gauge field by the parity of the originating site (Sec. 4.2).
// Here the user-facing layout is lexicographic AoS complex128; the kernels
// use even-odd SoA planes of 16-byte words (see common.cuh).  Lower-precision
// copies of the links (DF64, F32, REC12, BF16/F16 REC12) are derived from the
// FP64 master on demand and cached until the master changes.
#include <cmath>

#include "internal.h"

namespace lqcd {

template <class R> LQCD_DEV Cx<R> cx_from_d(double re, double im) {
  return {from_double<R>(re), from_double<R>(im)};
}

// lexicographic site i -> (parity, cb)
LQCD_DEV void parity_cb(const Geom &g, long i, int *p, int *cb) {
  int x = (int)(i % g.L[0]);
  long r = i / g.L[0];
  int y = (int)(r % g.L[1]);
  long zt = r / g.L[1];
  int z = (int)(zt % g.L[2]);
  int t = (int)(zt / g.L[2]);
  *p = (x + y + z + t) & 1;
  *cb = (int)(i >> 1);
}

// ---------------------------------------------------------------------------
// gauge: lexicographic [V][4][3][3] complex128 <-> master [p][mu][9][Vh]
// ---------------------------------------------------------------------------

__global__ void gauge_import_kernel(Geom g, const double2 *__restrict__ src,
                                    double2 *__restrict__ dst) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long V = 2L * g.Vh;
  if (i >= V) return;
  int p, cb;
  parity_cb(g, i, &p, &cb);
#pragma unroll
  for (int mu = 0; mu < 4; mu++)
#pragma unroll
    for (int k = 0; k < 9; k++)
      dst[(((size_t)p * 4 + mu) * 9 + k) * g.Vh + cb] = src[(i * 4 + mu) * 9 + k];
}

__global__ void gauge_export_kernel(Geom g, const double2 *__restrict__ src,
                                    double2 *__restrict__ dst) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long V = 2L * g.Vh;
  if (i >= V) return;
  int p, cb;
  parity_cb(g, i, &p, &cb);
#pragma unroll
  for (int mu = 0; mu < 4; mu++)
#pragma unroll
    for (int k = 0; k < 9; k++)
      dst[(i * 4 + mu) * 9 + k] = src[(((size_t)p * 4 + mu) * 9 + k) * g.Vh + cb];
}

// Largest deviation from SU(3) (|U U^+ - 1|_max and |det U - 1|) per block.
__global__ void su3_deviation_kernel(Geom g, const double2 *__restrict__ m, double *partials) {
  __shared__ double sh[256];
  size_t nl = (size_t)2 * 4 * g.Vh;
  size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  double dev = 0.0;
  if (l < nl) {
    size_t blk = l / g.Vh, cb = l % g.Vh;
    double2 u[9];
    for (int k = 0; k < 9; k++) u[k] = m[(blk * 9 + k) * g.Vh + cb];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double re = 0, im = 0;
        for (int c = 0; c < 3; c++) {
          double2 x = u[3 * a + c], y = u[3 * b + c];
          re += x.x * y.x + x.y * y.y;
          im += x.y * y.x - x.x * y.y;
        }
        dev = fmax(dev, fabs(re - (a == b)) + fabs(im));
      }
    // det by cofactors of row 0
    double c0r = u[4].x * u[8].x - u[4].y * u[8].y - (u[5].x * u[7].x - u[5].y * u[7].y);
    double c0i = u[4].x * u[8].y + u[4].y * u[8].x - (u[5].x * u[7].y + u[5].y * u[7].x);
    double c1r = u[5].x * u[6].x - u[5].y * u[6].y - (u[3].x * u[8].x - u[3].y * u[8].y);
    double c1i = u[5].x * u[6].y + u[5].y * u[6].x - (u[3].x * u[8].y + u[3].y * u[8].x);
    double c2r = u[3].x * u[7].x - u[3].y * u[7].y - (u[4].x * u[6].x - u[4].y * u[6].y);
    double c2i = u[3].x * u[7].y + u[3].y * u[7].x - (u[4].x * u[6].y + u[4].y * u[6].x);
    double dr = u[0].x * c0r - u[0].y * c0i + u[1].x * c1r - u[1].y * c1i + u[2].x * c2r - u[2].y * c2i;
    double di = u[0].x * c0i + u[0].y * c0r + u[1].x * c1i + u[1].y * c1r + u[2].x * c2i + u[2].y * c2r;
    dev = fmax(dev, fabs(dr - 1.0) + fabs(di));
    if (!isfinite(dev)) dev = INFINITY;
  }
  sh[threadIdx.x] = dev;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// master -> copy in (prec, recon)
template <int PREC, int RECON>
__global__ void gauge_copy_kernel(Geom g, const double2 *__restrict__ m, char *__restrict__ dst) {
  size_t nl = (size_t)2 * 4 * g.Vh;
  size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (l >= nl) return;
  size_t blk = l / g.Vh, cb = l % g.Vh;  // blk = parity*4 + mu
  constexpr int NE = RECON == 18 ? 9 : 6;
  double2 u[9];
#pragma unroll
  for (int k = 0; k < 9; k++) u[k] = m[(blk * 9 + k) * g.Vh + cb];
  const size_t mu_stride = (size_t)g.Vh * link_bytes_per_site(PREC, RECON);
  char *base = dst + blk * mu_stride;
  if (PREC == LQCD_F64) {
    double2 *b = (double2 *)base;
#pragma unroll
    for (int k = 0; k < NE; k++) b[(size_t)k * g.Vh + cb] = u[k];
  } else if (PREC == LQCD_DF64) {
    float4 *b = (float4 *)base;
#pragma unroll
    for (int k = 0; k < NE; k++) {
      df re = df_from_double(u[k].x), im = df_from_double(u[k].y);
      b[(size_t)k * g.Vh + cb] = make_float4(re.hi, im.hi, re.lo, im.lo);
    }
  } else if (PREC == LQCD_F32) {
    float4 *b = (float4 *)base;
    constexpr int NW = RECON == 18 ? 4 : 3;
#pragma unroll
    for (int k = 0; k < NW; k++)
      b[(size_t)k * g.Vh + cb] = make_float4((float)u[2 * k].x, (float)u[2 * k].y,
                                             (float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
    if (RECON == 18) {
      float2 *t = (float2 *)(base + (size_t)4 * g.Vh * 16);
      t[cb] = make_float2((float)u[8].x, (float)u[8].y);
    }
  } else {  // 16-bit, recon 12
    uint32_t w[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      uint32_t lo, hi;
      if (PREC == LQCD_BF16S) {
        lo = Half16<__nv_bfloat16>::from_f((float)u[k].x);
        hi = Half16<__nv_bfloat16>::from_f((float)u[k].y);
      } else {
        lo = Half16<__half>::from_f((float)u[k].x);
        hi = Half16<__half>::from_f((float)u[k].y);
      }
      w[k] = lo | (hi << 16);
    }
    ((uint4 *)base)[cb] = make_uint4(w[0], w[1], w[2], w[3]);
    ((uint2 *)(base + (size_t)g.Vh * 16))[cb] = make_uint2(w[4], w[5]);
  }
}

// ---------------------------------------------------------------------------
// spinors: lexicographic [nrhs][V][12] complex128 <-> EO full field [nrhs][2][..]
// ---------------------------------------------------------------------------

template <int PREC>
__global__ void spinor_pack_kernel(Geom g, const double2 *__restrict__ src, char *dst, float *scale,
                                   size_t rs, size_t srs, size_t half_bytes, size_t half_floats,
                                   int nrhs) {
  using R = typename SpinorIO<PREC>::R;
  long V = 2L * g.Vh;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (i >= V || r >= nrhs) return;
  int p, cb;
  parity_cb(g, i, &p, &cb);
  Cx<R> s[12];
  const double2 *in = src + ((size_t)r * V + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 w = in[k];
    s[k] = cx_from_d<R>(w.x, w.y);
  }
  SpinorView v{dst + r * rs + p * half_bytes, scale ? scale + r * srs + p * half_floats : nullptr,
               g.Vh};
  SpinorIO<PREC>::store(v, cb, s);
}

template <int PREC>
__global__ void spinor_unpack_kernel(Geom g, const char *src, const float *scale, double2 *dst,
                                     size_t rs, size_t srs, size_t half_bytes, size_t half_floats,
                                     int nrhs) {
  using R = typename SpinorIO<PREC>::R;
  long V = 2L * g.Vh;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (i >= V || r >= nrhs) return;
  int p, cb;
  parity_cb(g, i, &p, &cb);
  Cx<R> s[12];
  SpinorView v{(void *)(src + r * rs + p * half_bytes),
               scale ? (float *)scale + r * srs + p * half_floats : nullptr, g.Vh};
  SpinorIO<PREC>::load(v, cb, s);
  double2 *out = dst + ((size_t)r * V + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) out[k] = make_double2(to_double(s[k].re), to_double(s[k].im));
}

// EO precision conversion of nh half fields (nrhs x parities), element-wise per site.
template <int PIN, int POUT>
__global__ void spinor_convert_kernel(int Vh, int nh, const char *in, const float *in_scale,
                                      size_t in_hb, size_t in_hf, char *out, float *out_scale,
                                      size_t out_hb, size_t out_hf) {
  int cb = blockIdx.x * blockDim.x + threadIdx.x;
  int h = blockIdx.y;
  if (cb >= Vh || h >= nh) return;
  typename SpinorIO<PIN>::R dummy;
  (void)dummy;
  Cx<typename SpinorIO<PIN>::R> a[12];
  SpinorView vi{(void *)(in + h * in_hb), in_scale ? (float *)in_scale + h * in_hf : nullptr, Vh};
  SpinorIO<PIN>::load(vi, cb, a);
  using RO = typename SpinorIO<POUT>::R;
  Cx<RO> b[12];
#pragma unroll
  for (int k = 0; k < 12; k++)
    b[k] = {from_double<RO>(to_double(a[k].re)), from_double<RO>(to_double(a[k].im))};
  SpinorView vo{out + h * out_hb, out_scale ? out_scale + h * out_hf : nullptr, Vh};
  SpinorIO<POUT>::store(vo, cb, b);
}

// ---------------------------------------------------------------------------
// host entry points used by api.cu
// ---------------------------------------------------------------------------

lqcd_status gauge_import_raw(lqcd_ctx *ctx, const lqcd_gauge *U, const void *src) {
  long V = 2L * U->g.Vh;
  gauge_import_kernel<<<(unsigned)((V + 127) / 128), 128, 0, ctx->stream>>>(
      U->g, (const double2 *)src, (double2 *)U->master);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status gauge_export_raw(lqcd_ctx *ctx, const lqcd_gauge *U, void *dst) {
  long V = 2L * U->g.Vh;
  gauge_export_kernel<<<(unsigned)((V + 127) / 128), 128, 0, ctx->stream>>>(
      U->g, (const double2 *)U->master, (double2 *)dst);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status gauge_su3_deviation(lqcd_ctx *ctx, const lqcd_gauge *U, double *dev) {
  size_t nl = (size_t)8 * U->g.Vh;
  int nb = (int)((nl + 255) / 256);
  LQCD_TRY(ensure_partials(ctx, nb));
  LQCD_TRY(ensure_pinned(ctx, nb));
  su3_deviation_kernel<<<nb, 256, 0, ctx->stream>>>(U->g, (const double2 *)U->master, ctx->partials);
  LQCD_CUDA(ctx, cudaGetLastError());
  LQCD_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, ctx->partials, nb * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
  LQCD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double m = 0.0;
  for (int k = 0; k < nb; k++) m = std::fmax(m, ctx->pinned[k]);
  *dev = m;
  return LQCD_OK;
}

lqcd_status gauge_view(lqcd_ctx *ctx, lqcd_gauge *U, int prec, int recon, GaugeView *out) {
  const size_t Vh = U->g.Vh;
  if ((prec == LQCD_BF16S || prec == LQCD_F16S) && recon != 12)
    return fail(ctx, LQCD_ERR_UNSUPPORTED, "16-bit links are stored in REC12 form only");
  size_t mu_stride = Vh * link_bytes_per_site(prec, recon);
  out->Vh = (int)Vh;
  out->mu_stride = mu_stride;
  out->parity_stride = 4 * mu_stride;
  if (prec == LQCD_F64 && recon == 18) {
    out->ptr = U->master;
    return LQCD_OK;
  }
  lqcd_gauge::Copy *c = nullptr;
  for (auto &k : U->copies)
    if (k.prec == prec && k.recon == recon) c = &k;
  if (!c) {
    U->copies.push_back(lqcd_gauge::Copy());
    c = &U->copies.back();
    c->prec = prec;
    c->recon = recon;
    void *p = nullptr;
    if (raw_alloc(ctx, U->A, &p, 2 * 4 * mu_stride) != LQCD_OK) {
      U->copies.pop_back();
      return fail(ctx, LQCD_ERR_OOM, "gauge copy allocation of %zu bytes failed", 8 * mu_stride);
    }
    c->ptr = p;
    c->version = 0;
  }
  if (c->version != U->version) {
    size_t nl = 8 * Vh;
    unsigned nb = (unsigned)((nl + 127) / 128);
    const double2 *m = (const double2 *)U->master;
    char *d = (char *)c->ptr;
#define LQCD_GC(P, RC) gauge_copy_kernel<P, RC><<<nb, 128, 0, ctx->stream>>>(U->g, m, d)
    switch (prec) {
      case LQCD_F64: LQCD_GC(LQCD_F64, 12); break;
      case LQCD_DF64: if (recon == 12) LQCD_GC(LQCD_DF64, 12); else LQCD_GC(LQCD_DF64, 18); break;
      case LQCD_F32: if (recon == 12) LQCD_GC(LQCD_F32, 12); else LQCD_GC(LQCD_F32, 18); break;
      case LQCD_BF16S: LQCD_GC(LQCD_BF16S, 12); break;
      case LQCD_F16S: LQCD_GC(LQCD_F16S, 12); break;
      default: return fail(ctx, LQCD_ERR_INVALID, "bad link precision %d", prec);
    }
#undef LQCD_GC
    LQCD_CUDA(ctx, cudaGetLastError());
    c->version = U->version;
  }
  out->ptr = c->ptr;
  return LQCD_OK;
}

lqcd_status spinor_pack_raw(lqcd_ctx *ctx, const Geom &g, const void *lexi, const HalfField &eo_full) {
  // eo_full: ptr of a FULL field; rhs_stride covers both parities
  size_t hb = spinor_half_bytes(eo_full.prec, g.Vh);
  size_t hf = eo_full.scale ? (size_t)g.Vh : 0;
  long V = 2L * g.Vh;
  dim3 grid((unsigned)((V + 127) / 128), eo_full.nrhs);
#define LQCD_PK(P) spinor_pack_kernel<P><<<grid, 128, 0, ctx->stream>>>(g, (const double2 *)lexi, \
      (char *)eo_full.ptr, eo_full.scale, eo_full.rhs_stride, eo_full.scale_rhs_stride, hb, hf, eo_full.nrhs)
  switch (eo_full.prec) {
    case LQCD_F64: LQCD_PK(LQCD_F64); break;
    case LQCD_DF64: LQCD_PK(LQCD_DF64); break;
    case LQCD_F32: LQCD_PK(LQCD_F32); break;
    case LQCD_BF16S: LQCD_PK(LQCD_BF16S); break;
    case LQCD_F16S: LQCD_PK(LQCD_F16S); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "bad precision");
  }
#undef LQCD_PK
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

lqcd_status spinor_unpack_raw(lqcd_ctx *ctx, const Geom &g, const HalfField &eo_full, void *lexi) {
  size_t hb = spinor_half_bytes(eo_full.prec, g.Vh);
  size_t hf = eo_full.scale ? (size_t)g.Vh : 0;
  long V = 2L * g.Vh;
  dim3 grid((unsigned)((V + 127) / 128), eo_full.nrhs);
#define LQCD_UPK(P) spinor_unpack_kernel<P><<<grid, 128, 0, ctx->stream>>>(g, (const char *)eo_full.ptr, \
      eo_full.scale, (double2 *)lexi, eo_full.rhs_stride, eo_full.scale_rhs_stride, hb, hf, eo_full.nrhs)
  switch (eo_full.prec) {
    case LQCD_F64: LQCD_UPK(LQCD_F64); break;
    case LQCD_DF64: LQCD_UPK(LQCD_DF64); break;
    case LQCD_F32: LQCD_UPK(LQCD_F32); break;
    case LQCD_BF16S: LQCD_UPK(LQCD_BF16S); break;
    case LQCD_F16S: LQCD_UPK(LQCD_F16S); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "bad precision");
  }
#undef LQCD_UPK
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

// Converts nh consecutive half fields (stride = one half field) between precisions.
lqcd_status spinor_convert_raw(lqcd_ctx *ctx, int Vh, int nh, const void *in, const float *in_scale,
                               int pin, void *out, float *out_scale, int pout) {
  size_t ihb = spinor_half_bytes(pin, Vh), ohb = spinor_half_bytes(pout, Vh);
  dim3 grid((unsigned)((Vh + 127) / 128), nh);
#define LQCD_CV(A, B) spinor_convert_kernel<A, B><<<grid, 128, 0, ctx->stream>>>(Vh, nh, \
      (const char *)in, in_scale, ihb, (size_t)Vh, (char *)out, out_scale, ohb, (size_t)Vh)
#define LQCD_CVROW(A)                                   \
  switch (pout) {                                       \
    case LQCD_F64: LQCD_CV(A, LQCD_F64); break;         \
    case LQCD_DF64: LQCD_CV(A, LQCD_DF64); break;       \
    case LQCD_F32: LQCD_CV(A, LQCD_F32); break;         \
    case LQCD_BF16S: LQCD_CV(A, LQCD_BF16S); break;     \
    case LQCD_F16S: LQCD_CV(A, LQCD_F16S); break;       \
    default: return fail(ctx, LQCD_ERR_INVALID, "bad precision"); \
  }
  switch (pin) {
    case LQCD_F64: LQCD_CVROW(LQCD_F64); break;
    case LQCD_DF64: LQCD_CVROW(LQCD_DF64); break;
    case LQCD_F32: LQCD_CVROW(LQCD_F32); break;
    case LQCD_BF16S: LQCD_CVROW(LQCD_BF16S); break;
    case LQCD_F16S: LQCD_CVROW(LQCD_F16S); break;
    default: return fail(ctx, LQCD_ERR_INVALID, "bad precision");
  }
#undef LQCD_CVROW
#undef LQCD_CV
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

}  // namespace lqcd
