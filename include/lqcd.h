/*
 * lqcd.h -- C ABI of the GB300 (sm_103a) twisted-mass Wilson library.
 *
 * The library implements the hot path of "Lattice QCD based on OpenCL"
 * (Bach, Lindenstruth, Philipsen, Pinke, arXiv:1209.5942):
 *   - the twisted-mass Wilson matrix (Sec. 2.1, eq. "D_tm")
 *         M = (1 + 2 i kappa mu gamma_5) - kappa H,
 *         H psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                         + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu),
 *     its even-odd Schur complement (Sec. 2.1, "even-odd preconditioning")
 *         Mhat = A_e - kappa^2 H_eo A_o^-1 H_oe,   A = 1 + 2 i kappa mu gamma_5,
 *   - the CG inversion of Mhat^+ Mhat (Sec. 2.1, eq. "solvereq"),
 *   - the fermion force, gauge force, Cabibbo-Marinari heatbath and HMC of
 *     Sec. 2.2.
 *
 * Conventions (the paper leaves them open; these are the library's readings):
 *   - site index i = x + Lx*(y + Ly*(z + Lz*t)); mu = 0,1,2,3 = x,y,z,t;
 *     every extent even; parity p(x) = (x+y+z+t) mod 2, even = 0;
 *     checkerboard index cb = i / 2.
 *   - chiral gamma basis, gamma_5 = gamma_x gamma_y gamma_z gamma_t =
 *     diag(1, 1, -1, -1); hopping prefactor kappa (not kappa/2).
 *   - links periodic; fermions periodic in space and, when
 *     geom.antiperiodic_t = 1, antiperiodic in time (hops across the time
 *     boundary carry -1; the sign is never folded into the links).
 *
 * Memory layouts.
 *   Lexicographic (LQCD_LAYOUT_LEXI), complex128, array of structures:
 *     gauge  [V][4][3][3],   spinor [V][4][3]   (spin, colour)
 *   Even-odd (LQCD_LAYOUT_EO), structure of arrays on 16-byte words
 *   (the paper's Sec. 4.2 SoA on a 16-byte base type), per right-hand side:
 *     full field  [parity 2][component 12][Vh]   (even half first)
 *     half field  [component 12][Vh]             (one parity)
 *   with component = 3*spin + colour, Vh = V/2, and per-precision words:
 *     LQCD_F64   complex128                        (16 B per component)
 *     LQCD_DF64  float-float complex {re_hi, im_hi, re_lo, im_lo}
 *                (16 B per component; value = hi + lo)
 *     LQCD_F32   complex64, components paired into 16-B words:
 *                [6][Vh] of {c0.re, c0.im, c1.re, c1.im}
 *     LQCD_BF16S / LQCD_F16S  16-bit reals with one float scale per site:
 *                [3][Vh] of 16 B (8 reals each, value = stored * scale)
 *                plus field.scale -> float [Vh] (per right-hand side)
 *   Multi-RHS fields (nrhs > 1) stack nrhs such fields contiguously.
 *   Algebra fields (momenta, forces dS/domega): float64 [4][V][8], lexicographic
 *   sites, coordinates w.r.t. T^a = lambda^a / 2, links varied as
 *   U -> exp(i omega^a T^a) U.
 *
 * Ownership: spinor, force and momentum buffers are device memory owned by
 * the caller; gauge fields are opaque objects owned by the library (freed with
 * lqcd_gauge_free); the library never frees caller memory.
 *
 * Streams: every call enqueues work on the context's stream and returns
 * without synchronising, except where it writes a host-visible result
 * (solver statistics, plaquette, Hamiltonian), which it documents.
 *
 * Errors: every entry point returns lqcd_status; arguments are validated
 * before any launch (null pointers, odd or non-positive extents, 16-byte
 * alignment, precision/layout combinations, aliasing, geometry mismatch);
 * lqcd_last_error() gives a message.  Nothing throws or exits.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LQCD_ABI_VERSION 2

typedef enum {
  LQCD_OK = 0,
  LQCD_ERR_INVALID = -1,     /* bad argument; nothing was launched */
  LQCD_ERR_CUDA = -2,        /* a CUDA call failed */
  LQCD_ERR_NOCONV = -3,      /* solver stopped at max_iter; stats are filled */
  LQCD_ERR_NONFINITE = -4,   /* NaN/Inf met in an input or a solver scalar */
  LQCD_ERR_TIMEOUT = -5,     /* a bounded device-side wait ran out */
  LQCD_ERR_OOM = -6,         /* device allocation failed */
  LQCD_ERR_UNSUPPORTED = -7, /* valid request that the library does not implement */
  LQCD_ERR_COMM = -8         /* a caller's communication hook reported a failure */
} lqcd_status;

typedef enum { LQCD_FULL = 0, LQCD_EVEN = 1, LQCD_ODD = 2 } lqcd_parity;

typedef enum {
  LQCD_F64 = 0,   /* IEEE binary64 storage and arithmetic */
  LQCD_DF64 = 1,  /* float-float storage and arithmetic (about 48-bit significand) */
  LQCD_F32 = 2,
  LQCD_BF16S = 3, /* bfloat16 + per-site float scale; FP32 arithmetic */
  LQCD_F16S = 4   /* binary16 + per-site float scale; FP32 arithmetic */
} lqcd_prec;

typedef enum { LQCD_LAYOUT_LEXI = 0, LQCD_LAYOUT_EO = 1 } lqcd_layout;

typedef struct {
  int32_t L[4];           /* extents x, y, z, t: all even, >= 2 */
  int32_t antiperiodic_t; /* 1: fermion boundary factor -1 across the time boundary */
} lqcd_geom;

/* A caller-owned device spinor field. */
typedef struct {
  void *ptr;      /* device pointer, 16-byte aligned */
  void *scale;    /* device float array [nrhs][Vh] (or [nrhs][2][Vh] for full
                     fields) for LQCD_BF16S / LQCD_F16S, else NULL */
  int32_t layout; /* lqcd_layout */
  int32_t prec;   /* lqcd_prec; LEXI layout requires LQCD_F64 */
  int32_t nrhs;   /* number of right-hand sides stacked in the buffer (>= 1) */
  int32_t reserved;
} lqcd_field;

typedef struct lqcd_ctx lqcd_ctx;
typedef struct lqcd_gauge lqcd_gauge;

/* ---------------------------------------------------------------- */
/* Context                                                           */
/* ---------------------------------------------------------------- */

int lqcd_abi_version(void);

/* Creates a context on CUDA device `device` that enqueues work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * context owns a stream-ordered device memory pool (see "Device memory") and
 * a small workspace (reduction partials, device scalars, a pinned host status
 * word) allocated here.  lqcd_destroy synchronises the stream, frees the
 * workspace and destroys the pool; memory of gauge fields not yet freed stays
 * valid until lqcd_gauge_free (through any context of the same device). */
int lqcd_create(lqcd_ctx **ctx, int device, void *cuda_stream);
int lqcd_destroy(lqcd_ctx *ctx);
int lqcd_set_stream(lqcd_ctx *ctx, void *cuda_stream);
/* Message of the last failed call on this context (never NULL). */
const char *lqcd_last_error(const lqcd_ctx *ctx);

/* Work counters of a context, accumulated by every kernel the library
 * enqueues (a CUDA-graph replay adds the counts of the captured launches).
 * bytes / flops are ALGORITHMIC counts: each input word read once, each
 * output written once (a half hop per output site: 8 links, the input
 * spinor, the output spinor and the optional aux spinor; 1320 flops per
 * site for the hop, plus 48 per fused epilogue term). */
typedef struct {
  uint64_t launches;      /* all kernels */
  uint64_t hop_launches;  /* hopping-term kernels only */
  double bytes;           /* algorithmic bytes of all counted kernels */
  double hop_bytes;       /* ... of the hopping-term kernels */
  double hop_flops;       /* algorithmic flops of the hopping-term kernels */
  double hop_sites;       /* output sites x right-hand sides of the hop kernels */
} lqcd_counters;
int lqcd_get_counters(const lqcd_ctx *ctx, lqcd_counters *out);
int lqcd_reset_counters(lqcd_ctx *ctx);

/* Measured arithmetic peaks of the context's GPU, for the roofline of the
 * ALU-bound kernels (the IEEE-FP64 hop is bound by the FP64 pipe, the
 * float-float hop by the FP32 pipe; Sec. 5.2 of the paper states its kernels'
 * performance against peaks too): two microbenchmark launches of 8
 * independent FMA chains per thread on 8 x 256 threads per SM, FP64 FMA and
 * packed FP32x2 FMA, timed with CUDA events after a warm-up launch (about
 * 30 ms in all).  *fp64_tflops and *fp32_tflops (host) receive 2 flops per FMA per
 * second in TFLOP/s.  Synchronous.  NULL arguments: LQCD_ERR_INVALID. */
int lqcd_measure_peaks(lqcd_ctx *ctx, double *fp64_tflops, double *fp32_tflops);

/* Device memory.  By default the library allocates its workspace and gauge
 * fields from the context's own stream-ordered pool
 * (cudaMallocFromPoolAsync / cudaFreeAsync on the context's stream).  The
 * pool keeps memory that was freed mapped for later allocations of the
 * context (a solver's vectors, a re-imported gauge field) instead of
 * returning it to the driver at every synchronisation; it grows to the
 * context's peak use.  lqcd_trim_memory synchronises the stream and returns
 * every unused byte of the pool to the driver; lqcd_memory_stats writes the
 * bytes the pool holds (*reserved) and the bytes in live allocations (*used),
 * both host uint64.  NULL arguments: LQCD_ERR_INVALID.
 * lqcd_set_allocator routes every later device allocation of the context
 * (workspace, solver vectors, gauge fields imported afterwards and their
 * derived copies) through alloc(bytes, user) and free(ptr, user) instead --
 * e.g. PyTorch's caching allocator -- so one pool backs everything.  alloc
 * must return memory aligned to at least 256 bytes that may be used on the
 * context's stream, or NULL (the call then fails with LQCD_ERR_OOM).  Call it
 * before importing gauge fields: it releases the context's current workspace
 * (synchronising the stream) and reallocates it through the new pair.  A
 * gauge field keeps the pair it was imported with and is freed through it.
 * Passing NULL for both restores the default.  Mixing one non-NULL function
 * with a NULL one is LQCD_ERR_INVALID.  The library never frees memory it did
 * not allocate. */
typedef void *(*lqcd_alloc_fn)(size_t bytes, void *user);
typedef void (*lqcd_free_fn)(void *ptr, void *user);
int lqcd_set_allocator(lqcd_ctx *ctx, lqcd_alloc_fn alloc, lqcd_free_fn free_fn, void *user);
int lqcd_trim_memory(lqcd_ctx *ctx);
int lqcd_memory_stats(lqcd_ctx *ctx, uint64_t *reserved, uint64_t *used);

/* Launch-shape autotuner (on by default).  The first launch of each kernel
 * configuration (kernel, precision, link format, variant, lattice extents,
 * number of right-hand sides, GPU) made outside a stream capture times every
 * candidate block shape with CUDA events on the context's stream and keeps the
 * fastest; results never depend on the shape.  A hop configuration first met
 * inside a capture (the solvers capture their iterations in CUDA graphs) takes
 * the choice of a tuned configuration that differs from it only in the dagger,
 * reduction or epilogue variant, else the built-in default.  enable = 0 uses
 * the built-in defaults for configurations not yet tuned.  cache_path (may be NULL) names a
 * JSON file from which choices are loaded now and to which new ones are
 * written, so other processes skip the timing. */
int lqcd_set_autotune(lqcd_ctx *ctx, int enable, const char *cache_path);

/* Forces candidate number `choice` (taken modulo each configuration's
 * candidate count) for every tuned launch of this context, bypassing the
 * tuner and its cache; choice < 0 restores tuning.  For reproducible
 * performance experiments and for tests that every launch shape gives the
 * same bits.  Returns LQCD_ERR_INVALID for a NULL context. */
int lqcd_set_launch_choice(lqcd_ctx *ctx, int choice);

/* Bytes needed for a field of the given parity (LQCD_FULL or one parity),
 * precision and nrhs in the EO layout; *scale_bytes receives the size of the
 * scale array (0 for unscaled precisions).  Returns 0 on invalid input. */
size_t lqcd_field_bytes(const lqcd_geom *geom, int parity, int prec, int nrhs,
                        size_t *scale_bytes);

/* ---------------------------------------------------------------- */
/* Gauge fields (Sec. 2.1 links U_mu(x); Sec. 4.1 REC12;             */
/* Sec. 4.2 parity-split SoA storage)                                */
/* ---------------------------------------------------------------- */

/* Imports a device gauge field in the lexicographic layout (complex128
 * [V][4][3][3]) into a library-owned even-odd SoA field.  recon = 18 keeps
 * all 9 complex entries; recon = 12 keeps rows 0 and 1 and rebuilds row 2 as
 * conj(row0 x row1) in the kernels (requires SU(3) links; checked to 1e-12,
 * else LQCD_ERR_INVALID).  Lower-precision copies for mixed-precision solves
 * are derived on demand. Synchronous (validates on the host). */
int lqcd_gauge_import(lqcd_ctx *ctx, const void *U_lexi, const lqcd_geom *geom, int recon,
                      lqcd_gauge **out);
/* Writes the field back in the lexicographic layout (device pointer). */
int lqcd_gauge_export(lqcd_ctx *ctx, const lqcd_gauge *U, void *U_lexi);
int lqcd_gauge_free(lqcd_ctx *ctx, lqcd_gauge *U);

/* ---------------------------------------------------------------- */
/* Spinor layout and precision conversion                            */
/* ---------------------------------------------------------------- */

/* lexicographic complex128 [nrhs][V][4][3] <-> EO full field of any precision */
int lqcd_spinor_pack(lqcd_ctx *ctx, const lqcd_geom *geom, const void *lexi, lqcd_field eo);
int lqcd_spinor_unpack(lqcd_ctx *ctx, const lqcd_geom *geom, lqcd_field eo, void *lexi);
/* EO field precision conversion; parity selects a half field or the full one */
int lqcd_spinor_convert(lqcd_ctx *ctx, const lqcd_geom *geom, int parity, lqcd_field in,
                        lqcd_field out);

/* ---------------------------------------------------------------- */
/* Operators (Sec. 2.1, eq. "D_tm")                                  */
/* ---------------------------------------------------------------- */

/* Half hop ("Dslash"): out = H_{p,1-p} in (dagger = 0) or the adjoint
 * hop (dagger = 1, gamma_mu -> -gamma_mu), computed on the sites of
 * out_parity (LQCD_EVEN or LQCD_ODD) from `in` on the other parity.  Both
 * fields are EO half fields of the same precision (any lqcd_prec; nrhs >= 1
 * applies the link to every right-hand side). */
int lqcd_dslash(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                const lqcd_geom *geom, int out_parity, int dagger);

/* ---------------------------------------------------------------- */
/* Domain decomposition along t and z (Sec. 6: the hop over several */
/* GPUs)                                                             */
/* ---------------------------------------------------------------- */

/* A lattice of extent Lt in t split into nt domains of Lt / nt slices (one per
 * GPU or process).  Each domain is an ordinary field of this library on the
 * LOCAL geometry (local->L[3] = Lt / nt, which must be even so that local and
 * global parities agree; local->antiperiodic_t is ignored: the global
 * fermion boundary sign is passed to lqcd_dd_pack).  Of the half hop only the
 * t hops that cross a domain boundary need a neighbour's data, and only its
 * spin projection: a "face" of Vs/2 = Lx Ly Lz / 2 sites x 6 complex numbers in
 * the precision of the field ([6][Vs/2] words: complex128 for LQCD_F64,
 * float-float {re_hi, im_hi, re_lo, im_lo} for LQCD_DF64, complex64 for
 * LQCD_F32), indexed by a boundary site's checkerboard index within its t
 * slice.  One half hop on every domain is
 *   lqcd_dd_pack  (all domains) -> move the faces (caller: NCCL, peer copies)
 *   -> lqcd_dd_dslash (all domains),
 * and equals lqcd_dslash on the whole lattice.  Bytes of one face (0 for
 * invalid input): */
size_t lqcd_dd_face_bytes(const lqcd_geom *local, int prec);

/* Writes the two faces of this domain for a half hop onto out_parity
 * (dagger as in lqcd_dslash), from `in` (EO half field of the other parity,
 * LQCD_F64 / LQCD_DF64 / LQCD_F32, nrhs = 1; other precisions:
 * LQCD_ERR_UNSUPPORTED):
 *   face_to_prev (for the previous domain): (1 - s gamma_t) psi(y) for the
 *     sites y at local t = 0, projected to its two upper spin components;
 *   face_to_next (for the next domain): U_t(y)^+ (1 + s gamma_t) psi(y) for the
 *     sites y at local t = Lt/nt - 1, with this domain's links.
 * negate_to_prev / negate_to_next != 0 multiply a face by -1: set them where
 * its hop crosses the global t boundary of an antiperiodic lattice (the first
 * domain's face_to_prev, the last domain's face_to_next).  Device buffers of
 * lqcd_dd_face_bytes each, 16-byte aligned, not aliasing.  Asynchronous. */
int lqcd_dd_pack(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, void *face_to_prev, void *face_to_next,
                 const lqcd_geom *local, int out_parity, int dagger, int negate_to_prev, int negate_to_next);

/* The half hop of this domain: out = H in on the sites of out_parity, where
 * the +t hop of a site at local t = Lt/nt - 1 takes face_from_next (the next
 * domain's face_to_prev) times this domain's U_t(x), and the -t hop of a site
 * at local t = 0 takes face_from_prev (the previous domain's face_to_next);
 * with nt = 1 the domain's own faces give lqcd_dslash.  Same fields and
 * errors as lqcd_dd_pack; in and out must not alias.  Asynchronous. */
int lqcd_dd_dslash(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out, const void *face_from_next,
                   const void *face_from_prev, const lqcd_geom *local, int out_parity, int dagger);

/* Split along z as well: a grid of nz x nt domains, domain dz + nz dt
 * holding z in [dz Lz/nz, (dz+1) Lz/nz) and t in [dt Lt/nt, (dt+1) Lt/nt),
 * on the local geometry (Lx, Ly, Lz/nz, Lt/nt), both split extents even.
 * The z hops that cross a domain boundary take faces as the t hops do: along
 * mu = 2 a face holds Lx Ly (Lt/nt) / 2 sites x 6 complex numbers, indexed by
 * (x/2) + Lx/2 (y + Ly t) within the boundary z slice (along mu = 3 by
 * (x/2) + Lx/2 (y + Ly z) within the t slice, as above).  z is periodic: no z
 * face is negated.  Bytes of one face along mu = 2 or 3 (0 for invalid
 * input; lqcd_dd_face_bytes is mu = 3): */
size_t lqcd_dd_face_bytes_dir(const lqcd_geom *local, int mu, int prec);

/* lqcd_dd_pack for the two faces along mu = 2 (z: the sites at local z = 0
 * and, times U_z^+, at z = Lz/nz - 1) or mu = 3 (t: lqcd_dd_pack itself);
 * buffers of lqcd_dd_face_bytes_dir(local, mu, prec) each.  Same fields and
 * errors as lqcd_dd_pack; mu other than 2 or 3: LQCD_ERR_INVALID. */
int lqcd_dd_pack_dir(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, int mu, void *face_to_prev,
                     void *face_to_next, const lqcd_geom *local, int out_parity, int dagger, int negate_to_prev,
                     int negate_to_next);

/* The half hop of a domain of an nz x nt grid: lqcd_dd_dslash with the t
 * faces t_from_next / t_from_prev, and the z hops across the domain's z
 * boundaries from z_from_next (the next z domain's z face_to_prev) and
 * z_from_prev (the previous one's face_to_next); both z faces NULL: z is not
 * split (lqcd_dd_dslash).  Asynchronous. */
int lqcd_dd_dslash_zt(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out, const void *t_from_next,
                      const void *t_from_prev, const void *z_from_next, const void *z_from_prev,
                      const lqcd_geom *local, int out_parity, int dagger);

/* parity = LQCD_FULL: out = M in on the whole lattice (fields LEXI or EO full).
 * parity = LQCD_EVEN: out = Mhat in on the even sites (EO half fields).
 * parity = LQCD_ODD : the odd-site Schur complement A_o - kappa^2 H_oe A_e^-1 H_eo.
 * in and out must not alias.  Precision: LQCD_F64, LQCD_DF64 or LQCD_F32
 * (EO), LQCD_F64 (LEXI). */
int lqcd_apply_M(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                 const lqcd_geom *geom, double kappa, double mu, int parity);
/* Same with M^+ = (1 - 2 i kappa mu gamma_5) - kappa H^+ (Mhat^+ for one parity). */
int lqcd_apply_Mdag(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field in, lqcd_field out,
                    const lqcd_geom *geom, double kappa, double mu, int parity);

/* ---------------------------------------------------------------- */
/* Solver (Sec. 2.1: "D phi = psi", CG; even-odd preconditioning)    */
/* ---------------------------------------------------------------- */

typedef struct {
  double tol;             /* target relative true residual ||b - M x|| / ||b|| */
  int32_t max_iter;       /* cap on inner iterations (all cycles together) */
  int32_t outer_prec;     /* LQCD_F64 or LQCD_DF64: precision of x, of the
                             reliable-update residuals and of the plain solve */
  int32_t inner_prec;     /* == outer_prec: plain CG; LQCD_F32 / LQCD_BF16S /
                             LQCD_F16S: mixed precision with reliable updates */
  double delta;           /* reliable-update trigger: ||s|| < delta * max ||s||
                             since the last update (<= 0 selects 0.003 for an
                             LQCD_F32 inner format, whose updates cost more than
                             its drift, and 0.1 for the 16-bit ones); with a
                             LQCD_BF16S inner format the CG also updates every
                             8 iterations, which bounds the drift of the 8-bit
                             recursion from the true residual */
  int32_t max_restarts;   /* outer iterative-refinement cycles on the true residual */
  int32_t check_every;    /* host polls convergence every this many iterations */
  int32_t use_graph;      /* 1: capture check_every iterations in a CUDA graph */
  int32_t sloppy_recon;   /* 18 or 12: link format of the inner operator */
  int32_t solver;         /* LQCD_SOLVER_CG (default) or LQCD_SOLVER_BICGSTAB */
  double inner_tol;       /* BiCGStab with inner_prec != outer_prec, and the
                             domain-decomposed CG with an F32 inner format:
                             relative residual each refinement cycle reaches
                             in the inner format (0 selects 1e-5) */
} lqcd_cg_params;
enum { LQCD_SOLVER_CG = 0, LQCD_SOLVER_BICGSTAB = 1 };

typedef struct {
  int32_t iters;            /* inner iterations (each: 2 Mhat + 2 Mhat^+ ... = 4 half hops x2) */
  int32_t reliable_updates; /* FP64-class residual recomputations */
  int32_t restarts;         /* outer refinement cycles after the first */
  int32_t converged;        /* 1 if true_resid <= tol */
  double true_resid;        /* ||b - M x|| / ||b|| recomputed in IEEE FP64 with full M */
  double seconds;           /* wall time of the call */
} lqcd_cg_stats;

/* Solves M x = b (FULL fields, LEXI or EO, LQCD_F64) through CG on
 * Mhat^+ Mhat on the even sites (CGLS form), or with params->solver =
 * LQCD_SOLVER_BICGSTAB through BiCGStab on Mhat itself (Sec. 2.1 names CG and
 * BiCGStab; nrhs = 1 only, else LQCD_ERR_UNSUPPORTED; a mixed-precision
 * BiCGStab runs in inner_prec to inner_tol per cycle and the FP64 true
 * residual drives outer refinement), with source preparation
 *   bhat_e = b_e + kappa H_eo A_o^-1 b_o
 * and reconstruction x_o = A_o^-1 (b_o + kappa H_oe x_e), both in the outer
 * format (IEEE FP64 or float-float); the true residual ||b - M x|| / ||b||
 * is always recomputed in IEEE FP64.  nrhs > 1 solves
 * the right-hand sides together (one multi-RHS operator per iteration,
 * per-RHS scalars and convergence); stats then points to nrhs entries.
 * Synchronous: returns after the true residual is known.  Returns
 * LQCD_ERR_NOCONV (stats filled) when tol is not reached. */
int lqcd_cg_solve(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field b, lqcd_field x,
                  const lqcd_geom *geom, double kappa, double mu, const lqcd_cg_params *params,
                  lqcd_cg_stats *stats);

/* Communication of a domain-decomposed solve (lqcd_dd_cg_solve), called by
 * the library from the calling thread between its launches:
 *   exchange(user, t_bytes, z_bytes): every held domain's to_prev and to_next
 *     faces are written in their leading t_bytes (t faces) and z_bytes (z
 *     faces; 0 when z is not split) bytes: lqcd_dd_face_bytes_dir of the
 *     format of that half hop, LQCD_F64 for the FP64 steps and the inner
 *     format for the inner ones (the library's stream has been
 *     synchronised); the hook delivers those bytes of each to_prev face to
 *     the from_next buffer of the previous domain along the same direction
 *     and of each to_next face to the next domain's from_prev buffer, and
 *     returns once they are in place;
 *   allreduce(user, vals, n): sums n host doubles over all processes of the
 *     solve, in place (NULL: a single process).
 * Both return 0 on success; anything else ends the solve with LQCD_ERR_COMM. */
typedef struct {
  void *user;
  int (*exchange)(void *user, size_t t_bytes, size_t z_bytes);
  int (*allreduce)(void *user, double *vals, int n);
} lqcd_dd_comm;

/* The even-odd CG of lqcd_cg_solve (CGLS on Mhat^+ Mhat, source preparation,
 * reconstruction, FP64 true residual and outer refinement; one right-hand
 * side) on a lattice split into an nz x nt grid of domains as for
 * lqcd_dd_dslash_zt (nz = 1: along t only; Sec. 6 outlook: the solver over
 * several GPUs).  This call holds nd consecutive domains, first_domain ..
 * first_domain + nd - 1 (domain dz + nz dt), each on the local geometry
 * `local` (local->L[2] = Lz / nz, local->L[3] = Lt / nt, both even; local
 * must match the gauge fields' geometry): U[k] its gauge field, b[k] and x[k]
 * EO full fields (LQCD_F64, nrhs = 1; x is overwritten), and its face
 * buffers (device, 16-byte aligned, lqcd_dd_face_bytes_dir(local, mu,
 * LQCD_F64) each): with F = 4 (nz = 1) or 8, faces[F k .. F k + 3] its t
 * to_prev, to_next, from_next and from_prev faces and, if nz > 1,
 * faces[F k + 4 .. F k + 7] the same four along z.  Every half hop
 * packs the faces of all held domains, moves them and runs the domain hops
 * with the operator's diagonal epilogue; every norm is summed in a fixed
 * order on each domain, over the held domains in order, then over
 * processes.  Mixed precision (Sec. 3) as defect correction: with inner_prec
 * LQCD_F32 or LQCD_DF64 each refinement cycle runs the CGLS in that format
 * (links in sloppy_recon's format, 0: the field's) on its cycle's prepared
 * residual, until the residual has dropped by inner_tol (F32; 0 selects
 * 1e-5) or, for LQCD_DF64, to the tolerance; the source preparation, the
 * correction, the reconstruction and the true residual stay IEEE FP64.
 * comm = NULL: the call holds every domain (nd = nz nt, first_domain = 0) and
 * the library moves the faces by device copies; otherwise comm->exchange
 * moves them and comm->allreduce sums the norms.  antiperiodic_t: the
 * fermion boundary of the whole lattice.  params: tol, max_iter,
 * max_restarts, inner_tol, sloppy_recon (outer_prec LQCD_F64, inner_prec
 * LQCD_F64, LQCD_DF64 or LQCD_F32, solver CG, else LQCD_ERR_UNSUPPORTED).
 * stats: one entry; true_resid is that of the whole lattice.  Synchronous;
 * LQCD_ERR_NOCONV (stats filled) when tol is not reached. */
int lqcd_dd_cg_solve(lqcd_ctx *ctx, int nd, const lqcd_gauge *const *U, const lqcd_field *b,
                     const lqcd_field *x, void *const *faces, const lqcd_geom *local, int first_domain,
                     int nz, int nt, int antiperiodic_t, double kappa, double mu, const lqcd_cg_params *params,
                     const lqcd_dd_comm *comm, lqcd_cg_stats *stats);

/* Solves n independent systems M_k x_k = b_k on lattices of different sizes
 * (each b_k, x_k: FULL EO LQCD_F64 fields on U_k's geometry) with one
 * persistent kernel per operator stage working through a queue of tiles over
 * all lattices.  stats points to n entries.  Synchronous. */
int lqcd_cg_solve_batch(lqcd_ctx *ctx, int n, const lqcd_gauge *const *U, const lqcd_field *b,
                        const lqcd_field *x, const double *kappa, const double *mu,
                        const lqcd_cg_params *params, lqcd_cg_stats *stats);

/* ---------------------------------------------------------------- */
/* Forces, actions, heatbath, HMC (Sec. 2.2)                          */
/* ---------------------------------------------------------------- */

/* dS/domega for S = phi^+ (Mhat^+ Mhat)^-1 phi (phi: EO half field on the
 * even sites, LQCD_F64), through dD^-1 = -D^-1 dD D^-1:
 *   X = (Mhat^+ Mhat)^-1 phi (CG), Y = Mhat X, then one adjoint kernel over
 *   all links.  dSdw: device float64 [4][V][8], or NULL to compute the action
 *   alone (no force kernel; S_out must then be non-NULL, else
 *   LQCD_ERR_INVALID).  If X_cache is non-NULL and X_cache->reserved == 1 the
 *   stored X is reused, otherwise X is solved and, when X_cache is non-NULL,
 *   stored there (reserved set to 1).
 *   *S_out (host, may be NULL) receives S = Re phi^+ X.  Synchronous. */
int lqcd_fermion_force(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field phi, double *dSdw,
                       lqcd_field *X_cache, const lqcd_geom *geom, double kappa, double mu,
                       const lqcd_cg_params *params, lqcd_cg_stats *stats, double *S_out);

/* Mass preconditioning with a heavier twisted mass (Sec. 2.2: det D =
 * det A det(D / A) with a second fermion matrix A): for W = Mhat(mu2) the
 * ratio action
 *   S2 = phi2^+ W (Mhat^+ Mhat)^-1 W^+ phi2     (Mhat = Mhat(mu))
 * and its derivative -2 Re[Y^+ dMhat(mu) X] + 2 Re[phi2^+ dW X] with
 * X = (Mhat^+ Mhat)^-1 W^+ phi2 (CG with params), Y = Mhat X, into dSdw
 * (device float64 [4][V][8]).  phi2: EO half field of the even sites,
 * LQCD_F64.  *S_out (host, may be NULL) receives S2.  Synchronous. */
int lqcd_fermion_force_ratio(lqcd_ctx *ctx, const lqcd_gauge *U, lqcd_field phi2, double *dSdw,
                             const lqcd_geom *geom, double kappa, double mu, double mu2,
                             const lqcd_cg_params *params, lqcd_cg_stats *stats, double *S_out);

/* Gauge action (Sec. 2.1, eq. "S_tlsym")
 *   S_g = (beta/3) sum_x [ c0 sum_{mu<nu} (3 - Re Tr P_munu(x))
 *                        + c1 sum_{mu != nu} (3 - Re Tr R_munu(x)) ],
 * c0 = 1 - 8 c1, P the plaquette, R the 2x1 loop (two links along mu, one
 * along nu); c1 = 0 is the Wilson action, c1 = -1/12 tree-level Symanzik.
 * dSdw (device float64 [4][V][8]) receives the derivative
 *   dS_g/domega^a = -(beta/3) Re Tr[i T^a U_mu(x) W_mu(x)],
 * W = c0 (6 plaquette staples) + c1 (18 rectangle staples).  prec selects
 * the arithmetic of the staples and products: LQCD_F64 (IEEE FP64) or
 * LQCD_DF64 (float-float from the field's DF64 copy, FP64-class accuracy; the
 * action is always summed in FP64).  *S_out host (may be NULL, then the call
 * is asynchronous).  Non-finite beta or c1: LQCD_ERR_NONFINITE; other prec:
 * LQCD_ERR_INVALID. */
int lqcd_gauge_force(lqcd_ctx *ctx, const lqcd_gauge *U, double beta, double c1, int prec, double *dSdw,
                     double *S_out);

/* Plaquette (1/(6V)) sum_{x, mu<nu} (1/3) Re Tr U_munu(x) in FP64.  Synchronous. */
int lqcd_plaquette(lqcd_ctx *ctx, const lqcd_gauge *U, double *plaq_out);

/* One Cabibbo-Marinari heatbath sweep at coupling beta: for mu = 0..3 and
 * parity even, odd, every link of that class is updated in parallel over the
 * SU(2) subgroups (0,1), (1,2), (0,2) with the exact SU(2) update (Creutz for
 * b < 1.5, Kennedy-Pendleton above, b = 2 beta k / 3).  Random numbers:
 * Philox4x32-10 keyed by seed, counter (site, sweep_idx, mu | g<<2 | tag<<8,
 * draw).  Then n_or overrelaxation passes (0 <= n_or <= 64, else
 * LQCD_ERR_INVALID): the same checkerboard order, each SU(2) subgroup
 * replaced by its reflection v = (w^+/k)^2 (microcanonical: the action is
 * unchanged).  prec = LQCD_F64 updates the FP64 field in place (the SU(2)
 * left multiplications keep it unitary to rounding; a field imported with
 * recon = 12 is updated through its 12-real FP64 copy, the third row rebuilt
 * on every load, Sec. 4.1, and written back with the third row rebuilt);
 * prec = LQCD_DF64 runs the FP64 sweep with its staple sums in float-float
 * arithmetic on the FP32 pipe (2^-46 relative, from the field's 18-real
 * float-float copy, which the sweep keeps current; the SU(2) samplers, the
 * subgroup products and the links stay in IEEE FP64; 18-real links whatever
 * the import format); prec = LQCD_F32 runs
 * the same sweep in single precision on the field's FP32 copy (12-real links
 * with the third row rebuilt, Sec. 4.1, if the field was imported with
 * recon = 12) and writes the result back into the FP64 field, reunitarised
 * by a Gram-Schmidt in float-float arithmetic (|U U^+ - 1| below 1e-13), and
 * keeps the FP32 copy current for the next sweep (Sec. 5.1 measures the
 * single-precision kernels).  Other prec: LQCD_ERR_INVALID.
 * Asynchronous. */
int lqcd_heatbath_sweep(lqcd_ctx *ctx, lqcd_gauge *U, double beta, uint64_t seed,
                        uint64_t sweep_idx, int n_or, int prec);

/* n_or overrelaxation passes alone (Sec. 2.2: the alternative update of the
 * heatbath figure; 1 <= n_or <= 64, else LQCD_ERR_INVALID), in the
 * checkerboard order of lqcd_heatbath_sweep, with the same arithmetic and link
 * formats per prec: for each link and SU(2) subgroup (0,1), (1,2), (0,2) in
 * turn, w_hat = the unit quaternion part of the subgroup block of U A (A the
 * staple sum) and U <- V U with v = (w_hat^+)^2.  Deterministic (no random
 * numbers); the action is unchanged to rounding.  Asynchronous. */
int lqcd_overrelax_sweep(lqcd_ctx *ctx, lqcd_gauge *U, int n_or, int prec);

/* Gaussian momenta p^a ~ N(0,1) into P (device float64 [4][V][8]) from the
 * Philox stream (site, traj, mu | 1<<8, k). Asynchronous. */
int lqcd_momenta_gaussian(lqcd_ctx *ctx, const lqcd_geom *geom, double *P, uint64_t seed,
                          uint32_t traj);
/* Gaussian spinor eta (density exp(-eta^+ eta)) on the sites of `parity`
 * (LQCD_FULL, LQCD_EVEN) into an EO LQCD_F64 field, stream (site, traj, 2<<8, k). */
int lqcd_spinor_gaussian(lqcd_ctx *ctx, const lqcd_geom *geom, lqcd_field eta, int parity,
                         uint64_t seed, uint32_t traj);

/* U_mu(x) <- exp(i eps P_mu(x)) U_mu(x) for every link (exact 3x3 exponential
 * in FP64), then FP64 reunitarisation. Asynchronous. */
int lqcd_gauge_update(lqcd_ctx *ctx, lqcd_gauge *U, const double *P, double eps);
/* The same update in the arithmetic prec: LQCD_F64 (as lqcd_gauge_update) or
 * LQCD_DF64 -- the algebra element, the exponential, E U and the
 * reunitarisation in float-float (about 2^-46 relative, on the FP32 pipe;
 * GB300's FP64 pipe is 1/64 of its rate), P read and U read and written in
 * FP64.  Other prec: LQCD_ERR_INVALID.  Asynchronous. */
int lqcd_gauge_update_prec(lqcd_ctx *ctx, lqcd_gauge *U, const double *P, double eps, int prec);
/* P <- P - eps * dSdw (the leapfrog momentum step, F = -dS/domega). */
int lqcd_momenta_update(lqcd_ctx *ctx, const lqcd_geom *geom, double *P, const double *dSdw,
                        double eps);
/* 1/2 sum p^2 in FP64 (host result).  Synchronous. */
int lqcd_momenta_kinetic(lqcd_ctx *ctx, const lqcd_geom *geom, const double *P, double *K_out);
/* Copies U_src into U_dst (same geometry). */
int lqcd_gauge_copy(lqcd_ctx *ctx, const lqcd_gauge *U_src, lqcd_gauge *U_dst);

typedef struct {
  double beta, kappa, mu;
  double tau;          /* trajectory length */
  int32_t nsteps;      /* leapfrog steps, or 2MN steps of the outer (fermion) scale */
  int32_t nf;          /* 0: pure gauge, 1: one twisted-mass doublet (phi = Mhat^+ eta) */
  uint64_t seed;
  uint32_t traj;       /* trajectory number (Philox counter word) */
  int32_t integrator;  /* LQCD_LEAPFROG or LQCD_2MN (two time scales) */
  double c1;           /* rectangle coefficient of the gauge action (0: Wilson) */
  int32_t nsteps_gauge;/* 2MN: inner gauge steps per outer position update (>= 1) */
  int32_t force_prec;  /* arithmetic of the gauge force and of the link update
                          U <- exp(i h P) U: LQCD_F64 (default) or LQCD_DF64
                          (float-float, FP64-class; H and dH stay IEEE FP64) */
  double lambda;       /* 2MN parameter; 0 selects 0.1931833275037836 */
  double mu2;          /* mass preconditioning (nf = 1): 0 = off; else the heavier twisted
                          mass of W = Mhat(mu2), S_f = phi1^+ (W^+ W)^-1 phi1
                          + phi2^+ W (Mhat^+ Mhat)^-1 W^+ phi2 */
  int32_t nsteps_mid;  /* 2MN with mu2: steps of the W force per outer position update */
  int32_t reserved;
  lqcd_cg_params cg;   /* solver used for every force and action evaluation */
} lqcd_hmc_params;
enum { LQCD_LEAPFROG = 0, LQCD_2MN = 1 };

typedef struct {
  double dH, H0, H1;
  double plaquette;    /* after the trajectory (of the accepted field) */
  int32_t accepted;
  int32_t cg_iters;    /* total inner CG iterations */
  double seconds;
} lqcd_hmc_stats;

/* One HMC trajectory (Sec. 2.2): momenta and eta drawn from Philox, phi =
 * Mhat^+ eta, molecular dynamics with F = -dS/domega, H in FP64 and the
 * Metropolis test exp(-dH) against a Philox uniform (counter (0, traj, 4<<8,
 * 0)).  On rejection U is restored.
 *   LQCD_LEAPFROG: nsteps steps of eps = tau/nsteps, gauge and fermion force
 *     together:  P -= eps/2 dS; (U <- exp(i eps P) U; P -= eps dS) ...
 *   LQCD_2MN (Sec. 2.2 "2MN", "multiple timescales"; Sec. 5.3): the
 *     minimum-norm step  P -= l e dS; Q(e/2); P -= (1-2l) e dS; Q(e/2);
 *     P -= l e dS  on nested scales: the fermion force with nsteps steps of
 *     e = tau/nsteps outside, and every position update Q(h) an inner 2MN
 *     integration of the gauge force over h with nsteps_gauge steps.  With
 *     mu2 != 0 (mass preconditioning, Sec. 2.2) the ratio force is outside
 *     (nsteps), the W force in the middle (nsteps_mid per outer position
 *     update) and the gauge force inside; eta2 for phi2 = W^-+ Mhat^+ eta2 is
 *     drawn from the stream of seed ^ 0x9E3779B97F4A7C15.  Pure gauge (nf = 0)
 *     runs the gauge scale alone with 2 nsteps nsteps_gauge steps.
 * Momentum updates at the same links are merged, so each force is
 * evaluated once per distinct field.  Every force solve after the first of a
 * trajectory starts from the solution of the previous one (a chronological
 * initial guess for the same pseudofermion); its stopping test stays relative
 * to |phi|.  Synchronous. */
int lqcd_hmc_trajectory(lqcd_ctx *ctx, lqcd_gauge *U, const lqcd_hmc_params *params,
                        lqcd_hmc_stats *stats);

/* ---------------------------------------------------------------- */
/* No-allocation entry point (the paper has no counterpart)          */
/* ---------------------------------------------------------------- */

/* Plaquette (1/(6V)) sum_{x, mu<nu} (1/3) Re Tr U_munu(x) of a lexicographic
 * complex128 gauge field [V][4][3][3] (device pointer, 16-byte aligned),
 * written to *plaq_dev (device pointer to one double), for callers that
 * cannot allocate device memory (their allocator belongs to another
 * framework, their memory budget is fixed, or allocation is off limits while
 * they record work).  It needs no context and allocates nothing: the block
 * partial sums go to a fixed file-scope device array of 32768 doubles
 * (256 KiB) that each GPU using the library keeps until the process exits,
 * so V <= 4194304 sites; larger lattices, odd extents and misaligned or NULL
 * pointers return LQCD_ERR_INVALID without launching anything.  Work is
 * enqueued on cuda_stream (a cudaStream_t; NULL = legacy default stream) and
 * the call returns without synchronising.  All calls share the one array,
 * which keeps the last call's partial sums (each call overwrites every slot
 * it reads, so nothing needs clearing): calls whose work overlaps on the GPU
 * race, so order them on one stream.  Every call made outside a stream
 * capture looks up the array's device address afresh (cudaGetSymbolAddress),
 * so calls after cudaDeviceReset, which reloads the module and moves the
 * array, stay correct; a call whose stream is capturing reuses the address of
 * the last call on the same device and returns LQCD_ERR_CUDA if there was
 * none, so make one call on each device outside any capture first. */
int lqcd_plaquette_noalloc(const void *U_lexi, const lqcd_geom *geom, double *plaq_dev,
                           void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
