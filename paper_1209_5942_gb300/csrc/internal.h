// internal.h -- host-side structures of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/lqcd.h"
#include "common.cuh"

// caller-provided device allocator (lqcd_set_allocator); NULL: the context's
// stream-ordered memory pool
struct DevAllocator {
  lqcd_alloc_fn alloc = nullptr;
  lqcd_free_fn free = nullptr;
  void *user = nullptr;
};

struct lqcd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 152;
  DevAllocator A;
  // Stream-ordered pool of the default allocator.  Its release threshold is
  // unlimited: memory freed by one solve stays mapped for the next instead
  // of going back to the driver at every synchronisation (which the device's
  // default pool does, and which cost ~2 ms of page mapping per 24^3 x 48
  // solve).  lqcd_trim_memory returns it; lqcd_destroy destroys the pool.
  cudaMemPool_t pool = nullptr;
  std::string err;
  // reduction workspace: partial sums [slots][nblocks] and per-slot results
  double *partials = nullptr;
  size_t partials_cap = 0;  // doubles
  double *pinned = nullptr; // host pinned scratch for status read-back
  size_t pinned_cap = 0;
  // solver device state (see cg.cu)
  void *solver_state = nullptr;
  size_t solver_state_cap = 0;
  // algorithmic work counters (lqcd_get_counters)
  lqcd_counters cnt{};
  // launch-shape autotuner (tune.cu)
  // plaquette-staple workspace of the tlSym gauge force (gauge.cu)
  void *staples = nullptr;
  size_t staple_cap = 0;
  int autotune = 1;
  int forced_choice = -1;  // lqcd_set_launch_choice: >= 0 overrides the tuner
  std::string tune_path;
  std::string gpu_name;
  std::map<std::string, int> tuned;
};

struct lqcd_gauge {
  lqcd_geom geom;
  lqcd::Geom g;
  int recon = 18;            // link format of the FP64-class operator
  void *master = nullptr;    // FP64, recon 18, [parity][mu][9][Vh] complex128
  uint64_t version = 1;      // bumped whenever master changes
  struct Copy {
    void *ptr = nullptr;
    int prec = -1, recon = 0;
    uint64_t version = 0;
  };
  std::vector<Copy> copies;  // derived precisions / formats
  DevAllocator A;            // allocator of master and copies (the importing context's)
};

namespace lqcd {

// Launches `kernel` on `st` with programmatic stream serialization: it may
// start while the previous kernel in the stream runs and must call pdl_wait()
// first (common.cuh).  Inside a stream capture this records a programmatic
// dependency edge.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// status helpers
lqcd_status fail(lqcd_ctx *ctx, lqcd_status s, const char *fmt, ...);
// device memory through an allocator (the context's, or a gauge field's)
lqcd_status raw_alloc(lqcd_ctx *ctx, const DevAllocator &A, void **p, size_t bytes);
void raw_free(lqcd_ctx *ctx, const DevAllocator &A, void *p);
lqcd_status cuda_check(lqcd_ctx *ctx, cudaError_t e, const char *what);
#define LQCD_CUDA(ctx, call)                                           \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return lqcd::cuda_check((ctx), e_, #call);  \
  } while (0)
#define LQCD_TRY(expr)                          \
  do {                                          \
    lqcd_status s_ = (expr);                    \
    if (s_ != LQCD_OK) return s_;               \
  } while (0)

Geom make_geom(const lqcd_geom &g);
bool geom_equal(const lqcd_geom &a, const lqcd_geom &b);
size_t spinor_half_bytes(int prec, int Vh);   // one parity, one rhs
size_t spinor_scale_half_bytes(int prec, int Vh);

// device buffers (stream-ordered allocation on the context stream)
lqcd_status dalloc(lqcd_ctx *ctx, void **p, size_t bytes);
void dfree(lqcd_ctx *ctx, void *p);
lqcd_status ensure_partials(lqcd_ctx *ctx, size_t doubles);
lqcd_status ensure_pinned(lqcd_ctx *ctx, size_t doubles);
struct DBuf {  // device scratch freed on scope exit
  lqcd_ctx *ctx;
  void *p = nullptr;
  explicit DBuf(lqcd_ctx *c) : ctx(c) {}
  ~DBuf() { dfree(ctx, p); }
  lqcd_status alloc(size_t n) { return dalloc(ctx, &p, n); }
};

// A half field (one parity) with nrhs right-hand sides in the EO layout.
struct HalfField {
  void *ptr = nullptr;
  float *scale = nullptr;
  int prec = LQCD_F64;
  int nrhs = 1;
  size_t rhs_stride = 0;        // bytes between right-hand sides
  size_t scale_rhs_stride = 0;  // floats between right-hand sides
};

// batched hop (dslash.cu): descs = device HopArgs[nsys], tiles = device int2[ntiles]
struct HopLaunch;
lqcd_status launch_hop_batched(lqcd_ctx *ctx, int prec, int recon, bool dagger, bool reduce,
                               const void *descs, const void *tiles, int ntiles, int grid, const int *halt);
size_t hop_args_size();
void hop_args_fill(const Geom &g, const HopLaunch &L, void *dst);

// Autotuner (tune.cu): returns the index of the fastest of `ncand` launch
// shapes for `key`, timing run(i) (which enqueues one launch of candidate i on
// ctx->stream) with CUDA events the first time the key is seen outside a
// stream capture; returns `fallback` when tuning is off or not possible.
int tune_choice(lqcd_ctx *ctx, const std::string &key, int ncand, int fallback,
                const std::function<void(int)> &run);
void tune_load(lqcd_ctx *ctx);

// A BF16 recursion (8-bit significand, storage error ~2^-9 per operator
// application) drifts from the true residual while its own |s| keeps
// falling: on the 32^3 x 64 heatbath field it took 699 iterations at
// delta = 0.1 against 209 for FP32, and a trigger on the stagnation of |s|
// did not help, because |s| does not stagnate.  What bounds the drift is the
// number of iterations between updates, so BF16 inner solves also update
// after kBf16Gap iterations; other formats update only by delta.  Both CG
// drivers (single and batched systems) use this gap.
constexpr int kBf16Gap = 8;

// Reliable-update trigger when the caller leaves delta <= 0.  A reliable
// update costs two outer-precision (IEEE FP64 or float-float) Schur
// operators, and GB300's FP64 pipe runs at 1/64 of the FP32 rate, so with an
// FP32 recursion, whose residual stays faithful over a long drop, fewer
// updates pay: on the 24^3 x 48 bench field and the 32^3 x 64 heatbath field
// delta = 0.003 kept the iteration counts of delta = 0.1 with 4 updates
// instead of 10 (DF64/F32 15.9 -> 13.5 ms and 146 -> 139 ms, FP64/F32 23.4 ->
// 16.4 ms and 169 -> 148 ms, the 12-RHS DF64/F32 solve 139 -> 115 ms).  The
// 16-bit recursions keep 0.1: with FP16 a smaller delta took the heatbath
// field from 231 to 317-781 iterations.
inline double default_delta(int inner) { return inner == LQCD_F32 ? 0.003 : 0.1; }

// work counters: one launch moving `bytes` algorithmic bytes
inline void count_launch(lqcd_ctx *ctx, double bytes) {
  ctx->cnt.launches += 1;
  ctx->cnt.bytes += bytes;
}

// Work of the iterations a chunk of captured solver iterations really ran.
// Every kernel of a chunk returns at once after a device flag halts the
// solve (convergence, a reliable update), so a chunk of k iterations does
// the work of n <= k of them, the last one only up to the reduction that
// set the flag.  `full` is one iteration's count and `first` its part up to
// that reduction (both recorded while the first iteration is enqueued).
// Launches are counted for the whole chunk: halted kernels still launch.
struct IterWork {
  lqcd_counters full{}, first{};
  bool known = false;
};
inline lqcd_counters cnt_sub(const lqcd_counters &a, const lqcd_counters &b) {
  lqcd_counters d{};
  d.launches = a.launches - b.launches;
  d.hop_launches = a.hop_launches - b.hop_launches;
  d.bytes = a.bytes - b.bytes;
  d.hop_bytes = a.hop_bytes - b.hop_bytes;
  d.hop_flops = a.hop_flops - b.hop_flops;
  d.hop_sites = a.hop_sites - b.hop_sites;
  return d;
}
inline void add_work(lqcd_counters &c, const lqcd_counters &d, double times) {
  c.bytes += times * d.bytes;
  c.hop_bytes += times * d.hop_bytes;
  c.hop_flops += times * d.hop_flops;
  c.hop_sites += times * d.hop_sites;
}
// Executable graph of a solver's iterations (cg.cu).  Preferred form: a
// conditional while node whose body is one iteration followed by a
// one-thread control kernel, which ends the loop once the solver's halt word
// is set or after `chunk` passes, so a launch runs exactly the iterations up
// to the next halt (convergence, a reliable update) and no halted
// iterations.  If the driver rejects that graph, `chunk` iterations unrolled
// (whose kernels return at once after a halt).  per_pass: launch counts of
// one loop pass, or of the whole unrolled chunk.
struct SolverGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool loop = false;
  lqcd_counters per_pass{};
  SolverGraph() = default;
  SolverGraph(const SolverGraph &) = delete;
  SolverGraph &operator=(const SolverGraph &) = delete;
  ~SolverGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  // launch counts of a launch that began n iterations
  lqcd_counters launches(int n) const {
    lqcd_counters c{};
    const uint64_t k = loop ? (uint64_t)(n > 1 ? n : 1) : 1;
    c.launches = k * per_pass.launches;
    c.hop_launches = k * per_pass.hop_launches;
    return c;
  }
};
// halt, loops: device words of the solver's state (loops: the loop's pass
// counter, zero between launches).  Counters are left as they were.
lqcd_status build_solver_graph(lqcd_ctx *ctx, int chunk, const int *halt, int *loops,
                               const std::function<lqcd_status()> &iteration, SolverGraph *G);

// launches: the chunk's launch counts; n: iterations begun; halted: the last
// of them stopped at its halting reduction
inline void count_chunk(lqcd_ctx *ctx, const IterWork &w, const lqcd_counters &launches, int n, bool halted) {
  ctx->cnt.launches += launches.launches;
  ctx->cnt.hop_launches += launches.hop_launches;
  if (n <= 0) return;
  add_work(ctx->cnt, w.full, halted ? n - 1 : n);
  if (halted) add_work(ctx->cnt, w.first, 1.0);
}
inline double spinor_site_bytes(int prec) {
  return (double)spinor_bytes_per_site(prec) + ((prec == LQCD_BF16S || prec == LQCD_F16S) ? 4.0 : 0.0);
}

// gauge copies
lqcd_status gauge_view(lqcd_ctx *ctx, lqcd_gauge *U, int prec, int recon, GaugeView *out);

// ---------------------------------------------------------------------------
// hop kernel launch (dslash.cu)
// ---------------------------------------------------------------------------
struct HopLaunch {
  int prec = LQCD_F64;  // spinor precision == arithmetic class
  int recon = 18;
  GaugeView U{};
  HalfField in, out, aux;  // in: parity 1-p; out, aux: parity p
  int out_parity = 0;      // 0 or 1
  int dagger = 0;
  HostC c_up{1, 0}, c_dn{1, 0};  // out = c * H in + d * aux (per chirality)
  HostC d_up{0, 0}, d_dn{0, 0};
  bool has_aux = false;
  double *partials = nullptr;  // if set: |out|^2 partials [nrhs][nblocks]
  int *halt = nullptr;         // if set and *halt != 0 the kernel does nothing
};
lqcd_status launch_hop(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, int *nblocks_out);
int hop_blocks(const Geom &g, int nrhs);
// domain decomposition along t and z (dd.cu): dd_pack writes the two faces
// along mu = 2 (z) or 3 (t) (f0 = for the previous domain, f1 = for the next;
// n0/n1: negate them); dd_hop runs the domain's half hop with the faces
// received from the next and previous domains along t and, if z_next is not
// null, along z
lqcd_status dd_pack(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, int mu, void *f0, void *f1, int n0, int n1);
lqcd_status dd_hop(lqcd_ctx *ctx, const Geom &g, const HopLaunch &L, const void *t_next, const void *t_prev,
                   const void *z_next, const void *z_prev);
size_t dd_face_word_bytes(int prec);
int dd_face_sites(const Geom &g, int mu);  // sites of one parity in a boundary slice along mu
// domain-decomposed CG (dd_cg.cu): nd held domains of an nz x nt grid
// (domain dz + nz dt), the first of global index `first`; U: FP64 links, Ui:
// links of the inner format (prm.inner_prec F64: unused); b_full / x_full: EO
// full fields of each held domain; faces: per held domain to_prev, to_next,
// from_next, from_prev along t, then (nz > 1) the same four along z
lqcd_status dd_cg_solve(lqcd_ctx *ctx, int nd, int first, int nz, int nt, int antiper, const Geom &g, int recon,
                        const std::vector<GaugeView> &U, int recon_i, const std::vector<GaugeView> &Ui,
                        const std::vector<HalfField> &b_full, const std::vector<HalfField> &x_full,
                        const std::vector<void *> &faces, const lqcd_dd_comm *comm, double kappa, double mu,
                        const lqcd_cg_params &prm, lqcd_cg_stats *st);

// Operators assembled from hop launches (cg.cu)
struct Op {
  lqcd_ctx *ctx;
  Geom g;
  GaugeView U;
  int prec, recon;
  double kappa, mu;
};
// out_p = Mhat (or Mhat^+) in_p on parity p; tmp: half field of parity 1-p.
lqcd_status apply_schur(const Op &op, const HalfField &in, const HalfField &out, const HalfField &tmp,
                        int p, bool dagger, double *partials, int *nb, int *halt);
// full M (or M^+) on both parities of an EO field
lqcd_status apply_full(const Op &op, const HalfField &in_e, const HalfField &in_o, const HalfField &out_e,
                       const HalfField &out_o, bool dagger, double *partials_e, double *partials_o,
                       int *nb);
lqcd_status lincomb(lqcd_ctx *ctx, int Vh, const HalfField &out, const HalfField &x, const HalfField *y,
                    HostC ca_up, HostC ca_dn, HostC cb_up, HostC cb_dn, double *partials, int *nb_out);
lqcd_status spinor_convert_raw(lqcd_ctx *ctx, int Vh, int nh, const void *in, const float *in_scale,
                               int pin, void *out, float *out_scale, int pout);
lqcd_status spinor_pack_raw(lqcd_ctx *ctx, const Geom &g, const void *lexi, const HalfField &eo_full);
lqcd_status spinor_unpack_raw(lqcd_ctx *ctx, const Geom &g, const HalfField &eo_full, void *lexi);

}  // namespace lqcd
