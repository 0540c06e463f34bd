// noalloc.cu -- plaquette of a gauge field for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code running where the CUDA
// allocator is owned by someone else (a host framework's memory pool that
// forbids side allocations, a process whose memory budget is fixed up front,
// or work recorded into a larger graph while allocation is off limits).  For
// them lqcd_plaquette_noalloc computes the plaquette of a lexicographic gauge
// field without creating a context and without allocating: the per-block
// partial sums live in a fixed file-scope device array that every GPU which
// loads the library holds until the process exits.
//
// Scratch contract:
//   - lqcd_noalloc_partials holds LQCD_NOALLOC_MAX_BLOCKS doubles (256 KiB);
//     one block of 128 threads covers 128 sites, so V <= 128 * 32768 =
//     4194304 sites (e.g. 64^3 x 16 or 32^3 x 128); larger lattices are
//     rejected with LQCD_ERR_INVALID before anything is launched.
//   - every call writes partial slots 0..nblocks-1 before reading them, so
//     nothing has to start at zero; the array keeps the last call's values.
//   - all calls on a device share the one array: calls whose kernels overlap
//     on the GPU (different streams, no ordering between them) race and give
//     wrong results.  Order them on one stream or synchronise between them.
//   - the array's device address is looked up with cudaGetSymbolAddress on
//     every call made outside a stream capture, so a call after the device's
//     primary context was torn down and recreated (cudaDeviceReset), which
//     loads the module and its array afresh, never uses an address of the
//     old context.  A call made while its stream is capturing uses the address
//     of the last call on that device instead (no lookup inside a capture),
//     so one call outside a capture must come first on each device.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lqcd.h"

#define LQCD_NOALLOC_MAX_BLOCKS 32768
#define LQCD_NOALLOC_BLOCK 128

static __device__ __align__(256) double lqcd_noalloc_partials[LQCD_NOALLOC_MAX_BLOCKS];

namespace {

struct C2 {
  double re, im;
};
__device__ __forceinline__ C2 cmulc(C2 a, C2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C2 caddc(C2 a, C2 b) { return {a.re + b.re, a.im + b.im}; }

// 3x3 product a * b (dag_b: b^+), row-major complex128
__device__ void m3(const double2 *a, const double2 *b, bool dag_b, C2 *out) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      C2 s{0.0, 0.0};
      for (int k = 0; k < 3; k++) {
        C2 x{a[3 * i + k].x, a[3 * i + k].y};
        C2 y = dag_b ? C2{b[3 * j + k].x, -b[3 * j + k].y} : C2{b[3 * k + j].x, b[3 * k + j].y};
        s = caddc(s, cmulc(x, y));
      }
      out[3 * i + j] = s;
    }
}

// Sum over the block's sites of sum_{mu<nu} Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
// for a lexicographic field U[V][4][3][3]; one partial per block into `partials`.
__global__ void __launch_bounds__(LQCD_NOALLOC_BLOCK) plaquette_lexi_partials(const double2 *U, int Lx, int Ly,
                                                                             int Lz, int Lt, double *partials) {
  __shared__ double sh[LQCD_NOALLOC_BLOCK / 32];
  const long V = (long)Lx * Ly * Lz * Lt;
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < V) {
    const int L[4] = {Lx, Ly, Lz, Lt};
    int c[4];
    long r = i;
    for (int d = 0; d < 4; d++) {
      c[d] = (int)(r % L[d]);
      r /= L[d];
    }
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        int a[4] = {c[0], c[1], c[2], c[3]}, b[4] = {c[0], c[1], c[2], c[3]};
        a[mu] = (a[mu] + 1) % L[mu];
        b[nu] = (b[nu] + 1) % L[nu];
        long ia = a[0] + (long)Lx * (a[1] + (long)Ly * (a[2] + (long)Lz * a[3]));
        long ib = b[0] + (long)Lx * (b[1] + (long)Ly * (b[2] + (long)Lz * b[3]));
        C2 t1[9], t2[9], t3[9];
        double2 w1[9], w2[9];
        m3(U + (i * 4 + mu) * 9, U + (ia * 4 + nu) * 9, false, t1);   // U_mu(x) U_nu(x+mu)
        m3(U + (i * 4 + nu) * 9, U + (ib * 4 + mu) * 9, false, t2);   // U_nu(x) U_mu(x+nu)
        for (int k = 0; k < 9; k++) {
          w1[k] = make_double2(t1[k].re, t1[k].im);
          w2[k] = make_double2(t2[k].re, t2[k].im);
        }
        m3(w1, w2, true, t3);
        acc += t3[0].re + t3[4].re + t3[8].re;
      }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < LQCD_NOALLOC_BLOCK / 32; w++) t += sh[w];
    partials[blockIdx.x] = t;
  }
}

// One block: fixed-order sum of nb partials, normalised to the plaquette.
__global__ void plaquette_finish(const double *partials, int nb, double norm, double *out) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) t += partials[k];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] * norm;
}

std::mutex g_setup_mutex;
void *g_scratch[256];  // last looked-up device address of lqcd_noalloc_partials per device ordinal

// The device address of the array on the current device (dev): looked up on
// every call outside a capture; inside a capture of `st` the last address
// looked up on this device, or an error if there is none yet.
cudaError_t scratch_address(int dev, cudaStream_t st, double **ptr) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cs == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, lqcd_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  } else if (!g_scratch[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *ptr = (double *)g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int lqcd_plaquette_noalloc(const void *U_lexi, const lqcd_geom *geom, double *plaq_dev,
                                      void *cuda_stream) {
  if (!U_lexi || !geom || !plaq_dev) return LQCD_ERR_INVALID;
  if (((uintptr_t)U_lexi & 15u) || ((uintptr_t)plaq_dev & 7u)) return LQCD_ERR_INVALID;
  long V = 1;
  for (int k = 0; k < 4; k++) {
    if (geom->L[k] < 2 || (geom->L[k] & 1)) return LQCD_ERR_INVALID;
    V *= geom->L[k];
  }
  const long nb = (V + LQCD_NOALLOC_BLOCK - 1) / LQCD_NOALLOC_BLOCK;
  if (nb > LQCD_NOALLOC_MAX_BLOCKS) return LQCD_ERR_INVALID;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return LQCD_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *scratch = nullptr;
  if (scratch_address(dev, st, &scratch) != cudaSuccess) {
    cudaGetLastError();
    return LQCD_ERR_CUDA;
  }
  plaquette_lexi_partials<<<(unsigned)nb, LQCD_NOALLOC_BLOCK, 0, st>>>(
      (const double2 *)U_lexi, geom->L[0], geom->L[1], geom->L[2], geom->L[3], scratch);
  plaquette_finish<<<1, 256, 0, st>>>(scratch, (int)nb, 1.0 / (3.0 * 6.0 * (double)V), plaq_dev);
  if (cudaGetLastError() != cudaSuccess) return LQCD_ERR_CUDA;
  return LQCD_OK;
}
