// tune.cu -- the project's launch-shape autotuner.
//
// The paper tuned its Dslash "memory stride" by hand for one GPU (Sec. 5.2)
// and compiled run-time parameters into the kernels (Sec. 4).  Here every
// kernel configuration (kernel, precision, link format, dagger/epilogue
// variant, lattice extents, number of right-hand sides, GPU) gets its launch
// shape from a table: the first time a configuration is launched outside a
// stream capture, each candidate shape is run once to warm up and three times
// under CUDA events on the context's stream, and the fastest is kept (inside
// a capture an untuned hop configuration borrows a tuned sibling's choice).  The
// table can be persisted as a small JSON object {"key": choice, ...} in the
// file given to lqcd_set_autotune (or the LQCD_TUNE_CACHE environment
// variable), so later processes skip the timing.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>

#include "internal.h"

namespace lqcd {

void tune_load(lqcd_ctx *ctx) {
  if (ctx->tune_path.empty()) return;
  std::ifstream f(ctx->tune_path);
  if (!f) return;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  while ((i = s.find('"', i)) != std::string::npos) {
    size_t j = s.find('"', i + 1);
    if (j == std::string::npos) break;
    std::string key = s.substr(i + 1, j - i - 1);
    size_t c = s.find(':', j);
    if (c == std::string::npos) break;
    int v = std::atoi(s.c_str() + c + 1);
    ctx->tuned[key] = v;
    i = s.find_first_of(",}", c);
    if (i == std::string::npos) break;
  }
}

static void tune_save(lqcd_ctx *ctx) {
  if (ctx->tune_path.empty()) return;
  std::string tmp = ctx->tune_path + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t n = 0;
  for (const auto &kv : ctx->tuned)
    std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++n < ctx->tuned.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), ctx->tune_path.c_str());
}

// A hop configuration first met inside a stream capture (the reducing hop
// of a CG iteration is launched only inside the captured iteration) cannot
// be timed.  Its siblings -- the same kernel family, precision, links,
// extents and RHS count, differing only in the dagger, reduction or
// epilogue flags -- share its candidate list, so it takes the choice of the
// nearest tuned sibling (flags flipped one at a time, then two, then all).
static int sibling_choice(const lqcd_ctx *ctx, const std::string &key, int ncand) {
  const char *flags[3] = {"|d", "|red", "|aux"};
  size_t pos[3];
  for (int f = 0; f < 3; f++) {
    pos[f] = key.find(flags[f]);
    if (pos[f] == std::string::npos) return -1;
    pos[f] += std::char_traits<char>::length(flags[f]);
    if (pos[f] >= key.size() || (key[pos[f]] != '0' && key[pos[f]] != '1')) return -1;
  }
  static const int order[7] = {1, 2, 4, 3, 5, 6, 7};  // bit f flips flag f; fewest flips first
  for (int m : order) {
    std::string k = key;
    for (int f = 0; f < 3; f++)
      if (m & (1 << f)) k[pos[f]] = k[pos[f]] == '0' ? '1' : '0';
    auto it = ctx->tuned.find(k);
    if (it != ctx->tuned.end() && it->second >= 0 && it->second < ncand) return it->second;
  }
  return -1;
}

int tune_choice(lqcd_ctx *ctx, const std::string &key0, int ncand, int fallback,
                const std::function<void(int)> &run) {
  if (ctx->forced_choice >= 0) return ncand > 0 ? ctx->forced_choice % ncand : fallback;
  const std::string key = ctx->gpu_name + "|" + key0;
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end() && it->second >= 0 && it->second < ncand) return it->second;
  if (!ctx->autotune || ncand <= 1) return fallback;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    const int sib = key0.compare(0, 3, "hop") == 0 ? sibling_choice(ctx, key, ncand) : -1;
    return sib >= 0 ? sib : fallback;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fallback;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fallback;
  }
  int best = fallback;
  float best_ms = 1e30f;
  // the timing launches are not the caller's work: keep them out of the counters
  const lqcd_counters saved = ctx->cnt;
  for (int c = 0; c < ncand; c++) {
    run(c);
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3; r++) run(c);
    cudaEventRecord(e1, ctx->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaGetLastError() != cudaSuccess) continue;  // a shape that failed to launch is skipped
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->cnt = saved;
  ctx->tuned[key] = best;
  tune_save(ctx);
  return best;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_set_autotune(lqcd_ctx *ctx, int enable, const char *cache_path) {
  if (!ctx) return LQCD_ERR_INVALID;
  ctx->autotune = enable ? 1 : 0;
  if (cache_path) {
    ctx->tune_path = cache_path;
    tune_load(ctx);
  }
  return LQCD_OK;
}

extern "C" int lqcd_set_launch_choice(lqcd_ctx *ctx, int choice) {
  if (!ctx) return LQCD_ERR_INVALID;
  ctx->forced_choice = choice < 0 ? -1 : choice;
  return LQCD_OK;
}
