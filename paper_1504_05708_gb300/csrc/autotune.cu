// autotune.cu -- launch-shape autotuner of the CTA engine (uneven batches).
//
// For a mix of problems it times short fixed-count solves of a sample of the
// instances under each candidate (block size, shared-memory cap) with CUDA
// events on the context's stream and keeps the fastest.  The shared-memory
// cap trades staging Q, G, G' on chip against blocks resident per SM.  The
// choice is stored on the context under a signature of the size histogram
// (precision, per-bucket share of variables) and persisted to a text file
// (DQ_AUTOTUNE_CACHE or autotune.txt next to the library), so later runs of
// the same mix start tuned.
#include <dlfcn.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dq_host.h"

namespace dq {

std::string cta_signature(dq_problem* const* probs, int count) {
  // share of instances per n-bucket of width 64 (up to 1024), rounded to 5%
  int hist[17] = {0};
  int tot = 0;
  for (int i = 0; i < count; ++i) {
    const int bkt = std::min(probs[i]->n / 64, 16);
    hist[bkt] += probs[i]->batch;
    tot += probs[i]->batch;
  }
  std::string s = probs[0]->prec == DQ_FP64 ? "f64" : "f32";
  for (int k = 0; k < 17; ++k) {
    const int pct = tot ? (int)lround(20.0 * hist[k] / tot) : 0;
    s += ":" + std::to_string(pct);
  }
  return s;
}

static std::string cache_path() {
  const char* env = getenv("DQ_AUTOTUNE_CACHE");
  if (env && *env) return env;
  Dl_info info;
  if (dladdr((void*)&cache_path, &info) && info.dli_fname) {
    std::string f = info.dli_fname;
    const size_t slash = f.rfind('/');
    if (slash != std::string::npos) return f.substr(0, slash + 1) + "autotune.txt";
  }
  return "autotune.txt";
}

static void load_cache(dq_context* ctx) {
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return;
  char sig[512];
  int th, sm;
  while (fscanf(f, "%511s %d %d", sig, &th, &sm) == 3) ctx->tuned[sig] = {th, sm};
  fclose(f);
}

static void save_cache(const dq_context* ctx) {
  FILE* f = fopen(cache_path().c_str(), "w");
  if (!f) return;
  for (const auto& kv : ctx->tuned) fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
  fclose(f);
}

}  // namespace dq

using namespace dq;

extern "C" dq_status dq_autotune(dq_problem* const* probs, int32_t count, const dq_solve_opts* opts, int32_t sample,
                                 int32_t* threads_out, int32_t* smem_cap_out) {
  if (!probs || count < 1 || !opts) {
    set_error("dq_autotune needs problems and options");
    return DQ_ERR_INVALID;
  }
  dq_context* ctx = probs[0]->ctx;
  for (int i = 0; i < count; ++i)
    if (!probs[i] || probs[i]->ctx != ctx || probs[i]->prec != probs[0]->prec || probs[i]->prec == DQ_BF16X3) {
      set_error("dq_autotune needs FP64 or FP32 problems of one precision and one context");
      return DQ_ERR_INVALID;
    }
  DQ_CK(cudaSetDevice(ctx->device));
  const std::string sig = cta_signature(probs, count);
  if (ctx->tuned.empty()) load_cache(ctx);
  auto hit = ctx->tuned.find(sig);
  if (hit != ctx->tuned.end()) {
    if (threads_out) *threads_out = hit->second.first;
    if (smem_cap_out) *smem_cap_out = hit->second.second;
    return DQ_OK;
  }
  // sample spread over the mix, short fixed-count solves
  const int ns = std::max(1, std::min(sample > 0 ? sample : 256, count));
  std::vector<dq_problem*> sp(ns);
  std::vector<SolveCfg> cf(ns);
  for (int i = 0; i < ns; ++i) {
    const int idx = (int)((long long)i * count / ns);
    sp[i] = probs[idx];
    dq_status s = resolve_opts(sp[i], &opts[idx], &cf[i]);
    if (s != DQ_OK) return s;
    cf[i].fixed_outer = 2;
    cf[i].fixed_inner = 25;
    cf[i].inner_stop = DQ_INNER_FIXED;
    cf[i].warm_start = 0;
  }
  int total = 0;
  for (auto* p : sp) total += p->batch;
  std::vector<dq_result> res(total);
  const int cand_threads[3] = {128, 256, 512};
  const int cand_smem[3] = {48 * 1024, 112 * 1024, 0};
  cudaEvent_t e0, e1;
  DQ_CK(cudaEventCreate(&e0));
  DQ_CK(cudaEventCreate(&e1));
  float best = INFINITY;
  int bt = 256, bs = 0;
  // warm-up (constants computed once and cached on the handles)
  cta_solve_problems(sp.data(), ns, cf.data(), nullptr, res.data(), 0, 256, false);
  for (int t : cand_threads) {
    for (int sm : cand_smem) {
      cudaEventRecord(e0, ctx->stream);
      const dq_status s = cta_solve_problems(sp.data(), ns, cf.data(), nullptr, res.data(), sm, t, false);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      if (s < 0) {
        cudaGetLastError();
        continue;  // e.g. a cap below the vectors' needs
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bt = t;
        bs = sm;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!(best < INFINITY)) {
    set_error("dq_autotune: no candidate configuration ran");
    return DQ_ERR_CUDA;
  }
  ctx->tuned[sig] = {bt, bs};
  save_cache(ctx);
  if (threads_out) *threads_out = bt;
  if (smem_cap_out) *smem_cap_out = bs;
  return DQ_OK;
}
