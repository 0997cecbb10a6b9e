// cta_launch.cu -- host side of the whole-solve-per-CTA engine: builds the
// instance descriptors of one or many problems (shared-matrix batches expand
// to one descriptor per instance), orders them longest-first for the device
// work queue, sizes shared memory and launches one persistent grid.  The
// launch (descriptor upload, queue reset, kernel, result download) can run as
// a captured CUDA graph that is replayed while the inputs stay the same.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "cta_engine.cuh"
#include "dq_host.h"

namespace dq {

template <typename T>
static const void* kernel_fn(int threads) {
  switch (threads) {
    case 128: return (const void*)cta_solve_kernel<T, 128>;
    case 512: return (const void*)cta_solve_kernel<T, 512>;
    default: return (const void*)cta_solve_kernel<T, 256>;
  }
}

template <typename T>
static void launch(int threads, int grid, size_t smem, cudaStream_t st, const CtaInst<T>* insts, const int* order,
                   int count, int* next) {
  switch (threads) {
    case 128: cta_solve_kernel<T, 128><<<grid, 128, smem, st>>>(insts, order, count, next, smem); break;
    case 512: cta_solve_kernel<T, 512><<<grid, 512, smem, st>>>(insts, order, count, next, smem); break;
    default: cta_solve_kernel<T, 256><<<grid, 256, smem, st>>>(insts, order, count, next, smem); break;
  }
}

static uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < bytes; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

static dq_status pinned_scratch(dq_context* ctx, size_t bytes, void** out) {
  if (bytes > ctx->pinned_bytes) {
    if (ctx->pinned) {
      DQ_CK(cudaStreamSynchronize(ctx->stream));
      if (ctx->gstream) DQ_CK(cudaStreamSynchronize(ctx->gstream));
      cudaFreeHost(ctx->pinned);
      ctx->pinned = nullptr;
      ctx->pinned_bytes = 0;
      if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
        ctx->gkey = 0;
      }
    }
    const size_t b = std::max(bytes, size_t(1) << 20);
    if (cudaMallocHost(&ctx->pinned, b) != cudaSuccess) {
      cudaGetLastError();
      set_error("pinned staging allocation of %zu bytes failed", b);
      return DQ_ERR_NOMEM;
    }
    ctx->pinned_bytes = b;
  }
  *out = ctx->pinned;
  return DQ_OK;
}

template <typename T>
static dq_status run(dq_problem* const* probs, int count, const SolveCfg* cfgs, const dq_outputs* outs,
                     dq_result* results, int smem_cap, int threads, bool use_graph) {
  dq_context* ctx = probs[0]->ctx;
  cudaStream_t st = ctx->stream;
  size_t total = 0;
  for (int i = 0; i < count; ++i) total += probs[i]->batch;
  // device scratch: insts | order | counter | results | consts | host-output staging
  size_t stage_elems = 0;
  for (int i = 0; i < count; ++i) {
    const dq_outputs* o = outs ? &outs[i] : nullptr;
    if (o && o->memory == DQ_HOST)
      stage_elems += (size_t)probs[i]->batch * (2 * probs[i]->n + std::max(probs[i]->p, 1));
  }
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_inst = a256(total * sizeof(CtaInst<T>));
  const size_t b_order = a256(total * sizeof(int));
  const size_t b_cnt = 256;
  const size_t b_res = a256(total * sizeof(DevResult));
  const size_t b_con = a256(total * 6 * sizeof(double));
  const size_t b_stage = a256(stage_elems * sizeof(T));
  const size_t b_all = b_inst + b_order + b_cnt + b_res + b_con + b_stage;
  void* scratch = nullptr;
  dq_status s = ctx_scratch(ctx, b_all, &scratch);
  if (s != DQ_OK) return s;
  void* hbuf = nullptr;  // pinned mirror of the same layout
  if ((s = pinned_scratch(ctx, b_all, &hbuf)) != DQ_OK) return s;
  char* base = (char*)scratch;
  char* hbase = (char*)hbuf;
  CtaInst<T>* d_inst = (CtaInst<T>*)base;
  int* d_order = (int*)(base + b_inst);
  int* d_cnt = (int*)(base + b_inst + b_order);
  DevResult* d_res = (DevResult*)(base + b_inst + b_order + b_cnt);
  double* d_con = (double*)(base + b_inst + b_order + b_cnt + b_res);
  T* d_stage = (T*)(base + b_inst + b_order + b_cnt + b_res + b_con);
  CtaInst<T>* hi = (CtaInst<T>*)hbase;
  int* h_order = (int*)(hbase + b_inst);
  DevResult* h_res = (DevResult*)(hbase + b_inst + b_order + b_cnt);
  double* h_con = (double*)(hbase + b_inst + b_order + b_cnt + b_res);
  T* h_stage = (T*)(hbase + b_inst + b_order + b_cnt + b_res + b_con);

  std::vector<double> cost(total);
  size_t vec_max = 0, want_max = 0, k = 0, so = 0;
  std::vector<size_t> stage_off(count, 0);
  for (int i = 0; i < count; ++i) {
    dq_problem* P = probs[i];
    const SolveCfg& c = cfgs[i];
    const dq_outputs* o = outs ? &outs[i] : nullptr;
    const bool host_out = o && o->memory == DQ_HOST;
    const size_t n = P->n, p = P->p, pn = std::max<size_t>(p, 1);
    stage_off[i] = so;
    const bool warm = c.warm_start && P->has_state;
    const double lmin = P->lmin_Q;
    for (int b = 0; b < P->batch; ++b, ++k) {
      CtaInst<T>& I = hi[k];
      memset(&I, 0, sizeof(I));
      I.n = (int)n;
      I.p = (int)p;
      I.cone = P->cone;
      I.alg = c.alg;
      I.Q = (const T*)P->Q;
      I.G = (const T*)P->G;
      I.GT = (const T*)P->GT;
      I.q = (const T*)P->q + b * n;
      I.g = (const T*)P->g + b * p;
      I.lb = (const T*)P->lb;
      I.ub = (const T*)P->ub;
      I.lmax_Q = c.fresh ? P->lmax_given : P->lmax_Q;
      I.lmin_Q = lmin;
      I.normG2 = c.fresh ? P->normG2_given : P->normG2;
      I.lip_bound = P->lip_bound;
      I.stop_fstar = c.stop_fstar;
      I.f_star = c.f_star;
      I.rho = c.rho;
      I.LL = c.LL;
      I.sigma = c.sigma;
      I.Ld = c.Ld;
      I.inner_fixed = c.fixed_inner;
      I.inner_check_every = c.inner_check_every;
      I.cert_step = c.inner_cert == DQ_CERT_STEP;  // DQ_CERT_AUTO: the point certificate here
      I.max_inner = c.max_inner;
      I.eps_in = c.eps_in;
      I.outer_fixed = c.fixed_outer;
      I.check_every = c.check_every;
      I.max_outer = c.max_outer;
      I.eps_out = c.eps_out;
      I.want_last = (c.output & DQ_OUT_LAST) != 0;
      I.want_avg = (c.output & DQ_OUT_AVERAGE) != 0;
      I.kd_plus = !(c.kd_literal && !(lmin > 0.0));
      I.x0 = warm ? (const T*)P->x_state + b * n : nullptr;
      I.lam0 = warm ? (const T*)P->lam_state + b * p : nullptr;
      I.x_state = (T*)P->x_state + b * n;
      I.lam_state = (T*)P->lam_state + b * p;
      if (o && o->memory == DQ_DEVICE) {
        I.x_last = o->x_last ? (T*)o->x_last + b * n : nullptr;
        I.x_avg = o->x_avg ? (T*)o->x_avg + b * n : nullptr;
        I.lam_out = o->lambda ? (T*)o->lambda + b * p : nullptr;
      } else if (host_out) {
        I.x_last = d_stage + so;
        I.x_avg = d_stage + so + n;
        I.lam_out = d_stage + so + 2 * n;
        so += 2 * n + pn;
      }
      I.res = d_res + k;
      I.consts_out = d_con + 6 * k;
      const size_t vb = cta_vec_bytes<T>((int)n, (int)p);
      vec_max = std::max(vec_max, vb);
      want_max = std::max(want_max, vb + cta_mat_bytes<T>((int)n, (int)p));
      cost[k] = double(n) * n + 2.0 * double(n) * p;
    }
  }
  const void* kfn = kernel_fn<T>(threads);
  const size_t dmax = max_dynamic_smem(kfn, ctx->smem_optin);
  const size_t cap = smem_cap > 0 ? std::min<size_t>(smem_cap, dmax) : dmax;
  if (vec_max > dmax) {
    set_error("instance too large for the CTA engine (needs %zu bytes of shared memory)", vec_max);
    return DQ_ERR_INVALID;
  }
  const size_t smem = std::max(vec_max, std::min(want_max, cap));
  std::iota(h_order, h_order + total, 0);
  std::stable_sort(h_order, h_order + total, [&](int a, int b) { return cost[a] > cost[b]; });

  DQ_CK(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  DQ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, threads, smem));
  if (occ < 1) {
    set_error("CTA engine cannot be resident with %zu bytes of shared memory", smem);
    return DQ_ERR_CUDA;
  }
  const int grid = (int)std::min<size_t>(total, (size_t)ctx->num_sms * occ);
  // the whole launch as one stream-ordered sequence
  auto enqueue = [&](cudaStream_t q) -> cudaError_t {
    cudaMemcpyAsync(d_inst, hi, b_inst + b_order, cudaMemcpyHostToDevice, q);
    cudaMemsetAsync(d_cnt, 0, sizeof(int), q);
    launch<T>(threads, grid, smem, q, d_inst, d_order, (int)total, d_cnt);
    cudaMemcpyAsync(h_res, d_res, b_res + b_con + b_stage, cudaMemcpyDeviceToHost, q);
    return cudaGetLastError();
  };
  ++ctx->launches;
  if (use_graph) {
    uint64_t key = fnv1a(hi, total * sizeof(CtaInst<T>));
    key = fnv1a(h_order, total * sizeof(int), key);
    const uint64_t shape[6] = {(uint64_t)total, (uint64_t)smem, (uint64_t)threads, (uint64_t)grid,
                               (uint64_t)(uintptr_t)scratch, (uint64_t)(uintptr_t)hbuf};
    key = fnv1a(shape, sizeof(shape), key);
    if (!ctx->gstream) DQ_CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    if (!ctx->gev[0]) {
      DQ_CK(cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming));
      DQ_CK(cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming));
    }
    if (!ctx->gexec || ctx->gkey != key) {
      if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
      }
      cudaGraph_t g;
      DQ_CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = enqueue(ctx->gstream);
      cudaError_t ce2 = cudaStreamEndCapture(ctx->gstream, &g);
      if (ce != cudaSuccess || ce2 != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
        return DQ_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&ctx->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        set_error("graph instantiation failed: %s", cudaGetErrorString(ce));
        return DQ_ERR_CUDA;
      }
      ctx->gkey = key;
    }
    DQ_CK(cudaEventRecord(ctx->gev[0], st));
    DQ_CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
    DQ_CK(cudaGraphLaunch(ctx->gexec, ctx->gstream));
    DQ_CK(cudaEventRecord(ctx->gev[1], ctx->gstream));
    DQ_CK(cudaStreamWaitEvent(st, ctx->gev[1], 0));
    DQ_CK(cudaStreamSynchronize(ctx->gstream));
  } else {
    DQ_CK(enqueue(st));
    DQ_CK(cudaStreamSynchronize(st));
  }

  dq_status worst = DQ_OK;
  k = 0;
  for (int i = 0; i < count; ++i) {
    dq_problem* P = probs[i];
    const size_t n = P->n, p = P->p, pn = std::max<size_t>(p, 1);
    if (isnan(P->lmax_Q)) P->lmax_Q = h_con[6 * k + 0];
    if (isnan(P->normG2)) P->normG2 = h_con[6 * k + 1];
    P->has_state = true;
    const dq_outputs* o = outs ? &outs[i] : nullptr;
    const size_t off = stage_off[i];
    for (int b = 0; b < P->batch; ++b, ++k) {
      fill_result(&results[k], h_res[k], &h_con[6 * k], cfgs[i]);
      const dq_status st_i = (dq_status)h_res[k].status;
      if (st_i == DQ_ERR_INVALID) set_error("instance %zu: invalid constants (DGM/DFGM need lmin_Q > 0)", k);
      if (st_i == DQ_ERR_DIVERGED)
        set_error("instance %zu: infeasible (the certified dual lower bound passed the largest value of F on the box)",
                  k);
      if (st_i < 0 || worst < 0) worst = (st_i < worst) ? st_i : worst;
      else if (st_i > worst) worst = st_i;
      if (o && o->memory == DQ_HOST && st_i >= 0) {
        const T* src = h_stage + off + b * (2 * n + pn);
        if (o->x_last)
          for (size_t j = 0; j < n; ++j) ((double*)o->x_last)[b * n + j] = double(src[j]);
        if (o->x_avg)
          for (size_t j = 0; j < n; ++j) ((double*)o->x_avg)[b * n + j] = double(src[n + j]);
        if (o->lambda)
          for (size_t j = 0; j < p; ++j) ((double*)o->lambda)[b * p + j] = double(src[2 * n + j]);
      }
    }
  }
  return worst;
}

dq_status cta_solve_problems(dq_problem* const* probs, int count, const SolveCfg* cfgs,
                             const dq_outputs* outs, dq_result* results, int smem_cap, int threads,
                             bool graph) {
  for (int i = 0; i < count; ++i)
    if (probs[i]->sparse) {
      set_error("problem %d is sparse (CSR): sparse problems run on the grid engine (dq_solve)", i);
      return DQ_ERR_INVALID;
    }
  if (probs[0]->prec == DQ_FP64)
    return run<double>(probs, count, cfgs, outs, results, smem_cap, threads, graph);
  return run<float>(probs, count, cfgs, outs, results, smem_cap, threads, graph);
}

}  // namespace dq
