// cta_launch.cu -- host side of the whole-solve-per-CTA engine: builds the
// instance descriptors of one or many problems (shared-matrix batches expand
// to one descriptor per instance), orders them longest-first for the device
// work queue, sizes shared memory and launches one persistent grid.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "cta_engine.cuh"
#include "dq_host.h"

namespace dq {

template <typename T>
static dq_status run(dq_problem* const* probs, int count, const SolveCfg* cfgs, const dq_outputs* outs,
                     dq_result* results, int smem_cap, int threads) {
  dq_context* ctx = probs[0]->ctx;
  cudaStream_t st = ctx->stream;
  size_t total = 0;
  for (int i = 0; i < count; ++i) total += probs[i]->batch;
  // scratch layout: insts | order | counter | results | consts | host-output staging
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
  void* scratch = nullptr;
  dq_status s = ctx_scratch(ctx, b_inst + b_order + b_cnt + b_res + b_con + b_stage, &scratch);
  if (s != DQ_OK) return s;
  char* base = (char*)scratch;
  CtaInst<T>* d_inst = (CtaInst<T>*)base;
  int* d_order = (int*)(base + b_inst);
  int* d_cnt = (int*)(base + b_inst + b_order);
  DevResult* d_res = (DevResult*)(base + b_inst + b_order + b_cnt);
  double* d_con = (double*)(base + b_inst + b_order + b_cnt + b_res);
  T* d_stage = (T*)(base + b_inst + b_order + b_cnt + b_res + b_con);

  std::vector<CtaInst<T>> hi(total);
  std::vector<double> cost(total);
  size_t vec_max = 0, want_max = 0, k = 0, so = 0;
  struct Stage {
    int prob;
    size_t off;
  };
  std::vector<Stage> stages;
  for (int i = 0; i < count; ++i) {
    dq_problem* P = probs[i];
    const SolveCfg& c = cfgs[i];
    const dq_outputs* o = outs ? &outs[i] : nullptr;
    const bool host_out = o && o->memory == DQ_HOST;
    const size_t n = P->n, p = P->p, pn = std::max<size_t>(p, 1);
    if (host_out) stages.push_back({i, so});
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
      I.lmax_Q = P->lmax_Q;
      I.lmin_Q = lmin;
      I.normG2 = P->normG2;
      I.rho = c.rho;
      I.LL = c.LL;
      I.sigma = c.sigma;
      I.Ld = c.Ld;
      I.inner_fixed = c.fixed_inner;
      I.inner_check_every = c.inner_check_every;
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
  const size_t cap = smem_cap > 0 ? std::min<size_t>(smem_cap, ctx->smem_optin) : ctx->smem_optin;
  if (vec_max > ctx->smem_optin) {
    set_error("instance too large for the CTA engine (needs %zu bytes of shared memory)", vec_max);
    return DQ_ERR_INVALID;
  }
  const size_t smem = std::max(vec_max, std::min(want_max, cap));
  std::vector<int> order(total);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  auto kern = cta_solve_kernel<T>;
  DQ_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  DQ_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
  if (occ < 1) {
    set_error("CTA engine cannot be resident with %zu bytes of shared memory", smem);
    return DQ_ERR_CUDA;
  }
  const int grid = (int)std::min<size_t>(total, (size_t)ctx->num_sms * occ);
  DQ_CK(cudaMemcpyAsync(d_inst, hi.data(), total * sizeof(CtaInst<T>), cudaMemcpyHostToDevice, st));
  DQ_CK(cudaMemcpyAsync(d_order, order.data(), total * sizeof(int), cudaMemcpyHostToDevice, st));
  DQ_CK(cudaMemsetAsync(d_cnt, 0, sizeof(int), st));
  kern<<<grid, threads, smem, st>>>(d_inst, d_order, (int)total, d_cnt, smem);
  ++ctx->launches;
  DQ_CK(cudaGetLastError());

  std::vector<DevResult> hr(total);
  std::vector<double> hc(total * 6);
  DQ_CK(cudaMemcpyAsync(hr.data(), d_res, total * sizeof(DevResult), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaMemcpyAsync(hc.data(), d_con, total * 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
  std::vector<T> hs(stage_elems);
  if (stage_elems)
    DQ_CK(cudaMemcpyAsync(hs.data(), d_stage, stage_elems * sizeof(T), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaStreamSynchronize(st));

  dq_status worst = DQ_OK;
  k = 0;
  size_t si = 0;
  for (int i = 0; i < count; ++i) {
    dq_problem* P = probs[i];
    const size_t n = P->n, p = P->p, pn = std::max<size_t>(p, 1);
    if (isnan(P->lmax_Q)) P->lmax_Q = hc[6 * k + 0];
    if (isnan(P->normG2)) P->normG2 = hc[6 * k + 1];
    P->has_state = true;
    const dq_outputs* o = outs ? &outs[i] : nullptr;
    size_t off = 0;
    if (o && o->memory == DQ_HOST) off = stages[si++].off;
    for (int b = 0; b < P->batch; ++b, ++k) {
      fill_result(&results[k], hr[k], &hc[6 * k], cfgs[i]);
      const dq_status st_i = (dq_status)hr[k].status;
      if (st_i < 0 && st_i == DQ_ERR_INVALID)
        set_error("instance %zu: invalid constants (DGM/DFGM need lmin_Q > 0)", k);
      if (st_i < 0 || worst < 0) worst = (st_i < worst) ? st_i : worst;
      else if (st_i > worst) worst = st_i;
      if (o && o->memory == DQ_HOST && st_i >= 0) {
        const T* src = hs.data() + off + b * (2 * n + pn);
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
                             const dq_outputs* outs, dq_result* results, int smem_cap, int threads) {
  if (probs[0]->prec == DQ_FP64) return run<double>(probs, count, cfgs, outs, results, smem_cap, threads);
  return run<float>(probs, count, cfgs, outs, results, smem_cap, threads);
}

}  // namespace dq
