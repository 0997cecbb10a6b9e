// capi.cu -- the C ABI of include/duquad.h: contexts, the device problem
// store, option resolution and dispatch to the engines.
#include <math.h>
#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dq_host.h"

namespace dq {

static thread_local char g_err[512];

size_t max_dynamic_smem(const void* kernel, size_t optin) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess) {
    cudaGetLastError();
    return optin > 4096 ? optin - 4096 : optin;
  }
  return optin > a.sharedSizeBytes ? optin - a.sharedSizeBytes : 0;
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// ------------------------------------------------------------ small kernels

template <typename T>
__global__ void k_transpose(const T* __restrict__ in, T* __restrict__ out, int rows, int cols) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = bx + k, c = by + threadIdx.x;  // out is cols x rows
    if (r < cols && c < rows) out[(size_t)r * rows + c] = tile[threadIdx.x][k];
  }
}

__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, size_t m) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    out[i] = float(in[i]);
}

dq_status ctx_scratch(dq_context* ctx, size_t bytes, void** out) {
  if (bytes > ctx->scratch_bytes) {
    if (ctx->scratch) {
      DQ_CK(cudaStreamSynchronize(ctx->stream));
      cudaFree(ctx->scratch);
      ctx->scratch = nullptr;
      ctx->scratch_bytes = 0;
    }
    size_t b = std::max(bytes, size_t(1) << 20);
    if (cudaMalloc(&ctx->scratch, b) != cudaSuccess) {
      cudaGetLastError();
      set_error("scratch allocation of %zu bytes failed", b);
      return DQ_ERR_NOMEM;
    }
    ctx->scratch_bytes = b;
  }
  *out = ctx->scratch;
  return DQ_OK;
}

static dq_status dalloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed", bytes);
    return DQ_ERR_NOMEM;
  }
  return DQ_OK;
}

// Copy `m` elements into device array `dst` of the problem's element type.
// src: host double (memory = DQ_HOST) or device array of the element type.
static dq_status upload(dq_problem* P, void* dst, const void* src, size_t m, int memory) {
  cudaStream_t st = P->ctx->stream;
  if (m == 0) return DQ_OK;
  if (memory == DQ_DEVICE) {
    DQ_CK(cudaMemcpyAsync(dst, src, m * P->esz, cudaMemcpyDeviceToDevice, st));
    return DQ_OK;
  }
  if (P->esz == 8) {
    DQ_CK(cudaMemcpyAsync(dst, src, m * 8, cudaMemcpyHostToDevice, st));
    return DQ_OK;
  }
  void* tmp = nullptr;
  dq_status s = dalloc(&tmp, m * 8);
  if (s != DQ_OK) return s;
  cudaError_t e = cudaMemcpyAsync(tmp, src, m * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_d2f<<<1024, 256, 0, st>>>((const double*)tmp, (float*)dst, m);
    ++P->ctx->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) {
    set_error("upload failed: %s", cudaGetErrorString(e));
    return DQ_ERR_CUDA;
  }
  return DQ_OK;
}

static bool host_all_finite(const double* a, size_t m) {
  for (size_t i = 0; i < m; ++i)
    if (!isfinite(a[i])) return false;
  return true;
}

void fill_result(dq_result* r, const DevResult& d, const double* consts, const SolveCfg& c) {
  memset(r, 0, sizeof(*r));
  r->status = d.status;
  r->outer_iters = d.outer_iters;
  r->inner_iters = d.inner_iters;
  r->converged_last = d.converged_last;
  r->converged_avg = d.converged_avg;
  r->f_last = d.f_last;
  r->infeas_last = d.infeas_last;
  r->f_avg = d.f_avg;
  r->infeas_avg = d.infeas_avg;
  r->d_lb = d.d_lb;
  if (consts) {
    r->LL = consts[2];
    r->Ld = consts[3];
    r->sigma = consts[4];
    r->rho = consts[5];
    r->alpha = 1.0 / (2.0 * consts[3]);
  }
  (void)c;
}

dq_status resolve_opts(const dq_problem* P, const dq_solve_opts* o, SolveCfg* c) {
  if (!o) {
    set_error("opts is NULL");
    return DQ_ERR_INVALID;
  }
  if (o->alg < DQ_DGM || o->alg > DQ_ADFGM) {
    set_error("unknown algorithm %d", o->alg);
    return DQ_ERR_INVALID;
  }
  c->alg = o->alg;
  c->output = o->output ? o->output : DQ_OUT_BOTH;
  if (c->output < 1 || c->output > 3) {
    set_error("bad output selector %d", o->output);
    return DQ_ERR_INVALID;
  }
  c->inner_stop = o->inner_stop;
  c->engine = o->engine;
  c->eps_out = isnan(o->eps_out) || o->eps_out <= 0 ? 1e-3 : o->eps_out;
  c->eps_in = o->eps_in;  // NaN: derived on the device from eq. choose_ein
  c->rho = o->rho;
  if (!isnan(c->rho) && c->rho < 0) {
    set_error("rho must be >= 0");
    return DQ_ERR_INVALID;
  }
  if ((o->alg == DQ_DGM || o->alg == DQ_DFGM) && !isnan(c->rho) && c->rho != 0.0) {
    set_error("DGM/DFGM use rho = 0 (Case 1); use ADGM/ADFGM for rho > 0");
    return DQ_ERR_INVALID;
  }
  c->fixed_outer = o->fixed_outer > 0 ? o->fixed_outer : 0;
  c->fixed_inner = o->fixed_inner > 0 ? o->fixed_inner : 0;
  if (c->inner_stop == DQ_INNER_FIXED && c->fixed_inner <= 0) {
    set_error("DQ_INNER_FIXED needs fixed_inner > 0");
    return DQ_ERR_INVALID;
  }
  if (c->inner_stop != DQ_INNER_FIXED) c->fixed_inner = 0;
  c->max_outer = o->max_outer > 0 ? o->max_outer : 10000;
  c->max_inner = o->max_inner > 0 ? o->max_inner : 5000;
  c->check_every = o->check_every > 0 ? o->check_every : 1;
  c->inner_check_every = o->inner_check_every > 0 ? o->inner_check_every : 1;
  c->warm_start = o->warm_start;
  c->fresh = o->fresh_constants != 0;
  c->kd_literal = o->kd_literal;
  c->Ld = o->Ld;
  c->LL = o->LL;
  c->sigma = o->sigma;
  if (o->inner_cert < DQ_CERT_AUTO || o->inner_cert > DQ_CERT_STEP) {
    set_error("inner_cert must be DQ_CERT_AUTO, DQ_CERT_POINT or DQ_CERT_STEP");
    return DQ_ERR_INVALID;
  }
  c->inner_cert = o->inner_cert;
  (void)P;
  return DQ_OK;
}

}  // namespace dq

using namespace dq;

// ------------------------------------------------------------------ C ABI

extern "C" {

const char* dq_last_error(void) { return g_err; }

const char* dq_version(void) { return "duquad-gb300 0.1 (sm_103a)"; }

dq_status dq_theory(const dq_theory_in* in, dq_theory_out* out) {
  if (!in || !out) {
    set_error("NULL argument");
    return DQ_ERR_INVALID;
  }
  const bool fast = in->alg == DQ_DFGM || in->alg == DQ_ADFGM, aug = in->alg == DQ_ADGM || in->alg == DQ_ADFGM;
  auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
  if (in->alg < DQ_DGM || in->alg > DQ_ADFGM || !pos(in->eps) || !pos(in->Rd) || !pos(in->D_U) ||
      !std::isfinite(in->lmax_Q) || !std::isfinite(in->normG2) || in->normG2 < 0.0 || !(in->lmin_Q >= 0.0) ||
      !std::isfinite(in->lmin_Q)) {
    set_error("dq_theory: invalid algorithm, eps, R_d, D_U or constants");
    return DQ_ERR_INVALID;
  }
  const double rho = std::isnan(in->rho) ? (aug ? 8.0 * in->Rd * in->Rd / in->eps : 0.0) : in->rho;
  if (!(rho >= 0.0) || !std::isfinite(rho) || (!aug && rho != 0.0)) {
    set_error("dq_theory: rho must be >= 0 (and 0 for DGM/DFGM)");
    return DQ_ERR_INVALID;
  }
  const double LL = in->lmax_Q + rho * in->normG2, sigma = in->lmin_Q;
  const double den = in->lmin_Q + rho * in->normG2;
  if (!(LL > 0.0) || (in->normG2 > 0.0 && !(den > 0.0))) {
    set_error("dq_theory: L_d is undefined (DGM/DFGM need lmin_Q > 0)");
    return DQ_ERR_INVALID;
  }
  const double Ld = in->normG2 > 0.0 ? in->normG2 / den : 1.0;
  const double eps = in->eps, Rd = in->Rd, D2 = in->D_U * in->D_U;
  const double eps_in = fast ? eps * std::sqrt(eps) / (8.0 * Rd * std::sqrt(2.0 * Ld)) : eps / 4.0;
  const double kout = fast ? std::sqrt(8.0 * Ld * Rd * Rd / eps) : 8.0 * Ld * Rd * Rd / eps;
  const double kin = sigma > 0.0 ? std::sqrt(LL / sigma) * std::log(LL * D2 / eps_in) + 1.0
                                 : std::sqrt(2.0 * LL * D2 / eps_in);
  auto up = [](double v) { return (int64_t)std::max(1.0, std::ceil(v)); };
  out->rho = rho;
  out->LL = LL;
  out->sigma = sigma;
  out->Ld = Ld;
  out->eps_in = eps_in;
  out->k_out = up(kout);
  out->k_in = up(kin);
  out->k_total = out->k_out * out->k_in;
  return DQ_OK;
}

dq_status dq_context_profile(dq_context* ctx, int32_t enable) {
  if (!ctx) {
    set_error("NULL context");
    return DQ_ERR_INVALID;
  }
  ctx->profile = enable != 0;
  return DQ_OK;
}

dq_status dq_context_stats(dq_context* ctx, dq_stats* out, int32_t reset) {
  if (!ctx || !out) {
    set_error("NULL argument");
    return DQ_ERR_INVALID;
  }
  out->launches = ctx->launches;
  out->gemv_launches = ctx->gemv_launches;
  out->gemv_ms = ctx->gemv_ms;
  out->gemv_bytes = ctx->gemv_bytes;
  out->reduce_launches = ctx->reduce_launches;
  out->reduce_ms = ctx->reduce_ms;
  if (reset) {
    ctx->launches = ctx->gemv_launches = ctx->reduce_launches = 0;
    ctx->gemv_ms = ctx->gemv_bytes = ctx->reduce_ms = 0.0;
  }
  return DQ_OK;
}

dq_status dq_context_create(int device, void* cuda_stream, dq_context** out) {
  if (!out) {
    set_error("out is NULL");
    return DQ_ERR_INVALID;
  }
  *out = nullptr;
  int ndev = 0;
  DQ_CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    set_error("device %d out of range (%d devices)", device, ndev);
    return DQ_ERR_INVALID;
  }
  DQ_CK(cudaSetDevice(device));
  dq_context* c = new dq_context();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete c;
    set_error("cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    return DQ_ERR_CUDA;
  }
  c->num_sms = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  *out = c;
  return DQ_OK;
}

dq_status dq_serve_stop(dq_context* ctx);

static void context_free(dq_context* ctx) {
  cudaStreamSynchronize(ctx->stream);
  if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  for (cudaEvent_t e : ctx->gev)
    if (e) cudaEventDestroy(e);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->scratch) cudaFree(ctx->scratch);
  delete ctx;
}

dq_status dq_context_destroy(dq_context* ctx) {
  if (!ctx) return DQ_OK;
  if (ctx->serve) dq_serve_stop(ctx);
  if (ctx->live_problems > 0) {  // freed when the last problem handle goes
    ctx->destroy_requested = true;
    return DQ_OK;
  }
  context_free(ctx);
  return DQ_OK;
}

dq_status dq_problem_create(dq_context* ctx, const dq_problem_desc* d, dq_problem** out) {
  if (!ctx || !d || !out) {
    set_error("NULL argument");
    return DQ_ERR_INVALID;
  }
  *out = nullptr;
  if (d->n < 1 || d->p < 0 || d->batch < 1) {
    set_error("need n >= 1, p >= 0, batch >= 1 (got %d, %d, %d)", d->n, d->p, d->batch);
    return DQ_ERR_INVALID;
  }
  if (d->cone != DQ_CONE_INEQ && d->cone != DQ_CONE_EQ) {
    set_error("unknown cone %d", d->cone);
    return DQ_ERR_INVALID;
  }
  if (d->prec < DQ_FP64 || d->prec > DQ_BF16X3) {
    set_error("unknown precision %d", d->prec);
    return DQ_ERR_INVALID;
  }
  if (d->prec == DQ_BF16X3 && d->batch < 2) {
    set_error("DQ_BF16X3 is for shared-matrix batches (batch >= 2)");
    return DQ_ERR_INVALID;
  }
  if (d->memory != DQ_HOST && d->memory != DQ_DEVICE) {
    set_error("unknown memory kind %d", d->memory);
    return DQ_ERR_INVALID;
  }
  if (!d->Q || !d->q || !d->lb || !d->ub || (d->p > 0 && (!d->G || !d->g))) {
    set_error("NULL problem array");
    return DQ_ERR_INVALID;
  }
  const size_t n = d->n, p = d->p, B = d->batch;
  if (d->memory == DQ_HOST) {
    const double* lb = (const double*)d->lb;
    const double* ub = (const double*)d->ub;
    for (size_t i = 0; i < n; ++i)
      if (!(lb[i] <= ub[i])) {
        set_error("lb[%zu] > ub[%zu] or NaN", i, i);
        return DQ_ERR_INVALID;
      }
    if (!host_all_finite((const double*)d->Q, n * n) || !host_all_finite((const double*)d->q, B * n) ||
        (p && (!host_all_finite((const double*)d->G, p * n) || !host_all_finite((const double*)d->g, B * p))) ||
        !host_all_finite(lb, n) || !host_all_finite(ub, n)) {
      set_error("non-finite value in the problem data");
      return DQ_ERR_INVALID;
    }
  }
  if (!isnan(d->lmin_Q) && d->lmin_Q < 0) {
    set_error("lmin_Q must be a lower bound >= 0");
    return DQ_ERR_INVALID;
  }
  DQ_CK(cudaSetDevice(ctx->device));
  dq_problem* P = new dq_problem();
  P->ctx = ctx;
  ++ctx->live_problems;
  P->n = d->n;
  P->p = d->p;
  P->batch = d->batch;
  P->cone = d->cone;
  P->prec = d->prec;
  P->esz = d->prec == DQ_FP64 ? 8 : 4;
  P->lmax_Q = d->lmax_Q;
  P->lmin_Q = d->lmin_Q;
  P->normG2 = d->normG2;
  P->lmax_given = d->lmax_Q;
  P->normG2_given = d->normG2;
  dq_status s = DQ_OK;
  auto fail = [&](dq_status st) {
    dq_problem_destroy(P);
    return st;
  };
  const size_t e = P->esz;
  if (d->memory == DQ_DEVICE) {
    P->Q = (void*)d->Q;
    P->G = (void*)d->G;
  } else {
    if ((s = dalloc(&P->Q, n * n * e)) != DQ_OK) return fail(s);
    P->own_Q = true;
    if ((s = upload(P, P->Q, d->Q, n * n, DQ_HOST)) != DQ_OK) return fail(s);
    if (p) {
      if ((s = dalloc(&P->G, p * n * e)) != DQ_OK) return fail(s);
      P->own_G = true;
      if ((s = upload(P, P->G, d->G, p * n, DQ_HOST)) != DQ_OK) return fail(s);
    }
  }
  if (p) {
    if ((s = dalloc(&P->GT, p * n * e)) != DQ_OK) return fail(s);
    dim3 blk(32, 8), grd((unsigned)((n + 31) / 32), (unsigned)((p + 31) / 32));
    if (e == 8)
      k_transpose<double><<<grd, blk, 0, ctx->stream>>>((const double*)P->G, (double*)P->GT, (int)p, (int)n);
    else
      k_transpose<float><<<grd, blk, 0, ctx->stream>>>((const float*)P->G, (float*)P->GT, (int)p, (int)n);
    ++ctx->launches;
    if (cudaGetLastError() != cudaSuccess) {
      set_error("transpose launch failed");
      return fail(DQ_ERR_CUDA);
    }
  }
  if ((s = dalloc(&P->q, B * n * e)) != DQ_OK) return fail(s);
  if ((s = upload(P, P->q, d->q, B * n, d->memory)) != DQ_OK) return fail(s);
  if ((s = dalloc(&P->g, std::max<size_t>(B * p, 1) * e)) != DQ_OK) return fail(s);
  if (p && (s = upload(P, P->g, d->g, B * p, d->memory)) != DQ_OK) return fail(s);
  if ((s = dalloc(&P->lb, n * e)) != DQ_OK) return fail(s);
  if ((s = upload(P, P->lb, d->lb, n, d->memory)) != DQ_OK) return fail(s);
  if ((s = dalloc(&P->ub, n * e)) != DQ_OK) return fail(s);
  if ((s = upload(P, P->ub, d->ub, n, d->memory)) != DQ_OK) return fail(s);
  if ((s = dalloc(&P->x_state, B * n * e)) != DQ_OK) return fail(s);
  if ((s = dalloc(&P->lam_state, std::max<size_t>(B * p, 1) * e)) != DQ_OK) return fail(s);
  cudaError_t ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) {
    set_error("problem upload: %s", cudaGetErrorString(ce));
    return fail(DQ_ERR_CUDA);
  }
  *out = P;
  return DQ_OK;
}

dq_status dq_problem_set_vectors(dq_problem* P, const void* q, const void* g, int32_t memory) {
  if (!P) {
    set_error("NULL problem");
    return DQ_ERR_INVALID;
  }
  if (memory != DQ_HOST && memory != DQ_DEVICE) {
    set_error("unknown memory kind %d", memory);
    return DQ_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(P->mu);
  const size_t B = P->batch;
  if (memory == DQ_HOST) {
    if ((q && !host_all_finite((const double*)q, B * P->n)) ||
        (g && P->p && !host_all_finite((const double*)g, B * P->p))) {
      set_error("non-finite value in q or g");
      return DQ_ERR_INVALID;
    }
  }
  dq_status s;
  if (q && (s = upload(P, P->q, q, B * P->n, memory)) != DQ_OK) return s;
  if (g && P->p && (s = upload(P, P->g, g, B * P->p, memory)) != DQ_OK) return s;
  DQ_CK(cudaStreamSynchronize(P->ctx->stream));
  return DQ_OK;
}

dq_status dq_problem_constants(dq_problem* P, double* lmax_Q, double* lmin_Q, double* normG2) {
  if (!P) {
    set_error("NULL problem");
    return DQ_ERR_INVALID;
  }
  if (isnan(P->lmax_Q) || isnan(P->normG2)) {
    dq_status s = grid_constants(P);
    if (s != DQ_OK) return s;
  }
  if (lmax_Q) *lmax_Q = P->lmax_Q;
  if (lmin_Q) *lmin_Q = P->lmin_Q;
  if (normG2) *normG2 = P->normG2;
  return DQ_OK;
}

dq_status dq_problem_destroy(dq_problem* P) {
  if (!P) return DQ_OK;
  cudaStreamSynchronize(P->ctx->stream);
  if (P->own_Q && P->Q) cudaFree(P->Q);
  if (P->own_G && P->G) cudaFree(P->G);
  void* bufs[] = {P->GT, P->q, P->g, P->lb, P->ub, P->x_state, P->lam_state};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (P->gws) grid_free(P->gws);
  if (P->tws) tc_free(P->tws);
  dq_context* ctx = P->ctx;
  delete P;
  if (--ctx->live_problems == 0 && ctx->destroy_requested) context_free(ctx);
  return DQ_OK;
}

dq_status dq_solve(dq_problem* P, const dq_solve_opts* o, const dq_outputs* out, dq_result* results) {
  if (!P || !results) {
    set_error("NULL argument");
    return DQ_ERR_INVALID;
  }
  SolveCfg c;
  dq_status s = resolve_opts(P, o, &c);
  if (s != DQ_OK) return s;
  if (out && out->memory != DQ_HOST && out->memory != DQ_DEVICE) {
    set_error("unknown output memory kind %d", out->memory);
    return DQ_ERR_INVALID;
  }
  DQ_CK(cudaSetDevice(P->ctx->device));
  int engine = c.engine;
  if (engine == DQ_ENGINE_AUTO) {
    if (P->prec == DQ_BF16X3) engine = DQ_ENGINE_TC;
    else if (P->batch == 1 && P->n > 1024) engine = DQ_ENGINE_GRID;
    else engine = DQ_ENGINE_CTA;
  }
  if (P->prec == DQ_BF16X3 && engine != DQ_ENGINE_TC) {
    set_error("DQ_BF16X3 problems run on the tensor-core engine");
    return DQ_ERR_INVALID;
  }
  if (engine == DQ_ENGINE_TC) {
    if (P->prec != DQ_BF16X3) {
      set_error("the tensor-core engine needs a DQ_BF16X3 problem");
      return DQ_ERR_INVALID;
    }
    return tc_solve(P, c, out, results);
  }
  if (engine == DQ_ENGINE_GRID) {
    if (P->batch != 1) {
      set_error("the grid engine solves one instance (batch == 1)");
      return DQ_ERR_INVALID;
    }
    return grid_solve(P, c, out, results);
  }
  if (engine != DQ_ENGINE_CTA) {
    set_error("unknown engine %d", engine);
    return DQ_ERR_INVALID;
  }
  dq_problem* const probs[1] = {P};
  return cta_solve_problems(probs, 1, &c, out, results, 0, 256, false);
}

dq_status dq_solve_many(dq_problem* const* probs, int32_t count, const dq_solve_opts* opts,
                        const dq_outputs* outs, dq_result* results) {
  if (!probs || !opts || !results || count < 0) {
    set_error("NULL argument or negative count");
    return DQ_ERR_INVALID;
  }
  if (count == 0) return DQ_OK;
  std::vector<SolveCfg> cfgs(count);
  int prec = -1;
  dq_context* ctx = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!probs[i]) {
      set_error("problem %d is NULL", i);
      return DQ_ERR_INVALID;
    }
    if (prec < 0) {
      prec = probs[i]->prec;
      ctx = probs[i]->ctx;
    }
    if (probs[i]->prec != prec || probs[i]->ctx != ctx || probs[i]->prec == DQ_BF16X3) {
      set_error("dq_solve_many needs FP64 or FP32 problems of one precision and one context");
      return DQ_ERR_INVALID;
    }
    dq_status s = resolve_opts(probs[i], &opts[i], &cfgs[i]);
    if (s != DQ_OK) return s;
  }
  DQ_CK(cudaSetDevice(ctx->device));
  int threads = 256, smem_cap = 0;
  auto it = ctx->tuned.find(cta_signature(probs, count));
  if (it != ctx->tuned.end()) {
    threads = it->second.first;
    smem_cap = it->second.second;
  }
  return cta_solve_problems(probs, count, cfgs.data(), outs, results, smem_cap, threads, true);
}

}  // extern "C"
