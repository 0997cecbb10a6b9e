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

// Transposed copy of G (p x n -> n x p); flags non-finite entries of G.
template <typename T>
__global__ void k_transpose(const T* __restrict__ in, T* __restrict__ out, int rows, int cols, CheckFlags* f) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  bool bad = false;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) {
      const T v = in[(size_t)r * cols + c];
      bad |= !isfinite(v);
      tile[k][threadIdx.x] = v;
    }
  }
  if (bad) atomicOr(&f->nonfinite, 1);
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = bx + k, c = by + threadIdx.x;  // out is cols x rows
    if (r < cols && c < rows) out[(size_t)r * rows + c] = tile[threadIdx.x][k];
  }
}

// FP64 -> FP32 conversion of an uploaded chunk; flags non-finite values.
__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, size_t m, CheckFlags* f) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    bad |= !isfinite(v);
    out[i] = float(v);
  }
  if (bad) atomicOr(&f->nonfinite, 1);
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ a, size_t m, CheckFlags* f) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(a[i]);
  if (bad) atomicOr(&f->nonfinite, 1);
}

template <typename T>
__global__ void k_check_box(const T* __restrict__ lb, const T* __restrict__ ub, int n, CheckFlags* f) {
  bool bad = false, inv = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bad |= !isfinite(lb[i]) || !isfinite(ub[i]);
    inv |= !(lb[i] <= ub[i]);
  }
  if (bad) atomicOr(&f->nonfinite, 1);
  if (inv) atomicOr(&f->bad_box, 1);
}

// Symmetry and finiteness of Q (n x n row-major): block (I, J), J >= I, of
// 32 x 32 tiles compares Q[I, J] with Q[J, I]' through shared memory (both
// reads coalesced); a pair fails when |Q_ij - Q_ji| > tol sqrt(|Q_ii Q_jj|)
// (rounding of a symmetric Q computed as a product scales with its rows'
// norms, which sqrt(Q_ii Q_jj) is for a PSD Q).  One failing pair is kept.
template <typename T>
__global__ void k_check_sym(const T* __restrict__ Q, int n, double tol, CheckFlags* f) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (J < I) return;
  __shared__ T tb[32][33];
  const int i0 = I * 32, j0 = J * 32;
  bool bad = false;
  for (int k = threadIdx.y; k < 32; k += 8) {  // tb[k][c] = Q[j0 + k][i0 + c]
    const int r = j0 + k, c = i0 + threadIdx.x;
    if (r < n && c < n) {
      const T v = Q[(size_t)r * n + c];
      tb[k][threadIdx.x] = v;
      bad |= !isfinite(v);
    }
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {  // a = Q[i0 + k][j0 + c], b = Q[j0 + c][i0 + k]
    const int i = i0 + k, j = j0 + threadIdx.x;
    if (i < n && j < n) {
      const T a = Q[(size_t)i * n + j];
      const T b = tb[threadIdx.x][k];
      if (I != J) bad |= !isfinite(a);
      const double lim = tol * sqrt(fabs(double(Q[(size_t)i * n + i])) * fabs(double(Q[(size_t)j * n + j])));
      if (!(fabs(double(a) - double(b)) <= lim) && isfinite(a) && isfinite(b)) {
        if (atomicCAS(&f->asym, 0, 1) == 0) {
          f->asym_i = i;
          f->asym_j = j;
        }
      }
    }
  }
  if (bad) atomicOr(&f->nonfinite, 1);
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

// Upload resources of the context: staging halves of kStageChunk doubles, the
// copy stream, its events and the validation flags (created on first use).
static constexpr size_t kStageChunk = size_t(4) << 20;  // 32 MiB of doubles per half

// Symmetry tolerance of Q relative to sqrt(|Q_ii Q_jj|): rounding of the
// stored type (a symmetric FP64 Q rounds to a symmetric or one-ulp-apart
// FP32 pair) plus the rounding of a Q formed as a product in FP64.
static constexpr double kSymTol32 = 1e-6, kSymTol64 = 1e-10;

static dq_status upload_setup(dq_context* ctx, bool stage) {
  if (!ctx->dflags) {
    if (cudaMalloc(&ctx->dflags, sizeof(CheckFlags)) != cudaSuccess ||
        cudaMallocHost(&ctx->hflags, sizeof(CheckFlags)) != cudaSuccess) {
      cudaGetLastError();
      set_error("validation flag allocation failed");
      return DQ_ERR_NOMEM;
    }
  }
  if (stage && !ctx->stage) {
    if (cudaMalloc(&ctx->stage, 2 * kStageChunk * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      ctx->stage = nullptr;
      set_error("upload staging allocation failed");
      return DQ_ERR_NOMEM;
    }
    ctx->stage_bytes = 2 * kStageChunk * sizeof(double);
    DQ_CK(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ctx->cev) DQ_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  return DQ_OK;
}

// Copy `m` elements into device array `dst` of the problem's element type.
// src: host double (memory = DQ_HOST) or device array of the element type.
// Values are checked for finiteness on the device (flags in ctx->dflags).
// Host doubles for a float problem go through the context's staging halves
// in chunks: the copy of chunk k (copy stream) overlaps the conversion of
// chunk k - 1 (the context's stream); everything is ordered on the context's
// stream when this returns (no host synchronisation here).
static dq_status upload(dq_problem* P, void* dst, const void* src, size_t m, int memory) {
  dq_context* ctx = P->ctx;
  cudaStream_t st = ctx->stream;
  if (m == 0) return DQ_OK;
  CheckFlags* fl = (CheckFlags*)ctx->dflags;
  const unsigned grid = (unsigned)std::min<size_t>((m + 255) / 256, 2048);
  if (memory == DQ_DEVICE || P->esz == 8) {
    DQ_CK(cudaMemcpyAsync(dst, src, m * P->esz,
                          memory == DQ_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (P->esz == 8) k_check_finite<double><<<grid, 256, 0, st>>>((const double*)dst, m, fl);
    else k_check_finite<float><<<grid, 256, 0, st>>>((const float*)dst, m, fl);
    ++ctx->launches;
    DQ_CK(cudaGetLastError());
    return DQ_OK;
  }
  dq_status s = upload_setup(ctx, true);
  if (s != DQ_OK) return s;
  double* half[2] = {(double*)ctx->stage, (double*)ctx->stage + kStageChunk};
  cudaEvent_t* copied = ctx->cev;      // [0], [1]
  cudaEvent_t* freed = ctx->cev + 2;   // [2], [3]
  // the halves are free once earlier work on the context's stream is done
  DQ_CK(cudaEventRecord(freed[0], st));
  DQ_CK(cudaEventRecord(freed[1], st));
  for (size_t off = 0, k = 0; off < m; off += kStageChunk, ++k) {
    const size_t cnt = std::min(kStageChunk, m - off);
    const int b = (int)(k & 1);
    DQ_CK(cudaStreamWaitEvent(ctx->cstream, freed[b], 0));
    DQ_CK(cudaMemcpyAsync(half[b], (const double*)src + off, cnt * 8, cudaMemcpyHostToDevice, ctx->cstream));
    DQ_CK(cudaEventRecord(copied[b], ctx->cstream));
    DQ_CK(cudaStreamWaitEvent(st, copied[b], 0));
    k_d2f<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 4096), 256, 0, st>>>(half[b], (float*)dst + off, cnt, fl);
    ++ctx->launches;
    DQ_CK(cudaGetLastError());
    DQ_CK(cudaEventRecord(freed[b], st));
  }
  return DQ_OK;
}

// Clear the validation flags (before a create / set_vectors).
static dq_status flags_clear(dq_context* ctx) {
  dq_status s = upload_setup(ctx, false);
  if (s != DQ_OK) return s;
  DQ_CK(cudaMemsetAsync(ctx->dflags, 0, sizeof(CheckFlags), ctx->stream));
  return DQ_OK;
}

// Read the validation flags (synchronises the context's stream).
static dq_status flags_check(dq_context* ctx) {
  DQ_CK(cudaMemcpyAsync(ctx->hflags, ctx->dflags, sizeof(CheckFlags), cudaMemcpyDeviceToHost, ctx->stream));
  DQ_CK(cudaStreamSynchronize(ctx->stream));
  const CheckFlags& f = *(const CheckFlags*)ctx->hflags;
  if (f.nonfinite) {
    set_error("non-finite value in the problem data");
    return DQ_ERR_INVALID;
  }
  if (f.bad_box) {
    set_error("lb > ub for some coordinate");
    return DQ_ERR_INVALID;
  }
  if (f.asym) {
    set_error("Q is not symmetric: |Q[%d][%d] - Q[%d][%d]| exceeds the tolerance", f.asym_i, f.asym_j, f.asym_j,
              f.asym_i);
    return DQ_ERR_INVALID;
  }
  return DQ_OK;
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
  c->stop_fstar = o->stop_fstar != 0;
  c->f_star = o->f_star;
  if (c->stop_fstar && !std::isfinite(c->f_star)) {
    set_error("stop_fstar needs a finite f_star");
    return DQ_ERR_INVALID;
  }
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
  if (ctx->cstream) {
    cudaStreamSynchronize(ctx->cstream);
    cudaStreamDestroy(ctx->cstream);
  }
  for (cudaEvent_t e : ctx->cev)
    if (e) cudaEventDestroy(e);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->dflags) cudaFree(ctx->dflags);
  if (ctx->hflags) cudaFreeHost(ctx->hflags);
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
  if (d->lipschitz != DQ_LIP_LANCZOS && d->lipschitz != DQ_LIP_BOUND) {
    set_error("unknown lipschitz mode %d", d->lipschitz);
    return DQ_ERR_INVALID;
  }
  if (!d->Q || !d->q || !d->lb || !d->ub || (d->p > 0 && (!d->G || !d->g))) {
    set_error("NULL problem array");
    return DQ_ERR_INVALID;
  }
  const size_t n = d->n, p = d->p, B = d->batch;
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
  P->lip_bound = d->lipschitz == DQ_LIP_BOUND;
  dq_status s = DQ_OK;
  auto fail = [&](dq_status st) {
    dq_problem_destroy(P);
    return st;
  };
  if ((s = flags_clear(ctx)) != DQ_OK) return fail(s);
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
      k_transpose<double><<<grd, blk, 0, ctx->stream>>>((const double*)P->G, (double*)P->GT, (int)p, (int)n,
                                                         (CheckFlags*)ctx->dflags);
    else
      k_transpose<float><<<grd, blk, 0, ctx->stream>>>((const float*)P->G, (float*)P->GT, (int)p, (int)n,
                                                        (CheckFlags*)ctx->dflags);
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
  {  // lb <= ub and the symmetry of Q on the device (finiteness: checked by the copies above)
    CheckFlags* fl = (CheckFlags*)ctx->dflags;
    const unsigned gb = (unsigned)std::min<size_t>((n + 255) / 256, 1024);
    const dim3 blk(32, 8), grd((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    if (e == 8) {
      k_check_box<double><<<gb, 256, 0, ctx->stream>>>((const double*)P->lb, (const double*)P->ub, (int)n, fl);
      k_check_sym<double><<<grd, blk, 0, ctx->stream>>>((const double*)P->Q, (int)n, kSymTol64, fl);
    } else {
      k_check_box<float><<<gb, 256, 0, ctx->stream>>>((const float*)P->lb, (const float*)P->ub, (int)n, fl);
      k_check_sym<float><<<grd, blk, 0, ctx->stream>>>((const float*)P->Q, (int)n, kSymTol32, fl);
    }
    ctx->launches += 2;
    if (cudaGetLastError() != cudaSuccess) {
      set_error("validation launch failed");
      return fail(DQ_ERR_CUDA);
    }
  }
  cudaError_t ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) {
    set_error("problem upload: %s", cudaGetErrorString(ce));
    return fail(DQ_ERR_CUDA);
  }
  if ((s = flags_check(ctx)) != DQ_OK) return fail(s);
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
  dq_context* ctx = P->ctx;
  const size_t B = P->batch, bq = q ? B * P->n : 0, bg = (g && P->p) ? B * P->p : 0;
  // new vectors land in the context's scratch first and replace the handle's
  // only once they passed the finiteness check
  void* tmp = nullptr;
  dq_status s = ctx_scratch(ctx, (bq + bg) * P->esz + 256, &tmp);
  if (s != DQ_OK) return s;
  char* tq = (char*)tmp;
  char* tg = tq + ((bq * P->esz + 255) & ~size_t(255));
  if ((s = flags_clear(ctx)) != DQ_OK) return s;
  if (bq && (s = upload(P, tq, q, bq, memory)) != DQ_OK) return s;
  if (bg && (s = upload(P, tg, g, bg, memory)) != DQ_OK) return s;
  if ((s = flags_check(ctx)) != DQ_OK) return s;
  if (bq) DQ_CK(cudaMemcpyAsync(P->q, tq, bq * P->esz, cudaMemcpyDeviceToDevice, ctx->stream));
  if (bg) DQ_CK(cudaMemcpyAsync(P->g, tg, bg * P->esz, cudaMemcpyDeviceToDevice, ctx->stream));
  DQ_CK(cudaStreamSynchronize(ctx->stream));
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
  void* bufs[] = {P->GT, P->q, P->g, P->lb, P->ub, P->x_state, P->lam_state,
                  P->q_rp, P->q_ci, P->g_rp, P->g_ci, P->gt_rp, P->gt_ci};
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
  if (P->sparse) {  // CSR problems run on the grid engine's sparse products
    if (engine != DQ_ENGINE_AUTO && engine != DQ_ENGINE_GRID) {
      set_error("sparse (CSR) problems run on the grid engine");
      return DQ_ERR_INVALID;
    }
    return grid_solve(P, c, out, results);
  }
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

static dq_solve_opts default_opts(int alg) {
  dq_solve_opts o;
  memset(&o, 0, sizeof(o));
  o.alg = alg;
  o.output = DQ_OUT_BOTH;
  o.eps_out = 1e-3;
  o.eps_in = NAN;
  o.rho = NAN;
  o.Ld = o.LL = o.sigma = NAN;
  return o;
}

dq_status dq_solve_theory(dq_problem* P, const dq_theory_solve_opts* t, const dq_outputs* out, dq_result* result,
                          dq_theory_out* counts, double* Rd_used) {
  if (!P || !t || !result) {
    set_error("NULL argument");
    return DQ_ERR_INVALID;
  }
  if (P->batch != 1 || P->prec == DQ_BF16X3) {
    set_error("dq_solve_theory: one FP64 or FP32 instance (batch 1)");
    return DQ_ERR_INVALID;
  }
  if (!(std::isfinite(t->eps) && t->eps > 0.0) || t->alg < DQ_DGM || t->alg > DQ_ADFGM ||
      !(std::isnan(t->Rd) || (std::isfinite(t->Rd) && t->Rd > 0.0)) ||
      !(std::isnan(t->safety) || (std::isfinite(t->safety) && t->safety > 0.0)) || t->max_total < 0) {
    set_error("dq_solve_theory: invalid algorithm, eps, R_d, safety or max_total");
    return DQ_ERR_INVALID;
  }
  DQ_CK(cudaSetDevice(P->ctx->device));
  const size_t n = P->n, p = P->p;
  double Rd = t->Rd;
  dq_status s;
  if (std::isnan(Rd)) {  // R_d from the multipliers of a certified solve
    dq_solve_opts o = default_opts(t->alg);
    o.eps_out = t->eps;
    o.engine = t->engine;
    std::vector<double> lam(std::max<size_t>(p, 1));
    dq_outputs lo;
    memset(&lo, 0, sizeof(lo));
    lo.lambda = lam.data();
    lo.memory = DQ_HOST;
    dq_result r;
    s = dq_solve(P, &o, &lo, &r);
    if (s < 0) return s;
    double nl = 0.0;
    for (size_t j = 0; j < p; ++j) nl += lam[j] * lam[j];
    Rd = (std::isnan(t->safety) ? 2.0 : t->safety) * std::max(std::sqrt(nl), t->eps);
  }
  // D_U = ||ub - lb||_2 from the handle's device copies
  std::vector<double> lb(n), ub(n);
  if (P->esz == 8) {
    DQ_CK(cudaMemcpyAsync(lb.data(), P->lb, n * 8, cudaMemcpyDeviceToHost, P->ctx->stream));
    DQ_CK(cudaMemcpyAsync(ub.data(), P->ub, n * 8, cudaMemcpyDeviceToHost, P->ctx->stream));
    DQ_CK(cudaStreamSynchronize(P->ctx->stream));
  } else {
    std::vector<float> f(2 * n);
    DQ_CK(cudaMemcpyAsync(f.data(), P->lb, n * 4, cudaMemcpyDeviceToHost, P->ctx->stream));
    DQ_CK(cudaMemcpyAsync(f.data() + n, P->ub, n * 4, cudaMemcpyDeviceToHost, P->ctx->stream));
    DQ_CK(cudaStreamSynchronize(P->ctx->stream));
    for (size_t i = 0; i < n; ++i) {
      lb[i] = f[i];
      ub[i] = f[n + i];
    }
  }
  double D2 = 0.0;
  for (size_t i = 0; i < n; ++i) D2 += (ub[i] - lb[i]) * (ub[i] - lb[i]);
  dq_theory_in ti;
  ti.alg = t->alg;
  ti.eps = t->eps;
  ti.Rd = Rd;
  ti.D_U = std::sqrt(D2);
  ti.rho = t->rho;
  if ((s = dq_problem_constants(P, &ti.lmax_Q, &ti.lmin_Q, &ti.normG2)) != DQ_OK) return s;
  if (std::isnan(ti.lmin_Q)) ti.lmin_Q = 0.0;
  if (!(ti.D_U > 0.0)) ti.D_U = 1e-300;  // a box of one point: any count is enough
  dq_theory_out to;
  if ((s = dq_theory(&ti, &to)) != DQ_OK) return s;
  if (counts) *counts = to;
  if (Rd_used) *Rd_used = Rd;
  const int64_t cap = t->max_total > 0 ? t->max_total : 100000000LL;
  if (to.k_total > cap || to.k_out > INT32_MAX || to.k_in > INT32_MAX) {
    set_error("dq_solve_theory: k_out * k_in = %lld exceeds the cap %lld", (long long)to.k_total, (long long)cap);
    return DQ_ERR_INVALID;
  }
  dq_solve_opts o = default_opts(t->alg);
  o.inner_stop = DQ_INNER_FIXED;
  o.fixed_outer = (int32_t)to.k_out;
  o.fixed_inner = (int32_t)to.k_in;
  o.eps_out = t->eps;
  o.eps_in = to.eps_in;
  o.rho = to.rho;
  o.LL = to.LL;
  o.sigma = to.sigma;
  o.Ld = to.Ld;
  o.engine = t->engine;
  return dq_solve(P, &o, out, result);
}


}  // extern "C"
