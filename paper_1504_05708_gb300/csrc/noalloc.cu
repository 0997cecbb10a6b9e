// noalloc.cu -- dq_solve_noalloc: one QP solve that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a
// real-time control loop (for instance a model-predictive controller that
// solves one QP per sampling period) whose timing must not depend on the
// allocator, or an application whose memory pool has reserved the whole GPU
// up front so that an extra cudaMalloc would fail.  For them this entry point
// runs the CTA engine's whole-solve kernel on caller-provided device arrays and
// keeps its own scratch -- the instance descriptor, the work-queue counter,
// the result record, the constants and the transposed copy of G -- in one
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.  It calls no cudaMalloc, cudaFree or
// allocating library routine.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "cta_engine.cuh"
#include "dq_host.h"

namespace dq {

// Fixed scratch: 8 MiB per device.
static constexpr size_t kNoAllocBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Layout inside the scratch (offsets in bytes).
static constexpr size_t kOffInst = 0;        // CtaInst<T> (< 1 KiB)
static constexpr size_t kOffCounter = 1024;  // work-queue counter (int)
static constexpr size_t kOffResult = 1280;   // DevResult
static constexpr size_t kOffConsts = 1536;   // 6 doubles
static constexpr size_t kOffGT = 4096;       // G' (n x p elements)
static_assert(sizeof(CtaInst<double>) <= kOffCounter - kOffInst && sizeof(CtaInst<float>) <= kOffCounter - kOffInst,
              "the instance descriptor overlaps the work-queue counter");
static_assert(sizeof(int) <= kOffResult - kOffCounter, "the counter overlaps the result");
static_assert(sizeof(DevResult) <= kOffConsts - kOffResult, "the result overlaps the constants");
static_assert(6 * sizeof(double) <= kOffGT - kOffConsts, "the constants overlap G'");

// Host-side device address of the scratch, looked up once per device.
static constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

static dq_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("dq_solve_noalloc: device %d out of range", device);
    return DQ_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error("dq_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return DQ_ERR_CUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = (unsigned char*)g_scratch_addr[device];
  return DQ_OK;
}

template <typename T>
__global__ void k_noalloc_transpose(const T* __restrict__ in, T* __restrict__ out, int rows, int cols) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = bx + k, c = by + threadIdx.x;
    if (r < cols && c < rows) out[(size_t)r * rows + c] = tile[threadIdx.x][k];
  }
}

template <typename T>
static dq_status run_noalloc(int device, const dq_problem_desc* d, const SolveCfg& c, const dq_outputs* out,
                             dq_result* result, cudaStream_t st) {
  unsigned char* base = nullptr;
  dq_status s = scratch_address(device, &base);
  if (s != DQ_OK) return s;
  const size_t n = d->n, p = d->p;
  if (kOffGT + n * p * sizeof(T) > kNoAllocBytes) {
    set_error("dq_solve_noalloc: n * p = %zu elements of G' exceed the fixed scratch (%zu elements of %zu bytes)",
              n * p, (kNoAllocBytes - kOffGT) / sizeof(T), sizeof(T));
    return DQ_ERR_INVALID;
  }
  int optin = 0;
  DQ_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  const size_t dmax = max_dynamic_smem((const void*)cta_solve_kernel<T, 256>, (size_t)optin);
  if (cta_vec_bytes<T>(d->n, d->p) > dmax) {
    set_error("dq_solve_noalloc: the instance needs more shared memory than one thread block has");
    return DQ_ERR_INVALID;
  }
  CtaInst<T>* d_inst = (CtaInst<T>*)(base + kOffInst);
  int* d_cnt = (int*)(base + kOffCounter);
  DevResult* d_res = (DevResult*)(base + kOffResult);
  double* d_con = (double*)(base + kOffConsts);
  T* d_GT = (T*)(base + kOffGT);
  if (p > 0) {
    dim3 blk(32, 8), grd((unsigned)((n + 31) / 32), (unsigned)((p + 31) / 32));
    k_noalloc_transpose<T><<<grd, blk, 0, st>>>((const T*)d->G, d_GT, (int)p, (int)n);
    DQ_CK(cudaGetLastError());
  }
  CtaInst<T> I;
  memset(&I, 0, sizeof(I));
  I.n = d->n;
  I.p = d->p;
  I.cone = d->cone;
  I.alg = c.alg;
  I.Q = (const T*)d->Q;
  I.G = (const T*)d->G;
  I.GT = d_GT;
  I.q = (const T*)d->q;
  I.g = (const T*)d->g;
  I.lb = (const T*)d->lb;
  I.ub = (const T*)d->ub;
  I.lmax_Q = d->lmax_Q;
  I.lmin_Q = d->lmin_Q;
  I.normG2 = d->normG2;
  I.lip_bound = d->lipschitz == DQ_LIP_BOUND;
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
  I.kd_plus = !(c.kd_literal && !(d->lmin_Q > 0.0));
  I.x_last = out ? (T*)out->x_last : nullptr;
  I.x_avg = out ? (T*)out->x_avg : nullptr;
  I.lam_out = out ? (T*)out->lambda : nullptr;
  I.res = d_res;
  I.consts_out = d_con;
  // the descriptor and a zero work-queue counter; the result and constants are overwritten
  DQ_CK(cudaMemcpyAsync(d_inst, &I, sizeof(I), cudaMemcpyHostToDevice, st));
  DQ_CK(cudaMemsetAsync(d_cnt, 0, sizeof(int), st));
  const size_t want = cta_vec_bytes<T>(d->n, d->p) + cta_mat_bytes<T>(d->n, d->p);
  const size_t smem = std::max(cta_vec_bytes<T>(d->n, d->p), std::min<size_t>(want, dmax));
  DQ_CK(cudaFuncSetAttribute(cta_solve_kernel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cta_solve_kernel<T, 256><<<1, 256, smem, st>>>(d_inst, nullptr, 1, d_cnt, smem);
  DQ_CK(cudaGetLastError());
  DevResult hr;
  double hc[6];
  DQ_CK(cudaMemcpyAsync(&hr, d_res, sizeof(hr), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaMemcpyAsync(hc, d_con, sizeof(hc), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaStreamSynchronize(st));
  fill_result(result, hr, hc, c);
  if (hr.status == DQ_ERR_INVALID) set_error("dq_solve_noalloc: invalid constants (DGM/DFGM need lmin_Q > 0)");
  return (dq_status)hr.status;
}

}  // namespace dq

using namespace dq;

extern "C" dq_status dq_solve_noalloc(int device, const dq_problem_desc* desc, const dq_solve_opts* opts,
                                      const dq_outputs* out, dq_result* result, void* cuda_stream) {
  if (!desc || !opts || !result) {
    set_error("dq_solve_noalloc: NULL argument");
    return DQ_ERR_INVALID;
  }
  if (desc->memory != DQ_DEVICE || desc->batch != 1 || (desc->prec != DQ_FP64 && desc->prec != DQ_FP32) ||
      desc->n < 1 || desc->p < 0 || (out && out->memory != DQ_DEVICE) ||
      (desc->cone != DQ_CONE_INEQ && desc->cone != DQ_CONE_EQ) ||
      (desc->lipschitz != DQ_LIP_LANCZOS && desc->lipschitz != DQ_LIP_BOUND)) {
    set_error("dq_solve_noalloc: needs one FP64 or FP32 instance (batch 1) in device memory and device outputs");
    return DQ_ERR_INVALID;
  }
  if (!desc->Q || !desc->q || !desc->lb || !desc->ub || (desc->p > 0 && (!desc->G || !desc->g))) {
    set_error("dq_solve_noalloc: NULL problem array");
    return DQ_ERR_INVALID;
  }
  if (!isnan(desc->lmin_Q) && desc->lmin_Q < 0) {
    set_error("dq_solve_noalloc: lmin_Q must be a lower bound >= 0");
    return DQ_ERR_INVALID;
  }
  SolveCfg c;
  dq_status s = resolve_opts(nullptr, opts, &c);
  if (s != DQ_OK) return s;
  DQ_CK(cudaSetDevice(device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (desc->prec == DQ_FP64) return run_noalloc<double>(device, desc, c, out, result, st);
  return run_noalloc<float>(device, desc, c, out, result, st);
}
