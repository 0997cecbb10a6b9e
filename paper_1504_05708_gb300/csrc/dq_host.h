// dq_host.h -- host-side handle definitions shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "duquad.h"
#include "dq_common.cuh"

namespace dq {

void set_error(const char* fmt, ...);

// On failure: record the message, clear the runtime's last-error state (so a
// later cudaGetLastError check does not report this failure again) and return.
#define DQ_CK(call)                                                             \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      cudaGetLastError();                                                       \
      ::dq::set_error("%s failed: %s", #call, cudaGetErrorString(e_));          \
      return DQ_ERR_CUDA;                                                       \
    }                                                                           \
  } while (0)

// Largest dynamic shared memory a kernel can request: the per-block opt-in
// limit minus the kernel's static shared memory.
size_t max_dynamic_smem(const void* kernel, size_t optin);

struct GridWs;   // large-instance engine workspace (grid_engine.cu)
struct TcWs;     // tensor-core batch workspace (tc_engine.cu)
struct ServeState;

// Validation results of the problem-data checks on the device (dq_problem_create).
struct CheckFlags {
  int nonfinite;        // a NaN or Inf in Q, q, G, g, lb or ub
  int bad_box;          // lb_i > ub_i somewhere
  int asym;             // a pair |Q_ij - Q_ji| > tol sqrt(|Q_ii Q_jj|)
  int asym_i, asym_j;   // one such pair
};

// Resolved solve options (defaults applied; NaN kept where the device derives).
struct SolveCfg {
  int alg, output, inner_stop, engine;
  double eps_out, eps_in, rho;
  int fixed_outer, fixed_inner, max_outer, max_inner, check_every, inner_check_every;
  int warm_start, kd_literal, fresh;
  int inner_cert;  // dq_inner_cert
  double Ld, LL, sigma;
  int stop_fstar;  // outer stop on |F - f_star| (Sec. 6 experiments) instead of the certificate
  double f_star;
};

}  // namespace dq

struct dq_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  size_t smem_optin = 0;
  // grow-only scratch for per-call device arrays
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  dq::ServeState* serve = nullptr;
  // measurement
  int64_t launches = 0;
  bool profile = false;
  int64_t gemv_launches = 0;
  double gemv_ms = 0.0, gemv_bytes = 0.0;
  int64_t reduce_launches = 0;
  double reduce_ms = 0.0;
  // pinned staging and the captured graph of the last persistent launch
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec = nullptr;
  uint64_t gkey = 0;
  // autotuned CTA-engine configurations: size-histogram signature -> (threads, smem cap)
  std::map<std::string, std::pair<int, int>> tuned;
  // host -> device upload: a grow-only device staging buffer (two halves that
  // alternate), a copy stream that overlaps the copies with the conversion
  // kernels on `stream`, and the validation flags the device kernels set
  void* stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t cstream = nullptr;
  cudaEvent_t cev[4] = {nullptr, nullptr, nullptr, nullptr};
  int* dflags = nullptr;   // device dq::CheckFlags
  int* hflags = nullptr;   // pinned mirror
  // lifetime: problems keep their context alive; a destroy requested while
  // problems exist is carried out when the last one is destroyed
  int live_problems = 0;
  bool destroy_requested = false;
};

struct dq_problem {
  dq_context* ctx = nullptr;
  int n = 0, p = 0, batch = 1, cone = 0, prec = 0;
  size_t esz = 8;                  // element size of the device arrays
  void *Q = nullptr, *G = nullptr, *GT = nullptr;
  bool own_Q = false, own_G = false;
  void *q = nullptr, *g = nullptr, *lb = nullptr, *ub = nullptr;
  void *x_state = nullptr, *lam_state = nullptr;
  bool has_state = false;
  double lmax_Q = NAN, lmin_Q = NAN, normG2 = NAN;
  double lmax_given = NAN, normG2_given = NAN;  // as passed in dq_problem_desc
  int lip_bound = 0;                            // dq_problem_desc.lipschitz == DQ_LIP_BOUND
  // sparse (CSR) problems: Q, G, GT above hold the value arrays; row offsets
  // and column indices here (int32, device); solved by the grid engine only
  bool sparse = false;
  int *q_rp = nullptr, *q_ci = nullptr, *g_rp = nullptr, *g_ci = nullptr, *gt_rp = nullptr, *gt_ci = nullptr;
  long long nnzQ = 0, nnzG = 0;
  dq::GridWs* gws = nullptr;
  dq::TcWs* tws = nullptr;
  std::mutex mu;
};

namespace dq {
dq_status resolve_opts(const dq_problem* prob, const dq_solve_opts* o, SolveCfg* c);
dq_status ctx_scratch(dq_context* ctx, size_t bytes, void** out);
dq_status grid_solve(dq_problem* prob, const SolveCfg& c, const dq_outputs* out, dq_result* res);
void grid_free(GridWs* w);
dq_status grid_constants(dq_problem* prob);
dq_status tc_solve(dq_problem* prob, const SolveCfg& c, const dq_outputs* out, dq_result* res);
void tc_free(TcWs* w);
dq_status cta_solve_problems(dq_problem* const* probs, int count, const SolveCfg* cfgs,
                             const dq_outputs* outs, dq_result* results, int smem_cap,
                             int threads, bool graph);
std::string cta_signature(dq_problem* const* probs, int count);
void fill_result(dq_result* r, const DevResult& d, const double* consts, const SolveCfg& c);
}  // namespace dq
