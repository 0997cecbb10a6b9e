// serve.cu -- continuous-batching request loop (dq_serve_start / dq_submit /
// dq_poll / dq_serve_stop).
//
// A persistent grid of CTAs serves QP solve requests as they arrive: each CTA
// claims the next published request, runs the whole DFOM solve of that
// instance on-chip (the CTA engine), writes the outputs straight into
// host-mapped memory and claims the next one.  Requests of different n, p and
// algorithm overlap on the device; a request that arrives while others run is
// picked up by the first CTA that frees up.  Problem data (Q, G, G', box,
// warm-start lambda and x) stay resident on the device in their problem
// handles; a request carries only its new q and g.
//
// Host side: dq_submit validates and queues; a dispatcher thread admits
// queued requests into a ring of request entries while the device-memory
// footprint of the problems with requests in flight stays within the budget,
// publishes them (sequence numbers in host-mapped memory), collects finished
// entries and relaunches the request loop when it has gone idle.  Every
// device-side wait is bounded: an idle CTA exits after a timeout and the
// dispatcher relaunches the loop when work appears.
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <deque>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "cta_engine.cuh"
#include "dq_host.h"

namespace dq {

static constexpr int kSeqMap = 1 << 20;  // sequence -> entry map (power of two)

struct ServeShared {               // host-mapped control words
  volatile unsigned long long pub;  // number of published sequences
  volatile int stop;
  int pad;
  volatile int seq2entry[kSeqMap];
};

struct EntryIO {                   // host-mapped per-entry header
  CtaInst<float> inst;             // descriptor (device pointers)
  const float* q_stage;            // device view of the mapped q / g staging
  const float* g_stage;
  volatile unsigned long long done; // sequence + 1 when finished
};

__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(256) serve_kernel(EntryIO* ring, ServeShared* sh,
                                                    unsigned long long* claim, float* slot_q, float* slot_g,
                                                    int nmax, int pmax, size_t smem_bytes,
                                                    unsigned long long idle_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_seq;
  __shared__ int s_entry;
  __shared__ const float* s_hq;
  __shared__ const float* s_hg;
  __shared__ CtaInst<float> s_inst;
  unsigned long long t0 = gtimer_ns();
  for (;;) {
    if (threadIdx.x == 0) {
      long long got = -1;
      for (;;) {
        const unsigned long long pub = sh->pub;
        const unsigned long long c = *(volatile unsigned long long*)claim;
        if (c < pub) {
          if (atomicCAS(claim, c, c + 1) == c) {
            got = (long long)c;
            break;
          }
          continue;
        }
        if (sh->stop || gtimer_ns() - t0 > idle_ns) break;
        __nanosleep(1000);
      }
      s_seq = got;
      if (got >= 0) {
        __threadfence_system();
        const int e = sh->seq2entry[got & (kSeqMap - 1)];
        s_entry = e;
        s_inst = ring[e].inst;
        s_inst.q = slot_q + (size_t)e * nmax;
        s_inst.g = slot_g + (size_t)e * pmax;
        s_hq = ring[e].q_stage;
        s_hg = ring[e].g_stage;
      }
    }
    __syncthreads();
    const long long seq = s_seq;
    if (seq < 0) break;
    const int e = s_entry;
    // stage this request's q and g into device memory (read once over the host link)
    float* dq = slot_q + (size_t)e * nmax;
    float* dg = slot_g + (size_t)e * pmax;
    const float* hq = s_hq;
    const float* hg = s_hg;
    CtaInst<float> I = s_inst;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) dq[i] = hq[i];
    for (int j = threadIdx.x; j < I.p; j += blockDim.x) dg[j] = hg[j];
    __syncthreads();
    cta_solve<float>(I, smem, smem_bytes);
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) ring[e].done = (unsigned long long)seq + 1ull;
    __syncthreads();
    t0 = gtimer_ns();
  }
}

struct Ticket {
  dq_problem* prob = nullptr;
  int n = 0, p = 0;
  std::vector<float> q, g;         // request vectors (float)
  bool has_q = false, has_g = false;
  SolveCfg cfg;
  int entry = -1;
  unsigned long long seq = 0;
  bool done = false;
  DevResult res;
  double consts[6];
  std::vector<double> x_last, x_avg, lam;
};

struct ServeState {
  dq_context* ctx = nullptr;
  int R = 0, nmax = 0, pmax = 0;
  int64_t budget = 0, used = 0;
  size_t smem = 0;
  int grid = 0;
  ServeShared* sh_h = nullptr;
  ServeShared* sh_d = nullptr;
  EntryIO* io_h = nullptr;
  EntryIO* io_d = nullptr;
  float *qs_h = nullptr, *qs_d = nullptr, *gs_h = nullptr, *gs_d = nullptr;  // mapped staging
  float *out_h = nullptr, *out_d = nullptr;                                  // mapped outputs
  DevResult *res_h = nullptr, *res_d = nullptr;
  double *con_h = nullptr, *con_d = nullptr;
  unsigned long long* claim = nullptr;
  float *slot_q = nullptr, *slot_g = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t kdone = nullptr;
  bool kernel_live = false;
  std::mutex mu;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Ticket> tickets;
  std::vector<uint64_t> entry_ticket;  // 0 = free
  std::vector<int> free_entries;
  std::unordered_map<dq_problem*, int> inflight_per_prob;
  uint64_t next_ticket = 1;
  unsigned long long next_seq = 0;
  std::atomic<bool> running{false};
  std::thread worker;
  dq_status last_launch_error = DQ_OK;
};

static int64_t prob_bytes(const dq_problem* P) {
  const int64_t n = P->n, p = P->p, B = P->batch;
  return (int64_t)P->esz * (n * n + 2 * p * n + B * (2 * n + 2 * p) + 2 * n);
}

static size_t out_stride(const ServeState* S) { return 2 * (size_t)S->nmax + (size_t)std::max(S->pmax, 1); }

static void launch_loop(ServeState* S) {
  serve_kernel<<<S->grid, 256, S->smem, S->stream>>>(S->io_d, S->sh_d, S->claim, S->slot_q, S->slot_g, S->nmax,
                                                     std::max(S->pmax, 1), S->smem, 200000000ull /*0.2 s*/);
  ++S->ctx->launches;
  if (cudaGetLastError() != cudaSuccess) {
    S->last_launch_error = DQ_ERR_CUDA;
    return;
  }
  cudaEventRecord(S->kdone, S->stream);
  S->kernel_live = true;
}

// Fill entry e for ticket t (lock held).
static void fill_entry(ServeState* S, int e, Ticket& t) {
  EntryIO& io = S->io_h[e];
  dq_problem* P = t.prob;
  const SolveCfg& c = t.cfg;
  CtaInst<float>& I = io.inst;
  memset(&I, 0, sizeof(I));
  I.n = P->n;
  I.p = P->p;
  I.cone = P->cone;
  I.alg = c.alg;
  I.Q = (const float*)P->Q;
  I.G = (const float*)P->G;
  I.GT = (const float*)P->GT;
  I.q = nullptr;  // set on the device to the staged copy
  I.g = nullptr;
  I.lb = (const float*)P->lb;
  I.ub = (const float*)P->ub;
  I.lmax_Q = c.fresh ? P->lmax_given : P->lmax_Q;
  I.lmin_Q = P->lmin_Q;
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
  I.kd_plus = !(c.kd_literal && !(P->lmin_Q > 0.0));
  const bool warm = c.warm_start && P->has_state;
  I.x0 = warm ? (const float*)P->x_state : nullptr;
  I.lam0 = warm ? (const float*)P->lam_state : nullptr;
  I.x_state = (float*)P->x_state;
  I.lam_state = (float*)P->lam_state;
  float* od = S->out_d + (size_t)e * out_stride(S);
  I.x_last = od;
  I.x_avg = od + S->nmax;
  I.lam_out = od + 2 * S->nmax;
  I.res = S->res_d + e;
  I.consts_out = S->con_d + 6 * e;
  float* qh = S->qs_h + (size_t)e * S->nmax;
  float* gh = S->gs_h + (size_t)e * std::max(S->pmax, 1);
  const float* qsrc = t.has_q ? t.q.data() : nullptr;
  const float* gsrc = t.has_g ? t.g.data() : nullptr;
  if (qsrc) memcpy(qh, qsrc, sizeof(float) * P->n);
  if (gsrc) memcpy(gh, gsrc, sizeof(float) * P->p);
  io.q_stage = qsrc ? S->qs_d + (size_t)e * S->nmax : (const float*)P->q;
  io.g_stage = gsrc ? S->gs_d + (size_t)e * std::max(S->pmax, 1) : (const float*)P->g;
  io.done = 0;
  P->has_state = true;
}

static void collect(ServeState* S, int e) {
  const uint64_t tid = S->entry_ticket[e];
  auto it = S->tickets.find(tid);
  if (it != S->tickets.end()) {
    Ticket& t = it->second;
    const float* o = S->out_h + (size_t)e * out_stride(S);
    t.x_last.assign(o, o + t.n);
    t.x_avg.assign(o + S->nmax, o + S->nmax + t.n);
    t.lam.assign(o + 2 * S->nmax, o + 2 * S->nmax + t.p);
    t.res = S->res_h[e];
    memcpy(t.consts, S->con_h + 6 * e, sizeof(t.consts));
    t.done = true;
    dq_problem* P = t.prob;
    if (isnan(P->lmax_Q)) P->lmax_Q = t.consts[0];
    if (isnan(P->normG2)) P->normG2 = t.consts[1];
    if (--S->inflight_per_prob[P] == 0) {
      S->inflight_per_prob.erase(P);
      S->used -= prob_bytes(P);
    }
  }
  S->entry_ticket[e] = 0;
  S->free_entries.push_back(e);
}

static void worker_loop(ServeState* S) {
  cudaSetDevice(S->ctx->device);
  unsigned long long oldest_live = 0;
  while (S->running.load(std::memory_order_acquire)) {
    bool idle = true;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      // collect finished entries
      unsigned long long oldest = S->next_seq;
      for (int e = 0; e < S->R; ++e) {
        const uint64_t tid = S->entry_ticket[e];
        if (!tid) continue;
        const Ticket& t = S->tickets[tid];
        if (S->io_h[e].done == t.seq + 1) {
          std::atomic_thread_fence(std::memory_order_acquire);
          collect(S, e);
          idle = false;
        } else if (t.seq < oldest) {
          oldest = t.seq;
        }
      }
      oldest_live = oldest;
      // admit queued requests while entries and the footprint budget allow
      while (!S->pending.empty() && !S->free_entries.empty() &&
             S->next_seq - oldest_live < (unsigned long long)kSeqMap - 1) {
        const uint64_t tid = S->pending.front();
        Ticket& t = S->tickets[tid];
        const bool resident = S->inflight_per_prob.count(t.prob) > 0;
        const int64_t need = resident ? 0 : prob_bytes(t.prob);
        if (S->used + need > S->budget && !S->inflight_per_prob.empty()) break;  // wait for memory
        S->pending.pop_front();
        const int e = S->free_entries.back();
        S->free_entries.pop_back();
        fill_entry(S, e, t);
        S->used += need;
        S->inflight_per_prob[t.prob]++;
        t.entry = e;
        t.seq = S->next_seq++;
        S->entry_ticket[e] = tid;
        S->sh_h->seq2entry[t.seq & (kSeqMap - 1)] = e;
        std::atomic_thread_fence(std::memory_order_release);
        S->sh_h->pub = S->next_seq;
        idle = false;
      }
      // (re)launch the request loop when published work is waiting and it has exited
      if (S->kernel_live && cudaEventQuery(S->kdone) == cudaSuccess) S->kernel_live = false;
      bool waiting = false;
      for (int e = 0; e < S->R && !waiting; ++e) waiting = S->entry_ticket[e] != 0;
      if (waiting && !S->kernel_live) launch_loop(S);
    }
    if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

static void serve_free(ServeState* S) {
  if (S->sh_h) cudaFreeHost(S->sh_h);
  if (S->io_h) cudaFreeHost(S->io_h);
  if (S->qs_h) cudaFreeHost(S->qs_h);
  if (S->gs_h) cudaFreeHost(S->gs_h);
  if (S->out_h) cudaFreeHost(S->out_h);
  if (S->res_h) cudaFreeHost(S->res_h);
  if (S->con_h) cudaFreeHost(S->con_h);
  if (S->claim) cudaFree(S->claim);
  if (S->slot_q) cudaFree(S->slot_q);
  if (S->slot_g) cudaFree(S->slot_g);
  if (S->kdone) cudaEventDestroy(S->kdone);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // namespace dq

using namespace dq;

extern "C" {

dq_status dq_serve_stop(dq_context* ctx);

// Requests up to n = 512, p = 512 (FP32 problems) are served; the request
// loop's shared memory is sized for the largest.
dq_status dq_serve_start(dq_context* ctx, int32_t slots, int64_t hbm_budget_bytes) {
  if (!ctx || slots < 1 || hbm_budget_bytes <= 0) {
    set_error("dq_serve_start needs a context, slots >= 1 and a positive budget");
    return DQ_ERR_INVALID;
  }
  if (ctx->serve) {
    set_error("serving already started on this context");
    return DQ_ERR_INVALID;
  }
  DQ_CK(cudaSetDevice(ctx->device));
  ServeState* S = new ServeState();
  S->ctx = ctx;
  S->R = slots;
  S->nmax = 512;
  S->pmax = 1024;
  S->budget = hbm_budget_bytes;
  auto fail = [&](const char* what) {
    cudaGetLastError();
    set_error("dq_serve_start: %s", what);
    serve_free(S);
    return DQ_ERR_NOMEM;
  };
  const unsigned fl = cudaHostAllocMapped;
  const size_t R = S->R, nm = S->nmax, pm = S->pmax;
  if (cudaHostAlloc(&S->sh_h, sizeof(ServeShared), fl) != cudaSuccess) return fail("control block");
  memset((void*)S->sh_h, 0, sizeof(ServeShared));
  if (cudaHostAlloc(&S->io_h, R * sizeof(EntryIO), fl) != cudaSuccess) return fail("entries");
  memset((void*)S->io_h, 0, R * sizeof(EntryIO));
  if (cudaHostAlloc(&S->qs_h, R * nm * sizeof(float), fl) != cudaSuccess) return fail("q staging");
  if (cudaHostAlloc(&S->gs_h, R * pm * sizeof(float), fl) != cudaSuccess) return fail("g staging");
  if (cudaHostAlloc(&S->out_h, R * out_stride(S) * sizeof(float), fl) != cudaSuccess) return fail("outputs");
  if (cudaHostAlloc(&S->res_h, R * sizeof(DevResult), fl) != cudaSuccess) return fail("results");
  if (cudaHostAlloc(&S->con_h, R * 6 * sizeof(double), fl) != cudaSuccess) return fail("constants");
  cudaHostGetDevicePointer((void**)&S->sh_d, S->sh_h, 0);
  cudaHostGetDevicePointer((void**)&S->io_d, S->io_h, 0);
  cudaHostGetDevicePointer((void**)&S->qs_d, S->qs_h, 0);
  cudaHostGetDevicePointer((void**)&S->gs_d, S->gs_h, 0);
  cudaHostGetDevicePointer((void**)&S->out_d, S->out_h, 0);
  cudaHostGetDevicePointer((void**)&S->res_d, S->res_h, 0);
  cudaHostGetDevicePointer((void**)&S->con_d, S->con_h, 0);
  if (cudaMalloc(&S->claim, sizeof(unsigned long long)) != cudaSuccess) return fail("claim counter");
  if (cudaMemset(S->claim, 0, sizeof(unsigned long long)) != cudaSuccess) return fail("claim counter");
  if (cudaMalloc(&S->slot_q, R * nm * sizeof(float)) != cudaSuccess) return fail("slot q");
  if (cudaMalloc(&S->slot_g, R * pm * sizeof(float)) != cudaSuccess) return fail("slot g");
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) return fail("stream");
  if (cudaEventCreateWithFlags(&S->kdone, cudaEventDisableTiming) != cudaSuccess) return fail("event");
  S->smem = std::min<size_t>(max_dynamic_smem((const void*)serve_kernel, ctx->smem_optin), 96 * 1024);
  S->smem = std::max(S->smem, cta_vec_bytes<float>(S->nmax, S->pmax));
  auto kern = serve_kernel;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S->smem) != cudaSuccess)
    return fail("shared memory attribute");
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, S->smem);
  if (occ < 1) return fail("request loop cannot be resident");
  S->grid = std::min(S->R, ctx->num_sms * occ);
  S->entry_ticket.assign(S->R, 0);
  for (int e = S->R - 1; e >= 0; --e) S->free_entries.push_back(e);
  S->running = true;
  S->worker = std::thread(worker_loop, S);
  ctx->serve = S;
  return DQ_OK;
}

dq_status dq_submit(dq_context* ctx, dq_problem* prob, const dq_solve_opts* opts, const double* q,
                    const double* g, uint64_t* ticket) {
  if (!ctx || !ctx->serve || !prob || !ticket) {
    set_error("dq_submit needs a serving context, a problem and a ticket pointer");
    return DQ_ERR_INVALID;
  }
  ServeState* S = ctx->serve;
  if (prob->ctx != ctx || prob->prec != DQ_FP32 || prob->batch != 1 || prob->sparse) {
    set_error("served problems are single dense FP32 instances of this context");
    return DQ_ERR_INVALID;
  }
  if (prob->n > S->nmax || prob->p > S->pmax || prob_bytes(prob) > S->budget) {
    set_error("request (n=%d, p=%d) can never be admitted (limits n, p <= %d, %d; budget %lld bytes)", prob->n,
              prob->p, S->nmax, S->pmax, (long long)S->budget);
    return DQ_ERR_REJECTED;
  }
  Ticket t;
  t.prob = prob;
  t.n = prob->n;
  t.p = prob->p;
  dq_status s = resolve_opts(prob, opts, &t.cfg);
  if (s != DQ_OK) return s;
  if (q) {
    t.q.resize(t.n);
    for (int i = 0; i < t.n; ++i) {
      if (!isfinite(q[i])) {
        set_error("non-finite q");
        return DQ_ERR_INVALID;
      }
      t.q[i] = float(q[i]);
    }
    t.has_q = true;
  }
  if (g && t.p) {
    t.g.resize(t.p);
    for (int j = 0; j < t.p; ++j) {
      if (!isfinite(g[j])) {
        set_error("non-finite g");
        return DQ_ERR_INVALID;
      }
      t.g[j] = float(g[j]);
    }
    t.has_g = true;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  const uint64_t id = S->next_ticket++;
  S->tickets.emplace(id, std::move(t));
  S->pending.push_back(id);
  *ticket = id;
  return DQ_OK;
}

dq_status dq_poll(dq_context* ctx, uint64_t ticket, double* x_last, double* x_avg, double* lambda,
                  dq_result* result) {
  if (!ctx || !ctx->serve) {
    set_error("dq_poll needs a serving context");
    return DQ_ERR_INVALID;
  }
  ServeState* S = ctx->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->last_launch_error != DQ_OK) {
    set_error("the request loop failed to launch");
    return S->last_launch_error;
  }
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return DQ_ERR_INVALID;
  }
  Ticket& t = it->second;
  if (!t.done) return DQ_PENDING;
  if (t.res.status >= 0) {
    if (x_last) memcpy(x_last, t.x_last.data(), sizeof(double) * t.n);
    if (x_avg) memcpy(x_avg, t.x_avg.data(), sizeof(double) * t.n);
    if (lambda && t.p) memcpy(lambda, t.lam.data(), sizeof(double) * t.p);
  }
  if (result) fill_result(result, t.res, t.consts, t.cfg);
  const dq_status st = (dq_status)t.res.status;
  S->tickets.erase(it);
  return st;
}

dq_status dq_serve_stop(dq_context* ctx) {
  if (!ctx || !ctx->serve) return DQ_OK;
  ServeState* S = ctx->serve;
  S->sh_h->stop = 1;
  S->running = false;
  if (S->worker.joinable()) S->worker.join();
  cudaStreamSynchronize(S->stream);
  ctx->serve = nullptr;
  serve_free(S);
  return DQ_OK;
}

}  // extern "C"
