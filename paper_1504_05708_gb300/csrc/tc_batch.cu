// tc_batch.cu -- shared-matrix batches on the tensor cores (DQ_BF16X3).
//
// Instances that share Q and G and differ only in q and g (condensed MPC with
// a different initial state per instance) turn the matrix-vector products of
// Algorithm FOM (Sec. 2.1) and of the dual step of Algorithm DFOM (Sec. 3)
// into matrix-matrix products over the batch.  One thread block owns a tile
// of 128 instances and keeps the whole inner loop on chip:
//   * TMEM lane b holds instance b: columns hold D = Q x^k (the MMA
//     accumulator), x^k, x^{k-1}, Q x^{k-1} and c = q + G' mu, so every
//     per-instance quantity (step, projection, momentum, stopping certificate)
//     is local to one thread and needs no cross-thread reduction;
//   * each inner iteration is D = X Q' on tcgen05 with bf16 hi/lo split
//     operands (hi*hi + hi*lo + lo*hi) accumulated in FP32, X rewritten by the
//     epilogue threads straight into the operand layout;
//   * per outer iteration G ubar (dual gradient) and G' mu (next c) are two
//     more tensor-core products against G and G' tiles brought into shared
//     memory by bulk copies; lambda, lambda_prev, mu live in global memory.
// Stopping checks (eq. duquad_in for the inner loop per instance; the outer
// certificate with FP64-accurate residuals) follow the CTA engine's rules; the
// outer checks run between launches in a per-instance evaluation kernel.
// Limits: rho = 0 (DGM/DFGM), n <= 100 (TMEM columns), 1 CTA per SM.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "cta_engine.cuh"
#include "dq_host.h"
#include "tc_common.cuh"

namespace dq {

__global__ void k_pack_kmajor(const float* __restrict__ src, int R_valid, int K_valid, int ld, int R_pad, int K_pad,
                              uint4* __restrict__ hi, uint4* __restrict__ lo);

static constexpr int TM = 128;                        // instances per tile (TMEM lanes)
static constexpr unsigned long long kTcWaitNs = 2000000000ull;

struct TcArgs {
  int n, p, B, NPAD, NV, NC, KC, nchG, nchGT;
  const uint4 *Qhi, *Qlo, *Ghi, *Glo, *GThi, *GTlo;
  const float *q, *g, *lb, *ub;                       // q: B x n, g: B x p
  float *x, *xl, *usum, *lam, *lamp, *mun, *muk;      // B x n / B x p
  double *theta, *S;
  int* kout;
  long long* kin;
  int* active;
  float L, alpha;
  double sigma, beta_sigma, eps_in;
  int cone, kd_plus;
  int inner_fixed, inner_check_every, max_inner, nouter, mode, fast;
  int* err;
};

struct TcSmem {
  uint8_t *Qh, *Ql, *Xh, *Xl, *Gh, *Gl, *Mh, *Ml, *Bh, *Bl;
  float *lb, *ub;
};

__device__ __forceinline__ void tc_mma_tile(uint32_t d, const uint8_t* Ah, const uint8_t* Al, const uint8_t* Bh,
                                            const uint8_t* Bl, int Nrows, int K, bool accumulate) {
  const uint32_t idesc = tc::idesc_bf16_f32(TM, Nrows);
  const uint32_t la = tc::kmajor_lbo(TM), lb = tc::kmajor_lbo(Nrows);
  for (int s = 0; s < K / 16; ++s) {
    const uint64_t ah = tc::sdesc(tc::saddr(Ah) + s * 2 * la, la, 128);
    const uint64_t al = tc::sdesc(tc::saddr(Al) + s * 2 * la, la, 128);
    const uint64_t bh = tc::sdesc(tc::saddr(Bh) + s * 2 * lb, lb, 128);
    const uint64_t bl = tc::sdesc(tc::saddr(Bl) + s * 2 * lb, lb, 128);
    tc::mma_bf16(d, ah, bh, idesc, (accumulate || s > 0) ? 1u : 0u);
    tc::mma_bf16(d, ah, bl, idesc, 1u);
    tc::mma_bf16(d, al, bh, idesc, 1u);
  }
}

// Write 8 consecutive operand values (row r, columns k0..k0+7) as bf16 hi/lo.
__device__ __forceinline__ void put8(uint8_t* H, uint8_t* Lo, int r, int k0, const float* v) {
  uint4 h, l;
  tc::split8(v, h, l);
  const uint32_t off = tc::kmajor_off(r, k0, TM);
  *(uint4*)(H + off) = h;
  *(uint4*)(Lo + off) = l;
}

__global__ void __launch_bounds__(128, 1) k_tc_solve(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar_mma, bar_tx;
  __shared__ uint32_t s_taddr;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int NPAD = a.NPAD, NV = a.NV, n = a.n, p = a.p;
  // shared-memory carve (every region a multiple of 16 bytes)
  TcSmem S;
  size_t off = 0;
  auto take = [&](size_t b) {
    uint8_t* r = sm + off;
    off += (b + 127) & ~size_t(127);
    return r;
  };
  S.Qh = take((size_t)NPAD * NPAD * 2);
  S.Ql = take((size_t)NPAD * NPAD * 2);
  uint8_t* U = sm + off;
  const size_t uA = 2 * (size_t)TM * NPAD * 2 + 2 * (size_t)a.NC * NPAD * 2;
  const size_t uB = 2 * (size_t)TM * a.KC * 2 + 2 * (size_t)NPAD * a.KC * 2;
  S.Xh = U;
  S.Xl = U + (size_t)TM * NPAD * 2;
  S.Gh = S.Xl + (size_t)TM * NPAD * 2;
  S.Gl = S.Gh + (size_t)a.NC * NPAD * 2;
  S.Mh = U;
  S.Ml = U + (size_t)TM * a.KC * 2;
  S.Bh = S.Ml + (size_t)TM * a.KC * 2;
  S.Bl = S.Bh + (size_t)NPAD * a.KC * 2;
  off += (std::max(uA, uB) + 127) & ~size_t(127);
  S.lb = (float*)(sm + off);
  S.ub = S.lb + NV;
  for (int i = tid; i < NV; i += blockDim.x) {
    S.lb[i] = i < n ? a.lb[i] : 0.f;
    S.ub[i] = i < n ? a.ub[i] : 0.f;
  }
  if (tid == 0) {
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init(&bar_tx, 1);
    tc::mbar_init_fence();
    s_fail = 0;
  }
  __syncthreads();
  if (warp == 0) {
    tc::tmem_alloc(&s_taddr, 512);
    tc::tmem_relinquish();
  }
  uint32_t ph_mma = 0, ph_tx = 0;
  // Q operand (hi/lo) once per block
  if (tid == 0) {
    const uint32_t qb = (uint32_t)NPAD * NPAD * 2;
    tc::mbar_expect_tx(&bar_tx, 2 * qb);
    tc::bulk_g2s(S.Qh, a.Qhi, qb, &bar_tx);
    tc::bulk_g2s(S.Ql, a.Qlo, qb, &bar_tx);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  bool ok = tc::mbar_wait(&bar_tx, ph_tx, kTcWaitNs);
  ph_tx ^= 1;
  const uint32_t tm = s_taddr;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  const uint32_t cD = 0, cX = NPAD, cXP = NPAD + NV, cQP = NPAD + 2 * NV, cC = NPAD + 3 * NV;
  const uint32_t cR = (cXP + 31) / 32 * 32;  // 32-aligned accumulator for the dual products
  const float L = a.L;
  const double kap = a.sigma > 0.0 ? 1.0 / (2.0 * a.sigma) - 1.0 / (2.0 * (double)a.L) : 0.0;

  auto sync_mma = [&](void) -> bool {  // commit by thread 0 happened; all wait
    const bool w = tc::mbar_wait(&bar_mma, ph_mma, kTcWaitNs);
    ph_mma ^= 1;
    tc::fence_after();
    return w;
  };
  auto issue_fence = [&](void) {
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  };

  const int ntiles = (a.B + TM - 1) / TM;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int b = tile * TM + tid;  // this thread's instance
    const bool valid = b < a.B;
    int act = valid ? a.active[b] : 0;
    const float* qb = a.q + (size_t)(valid ? b : 0) * n;
    const float* gb = a.g + (size_t)(valid ? b : 0) * p;
    float* xb = a.x + (size_t)(valid ? b : 0) * n;
    // ---- load x into TMEM and the A operand; D = Q x
    {
      const float* src = a.mode == 1 ? xb : xb;
      for (int i0 = 0; i0 < NV; i0 += 8) {
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (valid && i0 + t < n) ? src[i0 + t] : 0.f;
        if (i0 + 8 <= NPAD) put8(S.Xh, S.Xl, tid, i0, v);
        float v4[4] = {v[0], v[1], v[2], v[3]};
        tc::tmem_st4(tm + lane_off + cX + i0, v4);
        if (i0 + 4 < NV) {
          float w4[4] = {v[4], v[5], v[6], v[7]};
          tc::tmem_st4(tm + lane_off + cX + i0 + 4, w4);
        }
      }
      for (int i0 = ((NV + 7) / 8) * 8; i0 < NPAD; i0 += 8) {
        float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        put8(S.Xh, S.Xl, tid, i0, z);
      }
      tc::tmem_st_wait();
    }
    issue_fence();
    if (tid == 0) {
      tc_mma_tile(tm + cD, S.Xh, S.Xl, S.Qh, S.Ql, NPAD, NPAD, false);
      tc::mma_commit(&bar_mma);
    }
    if (!sync_mma()) { ok = false; break; }

    // ---- c = q + G' m  with m = mu^k (mode 0) or lambda^k (mode 1)
    auto gtmu = [&](const float* mrow) -> bool {
      const uint32_t cAcc = cR;  // accumulator over the free x_{k-1} / Q x_{k-1} columns
      for (int ch = 0; ch < a.nchGT; ++ch) {
        const int j0 = ch * a.KC;
        for (int jj = 0; jj < a.KC; jj += 8) {
          float v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int j = j0 + jj + t;
            v[t] = (valid && j < p) ? mrow[j] : 0.f;
          }
          uint4 h, l;
          tc::split8(v, h, l);
          const uint32_t o = tc::kmajor_off(tid, jj, TM);
          *(uint4*)(S.Mh + o) = h;
          *(uint4*)(S.Ml + o) = l;
        }
        if (tid == 0) {
          const uint32_t bbytes = (uint32_t)NPAD * a.KC * 2;
          tc::mbar_expect_tx(&bar_tx, 2 * bbytes);
          tc::bulk_g2s(S.Bh, (const uint8_t*)a.GThi + (size_t)ch * bbytes, bbytes, &bar_tx);
          tc::bulk_g2s(S.Bl, (const uint8_t*)a.GTlo + (size_t)ch * bbytes, bbytes, &bar_tx);
        }
        issue_fence();
        if (!tc::mbar_wait(&bar_tx, ph_tx, kTcWaitNs)) return false;
        ph_tx ^= 1;
        if (tid == 0) {
          tc_mma_tile(tm + cAcc, S.Mh, S.Ml, S.Bh, S.Bl, NPAD, a.KC, ch > 0);
          tc::mma_commit(&bar_mma);
        }
        if (!sync_mma()) return false;
      }
      // c = acc + q  (zero when there are no constraints)
      for (int i0 = 0; i0 < NV; i0 += 4) {
        float c4[4];
        if (a.nchGT > 0) tc::tmem_ld4(tm + lane_off + cAcc + i0, c4);
        else c4[0] = c4[1] = c4[2] = c4[3] = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) c4[t] += (valid && i0 + t < n) ? qb[i0 + t] : 0.f;
        tc::tmem_st4(tm + lane_off + cC + i0, c4);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      return true;
    };
    {
      const float* m0 = a.mode == 1 ? a.lam + (size_t)(valid ? b : 0) * p : a.mun + (size_t)(valid ? b : 0) * p;
      if (!gtmu(m0)) { ok = false; break; }
    }

    const int nout = a.mode == 1 ? 1 : a.nouter;
    for (int o = 0; o < nout && ok; ++o) {
      if (!__syncthreads_or(act)) break;
      // ---- inner loop: Algorithm FOM from x^0 = ubar (x_{-1} = x^0)
      for (int i0 = 0; i0 < NV; i0 += 4) {
        float v[4], d[4];
        tc::tmem_ld4(tm + lane_off + cX + i0, v);
        tc::tmem_ld4(tm + lane_off + cD + i0, d);
        tc::tmem_st4(tm + lane_off + cXP + i0, v);
        tc::tmem_st4(tm + lane_off + cQP + i0, d);
      }
      tc::tmem_st_wait();
      const bool fgm_sigma = a.sigma > 0.0;
      double th_in = 1.0, beta = 0.0;
      int kin = 0, done_in = act ? 0 : 1, kstop = 0;
      const int m = a.inner_check_every > 0 ? a.inner_check_every : 1;
      const int kmax = a.inner_fixed > 0 ? a.inner_fixed : a.max_inner;
      for (;;) {
        ++kin;
        const float bt = (float)beta;
        // every lane runs the same tcgen05 instructions; lanes whose inner
        // loop has stopped write their unchanged values back.  The operand is
        // rewritten up to NPAD (zero padding) because the G' mu product
        // overlays it in shared memory.
        for (int i0 = 0; i0 < NPAD; i0 += 8) {
          float xn[8];
          for (int h = 0; h < 8; h += 4) {
            const int ii = i0 + h;
            if (ii >= NV) {
              xn[h] = xn[h + 1] = xn[h + 2] = xn[h + 3] = 0.f;
              continue;
            }
            float d[4], x[4], xp[4], qp[4], c[4];
            tc::tmem_ld4(tm + lane_off + cD + ii, d);
            tc::tmem_ld4(tm + lane_off + cX + ii, x);
            tc::tmem_ld4(tm + lane_off + cXP + ii, xp);
            tc::tmem_ld4(tm + lane_off + cQP + ii, qp);
            tc::tmem_ld4(tm + lane_off + cC + ii, c);
            float r4[4], nxp[4], nqp[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float y = x[t] + bt * (x[t] - xp[t]);
              const float qy = d[t] + bt * (d[t] - qp[t]);
              const float s = y - (qy + c[t]) / L;
              const float lo = S.lb[ii + t], hi = S.ub[ii + t];
              const float xnew = s < lo ? lo : (s > hi ? hi : s);
              r4[t] = done_in ? x[t] : xnew;
              nxp[t] = done_in ? xp[t] : x[t];
              nqp[t] = done_in ? qp[t] : d[t];
              xn[h + t] = r4[t];
            }
            tc::tmem_st4(tm + lane_off + cQP + ii, nqp);
            tc::tmem_st4(tm + lane_off + cXP + ii, nxp);
            tc::tmem_st4(tm + lane_off + cX + ii, r4);
          }
          put8(S.Xh, S.Xl, tid, i0, xn);
        }
        tc::tmem_st_wait();
        issue_fence();
        if (tid == 0) {
          tc_mma_tile(tm + cD, S.Xh, S.Xl, S.Qh, S.Ql, NPAD, NPAD, false);
          tc::mma_commit(&bar_mma);
        }
        if (!sync_mma()) { ok = false; break; }
        if (fgm_sigma) {
          beta = a.beta_sigma;
        } else {
          const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * th_in * th_in));
          beta = (th_in - 1.0) / t1;
          th_in = t1;
        }
        {
          bool stop = false;
          if (a.inner_fixed > 0) {
            stop = kin >= a.inner_fixed;
          } else {
            if (kin % m == 0) {  // certificate of eq. duquad_in at x^k (gradient Q x^k + c), all lanes
              double cert = 0.0;
              for (int i0 = 0; i0 < NV; i0 += 4) {
                float d[4], x[4], c[4];
                tc::tmem_ld4(tm + lane_off + cD + i0, d);
                tc::tmem_ld4(tm + lane_off + cX + i0, x);
                tc::tmem_ld4(tm + lane_off + cC + i0, c);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  if (i0 + t >= n) continue;
                  const double gd = (double)(d[t] + c[t]), xd = x[t];
                  const double lo = S.lb[i0 + t], hi = S.ub[i0 + t];
                  if (a.sigma > 0.0) {
                    const double xp = fmin(fmax(xd - gd / (double)L, lo), hi);
                    const double dd = xd - xp;
                    cert += gd * dd + ((double)L * dd) * ((double)L * dd) * kap;
                  } else {
                    const double u1 = gd * lo, u2 = gd * hi;
                    cert += gd * xd - (u1 < u2 ? u1 : u2);
                  }
                }
              }
              stop = cert <= a.eps_in;
            }
            stop = stop || kin >= a.max_inner;
          }
          if (stop && !done_in) {
            done_in = 1;
            kstop = kin;
          }
        }
        if (__syncthreads_and(done_in) || kin >= kmax) break;
      }
      if (!ok) break;
      if (act && valid) a.kin[b] += (kstop > 0 ? kstop : kin);
      if (a.mode == 1) break;
      // ---- dual step: lambda = [mu + (G ubar + g)/(2 L_d)]_{K_d}, momentum, averaging
      const double th = act ? a.theta[b] : 1.0;
      double beta_out = 0.0;
      if (a.fast) {
        const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * th * th));
        beta_out = (th - 1.0) / t1;
      }
      for (int ch = 0; ch < a.nchG; ++ch) {
        const int j0 = ch * a.NC;
        if (tid == 0) {
          const uint32_t bbytes = (uint32_t)a.NC * NPAD * 2;
          tc::mbar_expect_tx(&bar_tx, 2 * bbytes);
          tc::bulk_g2s(S.Gh, (const uint8_t*)a.Ghi + (size_t)ch * bbytes, bbytes, &bar_tx);
          tc::bulk_g2s(S.Gl, (const uint8_t*)a.Glo + (size_t)ch * bbytes, bbytes, &bar_tx);
        }
        issue_fence();
        if (!tc::mbar_wait(&bar_tx, ph_tx, kTcWaitNs)) { ok = false; break; }
        ph_tx ^= 1;
        if (tid == 0) {
          tc_mma_tile(tm + cR, S.Xh, S.Xl, S.Gh, S.Gl, a.NC, NPAD, false);
          tc::mma_commit(&bar_mma);
        }
        if (!sync_mma()) { ok = false; break; }
        {
          const bool upd = act && valid;
          const size_t rb = (size_t)(valid ? b : 0) * p;
          float* lr = a.lam + rb;
          float* lpr = a.lamp + rb;
          float* mr = a.mun + rb;
          float* mkr = a.muk + rb;
          for (int jj = 0; jj < a.NC && j0 + jj < p; jj += 4) {  // uniform tcgen05.ld, masked updates
            float r4[4];
            tc::tmem_ld4(tm + lane_off + cR + jj, r4);
            if (!upd) continue;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int j = j0 + jj + t;
              if (j >= p) break;
              const float mu = mr[j];
              const float l_old = lr[j];
              const float v = mu + a.alpha * (r4[t] + gb[j]);
              const float ln = (a.cone == CONE_EQ || !a.kd_plus) ? v : (v > 0.f ? v : 0.f);
              mkr[j] = mu;
              lpr[j] = l_old;
              lr[j] = ln;
              mr[j] = ln + (float)beta_out * (ln - l_old);
            }
          }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
      }
      if (!ok) break;
      {
        const bool upd = act && valid;
        float* us = a.usum + (size_t)(valid ? b : 0) * n;
        for (int i0 = 0; i0 < NV; i0 += 4) {  // uniform tcgen05.ld, masked updates
          float x[4];
          tc::tmem_ld4(tm + lane_off + cX + i0, x);
          if (!upd) continue;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (i0 + t < n) us[i0 + t] += (float)th * x[t];
        }
        if (upd) {
          a.S[b] += th;
          a.kout[b] += 1;
          if (a.fast) a.theta[b] = 0.5 * (1.0 + sqrt(1.0 + 4.0 * th * th));
        }
      }
      // next c = q + G' mu^{k+1}
      if (!gtmu(a.mun + (size_t)(valid ? b : 0) * p)) { ok = false; break; }
    }
    if (!ok) break;
    // ---- store x (mode 0: the warm-start chain; mode 1: the last-iterate output)
    float* dst = a.mode == 1 ? a.xl + (size_t)(valid ? b : 0) * n : xb;
    for (int i0 = 0; i0 < NV; i0 += 4) {
      float x[4];
      tc::tmem_ld4(tm + lane_off + cX + i0, x);
      if (valid && (act || a.mode == 1))
        for (int t = 0; t < 4; ++t)
          if (i0 + t < n) dst[i0 + t] = x[t];
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (!ok && tid == 0) atomicExch(a.err, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// Per-instance FP64-accurate evaluation for the outer certificate (same
// rules as the CTA engine): lower bound from (ubar, mu^k), outputs' F and
// dist_K, convergence flags.
struct TcEvalArgs {
  int n, p, B, cone;
  const float *Q, *G, *GT, *q, *g, *lb, *ub;
  const float *x, *xl, *usum, *lam, *muk;
  const double* S;
  float* xavg;
  double LL, sigma, eps_out;
  int want_last, want_avg, fast, fixed;
  int* active;
  DevResult* res;
};

__global__ void __launch_bounds__(128) k_tc_eval(TcEvalArgs e) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  if (b >= e.B) return;
  if (!e.active[b]) return;
  const int n = e.n, p = e.p;
  CtaWs<float> W;
  memset(&W, 0, sizeof(W));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* r = smem + off;
    off += (bytes + 15) & ~size_t(15);
    return r;
  };
  W.red = (double*)take(40 * sizeof(double));
  W.dn = (double*)take((size_t)n * sizeof(double));
  W.dp = (double*)take((size_t)(p > 0 ? p : 1) * sizeof(double));
  float* ua = (float*)take((size_t)n * sizeof(float));
  W.Q = e.Q;
  W.G = e.G;
  W.GT = e.GT;
  CtaInst<float> I;
  memset(&I, 0, sizeof(I));
  I.n = n;
  I.p = p;
  I.cone = e.cone;
  I.q = e.q + (size_t)b * n;
  I.g = e.g + (size_t)b * p;
  I.lb = e.lb;
  I.ub = e.ub;
  I.rho = 0.0;
  I.LL = e.LL;
  I.sigma = e.sigma;
  DevResult r = e.res[b];
  const float* xb = e.x + (size_t)b * n;
  const float* mk = e.muk + (size_t)b * p;
  bool mu_ok = true;
  if (e.cone == CONE_INEQ) {
    int neg = 0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) neg |= mk[j] < 0.f;
    mu_ok = !__syncthreads_or(neg);
  }
  if (mu_ok) {
    EvalOut v = cta_eval<float>(I, W, xb, mk);
    r.d_lb = fmax(r.d_lb, v.lagr - v.cert);
  }
  if (e.want_last) {
    if (e.fast) {
      const float* lb_ = e.lam + (size_t)b * p;
      bool lok = true;
      if (e.cone == CONE_INEQ) {
        int neg = 0;
        for (int j = threadIdx.x; j < p; j += blockDim.x) neg |= lb_[j] < 0.f;
        lok = !__syncthreads_or(neg);
      }
      EvalOut v = cta_eval<float>(I, W, e.xl + (size_t)b * n, lok ? lb_ : nullptr);
      if (lok) r.d_lb = fmax(r.d_lb, v.lagr - v.cert);
      r.f_last = v.F;
      r.infeas_last = v.infeas;
    } else {
      EvalOut v = cta_eval<float>(I, W, xb, (const float*)nullptr);
      r.f_last = v.F;
      r.infeas_last = v.infeas;
    }
  }
  if (e.want_avg) {
    const double Sb = e.S[b];
    for (int i = threadIdx.x; i < n; i += blockDim.x) ua[i] = (float)(e.usum[(size_t)b * n + i] / Sb);
    __syncthreads();
    EvalOut v = cta_eval<float>(I, W, ua, (const float*)nullptr);
    r.f_avg = v.F;
    r.infeas_avg = v.infeas;
    for (int i = threadIdx.x; i < n; i += blockDim.x) e.xavg[(size_t)b * n + i] = ua[i];
  }
  if (threadIdx.x == 0) {
    if ((e.want_last && !(isfinite(r.f_last) && isfinite(r.infeas_last))) ||
        (e.want_avg && !(isfinite(r.f_avg) && isfinite(r.infeas_avg)))) {
      r.status = ST_NONFINITE;
      e.active[b] = 0;
    } else if (!e.fixed) {
      r.converged_last = e.want_last && r.infeas_last <= e.eps_out && r.f_last - r.d_lb <= e.eps_out;
      r.converged_avg = e.want_avg && r.infeas_avg <= e.eps_out && r.f_avg - r.d_lb <= e.eps_out;
      if (r.converged_last || r.converged_avg) {
        r.status = ST_OK;
        e.active[b] = 0;
      }
    }
    e.res[b] = r;
  }
}

__global__ void k_tc_init(int B, int n, int p, float* x, const float* x0, const float* lb, const float* ub,
                          float* lam, float* lamp, float* mun, float* muk, const float* lam0, float* usum,
                          double* theta, double* S, int* kout, long long* kin, int* active, DevResult* res) {
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
  for (size_t k = tid; k < (size_t)B * n; k += nt) {
    const int i = (int)(k % n);
    x[k] = x0 ? x0[k] : fminf(fmaxf(0.f, lb[i]), ub[i]);
    usum[k] = 0.f;
  }
  for (size_t k = tid; k < (size_t)B * p; k += nt) {
    const float l = lam0 ? lam0[k] : 0.f;
    lam[k] = l;
    lamp[k] = l;
    mun[k] = l;
    muk[k] = l;
  }
  for (size_t b = tid; b < (size_t)B; b += nt) {
    theta[b] = 1.0;
    S[b] = 0.0;
    kout[b] = 0;
    kin[b] = 0;
    active[b] = 1;
    DevResult r;
    r.status = ST_NOT_CONVERGED;
    r.outer_iters = 0;
    r.inner_iters = 0;
    r.converged_last = r.converged_avg = 0;
    r.f_last = r.infeas_last = r.f_avg = r.infeas_avg = NAN;
    r.d_lb = -INFINITY;
    res[b] = r;
  }
}

__global__ void k_tc_finish(int B, const int* kout, const long long* kin, DevResult* res, int* count_active,
                            const int* active) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    res[b].outer_iters = kout[b];
    res[b].inner_iters = kin[b];
    if (active[b]) atomicAdd(count_active, 1);
  }
}

struct TcWs {
  int NPAD = 0, NV = 0, NC = 0, KC = 0, nchG = 0, nchGT = 0;
  void* mem = nullptr;
  uint4 *Qhi, *Qlo, *Ghi, *Glo, *GThi, *GTlo;
  float *x, *xl, *xa, *usum, *lam, *lamp, *mun, *muk;
  double *theta, *S;
  int *kout, *active, *err, *cnt;
  long long* kin;
  DevResult* res;
  bool packed = false;
};

void tc_free(TcWs* w) {
  if (!w) return;
  if (w->mem) cudaFree(w->mem);
  delete w;
}

static dq_status tc_ws(dq_problem* P, TcWs** out) {
  if (P->tws) {
    *out = P->tws;
    return DQ_OK;
  }
  TcWs* W = new TcWs();
  const int n = P->n, p = P->p, B = P->batch;
  W->NPAD = (n + 15) / 16 * 16;
  W->NV = (n + 3) / 4 * 4;
  W->NC = 192;
  W->KC = 64;
  W->nchG = (p + W->NC - 1) / W->NC;
  W->nchGT = (p + W->KC - 1) / W->KC;
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t qb = (size_t)W->NPAD * W->NPAD * 2, gb = (size_t)W->nchG * W->NC * W->NPAD * 2,
               gtb = (size_t)W->nchGT * W->NPAD * W->KC * 2;
  const size_t bn = (size_t)B * n * 4, bp = (size_t)std::max(B * p, 1) * 4;
  size_t total = 2 * a256(qb) + 2 * a256(gb) + 2 * a256(gtb) + 4 * a256(bn) + 4 * a256(bp) + 2 * a256((size_t)B * 8) +
                 3 * a256((size_t)B * 4) + a256((size_t)B * 8) + a256((size_t)B * sizeof(DevResult)) + 256;
  if (cudaMalloc(&W->mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete W;
    set_error("tensor-core workspace (%zu bytes) allocation failed", total);
    return DQ_ERR_NOMEM;
  }
  char* c = (char*)W->mem;
  auto take = [&](size_t b) {
    void* r = c;
    c += a256(b);
    return r;
  };
  W->Qhi = (uint4*)take(qb); W->Qlo = (uint4*)take(qb);
  W->Ghi = (uint4*)take(gb); W->Glo = (uint4*)take(gb);
  W->GThi = (uint4*)take(gtb); W->GTlo = (uint4*)take(gtb);
  W->x = (float*)take(bn); W->xl = (float*)take(bn); W->xa = (float*)take(bn); W->usum = (float*)take(bn);
  W->lam = (float*)take(bp); W->lamp = (float*)take(bp); W->mun = (float*)take(bp); W->muk = (float*)take(bp);
  W->theta = (double*)take((size_t)B * 8); W->S = (double*)take((size_t)B * 8);
  W->kout = (int*)take((size_t)B * 4); W->active = (int*)take((size_t)B * 4); W->err = (int*)take(4 * 64);
  W->cnt = W->err + 16;
  W->kin = (long long*)take((size_t)B * 8);
  W->res = (DevResult*)take((size_t)B * sizeof(DevResult));
  P->tws = W;
  *out = W;
  return DQ_OK;
}

static size_t tc_smem_bytes(const TcWs* W) {
  auto r128 = [](size_t b) { return (b + 127) & ~size_t(127); };
  const size_t q = 2 * r128((size_t)W->NPAD * W->NPAD * 2);
  const size_t uA = 2 * (size_t)TM * W->NPAD * 2 + 2 * (size_t)W->NC * W->NPAD * 2;
  const size_t uB = 2 * (size_t)TM * W->KC * 2 + 2 * (size_t)W->NPAD * W->KC * 2;
  return q + r128(std::max(uA, uB)) + 2 * (size_t)W->NV * 4 + 128;
}

dq_status tc_solve(dq_problem* P, const SolveCfg& c, const dq_outputs* out, dq_result* results) {
  std::lock_guard<std::mutex> lk(P->mu);
  if (c.alg != DQ_DGM && c.alg != DQ_DFGM) {
    set_error("the tensor-core engine runs DGM and DFGM (rho = 0); use the CTA engine for ADGM/ADFGM");
    return DQ_ERR_INVALID;
  }
  if (!isnan(c.rho) && c.rho != 0.0) {
    set_error("the tensor-core engine needs rho = 0");
    return DQ_ERR_INVALID;
  }
  const int n = P->n, p = P->p, B = P->batch;
  if ((n + 15) / 16 * 16 + 4 * ((n + 3) / 4 * 4) > 512) {
    set_error("the tensor-core engine holds n <= 100 variables per instance in tensor memory (n = %d)", n);
    return DQ_ERR_INVALID;
  }
  if (c.inner_stop == DQ_INNER_FIXED && c.fixed_inner <= 0) {
    set_error("fixed inner count needed");
    return DQ_ERR_INVALID;
  }
  dq_context* ctx = P->ctx;
  cudaStream_t st = ctx->stream;
  if (c.fresh) {
    P->lmax_Q = P->lmax_given;
    P->normG2 = P->normG2_given;
  }
  if (isnan(P->lmax_Q) || isnan(P->normG2)) {
    dq_status s = grid_constants(P);
    if (s != DQ_OK) return s;
  }
  TcWs* W;
  dq_status s = tc_ws(P, &W);
  if (s != DQ_OK) return s;
  const size_t smem = tc_smem_bytes(W);
  if (smem > max_dynamic_smem((const void*)k_tc_solve, ctx->smem_optin)) {
    set_error("tensor-core engine needs %zu bytes of shared memory", smem);
    return DQ_ERR_INVALID;
  }
  if (!W->packed) {
    k_pack_kmajor<<<64, 256, 0, st>>>((const float*)P->Q, n, n, n, W->NPAD, W->NPAD, W->Qhi, W->Qlo);
    for (int ch = 0; ch < W->nchG; ++ch) {
      const size_t o = (size_t)ch * W->NC * W->NPAD * 2 / 16;
      k_pack_kmajor<<<64, 256, 0, st>>>((const float*)P->G + (size_t)ch * W->NC * n, std::min(W->NC, p - ch * W->NC), n,
                                        n, W->NC, W->NPAD, W->Ghi + o, W->Glo + o);
    }
    for (int ch = 0; ch < W->nchGT; ++ch) {
      const size_t o = (size_t)ch * W->NPAD * W->KC * 2 / 16;
      k_pack_kmajor<<<64, 256, 0, st>>>((const float*)P->GT + (size_t)ch * W->KC, n, std::min(W->KC, p - ch * W->KC),
                                        p, W->NPAD, W->KC, W->GThi + o, W->GTlo + o);
    }
    ctx->launches += 1 + W->nchG + W->nchGT;
    DQ_CK(cudaGetLastError());
    W->packed = true;
  }
  const double lmin = isnan(P->lmin_Q) ? 0.0 : P->lmin_Q;
  const double rho = 0.0;
  const double LL = isnan(c.LL) ? P->lmax_Q : c.LL;
  const double sigma = isnan(c.sigma) ? lmin : c.sigma;
  double Ld = c.Ld;
  if (isnan(Ld)) Ld = P->normG2 > 0 ? (lmin > 0 ? P->normG2 / lmin : INFINITY) : 1.0;
  if (!(Ld < INFINITY)) {
    set_error("DGM/DFGM need lmin_Q > 0 (Case 1)");
    return DQ_ERR_INVALID;
  }
  const bool fast = c.alg == DQ_DFGM;
  const double eps_in = isnan(c.eps_in) ? (fast ? c.eps_out * sqrt(c.eps_out) / (8.0 * sqrt(2.0 * Ld)) : c.eps_out / 4.0)
                                        : c.eps_in;
  const bool warm = c.warm_start && P->has_state;
  k_tc_init<<<256, 256, 0, st>>>(B, n, p, W->x, warm ? (const float*)P->x_state : nullptr, (const float*)P->lb,
                                 (const float*)P->ub, W->lam, W->lamp, W->mun, W->muk,
                                 warm ? (const float*)P->lam_state : nullptr, W->usum, W->theta, W->S, W->kout, W->kin,
                                 W->active, W->res);
  ++ctx->launches;
  DQ_CK(cudaMemsetAsync(W->err, 0, 64 * 4, st));
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n; a.p = p; a.B = B; a.NPAD = W->NPAD; a.NV = W->NV; a.NC = W->NC; a.KC = W->KC;
  a.nchG = W->nchG; a.nchGT = W->nchGT;
  a.Qhi = W->Qhi; a.Qlo = W->Qlo; a.Ghi = W->Ghi; a.Glo = W->Glo; a.GThi = W->GThi; a.GTlo = W->GTlo;
  a.q = (const float*)P->q; a.g = (const float*)P->g; a.lb = (const float*)P->lb; a.ub = (const float*)P->ub;
  a.x = W->x; a.xl = W->xl; a.usum = W->usum; a.lam = W->lam; a.lamp = W->lamp; a.mun = W->mun; a.muk = W->muk;
  a.theta = W->theta; a.S = W->S; a.kout = W->kout; a.kin = W->kin; a.active = W->active;
  a.L = (float)LL; a.alpha = (float)(1.0 / (2.0 * Ld)); a.sigma = sigma;
  a.beta_sigma = sigma > 0 ? (sqrt(LL) - sqrt(sigma)) / (sqrt(LL) + sqrt(sigma)) : 0.0;
  a.eps_in = eps_in; a.cone = P->cone; a.kd_plus = !(c.kd_literal && !(lmin > 0.0));
  a.inner_fixed = c.fixed_inner; a.inner_check_every = c.inner_check_every; a.max_inner = c.max_inner;
  a.fast = fast; a.err = W->err;
  TcEvalArgs e;
  memset(&e, 0, sizeof(e));
  e.n = n; e.p = p; e.B = B; e.cone = P->cone;
  e.Q = (const float*)P->Q; e.G = (const float*)P->G; e.GT = (const float*)P->GT;
  e.q = (const float*)P->q; e.g = (const float*)P->g; e.lb = (const float*)P->lb; e.ub = (const float*)P->ub;
  e.x = W->x; e.xl = W->xl; e.usum = W->usum; e.lam = W->lam; e.muk = W->muk; e.S = W->S; e.xavg = W->xa;
  e.LL = LL; e.sigma = sigma; e.eps_out = c.eps_out;
  e.want_last = (c.output & DQ_OUT_LAST) != 0; e.want_avg = (c.output & DQ_OUT_AVERAGE) != 0; e.fast = fast;
  e.fixed = c.fixed_outer > 0; e.active = W->active; e.res = W->res;
  const size_t esmem = 40 * 8 + (size_t)n * 8 + (size_t)std::max(p, 1) * 8 + (size_t)n * 4 + 64;
  DQ_CK(cudaFuncSetAttribute(k_tc_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ntiles = (B + TM - 1) / TM;
  const int grid = std::min(ntiles, ctx->num_sms);
  const int kmax = c.fixed_outer > 0 ? c.fixed_outer : c.max_outer;
  const int step = c.fixed_outer > 0 ? c.fixed_outer : c.check_every;
  int k = 0, active_count = B;
  while (k < kmax && active_count > 0) {
    const int nout = std::min(step, kmax - k);
    a.mode = 0;
    a.nouter = nout;
    k_tc_solve<<<grid, TM, smem, st>>>(a);
    ++ctx->launches;
    k += nout;
    if (e.want_last && fast) {
      a.mode = 1;
      k_tc_solve<<<grid, TM, smem, st>>>(a);
      ++ctx->launches;
    } else {
      DQ_CK(cudaMemcpyAsync(W->xl, W->x, (size_t)B * n * 4, cudaMemcpyDeviceToDevice, st));
    }
    k_tc_eval<<<B, 128, esmem, st>>>(e);
    DQ_CK(cudaMemsetAsync(W->cnt, 0, 4, st));
    k_tc_finish<<<64, 256, 0, st>>>(B, W->kout, W->kin, W->res, W->cnt, W->active);
    ctx->launches += 2;
    DQ_CK(cudaGetLastError());
    int herr[2] = {0, 0};
    DQ_CK(cudaMemcpyAsync(&herr[0], W->err, 4, cudaMemcpyDeviceToHost, st));
    DQ_CK(cudaMemcpyAsync(&herr[1], W->cnt, 4, cudaMemcpyDeviceToHost, st));
    DQ_CK(cudaStreamSynchronize(st));
    if (herr[0]) {
      set_error("tensor-core engine: a device wait timed out");
      return DQ_ERR_TIMEOUT;
    }
    active_count = c.fixed_outer > 0 ? 0 : herr[1];
  }
  // results and outputs
  std::vector<DevResult> hr(B);
  DQ_CK(cudaMemcpyAsync(hr.data(), W->res, (size_t)B * sizeof(DevResult), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaMemcpyAsync(P->x_state, W->x, (size_t)B * n * 4, cudaMemcpyDeviceToDevice, st));
  if (p) DQ_CK(cudaMemcpyAsync(P->lam_state, W->lam, (size_t)B * p * 4, cudaMemcpyDeviceToDevice, st));
  P->has_state = true;
  if (out) {
    auto put = [&](void* dst, const float* src, size_t cnt) -> dq_status {
      if (!dst || !cnt) return DQ_OK;
      if (out->memory == DQ_DEVICE) {
        DQ_CK(cudaMemcpyAsync(dst, src, cnt * 4, cudaMemcpyDeviceToDevice, st));
      } else {
        std::vector<float> h(cnt);
        DQ_CK(cudaMemcpyAsync(h.data(), src, cnt * 4, cudaMemcpyDeviceToHost, st));
        DQ_CK(cudaStreamSynchronize(st));
        for (size_t i = 0; i < cnt; ++i) ((double*)dst)[i] = h[i];
      }
      return DQ_OK;
    };
    if ((s = put(out->x_last, W->xl, (size_t)B * n)) != DQ_OK) return s;
    if ((s = put(out->x_avg, W->xa, (size_t)B * n)) != DQ_OK) return s;
    if ((s = put(out->lambda, W->lam, (size_t)B * p)) != DQ_OK) return s;
  }
  DQ_CK(cudaStreamSynchronize(st));
  const double consts[6] = {P->lmax_Q, P->normG2, LL, Ld, sigma, rho};
  dq_status worst = DQ_OK;
  for (int b = 0; b < B; ++b) {
    if (c.fixed_outer > 0 && hr[b].status == ST_NOT_CONVERGED) hr[b].status = ST_OK;
    fill_result(&results[b], hr[b], consts, c);
    const dq_status sb = (dq_status)hr[b].status;
    if (sb < 0 || worst < 0) worst = sb < worst ? sb : worst;
    else if (sb > worst) worst = sb;
  }
  return worst;
}

}  // namespace dq
