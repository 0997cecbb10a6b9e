// tc_batch.cu -- shared-matrix batches on the tensor cores (DQ_BF16X3).
//
// Instances that share Q and G and differ only in q and g (condensed MPC with
// a different initial state per instance) turn the matrix-vector products of
// Algorithm FOM (Sec. 2.1) and of the dual step of Algorithm DFOM (Sec. 3)
// into matrix-matrix products over the batch.  One persistent thread block
// (256 threads, two per instance) takes a tile of 128 instances and runs its whole solve --
// every outer iteration, the inner loops, the outer stopping checks and the
// extra last-iterate solves -- without returning to the host:
//   * TMEM lane b holds instance b: four 16-aligned column regions hold
//     D (the MMA accumulator), y^k, x^k and c = q + G' mu, so every
//     per-instance quantity (step, projection, momentum, certificates,
//     residuals) is local to one thread and needs no cross-thread reduction;
//   * an inner iteration is D = Q y^k on tcgen05 with bf16 hi/lo split
//     operands (hi*hi + hi*lo + lo*hi) accumulated in FP32; the epilogue forms
//     x^{k+1} = [y^k - (D + c)/L]_U and y^{k+1}, and writes the next operand
//     straight into the K-major shared-memory layout.  At certificate
//     iterations the operand is x^{k+1} first (D = Q x^{k+1} for the
//     gradient-mapping bound of eq. duquad_in), then y^{k+1};
//   * per outer iteration G ubar (dual gradient) and G' mu (next c) are
//     chunked tensor-core products against pre-packed G and G' tiles brought
//     in by double-buffered bulk copies; lambda, lambda_prev, mu and the
//     averaging sum live in global memory, instance-minor
//     ([tile][element][lane]) so that a tile's 128 threads touch 512
//     contiguous bytes per element.
// The outer certificate (F(u) - d_lb <= eps, dist_K(Gu + g) <= eps) follows
// the thread-block engine's rules.  The split products carry a relative error
// near 2^-16, which is enough for G u (residuals) but not for F(u) = u'Qu/2 +
// q'u at eps = 1e-3 (the quadratic term is ~250 on the MPC workload), so F is
// evaluated per lane in FP32 from the FP32 Q (SIMT, symmetric half).  A lane
// whose instance has converged is frozen (its state no longer changes) and the
// tile ends when every lane is done.
// Limits: rho = 0 (DGM/DFGM), n <= 128 (four TMEM regions of 16-aligned n).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dq_common.cuh"
#include "dq_host.h"
#include "tc_common.cuh"

namespace dq {

__global__ void k_pack_kmajor(const float* __restrict__ src, int R_valid, int K_valid, int ld, int R_pad, int K_pad,
                              uint4* __restrict__ hi, uint4* __restrict__ lo);

static constexpr int TM = 128;                        // instances per tile (TMEM lanes, threads)
static constexpr int TC_KC = 64;                      // constraints per G' chunk (MMA K; 48 took 13 chunks at p = 600)
static constexpr unsigned long long kTcWaitNs = 2000000000ull;

struct TcArgs {
  int n, p, B, NPAD, NC, ntiles, nchG, nchGT;
  const uint4 *Qhi, *Qlo, *Ghi, *Glo, *GThi, *GTlo;   // packed K-major bf16 hi/lo
  const float* Qf;                                   // FP32 Q (n x n) for F(u)
  const float *qT, *gT;                              // instance-minor inputs
  const float *lb, *ub;                              // n (shared box)
  const float *x0T, *lam0T;                          // warm start, instance-minor (nullable)
  float *lam, *lamp, *mu, *usum, *save;              // instance-minor workspace
  float *xlT, *xaT, *xsT;                            // instance-minor outputs
  DevResult* res;
  float L, alpha;
  float sigma, beta_sigma, eps_in, eps_out;
  int cone, kd_plus, fast, want_last, want_avg;
  int inner_fixed, inner_check_every, max_inner, outer_fixed, max_outer, check_every;
  int* next;                                         // tile queue
  int* err;                                          // set when a bounded wait gave up
};

// Instance-minor index: element e of lane l in tile t.
__device__ __forceinline__ size_t im(int t, int E, int e, int l) { return ((size_t)t * E + e) * TM + l; }

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

__device__ __forceinline__ void kahan(float& s, float& c, float v) {
  const float y = v - c, t = s + y;
  c = (t - s) - y;
  s = t;
}

// Per-block state of the pipeline (uniform across the block's threads).  The
// block has 256 threads: thread (half h, lane l) works on TMEM lane l, columns
// 8h..8h+7 of every 16-column group (warps 4..7 reach the same TMEM lane
// quadrants as warps 0..3), so each lane's epilogue is split over two threads.
static constexpr int TC_THREADS = 2 * TM;

struct TcCtx {
  const TcArgs* a;
  uint8_t *Qh, *Ql, *Ah, *Al;
  uint8_t* B0;                  // chunk buffers: buffer b hi at B0 + 2 b bb, lo at B0 + (2 b + 1) bb
  size_t ab, bb;                // bytes of one operand half (hi or lo); of one chunk half
  float *lb, *ub;
  float* red;                   // [4][2][TM] per-lane partial sums of the two halves
  uint64_t *bar_mma, *bar_tx;   // [2] each
  uint32_t ph_mma, ph_tx;       // phase bit of barrier b at bit b
  uint32_t tm, lane_off;
  uint32_t rD, rY, rX, rC;       // TMEM column regions
  int tid, lane, half, NPAD;
  bool ok;

  __device__ void sync_async() {  // operand writes visible to the tensor core, TMEM ops ordered
    tc::tmem_st_wait();
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  // The two halves' partial sums of up to four per-lane values, added in half order.
  __device__ void combine(float (&v)[4], int cnt) {
    for (int i = 0; i < cnt; ++i) red[(i * 2 + half) * TM + lane] = v[i];
    __syncthreads();
    for (int i = 0; i < cnt; ++i) v[i] = red[(i * 2) * TM + lane] + red[(i * 2 + 1) * TM + lane];
    __syncthreads();
  }
  __device__ __forceinline__ uint8_t* Bh(int b) const { return B0 + (size_t)(2 * b) * bb; }
  __device__ __forceinline__ uint8_t* Bl(int b) const { return B0 + (size_t)(2 * b + 1) * bb; }
  __device__ __forceinline__ void wait_mma(int b) {
    ok = tc::mbar_wait(&bar_mma[b], (ph_mma >> b) & 1u, kTcWaitNs) && ok;
    ph_mma ^= 1u << b;
    tc::fence_after();
  }
  __device__ __forceinline__ void wait_tx(int b) {
    ok = tc::mbar_wait(&bar_tx[b], (ph_tx >> b) & 1u, kTcWaitNs) && ok;
    ph_tx ^= 1u << b;
  }
  __device__ __forceinline__ void issue_B(int b, const uint4* hi, const uint4* lo, uint32_t bytes) {  // thread 0
    tc::mbar_expect_tx(&bar_tx[b], 2 * bytes);
    tc::bulk_g2s(Bh(b), hi, bytes, &bar_tx[b]);
    tc::bulk_g2s(Bl(b), lo, bytes, &bar_tx[b]);
  }
  // D region = Q * operand (operand already written and synced by the caller)
  __device__ void mma_Q() {
    if (tid == 0) {
      tc_mma_tile(tm + rD, Ah, Al, Qh, Ql, NPAD, NPAD, false);
      tc::mma_commit(&bar_mma[0]);
    }
    wait_mma(0);
  }
  // this thread's 8 columns of group c0 of region r
  __device__ __forceinline__ void ld8(uint32_t r, int c0, uint32_t (&v)[8]) const {
    tc::tmem_ld8(tm + lane_off + r + c0 + 8 * half, v);
  }
  __device__ __forceinline__ void st8(uint32_t r, int c0, const uint32_t (&v)[8]) const {
    tc::tmem_st8(tm + lane_off + r + c0 + 8 * half, v);
  }
  // operand <- TMEM region r
  __device__ void operand_from(uint32_t r) {
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t v[8];
      ld8(r, c0, v);
      tc::tmem_ld_wait();
      float f[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) f[i] = __uint_as_float(v[i]);
      put8(Ah, Al, lane, c0 + 8 * half, f);
    }
  }
  // region dst <- region src
  __device__ void region_copy(uint32_t dst, uint32_t src) {
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t v[8];
      ld8(src, c0, v);
      tc::tmem_ld_wait();
      st8(dst, c0, v);
    }
  }

  // Chunked product G * operand (N = NC rows of G per chunk) into two
  // alternating accumulator slots (regions D and Y); epi(ch, slot) consumes
  // chunk ch.  Bulk copies of chunk ch+1 overlap the product of chunk ch.
  template <class Epi>
  __device__ void g_product(Epi epi) {
    const TcArgs& A = *a;
    const int nch = A.nchG;
    if (nch == 0) return;
    const uint32_t cb = (uint32_t)A.NC * NPAD * 2;  // bytes of one packed chunk (hi or lo)
    const uint32_t sdelta = rY - rD;                // accumulator slot b at rD + b * sdelta
    if (tid == 0) {
      issue_B(0, A.Ghi, A.Glo, cb);
      if (nch > 1) issue_B(1, A.Ghi + cb / 16, A.Glo + cb / 16, cb);
    }
    for (int ch = 0; ch < nch; ++ch) {
      const int b = ch & 1;
      wait_tx(b);
      if (tid == 0) {
        tc_mma_tile(tm + rD + b * sdelta, Ah, Al, Bh(b), Bl(b), A.NC, NPAD, false);
        tc::mma_commit(&bar_mma[b]);
      }
      if (ch >= 1) {
        wait_mma(b ^ 1);  // chunk ch-1: its buffer and accumulator slot are ready
        if (tid == 0 && ch + 1 < nch)
          issue_B(b ^ 1, A.Ghi + (size_t)(ch + 1) * cb / 16, A.Glo + (size_t)(ch + 1) * cb / 16, cb);
        epi(ch - 1, rD + (b ^ 1) * sdelta);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
      }
    }
    wait_mma((nch - 1) & 1);
    epi(nch - 1, rD + ((nch - 1) & 1) * sdelta);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }

  // c = q + G' m into region C, m instance-minor ([p][128] of this tile).
  // The A operand of each K-chunk (m split into bf16 hi/lo) is built by the
  // threads into a double buffer carved from the operand area.
  __device__ void gt_product(int tile, const float* m) {
    const TcArgs& A = *a;
    const int nch = A.nchGT, p = A.p;
    const uint32_t cb = (uint32_t)NPAD * TC_KC * 2;
    const size_t abytes = (size_t)TM * TC_KC * 2;  // chunk b: hi at Ah + 2 b abytes, lo next
    auto AH = [&](int b) { return Ah + (size_t)(2 * b) * abytes; };
    auto AL = [&](int b) { return Ah + (size_t)(2 * b + 1) * abytes; };
    auto build = [&](int ch, int b) {  // this half's 3 groups of 8: every load in flight before the stores
      const int j0 = ch * TC_KC;
      float v[TC_KC / 2];
#pragma unroll
      for (int g = 0; g < TC_KC / 16; ++g)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = j0 + 16 * g + 8 * half + i;
          v[8 * g + i] = j < p ? __ldcg(m + im(tile, p, j, lane)) : 0.f;
        }
#pragma unroll
      for (int g = 0; g < TC_KC / 16; ++g) put8(AH(b), AL(b), lane, 16 * g + 8 * half, v + 8 * g);
    };
    if (nch > 0) {
      build(0, 0);
      if (tid == 0) {
        issue_B(0, A.GThi, A.GTlo, cb);
        if (nch > 1) issue_B(1, A.GThi + cb / 16, A.GTlo + cb / 16, cb);
      }
      for (int ch = 0; ch < nch; ++ch) {
        const int b = ch & 1;
        sync_async();  // A chunk ch written by every thread
        wait_tx(b);
        if (tid == 0) {
          tc_mma_tile(tm + rC, AH(b), AL(b), Bh(b), Bl(b), NPAD, TC_KC, ch > 0);
          tc::mma_commit(&bar_mma[b]);
        }
        if (ch >= 1) {
          wait_mma(b ^ 1);  // product ch-1 done: buffers b^1 free
          if (tid == 0 && ch + 1 < nch)
            issue_B(b ^ 1, A.GThi + (size_t)(ch + 1) * cb / 16, A.GTlo + (size_t)(ch + 1) * cb / 16, cb);
        }
        if (ch + 1 < nch) build(ch + 1, b ^ 1);
      }
      wait_mma((nch - 1) & 1);
    }
    // c = acc + q
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t v[8];
      if (nch > 0) {
        ld8(rC, c0, v);
        tc::tmem_ld_wait();
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0u;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int col = c0 + 8 * half + i;
        const float qv = col < A.n ? A.qT[im(tile, A.n, col, lane)] : 0.f;
        v[i] = __float_as_uint(__uint_as_float(v[i]) + qv);
      }
      st8(rC, c0, v);
    }
    sync_async();
  }
};

// Algorithm FOM on L(., m) for every lane of the tile, from x = region X
// (warm start) with c = q + G' m in region C.  On return X = ubar, D = Q ubar,
// the operand holds ubar, and cert_out / kin_out hold the lane's final
// certificate and iteration count.  Lanes with active == false keep x.
__device__ __forceinline__ void tc_inner(TcCtx& C, bool active, float& cert_out, int& kin_out) {
  const TcArgs& A = *C.a;
  const int NPAD = C.NPAD, h8 = 8 * C.half;
  const float L = A.L;
  // the step 1/L as a multiplier: a correctly rounded FP32 division is about ten
  // instructions, and the epilogue takes 56 of them per thread per iteration at n = 100
  const float invL = 1.0f / L;
  // y^0 = x^0; D = Q x^0
  C.region_copy(C.rY, C.rX);
  C.operand_from(C.rX);
  C.sync_async();
  C.mma_Q();
  const bool fgm_sigma = A.sigma > 0.f;
  const float kap = A.sigma > 0.f ? 0.5f / A.sigma - 0.5f / L : 0.f;
  const int m = A.inner_check_every > 0 ? A.inner_check_every : 1;
  const int kmax = A.inner_fixed > 0 ? A.inner_fixed : A.max_inner;
  double th = 1.0;
  bool done = !active;
  int kin = 0;
  float cert = 0.f;
  for (int k = 1;; ++k) {
    const bool check = A.inner_fixed > 0 ? (k >= A.inner_fixed) : (k % m == 0 || k >= kmax);
    // weight of the next extrapolation (GM/FGM/FGM_sigma rules, Sec. 2.1)
    float beta;
    if (fgm_sigma) {
      beta = A.beta_sigma;
    } else {
      const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * th * th));
      beta = (float)((th - 1.0) / t1);
      th = t1;
    }
    // x^k = [y - (Q y + c)/L]_U,  y^k = x^k + beta (x^k - x^{k-1})
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t d[8], y[8], x[8], c[8];
      C.ld8(C.rD, c0, d);
      C.ld8(C.rY, c0, y);
      C.ld8(C.rX, c0, x);
      C.ld8(C.rC, c0, c);
      tc::tmem_ld_wait();
      uint32_t xn[8], yn[8];
      float op[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float yv = __uint_as_float(y[i]), xv = __uint_as_float(x[i]);
        const float s = yv - (__uint_as_float(d[i]) + __uint_as_float(c[i])) * invL;
        const float lo = C.lb[c0 + h8 + i], hi = C.ub[c0 + h8 + i];
        float xnew = s < lo ? lo : (s > hi ? hi : s);
        float ynew = xnew + beta * (xnew - xv);
        if (done) {
          xnew = xv;
          ynew = xv;
        }
        xn[i] = __float_as_uint(xnew);
        yn[i] = __float_as_uint(ynew);
        op[i] = check ? xnew : ynew;
      }
      C.st8(C.rX, c0, xn);
      C.st8(C.rY, c0, yn);
      put8(C.Ah, C.Al, C.lane, c0 + h8, op);
    }
    C.sync_async();
    C.mma_Q();
    if (__syncthreads_or(!C.ok)) break;  // a bounded wait gave up: leave with the error flag set
    if (!check) continue;
    // D = Q x^k: certificate of eq. duquad_in (gradient-mapping bound, or the
    // Frank-Wolfe gap when sigma = 0), compensated FP32 sums of the two halves
    float cs = 0.f, cc = 0.f;
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t d[8], x[8], c[8];
      C.ld8(C.rD, c0, d);
      C.ld8(C.rX, c0, x);
      C.ld8(C.rC, c0, c);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int col = c0 + h8 + i;
        if (col >= A.n) continue;
        const float gd = __uint_as_float(d[i]) + __uint_as_float(c[i]), xv = __uint_as_float(x[i]);
        const float lo = C.lb[col], hi = C.ub[col];
        if (fgm_sigma) {
          const float xp = fminf(fmaxf(xv - gd * invL, lo), hi);
          const float dd = xv - xp;
          kahan(cs, cc, gd * dd + (L * dd) * (L * dd) * kap);
        } else {
          const float u1 = gd * lo, u2 = gd * hi;
          kahan(cs, cc, gd * xv - (u1 < u2 ? u1 : u2));
        }
      }
    }
    float tot[4] = {cs - cc, 0.f, 0.f, 0.f};
    C.combine(tot, 1);
    const float cv = tot[0];
    const bool stop = A.inner_fixed > 0 || cv <= A.eps_in || k >= kmax;
    if (stop && !done) {
      done = true;
      kin = k;
      cert = cv;
    }
    if (__syncthreads_and(done)) break;
    // continue: frozen lanes present x (y = x), the others y^k
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t y[8], x[8];
      C.ld8(C.rY, c0, y);
      C.ld8(C.rX, c0, x);
      tc::tmem_ld_wait();
      float op[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (done) y[i] = x[i];
        op[i] = __uint_as_float(y[i]);
      }
      C.st8(C.rY, c0, y);
      put8(C.Ah, C.Al, C.lane, c0 + h8, op);
    }
    C.sync_async();
    C.mma_Q();
  }
  cert_out = cert;
  kin_out = active ? kin : 0;
}

// F(x) = x'Qx/2 + q'x of the lane's x (TMEM region rx), FP32 from the FP32 Q:
// Q is staged in the bulk-copy buffers and every lane's x in the operand area
// (instance-minor, conflict-free), both free at this point.  Rows alternate
// between the two halves; row sums use four accumulators over the upper
// triangle, rows are added with Kahan, and the halves are combined in order.
__device__ __forceinline__ float tc_F(TcCtx& C, int tile, uint32_t rx) {
  const TcArgs& A = *C.a;
  const int n = A.n, lane = C.lane;
  float* Xs = (float*)C.Ah;
  float* Qs = (float*)C.B0;
  {  // Q into shared memory, eight loads in flight per thread before the stores
    const int nn = n * n;
    for (int e0 = C.tid; e0 < nn; e0 += 8 * TC_THREADS) {
      float t8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t8[u] = e0 + u * TC_THREADS < nn ? __ldg(A.Qf + e0 + u * TC_THREADS) : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e0 + u * TC_THREADS < nn) Qs[e0 + u * TC_THREADS] = t8[u];
    }
  }
  for (int c0 = 0; c0 < C.NPAD; c0 += 16) {
    uint32_t x[8];
    C.ld8(rx, c0, x);
    tc::tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int col = c0 + 8 * C.half + i;
      if (col < n) Xs[col * TM + lane] = __uint_as_float(x[i]);
    }
  }
  __syncthreads();
  float s = 0.f, c = 0.f;
  for (int i = C.half; i < n; i += 2) {
    const float* Qr = Qs + (size_t)i * n;
    const float xi = Xs[i * TM + lane];
    float a0 = 0.5f * Qr[i] * xi, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int k = i + 1;
    for (; k + 4 <= n; k += 4) {
      a0 = fmaf(Qr[k], Xs[k * TM + lane], a0);
      a1 = fmaf(Qr[k + 1], Xs[(k + 1) * TM + lane], a1);
      a2 = fmaf(Qr[k + 2], Xs[(k + 2) * TM + lane], a2);
      a3 = fmaf(Qr[k + 3], Xs[(k + 3) * TM + lane], a3);
    }
    for (; k < n; ++k) a0 = fmaf(Qr[k], Xs[k * TM + lane], a0);
    kahan(s, c, xi * (((a0 + a1) + (a2 + a3)) + A.qT[im(tile, n, i, lane)]));
  }
  float v[4] = {s - c, 0.f, 0.f, 0.f};
  C.combine(v, 1);  // also orders the shared-memory reads before the buffers' next use
  return v[0];
}

// dist_K(Gx + g)^2 and sum_j m_j (Gx + g)_j for the operand x (m nullable);
// neg is set when some m_j < 0.
__device__ __forceinline__ void tc_resid(TcCtx& C, int tile, const float* m, float& inf2, float& lag, int& neg) {
  const TcArgs& A = *C.a;
  float is = 0.f, ic = 0.f, ls = 0.f, lc = 0.f;
  float ng = 0.f;
  C.g_product([&](int ch, uint32_t slot) {
    const int j0 = ch * A.NC;
    for (int c0 = 0; c0 < A.NC; c0 += 16) {
      uint32_t r[8];
      C.ld8(slot, c0, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = j0 + c0 + 8 * C.half + i;
        if (j >= A.p) continue;
        const float rv = __uint_as_float(r[i]) + A.gT[im(tile, A.p, j, C.lane)];
        const float dk = rv - proj_K(A.cone, rv);
        kahan(is, ic, dk * dk);
        if (m) {
          const float mj = m[im(tile, A.p, j, C.lane)];
          if (mj < 0.f) ng = 1.f;
          kahan(ls, lc, mj * rv);
        }
      }
    }
  });
  float v[4] = {is - ic, ls - lc, ng, 0.f};
  C.combine(v, 3);
  inf2 = v[0];
  lag = v[1];
  neg = v[2] > 0.f;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_solve(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar_mma[2], bar_tx[2], bar_q;
  __shared__ float s_red[4 * 2 * TM];
  __shared__ uint32_t s_taddr;
  __shared__ int s_tile;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int NPAD = a.NPAD, n = a.n, p = a.p;
  TcCtx C;
  C.a = &a;
  C.tid = tid;
  C.lane = tid & (TM - 1);
  C.half = tid / TM;
  C.NPAD = NPAD;
  C.ok = true;
  C.red = s_red;
  const int lane = C.lane, half = C.half, h8 = 8 * half;
  size_t off = 0;
  auto take = [&](size_t b) {
    uint8_t* r = sm + off;
    off += (b + 127) & ~size_t(127);
    return r;
  };
  const size_t qb = (size_t)NPAD * NPAD * 2;
  C.Qh = take(qb);
  C.Ql = take(qb);
  // operand area: [hi | lo] of the 128 x NPAD operand; also the G' mu chunk
  // double buffer (4 x 128 x KC bf16) and the FP32 x of every lane (tc_F)
  C.ab = std::max((size_t)TM * NPAD * 2, (size_t)2 * TM * TC_KC * 2);
  C.Ah = take(2 * C.ab);
  C.Al = C.Ah + C.ab;
  // bulk-copy chunk buffers, contiguous; also the FP32 Q (tc_F)
  C.bb = (std::max(std::max((size_t)a.NC * NPAD * 2, (size_t)NPAD * TC_KC * 2), (size_t)NPAD * NPAD) + 127) &
         ~size_t(127);
  C.B0 = take(4 * C.bb);
  C.lb = (float*)take((size_t)NPAD * 4);
  C.ub = (float*)take((size_t)NPAD * 4);
  for (int i = tid; i < NPAD; i += TC_THREADS) {
    C.lb[i] = i < n ? a.lb[i] : 0.f;
    C.ub[i] = i < n ? a.ub[i] : 0.f;
  }
  C.bar_mma = bar_mma;
  C.bar_tx = bar_tx;
  C.ph_mma = 0;
  C.ph_tx = 0;
  if (tid == 0) {
    tc::mbar_init(&bar_mma[0], 1);
    tc::mbar_init(&bar_mma[1], 1);
    tc::mbar_init(&bar_tx[0], 1);
    tc::mbar_init(&bar_tx[1], 1);
    tc::mbar_init(&bar_q, 1);
    tc::mbar_init_fence();
  }
  __syncthreads();
  if (warp == 0) {
    tc::tmem_alloc(&s_taddr, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {  // Q operand (hi/lo) once per block
    tc::mbar_expect_tx(&bar_q, 2 * (uint32_t)qb);
    tc::bulk_g2s(C.Qh, a.Qhi, (uint32_t)qb, &bar_q);
    tc::bulk_g2s(C.Ql, a.Qlo, (uint32_t)qb, &bar_q);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  C.ok = tc::mbar_wait(&bar_q, 0, kTcWaitNs);
  C.tm = s_taddr;
  C.lane_off = (uint32_t)((warp & 3) * 32) << 16;
  C.rD = 0;
  C.rY = NPAD;
  C.rX = 2 * NPAD;
  C.rC = 3 * NPAD;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.next, 1);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= a.ntiles || !C.ok) break;
    const int b = tile * TM + lane;
    const bool valid = b < a.B;
    // ---- x^0 = warm start or [0]_U; lambda^0 = mu^1 = warm start or 0
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int col = c0 + h8 + i;
        float x = 0.f;
        if (col < n) x = (valid && a.x0T) ? a.x0T[im(tile, n, col, lane)] : fminf(fmaxf(0.f, C.lb[col]), C.ub[col]);
        v[i] = __float_as_uint(x);
      }
      C.st8(C.rX, c0, v);
    }
    for (int j0 = 16 * half; j0 < p; j0 += 32) {
      float l0[16];
#pragma unroll
      for (int i = 0; i < 16; ++i)
        l0[i] = (valid && a.lam0T && j0 + i < p) ? __ldg(a.lam0T + im(tile, p, j0 + i, lane)) : 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (j0 + i >= p) continue;
        const size_t ix = im(tile, p, j0 + i, lane);
        a.lam[ix] = l0[i];
        a.lamp[ix] = l0[i];
        a.mu[ix] = l0[i];
      }
    }
    for (int i = half; i < n; i += 2) a.usum[im(tile, n, i, lane)] = 0.f;
    C.sync_async();
    C.gt_product(tile, a.mu);  // c = q + G' mu^1

    bool act = valid;
    double theta = 1.0, S = 0.0;
    long long kin_tot = 0;
    int conv_l = 0, conv_a = 0, status = ST_NOT_CONVERGED, kout = 0;
    float d_lb = -INFINITY, f_l = NAN, i_l = NAN, f_a = NAN, i_a = NAN;
    const int kmax = a.outer_fixed > 0 ? a.outer_fixed : a.max_outer;
    for (int k = 1; k <= kmax && C.ok; ++k) {
      if (!__syncthreads_or(act)) break;
      const bool eval = a.outer_fixed > 0 ? (k == kmax) : (k % a.check_every == 0 || k == kmax);
      // Step 1: ubar^k = FOM(L(., mu^k), U) from ubar^{k-1}
      float cert_u;
      int kin;
      tc_inner(C, act, cert_u, kin);
      kin_tot += kin;
      // Step 2: lambda^k = [mu^k + (G ubar + g)/(2 L_d)]_{K_d}; Step 3: mu^{k+1}
      double beta = 0.0, th_next = theta;
      if (a.fast) {
        th_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
        beta = (theta - 1.0) / th_next;
      }
      float is = 0.f, ic = 0.f, ls = 0.f, lc = 0.f, mneg = 0.f;
      C.g_product([&](int ch, uint32_t slot) {
        const int j0 = ch * a.NC;
        for (int c0 = 0; c0 < a.NC; c0 += 16) {
          uint32_t r[8];
          C.ld8(slot, c0, r);
          tc::tmem_ld_wait();
          if (!act) continue;
          // every load of this thread's 8 columns is issued before the first store
          float gv[8], mv[8], lv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int j = j0 + c0 + h8 + i;
            const size_t ix = im(tile, p, j < p ? j : 0, lane);
            gv[i] = __ldcg(a.gT + ix);
            mv[i] = __ldcg(a.mu + ix);
            lv[i] = __ldcg(a.lam + ix);
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int j = j0 + c0 + h8 + i;
            if (j >= p) continue;
            const size_t ix = im(tile, p, j, lane);
            const float rv = __uint_as_float(r[i]) + gv[i];
            const float muj = mv[i], lold = lv[i];
            if (eval) {
              kahan(ls, lc, muj * rv);
              if (muj < 0.f) mneg = 1.f;
              const float dk = rv - proj_K(a.cone, rv);
              kahan(is, ic, dk * dk);
            }
            const float ln = proj_Kd(a.cone, a.kd_plus != 0, muj + a.alpha * rv);
            a.lamp[ix] = lold;
            a.lam[ix] = ln;
            a.mu[ix] = ln + (float)beta * (ln - lold);
          }
        }
      });
      // averaging weight theta_k (eq. average_primal)
      for (int c0 = 0; c0 < NPAD; c0 += 16) {
        uint32_t x[8];
        C.ld8(C.rX, c0, x);
        tc::tmem_ld_wait();
        if (!act) continue;
        float us[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) us[i] = c0 + h8 + i < n ? __ldcg(a.usum + im(tile, n, c0 + h8 + i, lane)) : 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (c0 + h8 + i < n) a.usum[im(tile, n, c0 + h8 + i, lane)] = us[i] + (float)theta * __uint_as_float(x[i]);
      }
      if (act) {
        S += theta;
        theta = th_next;
        kout = k;
      }
      if (eval) {
        float ev[4] = {ls - lc, is - ic, mneg, 0.f};
        C.combine(ev, 3);
        // lower bound from (ubar^k, mu^k) when mu^k is a valid multiplier
        const float Fu = tc_F(C, tile, C.rX);
        if (act && (a.cone == CONE_EQ || !(ev[2] > 0.f))) d_lb = fmaxf(d_lb, Fu + ev[0] - cert_u);
        float fl = Fu, il = sqrtf(fmaxf(ev[1], 0.f));
        // save ubar (the warm-start chain continues from it)
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
          uint32_t x[8];
          C.ld8(C.rX, c0, x);
          tc::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (c0 + h8 + i < n) a.save[im(tile, n, c0 + h8 + i, lane)] = __uint_as_float(x[i]);
        }
        if (a.want_last) {
          if (a.fast) {  // ubar(lambda^k): extra inner solve at lambda^k from ubar^k
            C.gt_product(tile, a.lam);
            float cert_l;
            int kin_l;
            tc_inner(C, act, cert_l, kin_l);
            kin_tot += kin_l;
            float inf2, lag;
            int lneg;
            tc_resid(C, tile, a.lam, inf2, lag, lneg);
            fl = tc_F(C, tile, C.rX);
            il = sqrtf(fmaxf(inf2, 0.f));
            if (act && (a.cone == CONE_EQ || !lneg)) d_lb = fmaxf(d_lb, fl + lag - cert_l);
          }
          for (int c0 = 0; c0 < NPAD; c0 += 16) {
            uint32_t x[8];
            C.ld8(C.rX, c0, x);
            tc::tmem_ld_wait();
            if (!act) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (c0 + h8 + i < n) a.xlT[im(tile, n, c0 + h8 + i, lane)] = __uint_as_float(x[i]);
          }
          if (act) {
            f_l = fl;
            i_l = il;
          }
        }
        if (a.want_avg) {  // x_avg = usum / S, evaluated in region X
          // one FP64 division per lane, then FP32 products (an FP64 division per element
          // ran on the slow FP64 pipe)
          const float invS = S > 0.0 ? (float)(1.0 / S) : 0.f;
          for (int c0 = 0; c0 < NPAD; c0 += 16) {
            uint32_t v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int col = c0 + h8 + i;
              v[i] = __float_as_uint(col < n ? a.usum[im(tile, n, col, lane)] * invS : 0.f);
            }
            C.st8(C.rX, c0, v);
          }
          tc::tmem_st_wait();
          C.operand_from(C.rX);
          C.sync_async();
          float inf2, lag;
          int dummy;
          tc_resid(C, tile, nullptr, inf2, lag, dummy);
          const float fa = tc_F(C, tile, C.rX);
          if (act) {
            f_a = fa;
            i_a = sqrtf(fmaxf(inf2, 0.f));
            for (int i0 = 16 * half; i0 < n; i0 += 32) {
              float us[16];
#pragma unroll
              for (int i = 0; i < 16; ++i) us[i] = i0 + i < n ? __ldcg(a.usum + im(tile, n, i0 + i, lane)) : 0.f;
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (i0 + i < n) a.xaT[im(tile, n, i0 + i, lane)] = us[i] * invS;
            }
          }
        }
        // restore ubar into region X
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
          uint32_t v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int col = c0 + h8 + i;
            v[i] = __float_as_uint(col < n ? a.save[im(tile, n, col, lane)] : 0.f);
          }
          C.st8(C.rX, c0, v);
        }
        C.sync_async();
        if (act) {
          if ((a.want_last && !(isfinite(f_l) && isfinite(i_l))) || (a.want_avg && !(isfinite(f_a) && isfinite(i_a)))) {
            status = ST_NONFINITE;
            act = false;
          } else if (a.outer_fixed <= 0) {
            conv_l = a.want_last && i_l <= a.eps_out && f_l - d_lb <= a.eps_out;
            conv_a = a.want_avg && i_a <= a.eps_out && f_a - d_lb <= a.eps_out;
            if (conv_l || conv_a) {
              status = ST_OK;
              act = false;
            }
          }
        }
      }
      // next c = q + G' mu^{k+1}
      if (__syncthreads_or(act)) C.gt_product(tile, a.mu);
    }
    // ---- per-lane results and warm-start state
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      uint32_t x[8];
      C.ld8(C.rX, c0, x);
      tc::tmem_ld_wait();
      if (!valid) continue;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (c0 + h8 + i < n) a.xsT[im(tile, n, c0 + h8 + i, lane)] = __uint_as_float(x[i]);
    }
    if (valid && half == 0) {
      if (a.outer_fixed > 0 && status == ST_NOT_CONVERGED) status = ST_OK;
      DevResult r;
      r.status = status;
      r.outer_iters = kout;
      r.inner_iters = kin_tot;
      r.converged_last = conv_l;
      r.converged_avg = conv_a;
      r.f_last = f_l;
      r.infeas_last = i_l;
      r.f_avg = f_a;
      r.infeas_avg = i_a;
      r.d_lb = d_lb;
      a.res[b] = r;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (!C.ok && tid == 0) atomicExch(a.err, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(C.tm, 512);
}

// Row-major [B][E] -> instance-minor [tile][E][128] (zero for lanes past B).
__global__ void k_to_minor(const float* __restrict__ src, int B, int E, int ntiles, float* __restrict__ dst) {
  const size_t total = (size_t)ntiles * E * TM;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(k % TM);
    const size_t te = k / TM;
    const int e = (int)(te % E), t = (int)(te / E);
    const int b = t * TM + l;
    dst[k] = b < B ? src[(size_t)b * E + e] : 0.f;
  }
}
// Instance-minor -> row-major [B][E].
__global__ void k_from_minor(const float* __restrict__ src, int B, int E, float* __restrict__ dst) {
  const size_t total = (size_t)B * E;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(k / E), e = (int)(k % E);
    dst[k] = src[im(b / TM, E, e, b % TM)];
  }
}

struct TcWs {
  int NPAD = 0, NC = 0, ntiles = 0, nchG = 0, nchGT = 0;
  void* mem = nullptr;
  uint4 *Qhi, *Qlo, *Ghi, *Glo, *GThi, *GTlo;
  float *qT, *gT, *x0T, *lam0T, *lam, *lamp, *mu, *usum, *save, *xlT, *xaT, *xsT, *tmp;
  int *next, *err;
  DevResult* res;
  bool packed = false;
};

void tc_free(TcWs* w) {
  if (!w) return;
  if (w->mem) cudaFree(w->mem);
  delete w;
}

static size_t tc_smem_bytes(const TcWs* W) {
  auto r128 = [](size_t b) { return (b + 127) & ~size_t(127); };
  const size_t qb = (size_t)W->NPAD * W->NPAD * 2;
  const size_t ab = std::max((size_t)TM * W->NPAD * 2, (size_t)2 * TM * TC_KC * 2);
  const size_t bb = r128(std::max(std::max((size_t)W->NC * W->NPAD * 2, (size_t)W->NPAD * TC_KC * 2),
                                  (size_t)W->NPAD * W->NPAD));
  return 2 * r128(qb) + r128(2 * ab) + 4 * bb + 2 * r128((size_t)W->NPAD * 4) + 128;
}

static dq_status tc_ws(dq_problem* P, TcWs** out) {
  if (P->tws) {
    *out = P->tws;
    return DQ_OK;
  }
  TcWs* W = new TcWs();
  const int n = P->n, p = P->p, B = P->batch;
  W->NPAD = (n + 15) / 16 * 16;
  // G rows per chunk of the G ubar product: as many as shared memory allows (at most
  // NPAD, the accumulator slot's width): fewer chunks, each a bulk copy, an MMA and an
  // epilogue on the serial chain of every outer iteration (112 at n = 100: 6 chunks
  // instead of 10 for p = 600).  The chunking does not change any sum.
  W->NC = W->NPAD;
  const size_t smem_lim = max_dynamic_smem((const void*)k_tc_solve, P->ctx->smem_optin);
  while (W->NC > 16 && tc_smem_bytes(W) > smem_lim) W->NC -= 16;
  W->ntiles = (B + TM - 1) / TM;
  W->nchG = (p + W->NC - 1) / W->NC;
  W->nchGT = (p + TC_KC - 1) / TC_KC;
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t qb = (size_t)W->NPAD * W->NPAD * 2, gb = (size_t)W->nchG * W->NC * W->NPAD * 2,
               gtb = (size_t)W->nchGT * W->NPAD * TC_KC * 2;
  const size_t vn = (size_t)W->ntiles * TM * n * 4, vp = (size_t)W->ntiles * TM * std::max(p, 1) * 4;
  const size_t total = 2 * a256(qb) + 2 * a256(gb) + 2 * a256(gtb) + 8 * a256(vn) + 5 * a256(vp) +
                       a256(std::max(vn, vp)) + a256((size_t)B * sizeof(DevResult)) + 256;
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
  W->qT = (float*)take(vn); W->x0T = (float*)take(vn); W->usum = (float*)take(vn); W->save = (float*)take(vn);
  W->xlT = (float*)take(vn); W->xaT = (float*)take(vn); W->xsT = (float*)take(vn);
  W->gT = (float*)take(vp); W->lam0T = (float*)take(vp); W->lam = (float*)take(vp); W->lamp = (float*)take(vp);
  W->mu = (float*)take(vp);
  W->tmp = (float*)take(std::max(vn, vp));
  float* spare = (float*)take(vn);
  (void)spare;
  W->res = (DevResult*)take((size_t)B * sizeof(DevResult));
  W->next = (int*)take(256);
  W->err = W->next + 16;
  P->tws = W;
  *out = W;
  return DQ_OK;
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
  if (c.stop_fstar) {
    set_error("the tensor-core engine stops on the certificate only (no stop_fstar)");
    return DQ_ERR_INVALID;
  }
  const int n = P->n, p = P->p, B = P->batch;
  if ((n + 15) / 16 * 16 > 128) {
    set_error("the tensor-core engine holds n <= 128 variables per instance in tensor memory (n = %d)", n);
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
  const int NPAD = W->NPAD;
  if (!W->packed) {
    k_pack_kmajor<<<64, 256, 0, st>>>((const float*)P->Q, n, n, n, NPAD, NPAD, W->Qhi, W->Qlo);
    for (int ch = 0; ch < W->nchG; ++ch) {
      const size_t o = (size_t)ch * W->NC * NPAD * 2 / 16;
      k_pack_kmajor<<<64, 256, 0, st>>>((const float*)P->G + (size_t)ch * W->NC * n, std::min(W->NC, p - ch * W->NC), n,
                                        n, W->NC, NPAD, W->Ghi + o, W->Glo + o);
    }
    for (int ch = 0; ch < W->nchGT; ++ch) {
      const size_t o = (size_t)ch * NPAD * TC_KC * 2 / 16;
      k_pack_kmajor<<<64, 256, 0, st>>>((const float*)P->GT + (size_t)ch * TC_KC, n, std::min(TC_KC, p - ch * TC_KC),
                                        p, NPAD, TC_KC, W->GThi + o, W->GTlo + o);
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
  const int tg = std::max(1, std::min(4 * ctx->num_sms, (int)(((size_t)W->ntiles * TM * std::max(n, p) + 255) / 256)));
  k_to_minor<<<tg, 256, 0, st>>>((const float*)P->q, B, n, W->ntiles, W->qT);
  ++ctx->launches;
  if (p) {
    k_to_minor<<<tg, 256, 0, st>>>((const float*)P->g, B, p, W->ntiles, W->gT);
    ++ctx->launches;
  }
  if (warm) {
    k_to_minor<<<tg, 256, 0, st>>>((const float*)P->x_state, B, n, W->ntiles, W->x0T);
    ++ctx->launches;
    if (p) {
      k_to_minor<<<tg, 256, 0, st>>>((const float*)P->lam_state, B, p, W->ntiles, W->lam0T);
      ++ctx->launches;
    }
  }
  DQ_CK(cudaMemsetAsync(W->next, 0, 256, st));
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n; a.p = p; a.B = B; a.NPAD = NPAD; a.NC = W->NC; a.ntiles = W->ntiles; a.nchG = W->nchG; a.nchGT = W->nchGT;
  a.Qhi = W->Qhi; a.Qlo = W->Qlo; a.Ghi = W->Ghi; a.Glo = W->Glo; a.GThi = W->GThi; a.GTlo = W->GTlo;
  a.Qf = (const float*)P->Q;
  a.qT = W->qT; a.gT = W->gT; a.lb = (const float*)P->lb; a.ub = (const float*)P->ub;
  a.x0T = warm ? W->x0T : nullptr; a.lam0T = (warm && p) ? W->lam0T : nullptr;
  a.lam = W->lam; a.lamp = W->lamp; a.mu = W->mu; a.usum = W->usum; a.save = W->save;
  a.xlT = W->xlT; a.xaT = W->xaT; a.xsT = W->xsT; a.res = W->res;
  a.L = (float)LL; a.alpha = (float)(1.0 / (2.0 * Ld)); a.sigma = (float)sigma;
  a.beta_sigma = sigma > 0 ? (float)((sqrt(LL) - sqrt(sigma)) / (sqrt(LL) + sqrt(sigma))) : 0.f;
  a.eps_in = (float)eps_in; a.eps_out = (float)c.eps_out;
  a.cone = P->cone; a.kd_plus = !(c.kd_literal && !(lmin > 0.0)); a.fast = fast;
  a.want_last = (c.output & DQ_OUT_LAST) != 0; a.want_avg = (c.output & DQ_OUT_AVERAGE) != 0;
  a.inner_fixed = c.fixed_inner; a.inner_check_every = c.inner_check_every; a.max_inner = c.max_inner;
  a.outer_fixed = c.fixed_outer; a.max_outer = c.max_outer; a.check_every = c.check_every > 0 ? c.check_every : 1;
  a.next = W->next; a.err = W->err;
  DQ_CK(cudaFuncSetAttribute(k_tc_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(W->ntiles, ctx->num_sms);
  k_tc_solve<<<grid, TC_THREADS, smem, st>>>(a);
  ++ctx->launches;
  DQ_CK(cudaGetLastError());
  // warm-start state and outputs back to row-major
  const int og = std::max(1, std::min(4 * ctx->num_sms, (int)(((size_t)B * std::max(n, p) + 255) / 256)));
  k_from_minor<<<og, 256, 0, st>>>(W->xsT, B, n, (float*)P->x_state);
  ++ctx->launches;
  if (p) {
    k_from_minor<<<og, 256, 0, st>>>(W->lam, B, p, (float*)P->lam_state);
    ++ctx->launches;
  }
  P->has_state = true;
  std::vector<DevResult> hr(B);
  int herr = 0;
  DQ_CK(cudaMemcpyAsync(hr.data(), W->res, (size_t)B * sizeof(DevResult), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaMemcpyAsync(&herr, W->err, 4, cudaMemcpyDeviceToHost, st));
  if (out) {
    auto put = [&](void* dst, const float* srcT, int E) -> dq_status {
      if (!dst || !E) return DQ_OK;
      float* rowmajor = out->memory == DQ_DEVICE ? (float*)dst : W->tmp;
      k_from_minor<<<og, 256, 0, st>>>(srcT, B, E, rowmajor);
      ++ctx->launches;
      if (out->memory != DQ_DEVICE) {
        std::vector<float> h((size_t)B * E);
        DQ_CK(cudaMemcpyAsync(h.data(), W->tmp, h.size() * 4, cudaMemcpyDeviceToHost, st));
        DQ_CK(cudaStreamSynchronize(st));
        for (size_t i = 0; i < h.size(); ++i) ((double*)dst)[i] = h[i];
      }
      return DQ_OK;
    };
    if ((s = put(out->x_last, W->xlT, n)) != DQ_OK) return s;
    if ((s = put(out->x_avg, W->xaT, n)) != DQ_OK) return s;
    if ((s = put(out->lambda, W->lam, p)) != DQ_OK) return s;
  }
  DQ_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("tensor-core engine: a device wait timed out");
    return DQ_ERR_TIMEOUT;
  }
  const double consts[6] = {P->lmax_Q, P->normG2, LL, Ld, sigma, rho};
  dq_status worst = DQ_OK;
  for (int b = 0; b < B; ++b) {
    fill_result(&results[b], hr[b], consts, c);
    const dq_status sb = (dq_status)hr[b].status;
    if (sb < 0 || worst < 0) worst = sb < worst ? sb : worst;
    else if (sb > worst) worst = sb;
  }
  return worst;
}

}  // namespace dq
