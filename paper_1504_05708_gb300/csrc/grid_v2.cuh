// grid_v2.cuh -- single-pass inner iteration of the grid engine (FP32).
//
// One inner iteration of Algorithm FOM (Sec. 2.1) for a large dense instance
// reads every matrix element once:
//   * Q is stored once as its upper triangle (zeros left of the diagonal,
//     diagonal halved) in blocks of four rows: block b holds rows 4b..4b+3
//     from column 4b on, one float4 per column (the four rows' entries).  One
//     read of a block gives the four row dots (Q x)_{4b+r} += Qb[b,j].r x_j
//     and, because Q = Q', the column updates (Q x)_j += sum_r x_{4b+r}
//     Qb[b,j].r for j >= 4b.  Per-block work (waits, reductions) is shared by
//     four rows, and the four dot chains are independent.
//   * G is read once per iteration: row j's dot r_j = G_j x^k gives G x^k
//     (carried for the dual gradient) and, by linearity of G y in the
//     x-side form, w_j = [mu_j + rho (G y^{k+1} + g)_j]_+ of the next
//     iteration, so the same row (still in shared memory) adds w_j G_j to
//     G' w of the next iteration.
// A CTA is either a Q-CTA (blocks c, c + nQ, c + 2 nQ, ...: every Q-CTA gets
// the same mix of long and short blocks) or a G-CTA (a contiguous range of G
// rows).  Data streams through a ring of 16 KB shared-memory stages filled by
// bulk copies (full/empty mbarrier pairs): thread 0 fills the ring at the
// start, and refills a stage as soon as all 16 warps have released it, so up
// to 192 KB per SM are in flight.  (A separate producer warp would make 17
// warps per CTA and cut the register budget from 128 to 96 per thread.)  A
// chunk covers 1024 columns of a Q block (G: 1024 float4 of a row) at a fixed
// global position, which is two of each thread's register-resident column
// slots (Q: column t + 512 m; G: float4 column t + 512 m): the iterate x^k
// and the column partial sums never leave registers.  Each CTA writes one
// partial vector; k_v2_reduce adds the partial vectors in a fixed order
// (deterministic) and the row dots.  HBM bytes per iteration:
// 4 (n^2/2 + 2n + p n) instead of 4 (n^2 + 2 p n).
#pragma once
#include "dq_common.cuh"
#include "tc_common.cuh"

namespace dq {

struct V2Args {
  int n, p, n4;                       // n4 = n / 4 (n a multiple of 4)
  int nQ, nG;
  const int* grow;                    // nG + 1 row bounds of the G-CTAs
  const long long* boff;              // n/4 block offsets (float4 units)
  const float4* Qb;                   // blocked packed upper triangle
  const float* G;                     // p x n
  const float *x1, *x2, *qx1, *qx2;   // x^{k-1}, x^{k-2}, Q x^{k-1}, Q x^{k-2}
  const float* tn;                    // G' w(y^k) (rho > 0) or nullptr
  const float* addv;                  // q (rho > 0) or c = q + G' mu (rho = 0)
  const float *lb, *ub;
  const float *gx1, *mu, *g;          // G x^{k-1}, mu, g
  float beta_prev, beta_next, L, rho;
  int cone;
  float* xout;                        // x^k
  float* gxout;                       // G x^k
  float* dotQ;                        // row dots of the packed rows
  float4* partials;                   // (nQ + nG) x n4 (column-indexed)
  int* done;                          // inner loop finished (set by an earlier launch, or below)
  int* err;                           // set to 1 when a bounded wait gave up
  // step certificate (sigma > 0): this launch writes cpart[c] = sum over the
  // x-slice of Q-CTA c of (y_j - x_j)^2; at its start every CTA adds the
  // previous launch's cprev[0..nQ) in the same order, and stops the loop when
  // ccoef * sum <= eps_in (or kprev >= kmax): CTA 0 records cert and kstop.
  float* cpart;
  const float* cprev;
  float ccoef, eps_in;
  int kprev, kmax;
  int* kstop;
  double* cert;
};

static constexpr int V2_CONS = 512;                 // threads (16 warps), all consumers
static constexpr int V2_THREADS = V2_CONS;
static constexpr int V2_CH4 = 2 * V2_CONS;          // chunk: 1024 x 16 bytes (16 KB)
static constexpr int V2_STAGES = 12;                // ring depth (192 KB)
static constexpr int V2_RB = 16;                    // Q blocks (64 rows) between flushes of the row dots
static constexpr unsigned long long V2_WAIT_NS = 2000000000ull;

__device__ __forceinline__ void v2_consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(V2_CONS) : "memory"); }

// Warp sum (butterfly, every lane gets the total).  Each lane's value is
// already a compensated partial over its columns; the five pairwise levels
// add at most 5 roundings.
__device__ __forceinline__ float v2_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void v2_kahan(float& s, float& c, float v) {
  const float y = v - c, t = s + y;
  c = (t - s) - y;
  s = t;
}

// NPT (even) float4 column slots per thread for G rows (2 per G chunk); a Q
// block spans at most 2 NPT chunks (4 NPT scalar column slots per thread).
template <int NPT>
__global__ void __launch_bounds__(V2_THREADS, 1) k_v2_pass(V2Args a) {
  static_assert(NPT % 2 == 0 && NPT / 2 <= V2_STAGES, "chunk ring too shallow");
  constexpr int NQS = 4 * NPT;  // scalar column slots of a Q-CTA thread
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[V2_STAGES], empty[V2_STAGES];
  __shared__ float4 sdot[V2_RB][V2_CONS / 32];
  __shared__ float sred[2][V2_CONS / 32];
  __shared__ int s_stop;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (warp == 0) {  // loop control: done flag, or the step certificate of the previous launch
    int stop = a.done ? *(volatile const int*)a.done : 0;
    if (!stop && a.cprev) {
      float v = 0.f;
      for (int i = lane; i < a.nQ; i += 32) v += __ldcg(a.cprev + i);
      v = v2_warp_sum(v);  // butterfly: the same bits in every lane and every CTA
      const float ct = a.ccoef * v;
      if (ct <= a.eps_in || a.kprev >= a.kmax) {
        stop = 1;
        if (blockIdx.x == 0 && lane == 0) {
          *a.cert = (double)ct;
          *a.kstop = a.kprev;
          __threadfence();
          *(volatile int*)a.done = 1;
        }
      }
    }
    if (lane == 0) s_stop = stop;
  }
  __syncthreads();
  if (s_stop) return;
  const bool qcta = blockIdx.x < a.nQ;
  const int c = blockIdx.x, nQ = a.nQ, n = a.n, n4 = a.n4, nb = n4;
  const int klq = (n - 1) / V2_CH4;   // last chunk of every Q block
  const int klg = (n4 - 1) / V2_CH4;  // last chunk of every G row
  const int cnt = qcta ? (c < nb ? (nb - 1 - c) / nQ + 1 : 0) : 0;
  const int j0 = qcta ? 0 : a.grow[c - nQ], j1 = qcta ? 0 : a.grow[c - nQ + 1];
  float4* ring = (float4*)sm;
  // Q-CTA: the four x of each of its blocks; G-CTA: per-row constant of w
  float* xs = (float*)(sm + (size_t)V2_STAGES * V2_CH4 * 16);
  if (t == 0) {
    for (int s = 0; s < V2_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], V2_CONS / 32);
    }
    tc::mbar_init_fence();
  }
  __syncthreads();

  // Issue cursor (used by thread 0 only): chunk pk of this CTA's pr-th block
  // (Q) or row (G); chunk number pg goes to stage pg % STAGES.
  const int units = qcta ? cnt : j1 - j0;
  int pr = 0, pk = 0;
  uint32_t pg = 0;
  bool ok = true;
  auto first_chunk = [&](int r) { return qcta ? (4 * (c + r * nQ)) / V2_CH4 : 0; };
  auto issue_next = [&]() {  // thread 0: copy the cursor's chunk into stage pg % STAGES, advance
    const int f0 = qcta ? 4 * (c + pr * nQ) : 0;          // first column (Q) / float4 column (G)
    const int lim = qcta ? n : n4;
    const int b0 = max(pk * V2_CH4, f0), e0 = min((pk + 1) * V2_CH4, lim);
    // block offset in closed form: sum_{b' < b} (n - 4 b') = b n - 2 b (b - 1) (no load on the refill path)
    const long long blk = c + pr * nQ;
    const float4* src = qcta ? a.Qb + (blk * n - 2 * blk * (blk - 1)) + (b0 - f0)
                             : (const float4*)(a.G + (size_t)(j0 + pr) * n) + b0;
    const uint32_t bytes = (uint32_t)(e0 - b0) * 16u;
    const int s = (int)(pg % V2_STAGES);
    tc::mbar_expect_tx(&full[s], bytes);
    tc::bulk_g2s(ring + (size_t)s * V2_CH4 + (b0 - pk * V2_CH4), src, bytes, &full[s]);
    ++pg;
    if (++pk > (qcta ? klq : klg)) {
      ++pr;
      if (pr < units) pk = first_chunk(pr);
    }
  };
  if (t == 0 && units > 0) {
    pk = first_chunk(0);
    for (int s = 0; s < V2_STAGES && pr < units; ++s) issue_next();
  }
  // Release chunk gc (every warp, after its last read of the stage); thread 0
  // then waits for all 16 releases and refills the stage with the next chunk.
  auto release = [&](uint32_t gc) {
    const int s = (int)(gc % V2_STAGES);
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&empty[s]);
    if (t == 0 && pr < units) {
      ok = tc::mbar_wait(&empty[s], (gc / V2_STAGES) & 1, V2_WAIT_NS) && ok;
      issue_next();
    }
  };

  // ---------------- prologue: x^k = [y - grad(y)/L]_U for this thread's columns
  float xv[NQS], pv[NQS];  // G-CTA: float4 slot m is xv[4m..4m+3], pv[4m..4m+3]
  const float b = a.beta_prev;
  auto step = [&](int j, float& y) {
    const float x = a.x1[j], xp = a.x2[j], qx = a.qx1[j], qxp = a.qx2[j];
    y = x + b * (x - xp);
    const float qy = qx + b * (qx - qxp);
    const float s = y - (qy + a.addv[j] + (a.tn ? a.tn[j] : 0.f)) / a.L;
    const float l = a.lb[j], h = a.ub[j];
    return s < l ? l : (s > h ? h : s);
  };
  float csum = 0.f;  // step certificate: sum of (y_j - x_j)^2 over this CTA's x-slice
#pragma unroll
  for (int m = 0; m < NQS; ++m) pv[m] = 0.f;
  if (qcta) {
    const int per = (n + nQ - 1) / nQ;  // Q-CTA c stores the c-th slice of x^k
#pragma unroll
    for (int m = 0; m < NQS; ++m) {
      const int j = t + V2_CONS * m;
      float o = 0.f;
      if (j < n) {
        float y;
        o = step(j, y);
        if (j >= c * per && j < (c + 1) * per) {
          a.xout[j] = o;
          csum = fmaf(y - o, y - o, csum);
        }
        const int blk = j >> 2;
        if (blk >= c && (blk - c) % nQ == 0) xs[((blk - c) / nQ) * 4 + (j & 3)] = o;
      }
      xv[m] = o;
    }
  } else {
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      const int c4 = t + V2_CONS * m;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float y;
        xv[4 * m + u] = c4 < n4 ? step(4 * c4 + u, y) : 0.f;
      }
    }
    // w_j = [mu_j + rho (G y^{k+1} + g)_j]_+ with G y^{k+1} = (1 + beta) r_j - beta (G x^{k-1})_j,
    // r_j = (G x^k)_j: w_j = [A_j + rho (1 + beta) r_j]_+, A_j = mu_j + rho (g_j - beta (G x^{k-1})_j)
    for (int j = j0 + t; j < j1; j += V2_CONS) xs[j - j0] = a.mu[j] + a.rho * (a.g[j] - a.beta_next * a.gx1[j]);
  }
  if (qcta && a.cpart) {
    const float v = v2_warp_sum(csum);
    if (lane == 0) sred[0][warp] = v;  // sred is otherwise used by G-CTAs only
  }
  v2_consumer_sync();  // xs complete
  if (qcta && a.cpart && t == 0) {
    float v = 0.f;
    for (int w = 0; w < V2_CONS / 32; ++w) v += sred[0][w];
    a.cpart[c] = v;
  }

  uint32_t gc = 0;
  if (qcta) {
    for (int rb = 0; rb < cnt; rb += V2_RB) {
      const int re = min(cnt, rb + V2_RB);
      for (int idx = rb; idx < re; ++idx) {
        const int blk = c + idx * nQ;
        const int f0 = 4 * blk, kf = f0 / V2_CH4;
        const float4 xq = *(const float4*)(xs + 4 * idx);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * NPT; ++k) {
          if (k >= kf && k <= klq) {  // the same for every thread of the CTA
            const int s = (int)(gc % V2_STAGES);
            ok = tc::mbar_wait(&full[s], (gc / V2_STAGES) & 1, V2_WAIT_NS) && ok;
            const float4* ch = ring + (size_t)s * V2_CH4;  // column j at ch[j - k * V2_CH4]
            const int m0 = 2 * k, ja = t + V2_CONS * m0, jb = ja + V2_CONS;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 va = (ja >= f0 && ja < n) ? ch[ja - k * V2_CH4] : z4;
            const float4 vb = (jb >= f0 && jb < n) ? ch[jb - k * V2_CH4] : z4;
            const float xa = xv[m0], xb = xv[m0 + 1];
            // four independent row dots (Kahan per row, both columns folded in one step)
            v2_kahan(s0, e0, fmaf(va.x, xa, vb.x * xb));
            v2_kahan(s1, e1, fmaf(va.y, xa, vb.y * xb));
            v2_kahan(s2, e2, fmaf(va.z, xa, vb.z * xb));
            v2_kahan(s3, e3, fmaf(va.w, xa, vb.w * xb));
            // column updates x_{4b+r} Q[4b+r, j]
            pv[m0] = fmaf(xq.x, va.x, fmaf(xq.y, va.y, fmaf(xq.z, va.z, fmaf(xq.w, va.w, pv[m0]))));
            pv[m0 + 1] = fmaf(xq.x, vb.x, fmaf(xq.y, vb.y, fmaf(xq.z, vb.z, fmaf(xq.w, vb.w, pv[m0 + 1]))));
            release(gc);
            ++gc;
          }
        }
        const float4 tot = make_float4(v2_warp_sum(s0 - e0), v2_warp_sum(s1 - e1), v2_warp_sum(s2 - e2),
                                       v2_warp_sum(s3 - e3));
        if (lane == 0) sdot[idx - rb][warp] = tot;
      }
      v2_consumer_sync();
      if (t < 4 * (re - rb)) {  // row 4 (c + (rb + t/4) nQ) + t%4
        const int bl = t >> 2, r = t & 3;
        float sh = 0.f, sl = 0.f;  // compensated (TwoSum) sum of the 16 warp sums
        for (int w = 0; w < V2_CONS / 32; ++w) {
          const float4 q4 = sdot[bl][w];
          const float b2 = r == 0 ? q4.x : (r == 1 ? q4.y : (r == 2 ? q4.z : q4.w));
          const float s2 = sh + b2, bb = s2 - sh;
          sl += (sh - (s2 - bb)) + (b2 - bb);
          sh = s2;
        }
        a.dotQ[4 * (c + (rb + bl) * nQ) + r] = sh + sl;
      }
      v2_consumer_sync();
    }
  } else {
    for (int j = j0; j < j1; ++j) {
      const uint32_t g0 = gc;
      float sa = 0.f, comp = 0.f;
#pragma unroll
      for (int k = 0; k < NPT / 2; ++k) {
        if (k <= klg) {
          const uint32_t gk = g0 + k;
          const int s = (int)(gk % V2_STAGES);
          ok = tc::mbar_wait(&full[s], (gk / V2_STAGES) & 1, V2_WAIT_NS) && ok;
          const float4* ch = ring + (size_t)s * V2_CH4;
          const int m0 = 2 * k, c40 = t + V2_CONS * m0, c41 = c40 + V2_CONS;
          const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 v0 = c40 < n4 ? ch[c40 - k * V2_CH4] : z4;
          const float4 v1 = c41 < n4 ? ch[c41 - k * V2_CH4] : z4;
          float d0 = v0.x * xv[4 * m0], d1 = v1.x * xv[4 * m0 + 4];
          d0 = fmaf(v0.y, xv[4 * m0 + 1], d0);
          d1 = fmaf(v1.y, xv[4 * m0 + 5], d1);
          d0 = fmaf(v0.z, xv[4 * m0 + 2], d0);
          d1 = fmaf(v1.z, xv[4 * m0 + 6], d1);
          d0 = fmaf(v0.w, xv[4 * m0 + 3], d0);
          d1 = fmaf(v1.w, xv[4 * m0 + 7], d1);
          v2_kahan(sa, comp, d0 + d1);
        }
      }
      // one barrier per row: the 16 warp sums go to a buffer that alternates
      // with the row parity (a warp can only write the next row's buffer
      // after every warp has passed this row's barrier), and every warp adds
      // them itself (same order in every warp) to get r_j and w_j
      const float tot = v2_warp_sum(sa - comp);
      float* sr = sred[(j - j0) & 1];
      if (lane == 0) sr[warp] = tot;
      v2_consumer_sync();
      const float rf = v2_warp_sum(lane < V2_CONS / 32 ? sr[lane] : 0.f);
      // G x^k, and w of the next iteration (constant A_j precomputed in xs)
      const float wv = xs[j - j0] + a.rho * (1.f + a.beta_next) * rf;
      const float w = a.cone == CONE_EQ ? wv : (wv > 0.f ? wv : 0.f);
      if (t == 0) a.gxout[j] = rf;
#pragma unroll
      for (int k = 0; k < NPT / 2; ++k) {
        if (k <= klg) {
          const int s = (int)((g0 + k) % V2_STAGES);
          const float4* ch = ring + (size_t)s * V2_CH4;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = 2 * k + h, c4 = t + V2_CONS * m;
            if (c4 < n4) {
              const float4 gv = ch[c4 - k * V2_CH4];
              pv[4 * m + 0] = fmaf(w, gv.x, pv[4 * m + 0]);
              pv[4 * m + 1] = fmaf(w, gv.y, pv[4 * m + 1]);
              pv[4 * m + 2] = fmaf(w, gv.z, pv[4 * m + 2]);
              pv[4 * m + 3] = fmaf(w, gv.w, pv[4 * m + 3]);
            }
          }
          release(g0 + k);
        }
      }
      gc = g0 + klg + 1;
    }
  }
  if (!ok && a.err && lane == 0) atomicExch(a.err, 1);
  float* out = (float*)(a.partials + (size_t)c * n4);
  if (qcta) {
#pragma unroll
    for (int m = 0; m < NQS; ++m) {
      const int j = t + V2_CONS * m;
      if (j < n) out[j] = pv[m];
    }
  } else {
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      const int c4 = t + V2_CONS * m;
      if (c4 < n4) ((float4*)out)[c4] = make_float4(pv[4 * m], pv[4 * m + 1], pv[4 * m + 2], pv[4 * m + 3]);
    }
  }
}

// Step certificate of the last launched iteration, when the loop ran out of
// iterations before a later launch could read it (one warp).
__global__ void k_v2_final(const float* cprev, int nQ, float ccoef, int kprev, int* done, int* kstop,
                           double* cert) {
  if (*(volatile const int*)done) return;
  const int lane = threadIdx.x;
  float v = 0.f;
  for (int i = lane; i < nQ; i += 32) v += __ldcg(cprev + i);
  v = v2_warp_sum(v);
  if (lane == 0) {
    *cert = (double)(ccoef * v);
    *kstop = kprev;
    __threadfence();
    *(volatile int*)done = 1;
  }
}

// Q x^k = row dots + column partials of the Q-CTAs; G' w(y^{k+1}) = column
// partials of the G-CTAs.  A block owns 8 float4 columns (128 bytes of every
// partial vector); its 32 thread groups split the partial vectors: with both
// sums, groups 0..15 take the Q-CTA vectors c = g, g + 16, ... and groups
// 16..31 the G-CTA vectors, so both sums load at once (Kahan sums in FP32);
// the group sums are then added in group order: deterministic for a fixed
// grid split.
static constexpr int V2R_COLS = 8, V2R_GROUPS = 32;

__device__ __forceinline__ void v2r_kahan(float4& s, float4& e, const float4 v) {
  v2_kahan(s.x, e.x, v.x);
  v2_kahan(s.y, e.y, v.y);
  v2_kahan(s.z, e.z, v.z);
  v2_kahan(s.w, e.w, v.w);
}

__global__ void __launch_bounds__(V2R_COLS* V2R_GROUPS) k_v2_reduce(const float4* __restrict__ partials, int nQ,
                                                                     int nG, int n4, const float* __restrict__ dotQ,
                                                                     float* __restrict__ qxout,
                                                                     float* __restrict__ tnout, const int* done) {
  __shared__ float4 sh[2][V2R_GROUPS][V2R_COLS];
  if (done && *(volatile const int*)done) return;
  const int col = threadIdx.x % V2R_COLS, gi = threadIdx.x / V2R_COLS;
  const int c4 = blockIdx.x * V2R_COLS + col;
  const int ng = tnout ? V2R_GROUPS / 2 : V2R_GROUPS;  // groups per sum
  const int which = gi / ng, gl = gi % ng;
  const int c0 = which == 0 ? 0 : nQ, c1 = which == 0 ? nQ : nQ + nG;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f), e = s;
  if (c4 < n4) {
    int cc = c0 + gl;
    for (; cc + 3 * ng < c1; cc += 4 * ng) {  // four loads in flight, then the sums in order
      const float4 v0 = __ldcg(partials + (size_t)cc * n4 + c4);
      const float4 v1 = __ldcg(partials + (size_t)(cc + ng) * n4 + c4);
      const float4 v2 = __ldcg(partials + (size_t)(cc + 2 * ng) * n4 + c4);
      const float4 v3 = __ldcg(partials + (size_t)(cc + 3 * ng) * n4 + c4);
      v2r_kahan(s, e, v0);
      v2r_kahan(s, e, v1);
      v2r_kahan(s, e, v2);
      v2r_kahan(s, e, v3);
    }
    for (; cc < c1; cc += ng) v2r_kahan(s, e, __ldcg(partials + (size_t)cc * n4 + c4));
  }
  sh[0][gi][col] = s;
  sh[1][gi][col] = make_float4(-e.x, -e.y, -e.z, -e.w);
  __syncthreads();
  const int w = threadIdx.x / V2R_COLS, cw = blockIdx.x * V2R_COLS + threadIdx.x % V2R_COLS;
  if (w < (tnout ? 2 : 1) && cw < n4) {  // thread (w, col) adds the ng groups of sum w in order
    const int cl = threadIdx.x % V2R_COLS;
    double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    for (int q = w * ng; q < (w + 1) * ng; ++q) {
      const float4 h = sh[0][q][cl], l = sh[1][q][cl];
      r0 += double(h.x) + double(l.x);
      r1 += double(h.y) + double(l.y);
      r2 += double(h.z) + double(l.z);
      r3 += double(h.w) + double(l.w);
    }
    if (w == 0) {
      const float4 d = ((const float4*)dotQ)[cw];
      ((float4*)qxout)[cw] = make_float4(float(r0 + d.x), float(r1 + d.y), float(r2 + d.z), float(r3 + d.w));
    } else {
      ((float4*)tnout)[cw] = make_float4(float(r0), float(r1), float(r2), float(r3));
    }
  }
}

// Blocked packed upper triangle: block b holds rows 4b..4b+3 from column 4b
// on, one float4 (the four rows) per column; zeros left of the diagonal and
// half the diagonal.
__global__ void k_pack_qblocks(const float* __restrict__ Q, int n, const long long* __restrict__ boff,
                               float4* __restrict__ Qb) {
  for (int bl = blockIdx.x; bl < n / 4; bl += gridDim.x) {
    const int i0 = 4 * bl;
    float4* dst = Qb + boff[bl];
    for (int j = i0 + threadIdx.x; j < n; j += blockDim.x) {
      float v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + r;
        const float q = Q[(size_t)i * n + j];
        v[r] = j < i ? 0.f : (j == i ? 0.5f * q : q);
      }
      dst[j - i0] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

}  // namespace dq
