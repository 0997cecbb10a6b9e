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
// rows).  Data streams through a ring of six 32 KB shared-memory stages filled
// by bulk copies (full/empty mbarrier pairs): thread 0 fills the ring at the
// start, and refills a stage as soon as all 16 warps have released it, so up
// to 192 KB per SM are in flight.  (A separate producer warp would make 17
// warps per CTA and cut the register budget from 128 to 96 per thread.)  A
// chunk covers 2048 columns of a Q block (G: 2048 float4 of a row) at a fixed
// global position, which is four of each thread's register-resident column
// slots (Q: column t + 512 m; G: float4 column t + 512 m): the iterate x^k
// and the column partial sums never leave registers.  Each wait on a stage
// and each release serve four float4 per thread: with 16 KB chunks (two per
// thread) the loop control per byte was twice as large and the kernel ran at
// 0.73 of the measured HBM bandwidth instead of 0.90 at n = 20000 (0.98 once the
// Q-CTA / G-CTA split was re-tuned for this shape).  Each CTA writes one
// partial vector; k_v2_reduce adds the partial vectors in a fixed order
// (deterministic) and the row dots, and forms the next iterate x^{k+1} from
// them, so a pass reads only x^k besides the matrices.  HBM bytes per
// iteration: 4 (n^2/2 + 2n + p n) instead of 4 (n^2 + 2 p n).
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
  const float* xk;                    // x^k (formed by the previous reduction)
  const float *gx1, *mu, *g;          // G x^{k-1}, mu, g
  float beta_next, rho;
  int cone;
  float* gxout;                       // G x^k
  float* dotQ;                        // row dots of the packed rows
  float4* partials;                   // (nQ + nG) x n4 (column-indexed)
  int* done;                          // inner loop finished (set by an earlier launch, or below)
  int* err;                           // set to 1 when a bounded wait gave up
  // step certificate (sigma > 0) of x^{k-1}: the reduction that formed it
  // wrote one partial sum of (y_j - x_j)^2 per block, cprev[0..ncert); at its
  // start every CTA adds them in the same order and stops the loop when
  // ccoef * sum <= eps_in (or kprev >= kmax): CTA 0 records cert and kstop.
  const float* cprev;
  int ncert;
  float ccoef, eps_in;
  int kprev, kmax;
  int* kstop;
  double* cert;
};

static constexpr int V2_CONS = 512;                 // threads (16 warps), all consumers
static constexpr int V2_THREADS = V2_CONS;
static constexpr int V2_CW = 4;                     // float4 of a chunk per thread
static constexpr int V2_CH4 = V2_CW * V2_CONS;      // chunk: 2048 x 16 bytes (32 KB)
static constexpr int V2_STAGES = 6;                 // ring depth (192 KB), a compile-time constant
                                                    // (a depth passed at run time cost 8 %)
static constexpr int V2_RB = 16;                    // Q blocks (64 rows) between flushes of the row dots
static constexpr unsigned long long V2_WAIT_NS = 2000000000ull;

__device__ __forceinline__ void v2_consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(V2_CONS) : "memory"); }

// Warp sum (butterfly; every lane gets the same bits).  A lane's value is a
// short FP32 sum over its own columns (at most 2 NPT products per
// accumulator, each of them small next to the row's total for the dense
// workloads), so the rounding is dominated by the five pairwise levels here
// and the compensated sum over the 16 warps.
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

// NPT float4 column slots per thread for G rows (V2_CW of them per chunk); a
// Q-CTA thread holds 4 NPT scalar column slots (V2_CW per chunk).
template <int NPT>
__global__ void __launch_bounds__(V2_THREADS, 1) k_v2_pass(V2Args a) {
  constexpr int NQS = 4 * NPT;                          // scalar column slots of a Q-CTA thread
  constexpr int NQC = (NQS + V2_CW - 1) / V2_CW;        // chunk positions of a Q block
  constexpr int NGC = (NPT + V2_CW - 1) / V2_CW;        // chunk positions of a G row
  static_assert(NGC < V2_STAGES, "chunk ring too shallow");
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
      for (int i = lane; i < a.ncert; i += 32) v += __ldcg(a.cprev + i);
      v = v2_warp_sum(v);
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
  constexpr int nst = V2_STAGES;
  float* xs = (float*)(sm + (size_t)nst * V2_CH4 * 16);
  if (t == 0) {
    for (int s = 0; s < nst; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], V2_CONS / 32);
    }
    tc::mbar_init_fence();
  }
  __syncthreads();
  // Issue cursor (thread 0 only): chunk pk of this CTA's pr-th unit (Q block
  // or G row), whose data starts at u_src (column / float4 column u_f0).
  // Stages are refilled in the order they are released, so the chunk issued
  // after releasing stage s goes to stage s: no stage arithmetic here.
  const int units = qcta ? cnt : j1 - j0;
  const int lim = qcta ? n : n4, klast = qcta ? klq : klg;
  int pr = 0, pk = 0, u_f0 = 0;
  const float4* u_src = nullptr;
  bool ok = true;
  auto unit_begin = [&]() {
    if (qcta) {  // block offset in closed form: sum_{b' < b} (n - 4 b') = b n - 2 b (b - 1)
      const long long blk = c + (long long)pr * nQ;
      u_f0 = 4 * (int)blk;
      u_src = a.Qb + (blk * n - 2 * blk * (blk - 1));
      pk = u_f0 / V2_CH4;
    } else {
      u_f0 = 0;
      u_src = (const float4*)(a.G + (size_t)(j0 + pr) * n);
      pk = 0;
    }
  };
  auto issue_next = [&](int s) {  // copy the cursor's chunk into stage s, advance
    const int b0 = max(pk * V2_CH4, u_f0), e0 = min((pk + 1) * V2_CH4, lim);
    const uint32_t bytes = (uint32_t)(e0 - b0) * 16u;
    tc::mbar_expect_tx(&full[s], bytes);
    tc::bulk_g2s(ring + (size_t)s * V2_CH4 + (b0 - pk * V2_CH4), u_src + (b0 - u_f0), bytes, &full[s]);
    if (++pk > klast && ++pr < units) unit_begin();
  };
  if (t == 0 && units > 0) {
    unit_begin();
    for (int s = 0; s < nst && pr < units; ++s) issue_next(s);
  }
  // Release the chunk in stage rs (phase ph) after every warp's last read of
  // it; thread 0 then waits for all 16 releases and refills the stage with
  // the next chunk.
  auto release = [&](int rs, uint32_t ph) {
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&empty[rs]);
    if (t == 0 && pr < units) {
      ok = tc::mbar_wait(&empty[rs], ph, V2_WAIT_NS) && ok;
      issue_next(rs);
    }
  };

  // ---------------- prologue: x^k at this thread's columns (registers)
  float xv[NQS], pv[NQS];  // G-CTA: float4 slot m is xv[4m..4m+3], pv[4m..4m+3]
#pragma unroll
  for (int m = 0; m < NQS; ++m) pv[m] = 0.f;
  if (qcta) {
#pragma unroll
    for (int m = 0; m < NQS; ++m) {
      const int j = t + V2_CONS * m;
      xv[m] = j < n ? __ldcg(a.xk + j) : 0.f;
    }
    for (int i = t; i < 4 * cnt; i += V2_CONS) xs[i] = __ldcg(a.xk + 4 * (c + (i >> 2) * nQ) + (i & 3));
  } else {
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      const int c4 = t + V2_CONS * m;
      const float4 x4 = c4 < n4 ? __ldcg((const float4*)a.xk + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
      xv[4 * m] = x4.x;
      xv[4 * m + 1] = x4.y;
      xv[4 * m + 2] = x4.z;
      xv[4 * m + 3] = x4.w;
    }
    // w_j = [mu_j + rho (G y^{k+1} + g)_j]_+ with G y^{k+1} = (1 + beta) r_j - beta (G x^{k-1})_j,
    // r_j = (G x^k)_j: w_j = [A_j + rho (1 + beta) r_j]_+, A_j = mu_j + rho (g_j - beta (G x^{k-1})_j)
    for (int j = j0 + t; j < j1; j += V2_CONS) xs[j - j0] = a.mu[j] + a.rho * (a.g[j] - a.beta_next * a.gx1[j]);
  }
  v2_consumer_sync();  // xs complete

  // consumer cursor: stage and phase of the next chunk (chunk g sits in stage
  // g % STAGES with phase (g / STAGES) & 1)
  int rs = 0;
  uint32_t rph = 0;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (qcta) {
    for (int rb = 0; rb < cnt; rb += V2_RB) {
      const int re = min(cnt, rb + V2_RB);
      for (int idx = rb; idx < re; ++idx) {
        const int blk = c + idx * nQ;
        const int f0 = 4 * blk, kf = f0 / V2_CH4;
        const float4 xq = *(const float4*)(xs + 4 * idx);
        // four row dots, two FP32 accumulators each (even / odd slots of every
        // chunk): a thread adds at most 2 NPT small products per accumulator
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
#pragma unroll
        for (int k = 0; k < NQC; ++k) {
          if (k >= kf && k <= klq) {  // the same for every thread of the CTA
            ok = tc::mbar_wait(&full[rs], rph, V2_WAIT_NS) && ok;
            const float4* ch = ring + (size_t)rs * V2_CH4;
            const bool edge = (k == kf || k == klq);
#pragma unroll
            for (int h = 0; h < V2_CW; ++h) {
              const int m = V2_CW * k + h;
              if (m < NQS) {
                const int j = t + V2_CONS * m;
                float4 v = ch[t + V2_CONS * h];  // column k CH4 + t + CONS h = slot m
                if (edge && (j < f0 || j >= n)) v = z4;  // left of the block's first column, or past n
                const float xa = xv[m];
                if (h & 1) {
                  e0 = fmaf(v.x, xa, e0); e1 = fmaf(v.y, xa, e1); e2 = fmaf(v.z, xa, e2); e3 = fmaf(v.w, xa, e3);
                } else {
                  s0 = fmaf(v.x, xa, s0); s1 = fmaf(v.y, xa, s1); s2 = fmaf(v.z, xa, s2); s3 = fmaf(v.w, xa, s3);
                }
                // column update x_{4b+r} Q[4b+r, j]
                pv[m] = fmaf(xq.x, v.x, fmaf(xq.y, v.y, fmaf(xq.z, v.z, fmaf(xq.w, v.w, pv[m]))));
              }
            }
            release(rs, rph);
            if (++rs == nst) {
              rs = 0;
              rph ^= 1u;
            }
          }
        }
        const float4 tot = make_float4(v2_warp_sum(s0 + e0), v2_warp_sum(s1 + e1), v2_warp_sum(s2 + e2),
                                       v2_warp_sum(s3 + e3));
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
      const int rs0 = rs;  // the row's first chunk
      const uint32_t rph0 = rph;
      float sa = 0.f, sb = 0.f;
#pragma unroll
      for (int k = 0; k < NGC; ++k) {
        if (k <= klg) {
          ok = tc::mbar_wait(&full[rs], rph, V2_WAIT_NS) && ok;
          const float4* ch = ring + (size_t)rs * V2_CH4;
#pragma unroll
          for (int h = 0; h < V2_CW; ++h) {
            const int m = V2_CW * k + h;
            if (m < NPT) {
              const int c4 = t + V2_CONS * m;
              float4 v = ch[t + V2_CONS * h];
              if (k == klg && c4 >= n4) v = z4;
              if (h & 1) {
                sb = fmaf(v.x, xv[4 * m], sb); sb = fmaf(v.y, xv[4 * m + 1], sb);
                sb = fmaf(v.z, xv[4 * m + 2], sb); sb = fmaf(v.w, xv[4 * m + 3], sb);
              } else {
                sa = fmaf(v.x, xv[4 * m], sa); sa = fmaf(v.y, xv[4 * m + 1], sa);
                sa = fmaf(v.z, xv[4 * m + 2], sa); sa = fmaf(v.w, xv[4 * m + 3], sa);
              }
            }
          }
          if (++rs == nst) {
            rs = 0;
            rph ^= 1u;
          }
        }
      }
      // one barrier per row: the 16 warp sums go to a buffer that alternates
      // with the row parity (a warp can only write the next row's buffer
      // after every warp has passed this row's barrier), and every warp adds
      // them itself (same order in every warp) to get r_j and w_j
      const float tot = v2_warp_sum(sa + sb);
      float* sr = sred[(j - j0) & 1];
      if (lane == 0) sr[warp] = tot;
      v2_consumer_sync();
      const float rf = v2_warp_sum(lane < V2_CONS / 32 ? sr[lane] : 0.f);
      // G x^k, and w of the next iteration (constant A_j precomputed in xs)
      const float wv = xs[j - j0] + a.rho * (1.f + a.beta_next) * rf;
      const float w = a.cone == CONE_EQ ? wv : (wv > 0.f ? wv : 0.f);
      if (t == 0) a.gxout[j] = rf;
      int us = rs0;
      uint32_t uph = rph0;
#pragma unroll
      for (int k = 0; k < NGC; ++k) {
        if (k <= klg) {
          const float4* ch = ring + (size_t)us * V2_CH4;
#pragma unroll
          for (int h = 0; h < V2_CW; ++h) {
            const int m = V2_CW * k + h, c4 = t + V2_CONS * m;
            if (m < NPT && (k < klg || c4 < n4)) {
              const float4 gv = ch[t + V2_CONS * h];
              pv[4 * m + 0] = fmaf(w, gv.x, pv[4 * m + 0]);
              pv[4 * m + 1] = fmaf(w, gv.y, pv[4 * m + 1]);
              pv[4 * m + 2] = fmaf(w, gv.z, pv[4 * m + 2]);
              pv[4 * m + 3] = fmaf(w, gv.w, pv[4 * m + 3]);
            }
          }
          release(us, uph);
          if (++us == nst) {
            us = 0;
            uph ^= 1u;
          }
        }
      }
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

// The next iterate of Algorithm FOM in the x-side form, at four columns:
//   y = x^k + b (x^k - x^{k-1}),  Q y = Q x^k + b (Q x^k - Q x^{k-1}),
//   x^{k+1} = [y - (Q y + add + tn) / L]_U,
// with add = q (rho > 0; tn = G' w(y)) or c = q + G' mu (rho = 0; no tn).
// Returns the step certificate's sum of (y - x^{k+1})^2 over the four.
struct V2Step {
  const float *xk, *xkm1, *qxkm1, *addv, *lb, *ub;
  float b, L;
  float* xnext;
  float* cpart;  // one partial sum per block, or nullptr
};

__device__ __forceinline__ float v2_step4(const V2Step& st, int c4, const float4 qx, const float4 tn) {
  const float4 x = __ldcg((const float4*)st.xk + c4), xp = __ldcg((const float4*)st.xkm1 + c4);
  const float4 qp = __ldcg((const float4*)st.qxkm1 + c4), ad = __ldg((const float4*)st.addv + c4);
  const float4 lo = __ldg((const float4*)st.lb + c4), hi = __ldg((const float4*)st.ub + c4);
  const float b = st.b, L = st.L;
  float sq = 0.f;
  auto one = [&](float xv, float xpv, float q1, float q0, float a, float t, float l, float h) {
    const float y = xv + b * (xv - xpv);
    const float qy = q1 + b * (q1 - q0);
    const float st = (qy + a + t) / L, s = y - st;
    const float o = s < l ? l : (s > h ? h : s);
    // y - x^{k+1} is the step itself where the box is inactive (no cancellation
    // error of ulp(y), which L^2 / (2 sigma) would turn into a floor of the bound)
    const float d = (s > l && s < h) ? st : y - o;
    sq = fmaf(d, d, sq);
    return o;
  };
  float4 o;
  o.x = one(x.x, xp.x, qx.x, qp.x, ad.x, tn.x, lo.x, hi.x);
  o.y = one(x.y, xp.y, qx.y, qp.y, ad.y, tn.y, lo.y, hi.y);
  o.z = one(x.z, xp.z, qx.z, qp.z, ad.z, tn.z, lo.z, hi.z);
  o.w = one(x.w, xp.w, qx.w, qp.w, ad.w, tn.w, lo.w, hi.w);
  ((float4*)st.xnext)[c4] = o;
  return sq;
}

// Q x^k = row dots + column partials of the Q-CTAs; G' w(y^{k+1}) = column
// partials of the G-CTAs; then x^{k+1} from them.  A block owns 32 float4
// columns; its 16 thread groups split the partial vectors: with both sums,
// groups 0..7 take the Q-CTA vectors c = g, g + 8, ... and groups 8..15 the
// G-CTA vectors, so both sums load at once (Kahan sums in FP32); the group
// sums are then added in group order: deterministic for a fixed grid split.
// (1024-thread blocks with eight loads in flight ran at half the speed: one
// block per SM and a second wave; all of a thread's loads in flight at once
// ran at 12.9 against 10.6 us per launch at n = 20000.)
// Warp 0 forms x^{k+1} at the block's columns and the block's partial sum of
// the step certificate.
static constexpr int V2R_COLS = 32, V2R_GROUPS = 16;

__device__ __forceinline__ void v2r_kahan(float4& s, float4& e, const float4 v) {
  v2_kahan(s.x, e.x, v.x);
  v2_kahan(s.y, e.y, v.y);
  v2_kahan(s.z, e.z, v.z);
  v2_kahan(s.w, e.w, v.w);
}

__device__ __forceinline__ void v2_cert_store(const V2Step& st, float sq) {
  const float v = v2_warp_sum(sq);
  if (st.cpart && threadIdx.x == 0) st.cpart[blockIdx.x] = v;
}

__global__ void __launch_bounds__(V2R_COLS* V2R_GROUPS) k_v2_reduce(const float4* __restrict__ partials, int nQ,
                                                                     int nG, int n4, const float* __restrict__ dotQ,
                                                                     float* __restrict__ qxout,
                                                                     float* __restrict__ tnout, V2Step st,
                                                                     const int* done) {
  __shared__ float4 sh[2][V2R_GROUPS][V2R_COLS];
  __shared__ float4 sres[2][V2R_COLS];  // Q x^k, G' w(y^{k+1}) at the block's columns
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
  const int w = threadIdx.x / V2R_COLS;
  if (w < 2 && c4 < n4) {  // thread (w, col) adds the ng groups of sum w in order (w = 1: G' w, or zero)
    // compensated FP32 sums (TwoSum) of the groups' (sum, -error) pairs: FP64 adds run at a
    // small fraction of the FP32 rate on this GPU and were a visible part of this kernel
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    auto two_sum = [](float& sum, float& err, float v) {
      const float t = sum + v, bb = t - sum;
      err += (sum - (t - bb)) + (v - bb);
      sum = t;
    };
    if (w == 0 || tnout) {
      for (int q = w * ng; q < (w + 1) * ng; ++q) {
        const float4 h = sh[0][q][col], l = sh[1][q][col];
        two_sum(s[0], c[0], h.x); two_sum(s[0], c[0], l.x);
        two_sum(s[1], c[1], h.y); two_sum(s[1], c[1], l.y);
        two_sum(s[2], c[2], h.z); two_sum(s[2], c[2], l.z);
        two_sum(s[3], c[3], h.w); two_sum(s[3], c[3], l.w);
      }
    }
    float4 r;
    if (w == 0) {
      const float4 d = ((const float4*)dotQ)[c4];
      two_sum(s[0], c[0], d.x); two_sum(s[1], c[1], d.y); two_sum(s[2], c[2], d.z); two_sum(s[3], c[3], d.w);
      r = make_float4(s[0] + c[0], s[1] + c[1], s[2] + c[2], s[3] + c[3]);
      ((float4*)qxout)[c4] = r;
    } else {
      r = make_float4(s[0] + c[0], s[1] + c[1], s[2] + c[2], s[3] + c[3]);
      if (tnout) ((float4*)tnout)[c4] = r;
    }
    sres[w][col] = r;
  }
  __syncthreads();
  if (w == 0) {  // warp 0: x^{k+1} and the certificate's partial sum
    const float sq = c4 < n4 ? v2_step4(st, c4, sres[0][col], sres[1][col]) : 0.f;
    v2_cert_store(st, sq);
  }
}

// x^1 from x^0 (y^1 = x^0): the same step with Q x^0 and G' w(x^0) read from
// memory; blocks of 32 float4 columns like the reduction, one warp each.
__global__ void __launch_bounds__(32) k_v2_step(const float* __restrict__ qx, const float* __restrict__ tn, int n4,
                                               V2Step st) {
  const int c4 = blockIdx.x * 32 + threadIdx.x;
  float sq = 0.f;
  if (c4 < n4) {
    const float4 q4 = __ldcg((const float4*)qx + c4);
    const float4 t4 = tn ? __ldcg((const float4*)tn + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
    sq = v2_step4(st, c4, q4, t4);
  }
  v2_cert_store(st, sq);
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
