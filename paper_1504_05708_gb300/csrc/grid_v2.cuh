// grid_v2.cuh -- single-pass inner iteration of the grid engine (FP32).
//
// One inner iteration of Algorithm FOM (Sec. 2.1) for a large dense instance
// reads every matrix element once:
//   * Q is stored once as its upper triangle, row i from column 4*floor(i/4)
//     (16-byte aligned rows, zeros left of the diagonal, diagonal halved).  One
//     read of row segment i yields both the row dot (Q x)_i += Qp[i,:] x and
//     the column update (Q x)_j += x_i Qp[i,j], j >= i, because Q = Q'.
//   * G is read once per iteration: row j's dot r_j = G_j x^k gives G x^k
//     (carried for the dual gradient) and, by linearity of G y in the
//     x-side form, w_j = [mu_j + rho (G y^{k+1} + g)_j]_+ of the next
//     iteration, so the same row (still in shared memory) adds w_j G_j to
//     G' w of the next iteration.
// A CTA is either a Q-CTA (rows c, c + nQ, c + 2 nQ, ...: every Q-CTA gets
// the same mix of long and short rows) or a G-CTA (a contiguous range of G
// rows).  Rows stream through a ring of 16 KB shared-memory stages filled by
// bulk copies (full/empty mbarrier pairs): thread 0 fills the ring at the
// start, and refills a stage as soon as all 16 warps have released it, so up
// to 192 KB per SM are in flight.  (A separate producer warp would make 17
// warps per CTA and cut the register budget from 128 to 96 per thread.)  A
// chunk covers 1024 float4 columns at a fixed global position, which is two
// of each consumer thread's register-resident column slots (t + 512 m): the
// iterate x^k and the column partial sums never leave registers.  Each CTA
// writes one partial vector; k_v2_reduce adds the partial vectors in a fixed
// order (deterministic) and the row dots.  HBM bytes per iteration:
// 4 (n(n+1)/2 + p n) instead of 4 (n^2 + 2 p n).
#pragma once
#include "dq_common.cuh"
#include "tc_common.cuh"

namespace dq {

struct V2Args {
  int n, p, n4;                       // n4 = n / 4 (n a multiple of 4)
  int nQ, nG;
  const int* qrow;                    // unused (Q rows are dealt round-robin)
  const int* grow;                    // nG + 1 row bounds of the G-CTAs
  const long long* qoff;              // n packed-row offsets (floats, multiples of 4)
  const float* Qp;                    // packed upper triangle
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
  float4* partials;                   // (nQ + nG) x n4
  const int* done;
  int* err;                           // set to 1 when a bounded wait gave up
};

static constexpr int V2_CONS = 512;                 // threads (16 warps), all consumers
static constexpr int V2_THREADS = V2_CONS;
static constexpr int V2_CH4 = 2 * V2_CONS;          // float4 per chunk (16 KB)
static constexpr int V2_STAGES = 12;                // ring depth (192 KB)
static constexpr int V2_RB = 64;                    // rows between flushes of the row dots
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

// NPT (even) register slots of float4 columns per consumer thread; a row spans
// at most NPT / 2 <= V2_STAGES chunks.
template <int NPT>
__global__ void __launch_bounds__(V2_THREADS, 1) k_v2_pass(V2Args a) {
  static_assert(NPT % 2 == 0 && NPT / 2 <= V2_STAGES, "chunk ring too shallow");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[V2_STAGES], empty[V2_STAGES];
  __shared__ float sdot[V2_RB][V2_CONS / 32];
  __shared__ float sred[2][V2_CONS / 32];
  if (a.done && *(volatile const int*)a.done) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool qcta = blockIdx.x < a.nQ;
  const int c = blockIdx.x, nQ = a.nQ, n4 = a.n4;
  const int kl = (n4 - 1) / V2_CH4;  // last chunk of every row
  const int cnt = qcta ? (c < a.n ? (a.n - 1 - c) / nQ + 1 : 0) : 0;
  const int j0 = qcta ? 0 : a.grow[c - nQ], j1 = qcta ? 0 : a.grow[c - nQ + 1];
  float4* ring = (float4*)sm;
  // Q-CTA: x_i of its rows; G-CTA: per-row constant of w (see the G branch)
  float* xs = (float*)(sm + (size_t)V2_STAGES * V2_CH4 * 16);
  if (t == 0) {
    for (int s = 0; s < V2_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], V2_CONS / 32);
    }
    tc::mbar_init_fence();
  }
  __syncthreads();

  // Issue cursor (used by thread 0 only): chunk pk of this CTA's pr-th row;
  // chunk number pg (position in the CTA's sequence) goes to stage pg % STAGES.
  const int rows = qcta ? cnt : j1 - j0;
  int pr = 0, pk = 0;
  uint32_t pg = 0;
  bool ok = true;
  auto row_of = [&](int r) { return qcta ? c + r * nQ : j0 + r; };
  auto first_chunk = [&](int r) { return qcta ? (row_of(r) >> 2) / V2_CH4 : 0; };
  auto issue_next = [&]() {  // thread 0: copy the cursor's chunk into stage pg % STAGES, advance
    const int i = row_of(pr);
    const int f0 = qcta ? (i >> 2) : 0;
    const float* src = qcta ? a.Qp + a.qoff[i] + 4ll * (max(pk * V2_CH4, f0) - f0)
                            : a.G + (size_t)i * a.n + 4ll * (pk * V2_CH4);
    const int b4 = max(pk * V2_CH4, f0), e4 = min((pk + 1) * V2_CH4, n4);
    const uint32_t bytes = (uint32_t)(e4 - b4) * 16u;
    const int s = (int)(pg % V2_STAGES);
    tc::mbar_expect_tx(&full[s], bytes);
    tc::bulk_g2s(ring + (size_t)s * V2_CH4 + (b4 - pk * V2_CH4), src, bytes, &full[s]);
    ++pg;
    if (++pk > kl) {
      ++pr;
      if (pr < rows) pk = first_chunk(pr);
    }
  };
  if (t == 0 && rows > 0) {
    pk = first_chunk(0);
    for (int s = 0; s < V2_STAGES && pr < rows; ++s) issue_next();
  }
  // Release chunk gc (every warp, after its last read of the stage); thread 0
  // then waits for all 16 releases and refills the stage with the next chunk.
  auto release = [&](uint32_t gc) {
    const int s = (int)(gc % V2_STAGES);
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&empty[s]);
    if (t == 0 && pr < rows) {
      ok = tc::mbar_wait(&empty[s], (gc / V2_STAGES) & 1, V2_WAIT_NS) && ok;
      issue_next();
    }
  };

  // ---------------- consumers: prologue x^k = [y - grad(y)/L]_U for this thread's columns
  float4 xr[NPT];
  const float b = a.beta_prev;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int c4 = t + V2_CONS * m;
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c4 < n4) {
      const float4 x1 = ((const float4*)a.x1)[c4], x2 = ((const float4*)a.x2)[c4];
      const float4 q1 = ((const float4*)a.qx1)[c4], q2 = ((const float4*)a.qx2)[c4];
      const float4 ad = ((const float4*)a.addv)[c4];
      const float4 tw = a.tn ? ((const float4*)a.tn)[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 lo = ((const float4*)a.lb)[c4], hi = ((const float4*)a.ub)[c4];
      auto step = [&](float x, float xp, float qx, float qxp, float add, float tn_, float l, float h) {
        const float y = x + b * (x - xp);
        const float qy = qx + b * (qx - qxp);
        const float s = y - (qy + add + tn_) / a.L;
        return s < l ? l : (s > h ? h : s);
      };
      o.x = step(x1.x, x2.x, q1.x, q2.x, ad.x, tw.x, lo.x, hi.x);
      o.y = step(x1.y, x2.y, q1.y, q2.y, ad.y, tw.y, lo.y, hi.y);
      o.z = step(x1.z, x2.z, q1.z, q2.z, ad.z, tw.z, lo.z, hi.z);
      o.w = step(x1.w, x2.w, q1.w, q2.w, ad.w, tw.w, lo.w, hi.w);
      // every CTA computes x^k; CTA c stores the c-th slice
      const int per = (n4 + gridDim.x - 1) / gridDim.x;
      if (c4 >= c * per && c4 < (c + 1) * per) ((float4*)a.xout)[c4] = o;
      if (qcta) {
        const float xv[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * c4 + u;
          if (i >= c && (i - c) % nQ == 0) xs[(i - c) / nQ] = xv[u];
        }
      }
    }
    xr[m] = o;
  }
  float4 part[NPT];
#pragma unroll
  for (int m = 0; m < NPT; ++m) part[m] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!qcta) {
    // w_j = [mu_j + rho (G y^{k+1} + g)_j]_+ with G y^{k+1} = (1 + beta) r_j - beta (G x^{k-1})_j,
    // r_j = (G x^k)_j: w_j = [A_j + rho (1 + beta) r_j]_+, A_j = mu_j + rho (g_j - beta (G x^{k-1})_j)
    for (int j = j0 + t; j < j1; j += V2_CONS) xs[j - j0] = a.mu[j] + a.rho * (a.g[j] - a.beta_next * a.gx1[j]);
  }
  v2_consumer_sync();  // xs complete

  uint32_t gc = 0;
  if (qcta) {
    for (int rb = 0; rb < cnt; rb += V2_RB) {
      const int re = min(cnt, rb + V2_RB);
      for (int idx = rb; idx < re; ++idx) {
        const int i = c + idx * nQ;
        const int f0 = i >> 2, kf = f0 / V2_CH4;
        const float xi = xs[idx];
        float sa = 0.f, comp = 0.f;
#pragma unroll
        for (int k = 0; k < NPT / 2; ++k) {
          if (k >= kf && k <= kl) {  // the same for every thread of the CTA
            const int s = (int)(gc % V2_STAGES);
            ok = tc::mbar_wait(&full[s], (gc / V2_STAGES) & 1, V2_WAIT_NS) && ok;
            const float4* ch = ring + (size_t)s * V2_CH4;  // column c4 at ch[c4 - k * V2_CH4]
            // both of this thread's float4 of the chunk are loaded before use; their dots are
            // independent chains, and one Kahan step per chunk adds them to the row dot
            const int m0 = 2 * k, c40 = t + V2_CONS * m0, c41 = c40 + V2_CONS;
            const bool in0 = c40 >= f0 && c40 < n4, in1 = c41 >= f0 && c41 < n4;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 v0 = in0 ? ch[c40 - k * V2_CH4] : z4;
            const float4 v1 = in1 ? ch[c41 - k * V2_CH4] : z4;
            float d0 = v0.x * xr[m0].x, d1 = v1.x * xr[m0 + 1].x;
            d0 = fmaf(v0.y, xr[m0].y, d0);
            d1 = fmaf(v1.y, xr[m0 + 1].y, d1);
            d0 = fmaf(v0.z, xr[m0].z, d0);
            d1 = fmaf(v1.z, xr[m0 + 1].z, d1);
            d0 = fmaf(v0.w, xr[m0].w, d0);
            d1 = fmaf(v1.w, xr[m0 + 1].w, d1);
            {
              const float yk = (d0 + d1) - comp, tk = sa + yk;  // Kahan pair
              comp = (tk - sa) - yk;
              sa = tk;
            }
            part[m0].x = fmaf(xi, v0.x, part[m0].x);
            part[m0].y = fmaf(xi, v0.y, part[m0].y);
            part[m0].z = fmaf(xi, v0.z, part[m0].z);
            part[m0].w = fmaf(xi, v0.w, part[m0].w);
            part[m0 + 1].x = fmaf(xi, v1.x, part[m0 + 1].x);
            part[m0 + 1].y = fmaf(xi, v1.y, part[m0 + 1].y);
            part[m0 + 1].z = fmaf(xi, v1.z, part[m0 + 1].z);
            part[m0 + 1].w = fmaf(xi, v1.w, part[m0 + 1].w);
            release(gc);
            ++gc;
          }
        }
        const float tot = v2_warp_sum(sa - comp);
        if (lane == 0) sdot[idx - rb][warp] = tot;
      }
      v2_consumer_sync();
      if (t < re - rb) {
        float sh = 0.f, sl = 0.f;  // compensated (TwoSum) sum of the 16 warp sums
        for (int w = 0; w < V2_CONS / 32; ++w) {
          const float b2 = sdot[t][w], s2 = sh + b2, bb = s2 - sh;
          sl += (sh - (s2 - bb)) + (b2 - bb);
          sh = s2;
        }
        a.dotQ[c + (rb + t) * nQ] = sh + sl;
      }
      v2_consumer_sync();
    }
  } else {
    for (int j = j0; j < j1; ++j) {
      const uint32_t g0 = gc;
      float sa = 0.f, comp = 0.f;
#pragma unroll
      for (int k = 0; k < NPT / 2; ++k) {
        if (k <= kl) {
          const uint32_t gk = g0 + k;
          const int s = (int)(gk % V2_STAGES);
          ok = tc::mbar_wait(&full[s], (gk / V2_STAGES) & 1, V2_WAIT_NS) && ok;
          const float4* ch = ring + (size_t)s * V2_CH4;
          const int m0 = 2 * k, c40 = t + V2_CONS * m0, c41 = c40 + V2_CONS;
          const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 v0 = c40 < n4 ? ch[c40 - k * V2_CH4] : z4;
          const float4 v1 = c41 < n4 ? ch[c41 - k * V2_CH4] : z4;
          float d0 = v0.x * xr[m0].x, d1 = v1.x * xr[m0 + 1].x;
          d0 = fmaf(v0.y, xr[m0].y, d0);
          d1 = fmaf(v1.y, xr[m0 + 1].y, d1);
          d0 = fmaf(v0.z, xr[m0].z, d0);
          d1 = fmaf(v1.z, xr[m0 + 1].z, d1);
          d0 = fmaf(v0.w, xr[m0].w, d0);
          d1 = fmaf(v1.w, xr[m0 + 1].w, d1);
          const float yk = (d0 + d1) - comp, tk = sa + yk;
          comp = (tk - sa) - yk;
          sa = tk;
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
        if (k <= kl) {
          const int s = (int)((g0 + k) % V2_STAGES);
          const float4* ch = ring + (size_t)s * V2_CH4;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int m = 2 * k + h, c4 = t + V2_CONS * m;
            if (c4 < n4) {
              const float4 gv = ch[c4 - k * V2_CH4];
              part[m].x = fmaf(w, gv.x, part[m].x);
              part[m].y = fmaf(w, gv.y, part[m].y);
              part[m].z = fmaf(w, gv.z, part[m].z);
              part[m].w = fmaf(w, gv.w, part[m].w);
            }
          }
          release(g0 + k);
        }
      }
      gc = g0 + kl + 1;
    }
  }
  if (!ok && a.err && lane == 0) atomicExch(a.err, 1);
  float4* out = a.partials + (size_t)c * n4;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int c4 = t + V2_CONS * m;
    if (c4 < n4) out[c4] = part[m];
  }
}

// Q x^k = row dots + column partials of the Q-CTAs; G' w(y^{k+1}) = column
// partials of the G-CTAs.  A block owns 32 float4 columns; its 8 thread groups
// take the partial vectors c = gi, gi + 8, ... (Kahan sums in FP32), and the
// 8 group sums are added in group order: deterministic for a fixed grid split.
static constexpr int V2R_COLS = 32, V2R_GROUPS = 8;

__device__ __forceinline__ void v2r_kahan(float4& s, float4& e, const float4 v) {
  auto one = [](float& sv, float& ev, float x) {
    const float y = x - ev, tk = sv + y;
    ev = (tk - sv) - y;
    sv = tk;
  };
  one(s.x, e.x, v.x);
  one(s.y, e.y, v.y);
  one(s.z, e.z, v.z);
  one(s.w, e.w, v.w);
}

__global__ void __launch_bounds__(V2R_COLS* V2R_GROUPS) k_v2_reduce(const float4* __restrict__ partials, int nQ,
                                                                     int nG, int n4, const float* __restrict__ dotQ,
                                                                     float* __restrict__ qxout,
                                                                     float* __restrict__ tnout, const int* done) {
  __shared__ float4 sh[2][V2R_GROUPS][V2R_COLS];
  if (done && *(volatile const int*)done) return;
  const int col = threadIdx.x % V2R_COLS, gi = threadIdx.x / V2R_COLS;
  const int c4 = blockIdx.x * V2R_COLS + col;
  const bool in = c4 < n4;
  for (int which = 0; which < (tnout ? 2 : 1); ++which) {
    const int c0 = which == 0 ? 0 : nQ, c1 = which == 0 ? nQ : nQ + nG;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f), e = s;
    if (in)
      for (int cc = c0 + gi; cc < c1; cc += V2R_GROUPS) v2r_kahan(s, e, partials[(size_t)cc * n4 + c4]);
    sh[0][gi][col] = s;
    sh[1][gi][col] = make_float4(-e.x, -e.y, -e.z, -e.w);
    __syncthreads();
    if (gi == 0 && in) {
      double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
      for (int q = 0; q < V2R_GROUPS; ++q) {
        const float4 h = sh[0][q][col], l = sh[1][q][col];
        r0 += double(h.x) + double(l.x);
        r1 += double(h.y) + double(l.y);
        r2 += double(h.z) + double(l.z);
        r3 += double(h.w) + double(l.w);
      }
      if (which == 0) {
        const float4 d = ((const float4*)dotQ)[c4];
        ((float4*)qxout)[c4] = make_float4(float(r0 + d.x), float(r1 + d.y), float(r2 + d.z), float(r3 + d.w));
      } else {
        ((float4*)tnout)[c4] = make_float4(float(r0), float(r1), float(r2), float(r3));
      }
    }
    __syncthreads();
  }
}

// Packed upper triangle: row i holds columns 4 floor(i/4) .. n-1, zeros left of
// the diagonal, half the diagonal.
__global__ void k_pack_upper(const float* __restrict__ Q, int n, const long long* __restrict__ qoff,
                             float* __restrict__ Qp) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int i0 = i & ~3;
    float* dst = Qp + qoff[i];
    for (int j = i0 + threadIdx.x; j < n; j += blockDim.x) {
      const float v = Q[(size_t)i * n + j];
      dst[j - i0] = j < i ? 0.f : (j == i ? 0.5f * v : v);
    }
  }
}

}  // namespace dq
