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
//     iteration, so the same row (held in shared memory) adds w_j G_j to
//     G' w of the next iteration.  Rows arrive by double-buffered bulk copies.
// A CTA is either a Q-CTA (a contiguous range of packed rows with about the
// same element count as every other CTA) or a G-CTA (a range of G rows).
// Each keeps its column partial sums for the 512 threads' own columns in
// registers and writes one partial vector; k_v2_reduce adds the partial
// vectors in CTA order (deterministic) and the row dots.  HBM bytes per
// iteration: 4 (n(n+1)/2 + p n) instead of 4 (n^2 + 2 p n).
#pragma once
#include "dq_common.cuh"
#include "tc_common.cuh"

namespace dq {

struct V2Args {
  int n, p, n4;                       // n4 = n / 4 (n a multiple of 4)
  int nQ, nG;
  const int* qrow;                    // nQ + 1 row bounds of the Q-CTAs
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
};

static constexpr int V2_THREADS = 512;
static constexpr int V2_RB = 64;  // rows between flushes of the row-dot partials

template <int NPT>
__global__ void __launch_bounds__(V2_THREADS, 1) k_v2_pass(V2Args a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ float sdot[V2_RB][V2_THREADS / 32];
  __shared__ double sred[V2_THREADS / 32 + 1];
  if (a.done && *(volatile const int*)a.done) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool qcta = blockIdx.x < a.nQ;
  // prologue: x^k = [y - grad(y)/L]_U for this thread's columns (float4 units t + 512 m)
  float4 xr[NPT];
  const float b = a.beta_prev;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int c4 = t + V2_THREADS * m;
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c4 < a.n4) {
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
      const int per = (a.n4 + gridDim.x - 1) / gridDim.x;
      if (c4 >= blockIdx.x * per && c4 < (blockIdx.x + 1) * per) ((float4*)a.xout)[c4] = o;
    }
    xr[m] = o;
  }
  float4 part[NPT];
#pragma unroll
  for (int m = 0; m < NPT; ++m) part[m] = make_float4(0.f, 0.f, 0.f, 0.f);

  if (qcta) {
    // rows c, c + nQ, c + 2 nQ, ... (every CTA gets the same mix of long and
    // short rows), streamed through a double buffer of bulk copies
    const int c = blockIdx.x, nQ = a.nQ;
    const int cnt = c < a.n ? (a.n - 1 - c) / nQ + 1 : 0;
    float* xs = (float*)(sm + 2 * (size_t)a.n4 * 16);  // x_i of this CTA's rows
    auto qbuf = [&](int s) { return (const float4*)(sm + (size_t)s * a.n4 * 16); };
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      const int c4 = t + V2_THREADS * m;
      if (c4 < a.n4) {
        const float xv[4] = {xr[m].x, xr[m].y, xr[m].z, xr[m].w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * c4 + u;
          if (i >= c && (i - c) % nQ == 0) xs[(i - c) / nQ] = xv[u];
        }
      }
    }
    if (t == 0) {
      tc::mbar_init(&full[0], 1);
      tc::mbar_init(&full[1], 1);
      tc::mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int idx, int s) {
      const int i = c + idx * nQ;
      const uint32_t bytes = (uint32_t)(a.n - (i & ~3)) * 4u;
      tc::mbar_expect_tx(&full[s], bytes);
      tc::bulk_g2s((void*)qbuf(s), a.Qp + a.qoff[i], bytes, &full[s]);
    };
    if (t == 0)
      for (int s = 0; s < 2 && s < cnt; ++s) issue(s, s);
    for (int rb = 0; rb < cnt; rb += V2_RB) {
      const int re = min(cnt, rb + V2_RB);
      for (int idx = rb; idx < re; ++idx) {
        const int i = c + idx * nQ;
        const int s = idx & 1;
        tc::mbar_wait(&full[s], (idx >> 1) & 1, 2000000000ull);
        const float4* row = qbuf(s);
        const int f0 = i >> 2;  // first float4 column of the packed row
        const float xi = xs[idx];
        float sa = 0.f, comp = 0.f;
#pragma unroll
        for (int m = 0; m < NPT; ++m) {
          const int c4 = t + V2_THREADS * m;
          if (c4 >= f0 && c4 < a.n4) {
            const float4 v = row[c4 - f0];
            float d = v.x * xr[m].x;
            d = fmaf(v.y, xr[m].y, d);
            d = fmaf(v.z, xr[m].z, d);
            d = fmaf(v.w, xr[m].w, d);
            const float yk = d - comp, tk = sa + yk;  // Kahan pair
            comp = (tk - sa) - yk;
            sa = tk;
            part[m].x = fmaf(xi, v.x, part[m].x);
            part[m].y = fmaf(xi, v.y, part[m].y);
            part[m].z = fmaf(xi, v.z, part[m].z);
            part[m].w = fmaf(xi, v.w, part[m].w);
          }
        }
        double tot = double(sa) - double(comp);
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
        if (lane == 0) sdot[idx - rb][warp] = float(tot);
        __syncthreads();  // buffer s free again
        if (t == 0 && idx + 2 < cnt) issue(idx + 2, s);
      }
      if (t < re - rb) {
        double s = 0.0;
        for (int w = 0; w < V2_THREADS / 32; ++w) s += sdot[t][w];
        a.dotQ[c + (rb + t) * nQ] = float(s);
      }
      __syncthreads();
    }
  } else {
    // G rows through a double buffer of bulk copies
    const int gi = blockIdx.x - a.nQ;
    const int j0 = a.grow[gi], j1 = a.grow[gi + 1];
    auto buf = [&](int s) { return (float4*)(sm + (size_t)s * a.n4 * 16); };
    const uint32_t rowb = (uint32_t)a.n4 * 16;
    if (t == 0) {
      tc::mbar_init(&full[0], 1);
      tc::mbar_init(&full[1], 1);
      tc::mbar_init_fence();
    }
    __syncthreads();
    if (t == 0) {
      for (int s = 0; s < 2 && j0 + s < j1; ++s) {
        tc::mbar_expect_tx(&full[s], rowb);
        tc::bulk_g2s(buf(s), a.G + (size_t)(j0 + s) * a.n, rowb, &full[s]);
      }
    }
    bool ok = true;
    for (int j = j0; j < j1; ++j) {
      const int s = (j - j0) & 1;
      const uint32_t ph = ((j - j0) >> 1) & 1;
      ok = ok && tc::mbar_wait(&full[s], ph, 2000000000ull);
      float sacc = 0.f, comp = 0.f;
#pragma unroll
      for (int m = 0; m < NPT; ++m) {
        const int c4 = t + V2_THREADS * m;
        if (c4 < a.n4) {
          const float4 v = buf(s)[c4];
          float d = v.x * xr[m].x;
          d = fmaf(v.y, xr[m].y, d);
          d = fmaf(v.z, xr[m].z, d);
          d = fmaf(v.w, xr[m].w, d);
          const float yk = d - comp, tk = sacc + yk;
          comp = (tk - sacc) - yk;
          sacc = tk;
        }
      }
      double tot = double(sacc) - double(comp);
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
      if (lane == 0) sred[warp] = tot;
      __syncthreads();
      if (t == 0) {
        double r = 0.0;
        for (int w = 0; w < V2_THREADS / 32; ++w) r += sred[w];
        sred[V2_THREADS / 32] = r;
      }
      __syncthreads();
      const float r = float(sred[V2_THREADS / 32]);
      // G x^k, and w of the next iteration from G y^{k+1} = G x^k + beta (G x^k - G x^{k-1})
      const float gx1 = a.gx1[j];
      const float gy = r + a.beta_next * (r - gx1);
      const float v = a.mu[j] + a.rho * (gy + a.g[j]);
      const float w = a.cone == CONE_EQ ? v : (v > 0.f ? v : 0.f);
      if (t == 0) a.gxout[j] = r;
#pragma unroll
      for (int m = 0; m < NPT; ++m) {
        const int c4 = t + V2_THREADS * m;
        if (c4 < a.n4) {
          const float4 gv = buf(s)[c4];
          part[m].x = fmaf(w, gv.x, part[m].x);
          part[m].y = fmaf(w, gv.y, part[m].y);
          part[m].z = fmaf(w, gv.z, part[m].z);
          part[m].w = fmaf(w, gv.w, part[m].w);
        }
      }
      __syncthreads();  // buffer s free again
      if (t == 0 && j + 2 < j1) {
        tc::mbar_expect_tx(&full[s], rowb);
        tc::bulk_g2s(buf(s), a.G + (size_t)(j + 2) * a.n, rowb, &full[s]);
      }
    }
    (void)ok;
  }
  float4* out = a.partials + (size_t)blockIdx.x * a.n4;
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int c4 = t + V2_THREADS * m;
    if (c4 < a.n4) out[c4] = part[m];
  }
}

// Q x^k = row dots + column partials of the Q-CTAs; G' w(y^{k+1}) = column
// partials of the G-CTAs.  Partials are added in CTA order in FP64.
__global__ void k_v2_reduce(const float4* __restrict__ partials, int nQ, int nG, int n4,
                            const float* __restrict__ dotQ, float* __restrict__ qxout, float* __restrict__ tnout,
                            const int* done) {
  if (done && *(volatile const int*)done) return;
  for (int c4 = blockIdx.x * blockDim.x + threadIdx.x; c4 < n4; c4 += gridDim.x * blockDim.x) {
    double q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    for (int c = 0; c < nQ; ++c) {
      const float4 v = partials[(size_t)c * n4 + c4];
      q0 += v.x; q1 += v.y; q2 += v.z; q3 += v.w;
    }
    const float4 d = ((const float4*)dotQ)[c4];
    ((float4*)qxout)[c4] = make_float4(float(q0 + d.x), float(q1 + d.y), float(q2 + d.z), float(q3 + d.w));
    if (tnout) {
      double w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      for (int c = nQ; c < nQ + nG; ++c) {
        const float4 v = partials[(size_t)c * n4 + c4];
        w0 += v.x; w1 += v.y; w2 += v.z; w3 += v.w;
      }
      ((float4*)tnout)[c4] = make_float4(float(w0), float(w1), float(w2), float(w3));
    }
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
