// cta_engine.cuh -- whole-solve-per-thread-block engine.
//
// One CTA runs the complete Algorithm DFOM (arXiv 1504.05708, Sec. 3) for one
// QP instance: every inner Algorithm FOM iteration (Sec. 2.1), every dual
// update, the primal averaging (eq. average_primal), the last-iterate solve
// (eq. last_primal) and the stopping certificate, without returning to the
// host.  A persistent grid pulls instances from a device work queue, so one
// launch solves a batch of instances of different sizes and algorithms.
//
// Data layout: vectors live in shared memory; Q (n x n), G (p x n) and its
// transpose GT (n x p), row-major, are staged into shared memory when they
// fit and read through L2 otherwise.  Every matrix-vector product is written
// as out = M' v with one thread per output column, so each step of the
// reduction loop is a coalesced row read of M, and the summation order is
// fixed (results do not depend on which CTA runs the instance or what else
// is in the batch).
//
// Inner iteration in "x-side" form: the gradient of L_rho(., mu) at
// y = x^k + beta (x^k - x^{k-1}) needs Q y and G y, which are linear in y, so
// Q x^k and G x^k are carried and Q y = Q x^k + beta (Q x^k - Q x^{k-1}).  The
// matrix products per iteration are Q x^k, G x^k and G' w (rho > 0) or Q x^k
// alone (rho = 0, with c = q + G' mu formed once per outer iteration, the
// precomputation the paper's bottleneck section describes), and the gradient
// at x^k for the stopping certificate comes for free when rho = 0.
#pragma once
#include "dq_common.cuh"

namespace dq {

template <typename T>
struct CtaInst {
  int n, p, cone, alg;
  const T *Q, *G, *GT;            // device matrices
  const T *q, *g, *lb, *ub;       // device vectors
  double lmax_Q, lmin_Q, normG2;  // NaN lmax_Q / normG2: Lanczos estimate (or bound) on chip
  int lip_bound;                  // 1: guaranteed bounds instead of the Lanczos estimate
  int stop_fstar;                 // 1: outer stop on |F - f_star| instead of F - d_lb
  double f_star;
  double rho;                     // NaN: 0 for DGM/DFGM, 1/||G||^2 for ADGM/ADFGM
  double LL, sigma, Ld;           // NaN: derived (Sec. 3 Step 1, eq. Ld)
  int inner_fixed, inner_check_every, max_inner;
  int cert_step;                  // 1: step certificate of y^k -> x^k (FP64, sigma > 0)
  double eps_in;
  int outer_fixed, check_every, max_outer;
  double eps_out;
  int want_last, want_avg, kd_plus;
  const T *x0, *lam0;             // warm start (nullable)
  T *x_state, *lam_state;         // final ubar^k and lambda^k (nullable)
  T *x_last, *x_avg, *lam_out;    // outputs (nullable)
  DevResult *res;
  double *consts_out;             // nullable: lmax_Q, normG2, LL, Ld, sigma, rho
};

// out[i] = sum_j M[j*ld + i] v[j], i < cols, j < rows  (out = M' v).
// Work units of one lane: cpw columns 32 apart (cpw = 4 for cols >= 128, 2 for
// cols >= 64, else 1; a warp's load covers 128 contiguous bytes) over one of S
// contiguous row segments, S chosen for about 512 units (FP32: S = 1 for
// products of at most 4096 terms, where the split costs more than it saves;
// FP64: at least 256 units, because the FP64 pipe is slow and a long
// dependent chain per lane left most warps waiting at the next barrier, e.g.
// 64 lanes with 25 FMAs each at n = 50).  A unit walks its rows
// four at a time (16 loads in flight for cpw = 4), even rows into one
// accumulator and odd rows into another (four accumulators by row mod 4
// measured slower for FP64 at n = 50), and the S segment sums in `part`
// (at most 2048 elements) are added in segment order (FP32) or as a tree
// (FP64, where the add latency counts).  Every sum's order is fixed
// by (rows, cols) alone: results do not depend on the block size or on whether
// M sits in shared or global memory.
template <typename A, typename T, typename V>
__device__ __forceinline__ void mtv(const T* __restrict__ M, int rows, int cols, int ld,
                                    const V* __restrict__ v, A* __restrict__ out, A* __restrict__ part) {
  // FP64 (the small exact-parity instances) keeps one column per lane: four
  // columns of doubles would not stay in registers
  const int cpw = sizeof(T) == 8 ? 1 : (cols >= 128 ? 4 : (cols >= 64 ? 2 : 1));
  const int bw = 32 * cpw, units = ((cols + bw - 1) / bw) * 32;
  // small FP32 products (a few thousand terms) skip the segment split and its barrier
  const int S = sizeof(T) == 8 ? (units >= 256 ? 1 : min(8, 256 / units))
                               : ((units >= 512 || (long long)rows * cols <= 4096) ? 1 : min(8, 512 / units));
  for (int q = threadIdx.x; q < S * units; q += blockDim.x) {
    const int sg = q / units, rem = q - sg * units;
    const int cbase = (rem >> 5) * bw + (rem & 31);
    const int r0 = (int)((long long)rows * sg / S), r1 = (int)((long long)rows * (sg + 1) / S);
    A e[4], o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = o[u] = A(0);
    bool cv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) cv[u] = u < cpw && cbase + 32 * u < cols;
    int j = r0;
    for (; j + 4 <= r1; j += 4) {
      T m[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int u = 0; u < 4; ++u) m[r][u] = cv[u] ? M[(size_t)(j + r) * ld + cbase + 32 * u] : T(0);
      const A v0 = A(v[j]), v1 = A(v[j + 1]), v2 = A(v[j + 2]), v3 = A(v[j + 3]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        e[u] += A(m[0][u]) * v0;
        o[u] += A(m[1][u]) * v1;
        e[u] += A(m[2][u]) * v2;
        o[u] += A(m[3][u]) * v3;
      }
    }
    for (; j < r1; ++j) {
      const A vj = A(v[j]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const A mv = cv[u] ? A(M[(size_t)j * ld + cbase + 32 * u]) : A(0);
        if ((j - r0) & 1) o[u] += mv * vj;
        else e[u] += mv * vj;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!cv[u]) continue;
      const int c = cbase + 32 * u;
      if (S == 1) out[c] = e[u] + o[u];
      else part[sg * cols + c] = e[u] + o[u];
    }
  }
  if (S > 1) {
    __syncthreads();
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
      if constexpr (sizeof(A) == 8) {  // FP64: a three-level tree (zeros past S)
        A r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = k < S ? part[k * cols + c] : A(0);
        out[c] = ((r[0] + r[1]) + (r[2] + r[3])) + ((r[4] + r[5]) + (r[6] + r[7]));
      } else {
        A r = part[c];
        for (int sg = 1; sg < S; ++sg) r += part[sg * cols + c];
        out[c] = r;
      }
    }
  }
}

// Same product with the accurate accumulator of the element type (FP64 or Dot2).
template <typename T>
__device__ __forceinline__ void mtv_acc(const T* __restrict__ M, int rows, int cols, int ld,
                                        const T* __restrict__ v, double* __restrict__ out) {
  using Acc = typename AccurateAcc<T>::type;
  for (int i = threadIdx.x; i < cols; i += blockDim.x) {
    const T* col = M + i;
    Acc a;
    for (int j = 0; j < rows; ++j) a.add(col[(size_t)j * ld], v[j]);
    out[i] = a.get();
  }
}

template <typename T>
struct XState {  // three rotating buffers each for x, Q x, G x
  T *x, *xp, *xn;
  T *Qx, *Qxp, *Qxn;
  T *Gx, *Gxp, *Gxn;
};

template <typename T>
struct CtaWs {
  XState<T> A, B;        // main warm-start chain, extra last-iterate solve
  T *c, *tn, *w, *mu, *lam, *lamp, *ul, *uavg;
  double *usum, *dn, *dp, *red;
  T* part;               // 2048 partial sums of the segmented products
  const T *Q, *G, *GT;
};

template <typename T>
__device__ __forceinline__ void vcopy(T* __restrict__ d, const T* __restrict__ s, int m) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) d[i] = s[i];
}

// Certificate of eq. duquad_in at x (x, Q x, G x given): upper bound on
// L_rho(x, mu) - d_rho(mu).  sigma > 0: gradient-mapping bound
// <grad, x - x+> + ||L (x - x+)||^2 (1/(2 sigma) - 1/(2 L)); sigma = 0:
// Frank-Wolfe gap.  rho = 0 uses c = q + G' mu; rho > 0 forms G' w(x).
template <typename T>
__device__ double cta_cert(const CtaInst<T>& I, CtaWs<T>& W, const T* x, const T* Qx, const T* Gx,
                           const T* mu, bool c_valid) {
  const int n = I.n, p = I.p;
  const bool aug = I.rho > 0.0;
  const T rho = T(I.rho);
  if (aug) {
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      T v = mu[j] + rho * (Gx[j] + I.g[j]);
      W.w[j] = I.cone == CONE_EQ ? v : (v > T(0) ? v : T(0));
    }
    __syncthreads();
    mtv<T>(W.G, p, n, n, W.w, W.tn, W.part);
    __syncthreads();
  } else if (!c_valid) {
    mtv<T>(W.G, p, n, n, mu, W.tn, W.part);
    __syncthreads();
  }
  const double L = I.LL, sg = I.sigma;
  const double kap = sg > 0.0 ? 1.0 / (2.0 * sg) - 1.0 / (2.0 * L) : 0.0;
  double part = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T gr = aug ? (Qx[i] + I.q[i] + W.tn[i]) : (c_valid ? Qx[i] + W.c[i] : Qx[i] + I.q[i] + W.tn[i]);
    const double gd = double(gr), xd = double(x[i]);
    if (sg > 0.0) {
      const double xp = fmin(fmax(xd - gd / L, double(I.lb[i])), double(I.ub[i]));
      const double d = xd - xp;
      part += gd * d + (L * d) * (L * d) * kap;
    } else {
      const double a = gd * double(I.lb[i]), b = gd * double(I.ub[i]);
      part += gd * xd - (a < b ? a : b);
    }
  }
  return block_sum(part, W.red);
}

// Algorithm FOM on phi = L_rho(., mu) over the box, warm-started from S.x
// (with S.Qx and, for rho > 0, S.Gx valid).  On return S.x = ubar, S.Qx = Q ubar,
// S.Gx = G ubar.  Inner variant: FGM_sigma when sigma > 0, else FGM.
template <typename T>
__device__ int cta_fom(const CtaInst<T>& I, CtaWs<T>& W, XState<T>& S, const T* mu) {
  const int n = I.n, p = I.p;
  const bool aug = I.rho > 0.0;
  const T rho = T(I.rho), invL = T(1.0 / I.LL);
  if (!aug) {  // c = q + G' mu, fixed over the inner loop
    if (p > 0) {
      mtv<T>(W.G, p, n, n, mu, W.c, W.part);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) W.c[i] = (p > 0 ? W.c[i] : T(0)) + I.q[i];
  }
  vcopy(S.xp, S.x, n);
  vcopy(S.Qxp, S.Qx, n);
  if (aug) vcopy(S.Gxp, S.Gx, p);
  __syncthreads();
  const bool fgm_sigma = I.sigma > 0.0;
  const double beta_sigma = (sqrt(I.LL) - sqrt(I.sigma)) / (sqrt(I.LL) + sqrt(I.sigma));
  // theta: thread 0's copy of the FGM sequence.  The next weight beta_{k+1}
  // depends on theta_k alone, so thread 0 forms it during iteration k and
  // publishes it through W.red[38 + ((k + 1) & 1)] (double-buffered: the slot
  // it writes in iteration k + 1 was read before the barrier that follows
  // iteration k's step); every other thread skips the FP64 sqrt and
  // division, which a block of 8 to 16 warps would otherwise repeat on the
  // slow FP64 pipe each iteration.
  double theta = 1.0, beta = 0.0;
  const int m = I.inner_check_every > 0 ? I.inner_check_every : 1;
  int k = 0;
  for (;;) {
    ++k;
    const T b = T(beta);
    if (aug) {  // w = [mu + rho (G y + g)]_+ ,  tn = G' w
      for (int j = threadIdx.x; j < p; j += blockDim.x) {
        const T Gy = S.Gx[j] + b * (S.Gx[j] - S.Gxp[j]);
        const T v = mu[j] + rho * (Gy + I.g[j]);
        W.w[j] = I.cone == CONE_EQ ? v : (v > T(0) ? v : T(0));
      }
      __syncthreads();
      mtv<T>(W.G, p, n, n, W.w, W.tn, W.part);
      __syncthreads();
    }
    // step 1 of FOM: x^k = [y - grad phi(y) / L]_U
    auto plain_step = [&]() {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T y = S.x[i] + b * (S.x[i] - S.xp[i]);
        const T Qy = S.Qx[i] + b * (S.Qx[i] - S.Qxp[i]);
        const T gr = aug ? Qy + I.q[i] + W.tn[i] : Qy + W.c[i];
        S.xn[i] = clampT(y - gr * invL, I.lb[i], I.ub[i]);
      }
    };
    if constexpr (sizeof(T) == 8) {
      // FP64: the step certificate ||L (y^k - x^k)||^2 (1/(2 sigma) - 1/(2 L))
      // bounds phi(x^k) - phi* from the step itself; its sum waits in W.red[32].
      // (FP32 keeps the certificate at x^k: the extrapolated Q y carries about
      // (1 + 2 beta) times the rounding of one product, which the step
      // certificate squares.)
      if (I.cert_step && I.sigma > 0.0 && I.inner_fixed <= 0 && k % m == 0) {
        T sq = T(0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          const T y = S.x[i] + b * (S.x[i] - S.xp[i]);
          const T Qy = S.Qx[i] + b * (S.Qx[i] - S.Qxp[i]);
          const T gr = aug ? Qy + I.q[i] + W.tn[i] : Qy + W.c[i];
          const T st = gr * invL, s = y - st;
          const T xn = clampT(s, I.lb[i], I.ub[i]);
          S.xn[i] = xn;
          // y - x^k is the step itself where the box is inactive (no cancellation)
          const T d = (s > I.lb[i] && s < I.ub[i]) ? st : y - xn;
          sq += d * d;
        }
        block_sum(double(sq), W.red);
      } else {
        plain_step();
      }
    } else {
      plain_step();
    }
    if (!fgm_sigma && threadIdx.x == 0) {  // step 2 weight of the next iteration (Sec. 2.1)
      const double tn1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
      W.red[38 + ((k + 1) & 1)] = (theta - 1.0) / tn1;
      theta = tn1;
    }
    __syncthreads();
    mtv<T>(W.Q, n, n, n, S.xn, S.Qxn, W.part);
    if (aug) {
      __syncthreads();
      mtv<T>(W.GT, n, p, p, S.xn, S.Gxn, W.part);
    }
    __syncthreads();
    // step 2 weight beta_k (GM/FGM/FGM_sigma rules, Sec. 2.1)
    beta = fgm_sigma ? beta_sigma : W.red[38 + ((k + 1) & 1)];
    T* t;
    t = S.xp; S.xp = S.x; S.x = S.xn; S.xn = t;
    t = S.Qxp; S.Qxp = S.Qx; S.Qx = S.Qxn; S.Qxn = t;
    if (aug) { t = S.Gxp; S.Gxp = S.Gx; S.Gx = S.Gxn; S.Gxn = t; }
    if (I.inner_fixed > 0) {
      if (k >= I.inner_fixed) break;
    } else {
      if (k % m == 0) {
        double cert;
        if constexpr (sizeof(T) == 8) {
          cert = (I.cert_step && I.sigma > 0.0) ? I.LL * I.LL * (0.5 / I.sigma - 0.5 / I.LL) * W.red[32]
                                                : cta_cert(I, W, S.x, S.Qx, S.Gx, mu, !aug);
        } else {
          cert = cta_cert(I, W, S.x, S.Qx, S.Gx, mu, !aug);
        }
        if (cert <= I.eps_in) break;
      }
      if (k >= I.max_inner) break;
    }
  }
  if (!aug && p > 0) {  // G ubar for the dual gradient
    mtv<T>(W.GT, n, p, p, S.x, S.Gx, W.part);
    __syncthreads();
  }
  return k;
}

// FP64-accurate evaluation at u: F(u), dist_K(Gu + g) and, when mu is given,
// L_rho(u, mu) (eq. auglag1) and the inner certificate at (u, mu).
struct EvalOut {
  double F, infeas, lagr, cert;
};

template <typename T>
__device__ EvalOut cta_eval(const CtaInst<T>& I, CtaWs<T>& W, const T* u, const T* mu) {
  const int n = I.n, p = I.p;
  mtv_acc<T>(W.Q, n, n, n, u, W.dn);
  if (p > 0) mtv_acc<T>(W.GT, n, p, p, u, W.dp);
  __syncthreads();
  double pf = 0.0, pi = 0.0, pl = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    pf += 0.5 * double(u[i]) * W.dn[i] + double(I.q[i]) * double(u[i]);
  const double rho = I.rho;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double r = W.dp[j] + double(I.g[j]);
    const double d = r - proj_K(I.cone, r);
    pi += d * d;
    if (mu) {
      const double mj = double(mu[j]);
      if (rho > 0.0) {
        const double z = r + mj / rho;
        const double dz = z - proj_K(I.cone, z);
        pl += 0.5 * rho * dz * dz - mj * mj / (2.0 * rho);
      } else {
        pl += mj * r;
      }
    }
  }
  EvalOut e;
  e.F = block_sum(pf, W.red);
  e.infeas = sqrt(block_sum(pi, W.red));
  e.lagr = e.cert = NAN;
  if (!mu) return e;
  e.lagr = e.F + block_sum(pl, W.red);
  // gradient of L_rho(., mu) at u, accumulated accurately
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const double r = W.dp[j] + double(I.g[j]);
    const double mj = double(mu[j]);
    double w;
    if (rho > 0.0) {
      const double z = r + mj / rho;
      w = rho * (z - proj_K(I.cone, z));
    } else {
      w = mj;
    }
    W.dp[j] = w;
  }
  __syncthreads();
  using Acc = typename AccurateAcc<T>::type;
  const double L = I.LL, sg = I.sigma;
  const double kap = sg > 0.0 ? 1.0 / (2.0 * sg) - 1.0 / (2.0 * L) : 0.0;
  double pc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double gsum;
    if (sizeof(T) == 8) {
      double a = 0.0;
      for (int j = 0; j < p; ++j) a = fma(double(W.G[(size_t)j * n + i]), W.dp[j], a);
      gsum = a;
    } else {
      Acc a;
      for (int j = 0; j < p; ++j) {
        // split the FP64 weight into two floats so the product stays accurate
        const float hi = float(W.dp[j]);
        const float lo = float(W.dp[j] - double(hi));
        a.add(float(W.G[(size_t)j * n + i]), hi);
        a.add(float(W.G[(size_t)j * n + i]), lo);
      }
      gsum = a.get();
    }
    const double gd = W.dn[i] + double(I.q[i]) + gsum;
    const double xd = double(u[i]);
    if (sg > 0.0) {
      const double xp = fmin(fmax(xd - gd / L, double(I.lb[i])), double(I.ub[i]));
      const double d = xd - xp;
      pc += gd * d + (L * d) * (L * d) * kap;
    } else {
      const double a = gd * double(I.lb[i]), b = gd * double(I.ub[i]);
      pc += gd * xd - (a < b ? a : b);
    }
  }
  e.cert = block_sum(pc, W.red);
  return e;
}

// Bit-level helpers of the Sturm count: sign bit, biased exponent, and an
// exact zero, read from the representation (integer instructions: FP64
// comparisons issue on the FP64 pipe, which runs at 1/64 of the FP32 rate on
// this GPU).
__device__ __forceinline__ unsigned tri_sign(double v) { return (unsigned)__double2hiint(v) >> 31; }
__device__ __forceinline__ unsigned tri_sign(float v) { return __float_as_uint(v) >> 31; }
__device__ __forceinline__ int tri_exp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ __forceinline__ int tri_exp(float v) { return (int)((__float_as_uint(v) >> 23) & 0xff); }
__device__ __forceinline__ bool tri_zero(double v) { return ((unsigned long long)__double_as_longlong(v) << 1) == 0ull; }
__device__ __forceinline__ bool tri_zero(float v) { return (__float_as_uint(v) << 1) == 0u; }

// Number of eigenvalues below x of the symmetric tridiagonal matrix T with
// diagonal a and squared off-diagonal bq (bq[i] = b_i^2, b_i joining rows i
// and i + 1), in precision R and scaled so that |a_i|, |b_i| <= 1 (the FP32
// rounds read float copies: no conversion from FP64 per step): the number of
// sign changes along the leading principal
// minors p_0 = 1, p_1, ..., p_m of T - x I (Sturm), from the three-term
// recurrence p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2}, in precision R.
// No division (the pivot form d_i = p_i / p_{i-1} divides every step).  A
// step's roundings act as relative perturbations of a few units in the last
// place of a_i - x and b_{i-1}^2 (and a common factor of the tail of the
// sequence, which keeps its signs), so the count is exact for a nearby
// matrix, as for the pivot form.  With |a_i - x| <= 2 and b^2 <= 1 a minor
// grows at most threefold per step; the pair (p_{i-1}, p_i) is rescaled by
// 2^-+E when both fall below 2^-E or one rises above 2^E.  An exactly zero
// minor becomes -2^-40 p_{i-1} (a tiny negative pivot).
template <typename R>
__device__ __forceinline__ int tri_count_below(const R* a, const R* bq, int m, R x) {
  constexpr int bias = sizeof(R) == 8 ? 1023 : 127, E = sizeof(R) == 8 ? 400 : 40;
  const R up = sizeof(R) == 8 ? R(0x1p400) : R(0x1p40), dn = sizeof(R) == 8 ? R(0x1p-400) : R(0x1p-40);
  R q0 = R(0), q1 = R(1);
  int cnt = 0;
  for (int i = 0; i < m; ++i) {
    const R b2 = i > 0 ? bq[i - 1] : R(0);
    R pv = (a[i] - x) * q1 - b2 * q0;
    if (tri_zero(pv)) pv = -q1 * R(0x1p-40);
    cnt += (int)(tri_sign(pv) ^ tri_sign(q1));
    q0 = q1;
    q1 = pv;
    const int e = max(tri_exp(q0), tri_exp(q1));
    if (e < bias - E) {
      q0 *= up;
      q1 *= up;
    } else if (e > bias + E) {
      q0 *= dn;
      q1 *= dn;
    }
  }
  return cnt;
}

// One round of 33-way multisection of [lo, hi] (which holds the largest
// eigenvalue) by the 32 lanes of a warp: lane l tests lo + (hi - lo)(l + 1)/33.
template <typename R>
__device__ __forceinline__ void tri_multisect(const R* a, const R* bq, int m, R& lo, R& hi) {
  const int lane = threadIdx.x & 31;
  const R x = lo + (hi - lo) * (R(lane + 1) / R(33));
  const unsigned ball = __ballot_sync(0xffffffffu, tri_count_below<R>(a, bq, m, x) == m);  // x above all
  const int first = ball ? __ffs(ball) - 1 : 32;
  const R nhi = first < 32 ? __shfl_sync(0xffffffffu, x, first) : hi;
  const R nlo = first > 0 ? __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0) : lo;
  lo = nlo;
  hi = nhi;
}

// Largest eigenvalue theta of the m x m symmetric tridiagonal matrix (a, b)
// and |s_m|, the last component of its unit eigenvector, in FP64 (one warp;
// m <= 160).  a is first divided in place by the power of two s >= the
// Gershgorin bound (exact) and b (b[0..m-2]) replaced by (b_i / s)^2, with
// float copies in fa, fb (m floats each, caller's scratch) and the
// reciprocals s / b_i across the lanes; then: multisection on Sturm counts,
// in FP32 to a bracket of relative width 1e-6, then in FP64 from that bracket
// widened by 1e-5 (checked by two FP64 Sturm counts; the Gershgorin interval
// when the check fails) to 1e-13; then the three-term eigenvector recurrence
// (rescaled) at the bracket's upper end, taking b_{i-1} as
// b_{i-1}^2 (1 / b_{i-1}).  Results in out[0] (theta, unscaled), out[1].
__device__ inline void warp_tridiag_top(double* a, double* b, int m, double* out, float* fa, float* fb) {
  static_assert(kLzMaxSteps <= 160, "five reciprocals per lane");
  const int lane = threadIdx.x & 31;
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = lane; i < m; i += 32) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
    glo = fmin(glo, a[i] - r);
    ghi = fmax(ghi, a[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  const double M = fmax(fabs(glo), fabs(ghi));
  if (!(M < INFINITY)) {  // a non-finite recurrence: no estimate
    if (lane == 0) {
      out[0] = M;
      out[1] = 1.0;
    }
    __syncwarp();
    return;
  }
  int ex = 0;
  frexp(M, &ex);
  const double s = M > 0.0 ? ldexp(1.0, ex) : 1.0, inv_s = 1.0 / s;
  double rb[5];  // 1 / b_i for i = lane + 32 k
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = lane + 32 * k;
    rb[k] = 0.0;
    if (i < m) {
      const double as = a[i] * inv_s;
      a[i] = as;
      fa[i] = float(as);
      if (i + 1 < m) {
        const double bs = b[i] * inv_s, b2 = bs * bs;
        rb[k] = bs != 0.0 ? 1.0 / bs : 0.0;
        b[i] = b2;
        fb[i] = float(b2);
      }
    }
  }
  __syncwarp();
  glo *= inv_s;
  ghi *= inv_s;
  float flo = float(glo), fhi = float(ghi);
  for (int round = 0; round < 8; ++round) {
    tri_multisect<float>(fa, fb, m, flo, fhi);
    if (fhi - flo <= 1e-6f * fmaxf(fabsf(flo), fabsf(fhi))) break;
  }
  const double sc = fmax(fabs(double(flo)), fabs(double(fhi)));
  double lo = double(flo) - 1e-5 * sc - 1e-300, hi = double(fhi) + 1e-5 * sc + 1e-300;
  {  // lane 0: some eigenvalue is >= lo; lane 1: every eigenvalue is < hi
    const int c = tri_count_below<double>(a, b, m, lane == 0 ? lo : hi);
    const bool okl = __shfl_sync(0xffffffffu, c, 0) < m, okh = __shfl_sync(0xffffffffu, c, 1) == m;
    if (!(okl && okh)) {
      lo = glo;
      hi = ghi;
    }
  }
  for (int round = 0; round < 14; ++round) {
    if (hi - lo <= 1e-13 * fmax(fabs(lo), fabs(hi))) break;
    tri_multisect<double>(a, b, m, lo, hi);
  }
  // the recurrence, run by every lane alike (each holds part of the reciprocals)
  double upv = 0.0, u = 1.0, nrm2 = 1.0, rbp = 0.0;
  for (int i = 0; i + 1 < m; ++i) {
    const int k = i >> 5;
    const double rk = k == 0 ? rb[0] : k == 1 ? rb[1] : k == 2 ? rb[2] : k == 3 ? rb[3] : rb[4];
    const double rbi = __shfl_sync(0xffffffffu, rk, i & 31);
    const double bprev = i > 0 ? b[i - 1] * rbp : 0.0;  // b_{i-1} = b_{i-1}^2 / b_{i-1}
    rbp = rbi;
    if (tri_zero(rbi)) {  // b_i = 0: the matrix splits, the leading block's vector ends here
      upv = 0.0;
      u = 1.0;
      nrm2 = 1.0;
      continue;
    }
    const double un = ((hi - a[i]) * u - bprev * upv) * rbi;
    upv = u;
    u = un;
    nrm2 += u * u;
    if (tri_exp(nrm2) > 1023 + 660) {
      const double sq = 1.0 / sqrt(nrm2);
      upv *= sq;
      u *= sq;
      nrm2 = 1.0;
    }
  }
  if (lane == 0) {
    out[0] = hi * s;
    out[1] = fabs(u) / sqrt(nrm2);
  }
  __syncwarp();
}

// lambda_max of Q (which = 0) or G'G (which = 1) by the Lanczos method
// without reorthogonalisation (only the extreme Ritz value is used), from the
// SplitMix64 start vector, for lz_min_steps(n) steps (at most kLzMaxSteps;
// all n when n is smaller, the exhausted case): the top Ritz value theta of
// T_k and its residual r = beta_k |s_k| give lz_estimate (theta / (1 - eps)
// or theta + 2 r, whichever is larger).  Products in T, the three-term
// recurrence and the tridiagonal eigenproblem in FP64.
// Scratch: A.x, B.x, A.Qx, A.Gx, dn, usum (and A.xp, A.xn for the
// tridiagonal solve's float copies).
// The same Lanczos for FP32 instances with n, p <= 64, run by warp 0 alone
// (the block waits once): at these sizes the block version spent most of
// its time in the barriers of its block reductions (about nine per step).
// Lane l holds rows l and l + 32 of v and w; a product out = M' v reads
// column i of M (conflict-free in shared memory) with a sequential FP32 sum
// over the rows, as the block version's products, and the dot products are
// FP64 butterflies, so every sum has a fixed order.  Result in out[0].
__device__ inline void warp_lanczos(const CtaInst<float>& I, CtaWs<float>& W, int which, double* out) {
  const int n = I.n, p = I.p, lane = threadIdx.x & 31;
  float* v = W.A.x;   // the current Lanczos vector (every product reads all of it)
  float* t = W.A.Gx;  // G v (which = 1)
  double* al = W.dn;
  double* be = W.usum;
  auto wsum = [](double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  // out[i] = sum_j A[j * lda + i] x[j] over j < rows, this lane's i = l, l + 32
  auto prod = [&](const float* A, int rows, int cols, int lda, const float* x, double (&o)[2]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      float s = 0.f;
      if (i < cols)
        for (int j = 0; j < rows; ++j) s = fmaf(A[j * lda + i], x[j], s);
      o[h] = double(s);
    }
  };
  double vl[2], vpl[2] = {0.0, 0.0}, wl[2];
  double ps = 0.0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    vl[h] = i < n ? lz_start((unsigned long long)i) : 0.0;
    ps += vl[h] * vl[h];
  }
  const double inv = 1.0 / sqrt(wsum(ps));
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    vl[h] = i < n ? double(float(vl[h] * inv)) : 0.0;  // the vector the products see
    if (i < n) v[i] = float(vl[h]);
  }
  __syncwarp();
  const int ksteps = min(lz_min_steps(n), kLzMaxSteps);
  double beta_prev = 0.0, theta = 0.0, r = 0.0;
  bool exhausted = false;
  for (int j = 0; j < ksteps; ++j) {
    if (which == 0) {
      prod(W.Q, n, n, n, v, wl);
    } else {
      double tl[2];
      prod(W.GT, n, p, p, v, tl);  // t = G v (columns of G')
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (lane + 32 * h < p) t[lane + 32 * h] = float(tl[h]);
      __syncwarp();
      prod(W.G, p, n, n, t, wl);   // w = G' t
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) wl[h] = lane + 32 * h < n ? wl[h] : 0.0;
    const double alpha = wsum(vl[0] * wl[0] + vl[1] * wl[1]);
    double pb = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double rr = lane + 32 * h < n ? wl[h] - alpha * vl[h] - beta_prev * vpl[h] : 0.0;
      wl[h] = rr;
      pb += rr * rr;
    }
    const double beta = sqrt(wsum(pb));
    if (lane == 0) {
      al[j] = alpha;
      be[j] = beta;
    }
    const bool invariant = !(beta > 1e-300);
    if (invariant || j + 1 == ksteps) {
      __syncwarp();
      warp_tridiag_top(al, be, j + 1, W.red + 34, (float*)W.A.xp, (float*)W.A.xn);
      __syncwarp();
      theta = W.red[34];
      r = beta * W.red[35];
      exhausted = invariant || j + 1 == n;
      break;
    }
    __syncwarp();  // every lane has read v in its products
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      vpl[h] = vl[h];
      vl[h] = i < n ? double(float(wl[h] / beta)) : 0.0;
      if (i < n) v[i] = float(vl[h]);
    }
    beta_prev = beta;
    __syncwarp();
  }
  if (lane == 0) out[0] = lz_estimate(theta, r, exhausted, 6.0e-8);
}

template <typename T>
__device__ double cta_lanczos(const CtaInst<T>& I, CtaWs<T>& W, int which) {
  const int n = I.n, p = I.p;
  if constexpr (sizeof(T) == 4) {
    if (n <= 64 && p <= 64) {
      __syncthreads();
      if (threadIdx.x < 32) warp_lanczos(I, W, which, W.red + 36);
      __syncthreads();
      const double est = W.red[36];
      __syncthreads();
      return est;
    }
  }
  T* v = W.A.x;
  T* vp = W.B.x;
  T* w = W.A.Qx;
  T* t = W.A.Gx;
  double* al = W.dn;
  double* be = W.usum;
  double ps = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double s = lz_start((unsigned long long)i);
    ps += s * s;
  }
  const double inv = 1.0 / sqrt(block_sum(ps, W.red));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    v[i] = T(lz_start((unsigned long long)i) * inv);
    vp[i] = T(0);
  }
  __syncthreads();
  const int ksteps = min(lz_min_steps(n), kLzMaxSteps);
  double theta = 0.0, r = 0.0, beta_prev = 0.0;
  bool exhausted = false;
  for (int j = 0; j < ksteps; ++j) {
    if (which == 0) {
      mtv<T>(W.Q, n, n, n, v, w, W.part);
    } else {
      mtv<T>(W.GT, n, p, p, v, t, W.part);
      __syncthreads();
      mtv<T>(W.G, p, n, n, t, w, W.part);
    }
    __syncthreads();
    double pa = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) pa += double(v[i]) * double(w[i]);
    const double alpha = block_sum(pa, W.red);
    double pb = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double rr = double(w[i]) - alpha * double(v[i]) - beta_prev * double(vp[i]);
      w[i] = T(rr);
      pb += rr * rr;
    }
    const double bsq = block_sum(pb, W.red);
    // beta and 1/beta (no division): one chain each on lane 0 of two warps,
    // published through W.red[34..35], instead of every warp repeating both
    for (int t = threadIdx.x >> 5; t < 2; t += (blockDim.x + 31) >> 5)
      if ((threadIdx.x & 31) == 0) W.red[34 + t] = t ? rsqrt(bsq) : sqrt(bsq);
    __syncthreads();
    const double beta = W.red[34], rbeta = W.red[35];
    if (threadIdx.x == 0) {
      al[j] = alpha;
      be[j] = beta;
    }
    const bool invariant = !(beta > 1e-300);
    if (invariant || j + 1 == ksteps) {
      __syncthreads();
      if (threadIdx.x < 32) warp_tridiag_top(al, be, j + 1, W.red + 34, (float*)W.A.xp, (float*)W.A.xn);
      __syncthreads();
      theta = W.red[34];
      r = beta * W.red[35];
      exhausted = invariant || j + 1 == n;
      break;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      vp[i] = v[i];
      v[i] = T(double(w[i]) * rbeta);
    }
    beta_prev = beta;
    __syncthreads();
  }
  __syncthreads();
  return lz_estimate(theta, r, exhausted, sizeof(T) == 8 ? 1.2e-16 : 6.0e-8);
}

// Both Lanczos runs of an FP64 instance (Q and G'G) in one loop: each step
// makes the three products (Q v1 beside G v2, then G' (G v2)) and takes the two
// runs' dot products in shared block reductions, so the runs share every
// barrier and keep two independent product chains on the FP64 pipe (at
// n = 50 the two runs one after the other were 1.0 of the 1.4 ms of a solve,
// the FP64 pipe about a quarter busy and the warps mostly waiting at
// barriers), and the two tridiagonal eigenproblems run at once on two warps.
// Each run's arithmetic is the single run's (cta_lanczos): the same start
// vector, step count, products and estimate.  Extra buffers: the B chain's
// Q x slots hold the second run's alpha and beta (n doubles each), and A.Qxn
// and B.Qxn the float copies of the two tridiagonal solves.
// Two block sums at once where only threads below `act` hold nonzero values
// (vectors of length act < blockDim): the other warps skip the shuffles,
// which would only keep the SM's FP64 pipe busy with zeros, and warp 0 adds
// the warp sums as a butterfly tree.
__device__ __forceinline__ void block_sum2(double a, double b, int act, double* red, double* out) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nwa = (min(act, (int)blockDim.x) + 31) >> 5;
  if (w < nwa) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
  __syncthreads();
  if (w < nwa && l == 0) {
    red[w] = a;
    red[16 + w] = b;
  }
  __syncthreads();
  if (w == 0) {
    double sa = l < nwa ? red[l] : 0.0, sb = l < nwa ? red[16 + l] : 0.0;
    for (int o = 1; o < nwa; o <<= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (l == 0) {
      red[32] = sa;
      red[33] = sb;
    }
  }
  __syncthreads();
  out[0] = red[32];
  out[1] = red[33];
}

__device__ inline void cta_lanczos_pair(const CtaInst<double>& I, CtaWs<double>& W, double* lmax_Q, double* normG2) {
  const int n = I.n, p = I.p;
  double *v1 = W.A.x, *vp1 = W.B.x, *w1 = W.A.Qx;            // Q run
  double *v2 = W.A.xp, *vp2 = W.A.xn, *w2 = W.A.Qxp, *t = W.A.Gx;  // G'G run
  double *al1 = W.dn, *be1 = W.usum, *al2 = W.B.Qx, *be2 = W.B.Qxp;
  double ps = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double s = lz_start((unsigned long long)i);
    ps += s * s;
  }
  const double inv = 1.0 / sqrt(block_sum(ps, W.red));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    v1[i] = v2[i] = lz_start((unsigned long long)i) * inv;
    vp1[i] = vp2[i] = 0.0;
  }
  __syncthreads();
  const int ksteps = min(lz_min_steps(n), kLzMaxSteps);
  double bprev1 = 0.0, bprev2 = 0.0, beta1 = 0.0, beta2 = 0.0;
  int m1 = 0, m2 = 0;  // steps recorded by each run (a run stops at an invariant subspace)
  bool on1 = true, on2 = true;
  for (int j = 0; j < ksteps && (on1 || on2); ++j) {
    // Q v1 and G v2 read different vectors and write different outputs: no
    // barrier between them, each with its own half of `part` (an FP64 split
    // product holds at most 256 partial sums, see mtv)
    if (on1) mtv<double>(W.Q, n, n, n, v1, w1, W.part);
    if (on2) mtv<double>(W.GT, n, p, p, v2, t, W.part + 1024);
    __syncthreads();
    if (on2) mtv<double>(W.G, p, n, n, t, w2, W.part);
    __syncthreads();
    double pa1 = 0.0, pa2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (on1) pa1 += v1[i] * w1[i];
      if (on2) pa2 += v2[i] * w2[i];
    }
    double al[2];
    block_sum2(pa1, pa2, n, W.red, al);
    double pb1 = 0.0, pb2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (on1) {
        const double rr = w1[i] - al[0] * v1[i] - bprev1 * vp1[i];
        w1[i] = rr;
        pb1 += rr * rr;
      }
      if (on2) {
        const double rr = w2[i] - al[1] * v2[i] - bprev2 * vp2[i];
        w2[i] = rr;
        pb2 += rr * rr;
      }
    }
    double bb[2];
    block_sum2(pb1, pb2, n, W.red, bb);
    // beta and 1/beta of both runs: one chain each on lane 0 of four warps
    // (four schedulers), published through W.red[34..37], instead of every
    // warp repeating all four on the shared FP64 pipe
    for (int t = threadIdx.x >> 5; t < 4; t += (blockDim.x + 31) >> 5)
      if ((threadIdx.x & 31) == 0) W.red[34 + t] = (t & 1) ? rsqrt(bb[t >> 1]) : sqrt(bb[t >> 1]);
    __syncthreads();
    const bool last = j + 1 == ksteps;
    const double rb1 = W.red[35], rb2 = W.red[37];
    if (on1) {
      beta1 = W.red[34];
      if (threadIdx.x == 0) {
        al1[j] = al[0];
        be1[j] = beta1;
      }
      m1 = j + 1;
    }
    if (on2) {
      beta2 = W.red[36];
      if (threadIdx.x == 0) {
        al2[j] = al[1];
        be2[j] = beta2;
      }
      m2 = j + 1;
    }
    const bool go1 = on1 && !last && beta1 > 1e-300, go2 = on2 && !last && beta2 > 1e-300;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (go1) {
        vp1[i] = v1[i];
        v1[i] = w1[i] * rb1;
      }
      if (go2) {
        vp2[i] = v2[i];
        v2[i] = w2[i] * rb2;
      }
    }
    if (go1) bprev1 = beta1;
    if (go2) bprev2 = beta2;
    on1 = go1;
    on2 = go2;
    __syncthreads();
  }
  // the two tridiagonal problems at once, on warps 0 and 1 (two schedulers)
  __syncthreads();
  // float scratch: a free n-double buffer per run holds both copies (2m <= 2n floats)
  if (threadIdx.x < 32) warp_tridiag_top(al1, be1, m1, W.red + 34, (float*)W.A.Qxn, (float*)W.A.Qxn + m1);
  else if (threadIdx.x < 64) warp_tridiag_top(al2, be2, m2, W.red + 36, (float*)W.B.Qxn, (float*)W.B.Qxn + m2);
  __syncthreads();
  const double ex = 1.2e-16;
  *lmax_Q = lz_estimate(W.red[34], beta1 * W.red[35], !(beta1 > 1e-300) || m1 == n, ex);
  *normG2 = lz_estimate(W.red[36], beta2 * W.red[37], !(beta2 > 1e-300) || m2 == n, ex);
  __syncthreads();
}

// Guaranteed upper bounds (no estimate): lambda_max(Q) <= min(max_i sum_j |Q_ij|
// (Gershgorin), ||Q||_F) and ||G||^2 <= min(||G||_1 ||G||_inf, ||G||_F^2), from
// FP64 column sums (Q symmetric: column sums are row sums; GT's column sums
// are G's row sums).
template <typename T>
__device__ double cta_col_abs_max(const T* M, int rows, int cols, double* red, double* fro) {
  double mx = 0.0, f = 0.0;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < rows; ++r) {
      const double v = double(M[(size_t)r * cols + c]);
      s += fabs(v);
      f += v * v;
    }
    mx = fmax(mx, s);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  double m = 0.0;
  for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) m = fmax(m, red[i]);
  __syncthreads();
  *fro = block_sum(f, red);
  return m;
}

template <typename T>
__device__ double cta_bound(const CtaInst<T>& I, CtaWs<T>& W, int which) {
  const int n = I.n, p = I.p;
  double fro = 0.0;
  if (which == 0) {
    const double g = cta_col_abs_max<T>(W.Q, n, n, W.red, &fro);
    return fmin(g, sqrt(fro));
  }
  const double c1 = cta_col_abs_max<T>(W.G, p, n, W.red, &fro);  // ||G||_1
  double f2 = 0.0;
  const double ci = cta_col_abs_max<T>(W.GT, n, p, W.red, &f2);  // ||G||_inf
  return fmin(c1 * ci, fro);
}

__device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared-memory bytes for the vectors of an (n, p) instance.
template <typename T>
__host__ __device__ inline size_t cta_vec_bytes(int n, int p) {
  const size_t pn = p > 0 ? p : 1;
  auto a16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  size_t b = a16(40 * sizeof(double));
  b += 2 * a16(n * sizeof(double)) + a16(pn * sizeof(double));  // usum, dn, dp
  b += 2 * (6 * a16(n * sizeof(T)) + 3 * a16(pn * sizeof(T)));  // A, B states
  b += 4 * a16(n * sizeof(T));                                   // c, tn, ul, uavg
  b += 4 * a16(pn * sizeof(T));                                  // w, mu, lam, lamp
  b += a16(2048 * sizeof(T));                                    // part
  return b;
}
template <typename T>
__host__ __device__ inline size_t cta_mat_bytes(int n, int p) {
  return ((size_t)n * n + 2 * (size_t)n * p) * sizeof(T) + 64;
}

template <typename T>
__device__ void cta_solve(CtaInst<T>& I, unsigned char* smem, size_t smem_bytes) {
  const int n = I.n, p = I.p;
  const size_t pn = p > 0 ? p : 1;
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char* {
    unsigned char* ptr = smem + off;
    off += align16(bytes);
    return ptr;
  };
  CtaWs<T> W;
  W.red = (double*)take(40 * sizeof(double));
  W.usum = (double*)take(n * sizeof(double));
  W.dn = (double*)take(n * sizeof(double));
  W.dp = (double*)take(pn * sizeof(double));
  XState<T>* st[2] = {&W.A, &W.B};
  for (int s = 0; s < 2; ++s) {
    XState<T>& S = *st[s];
    S.x = (T*)take(n * sizeof(T)); S.xp = (T*)take(n * sizeof(T)); S.xn = (T*)take(n * sizeof(T));
    S.Qx = (T*)take(n * sizeof(T)); S.Qxp = (T*)take(n * sizeof(T)); S.Qxn = (T*)take(n * sizeof(T));
    S.Gx = (T*)take(pn * sizeof(T)); S.Gxp = (T*)take(pn * sizeof(T)); S.Gxn = (T*)take(pn * sizeof(T));
  }
  W.c = (T*)take(n * sizeof(T));
  W.tn = (T*)take(n * sizeof(T));
  W.ul = (T*)take(n * sizeof(T));
  W.uavg = (T*)take(n * sizeof(T));
  W.w = (T*)take(pn * sizeof(T));
  W.mu = (T*)take(pn * sizeof(T));
  W.lam = (T*)take(pn * sizeof(T));
  W.lamp = (T*)take(pn * sizeof(T));
  W.part = (T*)take(2048 * sizeof(T));
  W.Q = I.Q; W.G = I.G; W.GT = I.GT;
  // stage the matrices in shared memory when they fit
  const size_t nn = (size_t)n * n, np_ = (size_t)n * p;
  if (off + cta_mat_bytes<T>(n, p) <= smem_bytes) {
    T* Qs = (T*)take(nn * sizeof(T));
    T* Gs = (T*)take(np_ * sizeof(T));
    T* GTs = (T*)take(np_ * sizeof(T));
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x) Qs[i] = I.Q[i];
    for (size_t i = threadIdx.x; i < np_; i += blockDim.x) { Gs[i] = I.G[i]; GTs[i] = I.GT[i]; }
    W.Q = Qs; W.G = Gs; W.GT = GTs;
  }
  __syncthreads();
  // FP64 constants (a1): lambda_max(Q), ||G||^2, then L_L, sigma_L, L_d, rho
  if constexpr (sizeof(T) == 8) {  // both estimates wanted: the two Lanczos runs in one loop
    if (isnan(I.lmax_Q) && isnan(I.normG2) && p > 0 && !I.lip_bound) cta_lanczos_pair(I, W, &I.lmax_Q, &I.normG2);
  }
  if (isnan(I.lmax_Q)) I.lmax_Q = I.lip_bound ? cta_bound<T>(I, W, 0) : cta_lanczos<T>(I, W, 0);
  if (isnan(I.normG2)) I.normG2 = p > 0 ? (I.lip_bound ? cta_bound<T>(I, W, 1) : cta_lanczos<T>(I, W, 1)) : 0.0;
  const double lmin = isnan(I.lmin_Q) ? 0.0 : I.lmin_Q;
  if (isnan(I.rho)) I.rho = (I.alg == ALG_ADGM || I.alg == ALG_ADFGM) ? (I.normG2 > 0.0 ? 1.0 / I.normG2 : 1.0) : 0.0;
  if (isnan(I.LL)) I.LL = I.lmax_Q + I.rho * I.normG2;
  if (isnan(I.sigma)) I.sigma = lmin;
  if (isnan(I.Ld)) {
    const double den = lmin + I.rho * I.normG2;
    I.Ld = I.normG2 > 0.0 ? (den > 0.0 ? I.normG2 / den : INFINITY) : 1.0;
  }
  if (isnan(I.eps_in))  // eq. choose_ein with R_d = 1
    I.eps_in = (I.alg == ALG_DGM || I.alg == ALG_ADGM) ? I.eps_out / 4.0
                                                       : I.eps_out * sqrt(I.eps_out) / (8.0 * sqrt(2.0 * I.Ld));
  if (threadIdx.x == 0 && I.consts_out) {
    I.consts_out[0] = I.lmax_Q; I.consts_out[1] = I.normG2; I.consts_out[2] = I.LL;
    I.consts_out[3] = I.Ld; I.consts_out[4] = I.sigma; I.consts_out[5] = I.rho;
  }
  if (!(I.Ld < INFINITY) || !(I.LL > 0.0)) {  // DGM/DFGM need lambda_min(Q) > 0 (Case 1)
    if (threadIdx.x == 0 && I.res) {
      DevResult r = {};
      r.status = -1;
      r.f_last = r.infeas_last = r.f_avg = r.infeas_avg = r.d_lb = NAN;
      *I.res = r;
    }
    __syncthreads();
    return;
  }
  // initial point and multipliers (Algorithm DFOM: lambda^0 = mu^1 in K_d)
  XState<T>& A = W.A;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    A.x[i] = I.x0 ? I.x0[i] : clampT(T(0), I.lb[i], I.ub[i]);
    W.usum[i] = 0.0;
  }
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const T l0 = I.lam0 ? I.lam0[j] : T(0);
    W.lam[j] = l0; W.lamp[j] = l0; W.mu[j] = l0;
  }
  __syncthreads();
  mtv<T>(W.Q, n, n, n, A.x, A.Qx, W.part);
  if (p > 0) {
    __syncthreads();
    mtv<T>(W.GT, n, p, p, A.x, A.Gx, W.part);
  }
  __syncthreads();

  // Upper bound of F over the box, F(u) <= sum_i max(q_i lb_i, q_i ub_i) +
  // lambda_max(Q)/2 sum_i max(lb_i^2, ub_i^2) (twice the lambda_max estimate,
  // so a low estimate cannot spoil it).  When the certified lower bound d_lb on
  // F* passes it, no feasible point exists (weak duality): DQ_ERR_DIVERGED.
  double fub = 0.0;
  {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double qi = double(I.q[i]), l = double(I.lb[i]), u = double(I.ub[i]);
      a += fmax(qi * l, qi * u);
      b += fmax(l * l, u * u);
    }
    const double sa = block_sum(a, W.red), sb = block_sum(b, W.red);
    fub = sa + I.lmax_Q * sb;
    fub += 1e-9 * (fabs(fub) + 1.0);
  }
  const bool aug = I.rho > 0.0, fast = alg_fast(I.alg);
  const T alpha = T(1.0 / (2.0 * I.Ld));
  const T rho = T(I.rho);
  double theta = 1.0, S = 0.0;
  long long inner_total = 0;
  const int check_every = I.check_every > 0 ? I.check_every : 1;
  const int kmax = I.outer_fixed > 0 ? I.outer_fixed : I.max_outer;
  double d_lb = -INFINITY, f_last = NAN, i_last = NAN, f_avg = NAN, i_avg = NAN;
  int conv_last = 0, conv_avg = 0, status = ST_OK, k = 0;
  bool done = false, last_valid = false;

  while (k < kmax && !done) {
    ++k;
    // Step 1: ubar^k = FOM(L_rho(., mu^k), U), warm start ubar^{k-1}
    inner_total += cta_fom(I, W, A, W.mu);
    // Step 2: lambda^k = [mu^k + (G ubar + g - s(ubar, mu))/(2 L_d)]_{K_d}
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      const T r = A.Gx[j] + I.g[j];
      const T s = aug ? proj_K(I.cone, r + W.mu[j] / rho) : T(0);
      W.lam[j] = proj_Kd(I.cone, I.kd_plus != 0, W.mu[j] + alpha * (r - s));
    }
    // averaging weight theta_k (eq. average_primal)
    S += theta;
    for (int i = threadIdx.x; i < n; i += blockDim.x) W.usum[i] += theta * double(A.x[i]);
    double beta = 0.0;
    if (fast) {
      const double tn1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * theta * theta));
      beta = (theta - 1.0) / tn1;
      theta = tn1;
    }
    __syncthreads();
    const bool final_iter = (k == kmax);
    if (final_iter || (I.outer_fixed <= 0 && k % check_every == 0)) {
      bool mu_ok = aug || I.cone == CONE_EQ;
      if (!mu_ok) {
        int neg = 0;
        for (int j = threadIdx.x; j < p; j += blockDim.x) neg |= (W.mu[j] < T(0));
        mu_ok = !__syncthreads_or(neg);
      }
      if (mu_ok) {
        EvalOut e = cta_eval(I, W, A.x, W.mu);
        d_lb = fmax(d_lb, e.lagr - e.cert);
      }
      if (I.want_last) {
        if (fast) {  // ubar(lambda^k): extra warm-started inner solve at mu = lambda^k
          XState<T>& B = W.B;
          vcopy(B.x, A.x, n);
          vcopy(B.Qx, A.Qx, n);
          if (p > 0) vcopy(B.Gx, A.Gx, p);
          __syncthreads();
          inner_total += cta_fom(I, W, B, W.lam);
          vcopy(W.ul, B.x, n);
          __syncthreads();
          bool lam_ok = aug || I.cone == CONE_EQ;
          if (!lam_ok) {
            int neg = 0;
            for (int j = threadIdx.x; j < p; j += blockDim.x) neg |= (W.lam[j] < T(0));
            lam_ok = !__syncthreads_or(neg);
          }
          if (lam_ok) {
            EvalOut e = cta_eval(I, W, W.ul, W.lam);
            d_lb = fmax(d_lb, e.lagr - e.cert);
          }
        } else {
          vcopy(W.ul, A.x, n);
          __syncthreads();
        }
        EvalOut e = cta_eval(I, W, W.ul, (const T*)nullptr);
        f_last = e.F;
        i_last = e.infeas;
        last_valid = true;
      }
      if (I.want_avg) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) W.uavg[i] = T(W.usum[i] / S);
        __syncthreads();
        EvalOut e = cta_eval(I, W, W.uavg, (const T*)nullptr);
        f_avg = e.F;
        i_avg = e.infeas;
      }
      if ((I.want_last && !(isfinite(f_last) && isfinite(i_last))) ||
          (I.want_avg && !(isfinite(f_avg) && isfinite(i_avg)))) {
        status = ST_NONFINITE;
        done = true;
      } else if (d_lb > fub) {  // infeasible: the dual lower bound passed max_U F
        status = ST_DIVERGED;
        done = true;
      }
      if (I.outer_fixed <= 0 && !done) {
        // the certificate F - d_lb, or |F - F*| for a known F* (the paper's experiments)
        const double gl = I.stop_fstar ? fabs(f_last - I.f_star) : f_last - d_lb;
        const double ga = I.stop_fstar ? fabs(f_avg - I.f_star) : f_avg - d_lb;
        conv_last = I.want_last && i_last <= I.eps_out && gl <= I.eps_out;
        conv_avg = I.want_avg && i_avg <= I.eps_out && ga <= I.eps_out;
        done = conv_last || conv_avg;
      }
    }
    // Step 3: mu^{k+1} = lambda^k + beta_k (lambda^k - lambda^{k-1})
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      const T l = W.lam[j];
      const T mm = l + T(beta) * (l - W.lamp[j]);
      W.lamp[j] = l;
      W.mu[j] = mm;
    }
    __syncthreads();
  }
  if (!last_valid) {
    vcopy(W.ul, A.x, n);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (I.x_last) I.x_last[i] = W.ul[i];
    if (I.x_avg) I.x_avg[i] = T(W.usum[i] / S);
    if (I.x_state) I.x_state[i] = A.x[i];
  }
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    if (I.lam_out) I.lam_out[j] = W.lam[j];
    if (I.lam_state) I.lam_state[j] = W.lam[j];
  }
  if (threadIdx.x == 0 && I.res) {
    DevResult r;
    r.status = status != ST_OK ? status : ((I.outer_fixed > 0 || conv_last || conv_avg) ? ST_OK : ST_NOT_CONVERGED);
    r.outer_iters = k;
    r.inner_iters = inner_total;
    r.converged_last = conv_last;
    r.converged_avg = conv_avg;
    r.f_last = f_last; r.infeas_last = i_last; r.f_avg = f_avg; r.infeas_avg = i_avg; r.d_lb = d_lb;
    *I.res = r;
  }
  __syncthreads();
}

// Persistent kernel: CTAs pull instance indices (in `order`) from a device counter.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) cta_solve_kernel(const CtaInst<T>* __restrict__ insts,
                                                        const int* __restrict__ order, int count,
                                                        int* __restrict__ next, size_t smem_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(next, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= count) break;
    CtaInst<T> I = insts[order ? order[idx] : idx];
    cta_solve<T>(I, smem, smem_bytes);
  }
}

}  // namespace dq
