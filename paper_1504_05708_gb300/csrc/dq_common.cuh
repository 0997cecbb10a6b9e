// dq_common.cuh -- internal definitions shared by the solver engines.
//
// The method is DuQuad's inexact (augmented) dual first-order method DFOM
// (arXiv 1504.05708, Sec. 3) with the inner Algorithm FOM (Sec. 2.1).  This
// header holds only plumbing: result records, reductions and accumulators.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace dq {

// Per-instance result written by the device (mirrors dq_result's solver fields).
struct DevResult {
  int status;           // dq_status
  int outer_iters;
  long long inner_iters;
  int converged_last, converged_avg;
  double f_last, infeas_last, f_avg, infeas_avg, d_lb;
};

enum { ALG_DGM = 0, ALG_DFGM = 1, ALG_ADGM = 2, ALG_ADFGM = 3 };
enum { CONE_INEQ = 0, CONE_EQ = 1 };
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_NONFINITE = -4, ST_DIVERGED = -5, ST_TIMEOUT = -6 };

__host__ __device__ inline bool alg_fast(int alg) { return alg == ALG_DFGM || alg == ALG_ADFGM; }

// Projection onto K (R^p_- or {0}) and onto the dual cone K_d (Sec. 2).
template <typename T>
__device__ __forceinline__ T proj_K(int cone, T z) {
  return cone == CONE_EQ ? T(0) : (z < T(0) ? z : T(0));
}
template <typename T>
__device__ __forceinline__ T proj_Kd(int cone, bool kd_plus, T z) {
  if (cone == CONE_EQ || !kd_plus) return z;
  return z > T(0) ? z : T(0);
}
template <typename T>
__device__ __forceinline__ T clampT(T v, T lo, T hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Deterministic block-wide sum of one double per thread.  Lane 0 of warp w
// stores the warp's shuffle-tree sum; warp 0 adds the warp sums as a
// butterfly tree (three dependent FP64 adds for eight warps instead of eight:
// FP64 latency sets the cost of these sums).  The result depends only on the
// values and blockDim, never on scheduling.  `red` must hold 33 doubles of
// shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double s = l < nw ? red[l] : 0.0;
    for (int o = 1; o < nw; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProduct) and the
// compensated dot product Dot2 of Ogita, Rump and Oishi (SIAM J. Sci.
// Comput. 26(6), 2005): a float pair accumulates sum a_i b_i with the
// accuracy of twice the working precision.  Used where the paper's
// quantities need FP64-level accuracy from float data.
struct Dot2f {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float ep = fmaf(a, b, -p);
    const float t = s + p;
    const float z = t - s;
    const float es = (s - (t - z)) + (p - z);
    s = t;
    c += ep + es;
  }
  __device__ __forceinline__ void add1(float a) {
    const float t = s + a;
    const float z = t - s;
    c += (s - (t - z)) + (a - z);
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

struct Acc64 {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void add1(double a) { s += a; }
  __device__ __forceinline__ double get() const { return s; }
};

// Accurate accumulator per element type: double data uses FP64, float data
// uses Dot2 on the FP32 pipe.
template <typename T> struct AccurateAcc;
template <> struct AccurateAcc<double> { using type = Acc64; };
template <> struct AccurateAcc<float> { using type = Dot2f; };

// ---- Lanczos estimates of lambda_max(Q) and ||G||^2 = lambda_max(G'G) ------
//
// Entry i of the start vector: a value in [-1, 1) from the SplitMix64
// generator (Steele, Lea and Flood, OOPSLA 2014) at counter i.  A pseudo-random
// start has a component along the top eigenvector whatever structure Q has
// (an all-ones start is orthogonal to, e.g., a top eigenvector (1, -1, 0, ...)).
__host__ __device__ inline double lz_start(unsigned long long i) {
  unsigned long long z = 0x2545F4914F6CDD1DULL + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Relative margin eps and failure probability delta of the estimate.  For a
// start vector drawn uniformly from the sphere, the top Ritz value theta_k of
// k Lanczos steps satisfies P(theta_k < (1 - eps) lambda_max) <=
// 1.648 sqrt(n) exp(-sqrt(eps) (2k - 1)) (Kuczynski and Wozniakowski, SIAM J.
// Matrix Anal. Appl. 13(4), 1992).  After lz_min_steps(n) steps that is at
// most delta, so theta_k / (1 - eps) is an upper bound of lambda_max with
// probability >= 1 - delta (the SplitMix64 start stands in for the random one).
static constexpr double kLzEps = 0.01, kLzDelta = 1e-3;
static constexpr int kLzMaxSteps = 160;

__host__ __device__ inline int lz_min_steps(int n) {
  const double k = 0.5 * (log(1.648 * sqrt(double(n)) / kLzDelta) / sqrt(kLzEps) + 1.0);
  const int kk = int(ceil(k));
  return kk < n ? kk : n;
}

// The returned estimate: theta + 2 r (r = beta_k |s_k| is the residual of the
// Ritz pair, so an eigenvalue lies within r of theta) and at least
// theta / (1 - eps).  After n steps (or an invariant subspace, beta = 0) the
// Krylov space holds the top eigenvector and theta is exact up to the
// rounding `ulp_rel` of the products.
__host__ __device__ inline double lz_estimate(double theta, double r, bool exhausted, double ulp_rel) {
  if (exhausted) return theta + 2.0 * r + 64.0 * ulp_rel * fabs(theta);
  const double a = theta + 2.0 * r, b = theta / (1.0 - kLzEps);
  return a > b ? a : b;
}

}  // namespace dq
