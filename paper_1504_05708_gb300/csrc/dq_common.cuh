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
// stores the warp's shuffle-tree sum; thread 0 adds the warps in order.  The
// result depends only on the values and blockDim, never on scheduling.
// `red` must hold 33 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
    red[32] = s;
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

}  // namespace dq
