// csr.cuh -- sparse (CSR) matrix-vector products of the grid engine.
//
// For sparse Q and G the inner step of Algorithm FOM still needs only
// matrix-vector products (Sec. 5: the products dominate, and for sparse Q, G
// they cost O(nnz) instead of O(n^2)).  The grid engine's products take a
// prologue vector v (x, the extrapolated step, or w = [mu + rho (G y + g)]_+)
// and rows of one or two matrices; for CSR matrices the prologue is formed
// once into a global vector (a separate kernel) and k_csr_rows gathers it.
// Each row is summed by a group of TPR lanes of a warp, lane l taking the
// row's entries l, l + TPR, ... and the group adding its lanes in a fixed
// butterfly order, so the result depends on the row's structure only (not on
// the grid or on which rows share a warp).
#pragma once
#include <type_traits>

#include "dq_common.cuh"

namespace dq {

struct CsrRef {
  const int* rp;  // rows + 1 row offsets (int32: nnz < 2^31)
  const int* ci;  // column indices, strictly increasing within a row
};

// out1[r] = sum_e M1[e] v[ci1[e]] (+ add1[r]) for the R1 rows of M1, then
// out2 likewise for the R2 rows of M2.  ACC: Dot2-accurate FP64 outputs.
template <typename T, bool ACC, int TPR, typename Job>
__global__ void __launch_bounds__(256) k_csr_rows(Job J, CsrRef A1, CsrRef A2, const T* __restrict__ v) {
  static_assert(TPR >= 1 && TPR <= 32 && (32 % TPR) == 0, "TPR must divide the warp");
  if (J.done && *(volatile const int*)J.done) return;
  const int lane = threadIdx.x & 31, sub = lane % TPR;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int groups = (gridDim.x * blockDim.x) / TPR;
  const int g0 = (gtid - lane) / TPR, gi = lane / TPR;  // the warp's first group, this lane's group
  const int R = J.R1 + J.R2;
  // accurate mode: Dot2 per lane and FP64 lane sums; otherwise the row is
  // summed in T (FP64 arithmetic runs at a small fraction of the FP32 rate)
  using S = typename std::conditional<ACC, double, T>::type;
  for (int base = g0; base < R; base += groups) {  // the same trips for every lane of the warp
    const int r = base + gi;
    S tot = S(0);
    if (r < R) {
      const bool first = r < J.R1;
      const CsrRef A = first ? A1 : A2;
      const T* M = first ? J.M1 : J.M2;
      const int row = first ? r : r - J.R1;
      const int e0 = __ldg(A.rp + row), e1 = __ldg(A.rp + row + 1);
      if constexpr (ACC) {
        typename AccurateAcc<T>::type a;
        for (int e = e0 + sub; e < e1; e += TPR) a.add(__ldcs(M + e), __ldg(v + __ldcs(A.ci + e)));
        tot = a.get();
      } else {
        for (int e = e0 + sub; e < e1; e += TPR) tot = fma(__ldcs(M + e), __ldg(v + __ldcs(A.ci + e)), tot);
      }
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (r < R && sub == 0) {
      if (r < J.R1) {
        if constexpr (ACC) {
          double d = tot;
          if (J.add1) d += double(J.add1[r]);
          J.dout1[r] = d;
        } else {
          J.out1[r] = J.add1 ? tot + J.add1[r] : tot;
        }
      } else {
        if constexpr (ACC) J.dout2[r - J.R1] = tot; else J.out2[r - J.R1] = tot;
      }
    }
  }
}

}  // namespace dq
