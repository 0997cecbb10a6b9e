// tc_engine.cu -- tensor-core building blocks and their self-test.
#include <string.h>

#include "dq_host.h"
#include "duquad_testing.h"
#include "tc_common.cuh"

namespace dq {


// Pack an R x K row-major float matrix (rows >= R_valid and cols >= K_valid
// are zero) into bf16 hi and lo tiles of the K-major no-swizzle layout with
// R_pad rows and K_pad columns.
__global__ void k_pack_kmajor(const float* __restrict__ src, int R_valid, int K_valid, int ld, int R_pad, int K_pad,
                              uint4* __restrict__ hi, uint4* __restrict__ lo) {
  const int chunks = R_pad * (K_pad / 8);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += gridDim.x * blockDim.x) {
    const int r = c / (K_pad / 8), k0 = (c % (K_pad / 8)) * 8;
    float x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = (r < R_valid && k0 + t < K_valid) ? src[(size_t)r * ld + k0 + t] : 0.f;
    uint4 h, l;
    tc::split8(x, h, l);
    const uint32_t off = tc::kmajor_off(r, k0, R_pad) / 16;
    hi[off] = h;
    lo[off] = l;
  }
}

static constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__global__ void __launch_bounds__(128) k_tc_selftest(const float* __restrict__ A, const float* __restrict__ B,
                                                     const uint4* __restrict__ Bpk_hi, const uint4* __restrict__ Bpk_lo,
                                                     float* __restrict__ D, int N, int K, int split, int bulk,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_tx, bar_mma;
  __shared__ uint32_t s_taddr;
  constexpr int M = 128;
  const size_t a_bytes = (size_t)M * K * 2, b_bytes = (size_t)N * K * 2;
  unsigned char* A_hi = sm;
  unsigned char* A_lo = sm + a_bytes;
  unsigned char* B_hi = sm + 2 * a_bytes;
  unsigned char* B_lo = sm + 2 * a_bytes + b_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&bar_tx, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init_fence();
  }
  __syncthreads();
  if (warp == 0) {
    tc::tmem_alloc(&s_taddr, 256);
    tc::tmem_relinquish();
  }
  // operands into shared memory
  for (int k0 = 0; k0 < K; k0 += 8) {
    uint4 h, l;
    tc::split8(A + (size_t)tid * K + k0, h, l);
    if (!split) l = make_uint4(0, 0, 0, 0);
    *(uint4*)(A_hi + tc::kmajor_off(tid, k0, M)) = h;
    *(uint4*)(A_lo + tc::kmajor_off(tid, k0, M)) = l;
  }
  if (bulk) {
    if (tid == 0) {
      tc::mbar_expect_tx(&bar_tx, (uint32_t)(2 * b_bytes));
      tc::bulk_g2s(B_hi, Bpk_hi, (uint32_t)b_bytes, &bar_tx);
      tc::bulk_g2s(B_lo, Bpk_lo, (uint32_t)b_bytes, &bar_tx);
    }
  } else {
    for (int r = tid; r < N; r += blockDim.x)
      for (int k0 = 0; k0 < K; k0 += 8) {
        uint4 h, l;
        tc::split8(B + (size_t)r * K + k0, h, l);
        *(uint4*)(B_hi + tc::kmajor_off(r, k0, N)) = h;
        *(uint4*)(B_lo + tc::kmajor_off(r, k0, N)) = l;
      }
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  bool ok = true;
  if (bulk && !tc::mbar_wait(&bar_tx, 0, kWaitNs)) ok = false;
  const uint32_t taddr = s_taddr;
  if (tid == 0 && ok) {
    const uint32_t idesc = tc::idesc_bf16_f32(M, N);
    const uint32_t lboA = tc::kmajor_lbo(M), lboB = tc::kmajor_lbo(N);
    for (int s = 0; s < K / 16; ++s) {
      const uint64_t ah = tc::sdesc(tc::saddr(A_hi) + s * 2 * lboA, lboA, 128);
      const uint64_t al = tc::sdesc(tc::saddr(A_lo) + s * 2 * lboA, lboA, 128);
      const uint64_t bh = tc::sdesc(tc::saddr(B_hi) + s * 2 * lboB, lboB, 128);
      const uint64_t bl = tc::sdesc(tc::saddr(B_lo) + s * 2 * lboB, lboB, 128);
      tc::mma_bf16(taddr, ah, bh, idesc, s > 0 ? 1u : 0u);
      if (split) {
        tc::mma_bf16(taddr, ah, bl, idesc, 1u);
        tc::mma_bf16(taddr, al, bh, idesc, 1u);
      }
    }
    tc::mma_commit(&bar_mma);
  }
  __syncthreads();
  if (ok && !tc::mbar_wait(&bar_mma, 0, kWaitNs)) ok = false;
  tc::fence_after();
  if (!__syncthreads_and(ok)) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    const int row = warp * 32 + lane;
    for (int c = 0; c < N; c += 16) {
      uint32_t r[16];
      tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) D[(size_t)row * N + c + j] = __uint_as_float(r[j]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

}  // namespace dq

using namespace dq;

extern "C" dq_status dq_test_tc_gemm(const float* A, const float* B, float* D, int32_t M, int32_t N, int32_t K,
                                     int32_t split, int32_t bulk, void* stream) {
  if (!A || !B || !D || M != 128 || N < 16 || N > 256 || N % 16 || K < 16 || K > 128 || K % 16) {
    set_error("dq_test_tc_gemm: need M == 128, N in [16,256] and K in [16,128], multiples of 16");
    return DQ_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t a_bytes = (size_t)M * K * 2, b_bytes = (size_t)N * K * 2;
  const size_t smem = 2 * a_bytes + 2 * b_bytes + 16384;  // slack past the operands
  void *pk = nullptr, *errp = nullptr;
  DQ_CK(cudaMalloc(&pk, 2 * b_bytes));
  DQ_CK(cudaMalloc(&errp, sizeof(int)));
  DQ_CK(cudaMemsetAsync(errp, 0, sizeof(int), st));
  uint4* hi = (uint4*)pk;
  uint4* lo = (uint4*)((char*)pk + b_bytes);
  if (bulk) {
    k_pack_kmajor<<<64, 256, 0, st>>>(B, N, K, K, N, K, hi, lo);
    DQ_CK(cudaGetLastError());
  }
  DQ_CK(cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_tc_selftest<<<1, 128, smem, st>>>(A, B, hi, lo, D, N, K, split, bulk, (int*)errp);
  DQ_CK(cudaGetLastError());
  int herr = 0;
  DQ_CK(cudaMemcpyAsync(&herr, errp, sizeof(int), cudaMemcpyDeviceToHost, st));
  DQ_CK(cudaStreamSynchronize(st));
  cudaFree(pk);
  cudaFree(errp);
  if (herr) {
    set_error("dq_test_tc_gemm: a tensor-core wait timed out");
    return DQ_ERR_TIMEOUT;
  }
  return DQ_OK;
}

namespace dq {

// The engines' bounded wait (tc::mbar_wait on the global timer) on an
// mbarrier that expects one arrival.  complete != 0: thread 0 arrives first,
// so the wait ends at once; otherwise nothing arrives and the wait gives up
// after limit_ns.  No copy or MMA is in flight, so giving up is safe.
__global__ void k_wait_selftest(unsigned long long limit_ns, int complete, int* gave_up) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init_fence();
  }
  __syncthreads();
  if (complete && threadIdx.x == 0) tc::mbar_arrive(&bar);
  const bool ok = tc::mbar_wait(&bar, 0, limit_ns);
  if (!ok) atomicExch(gave_up, 1);
}

}  // namespace dq

extern "C" dq_status dq_test_bounded_wait(uint64_t limit_ns, int32_t complete, void* stream) {
  using namespace dq;
  if (limit_ns == 0 || limit_ns > 1000000000ull) {
    set_error("dq_test_bounded_wait: limit_ns must be in (0, 1e9]");
    return DQ_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* flag = nullptr;
  DQ_CK(cudaMalloc(&flag, sizeof(int)));
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 64, 0, st>>>((unsigned long long)limit_ns, complete, flag);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(flag);
  if (e != cudaSuccess) {
    set_error("dq_test_bounded_wait: %s", cudaGetErrorString(e));
    return DQ_ERR_CUDA;
  }
  if (h) {
    set_error("dq_test_bounded_wait: the wait gave up after %llu ns", (unsigned long long)limit_ns);
    return DQ_ERR_TIMEOUT;
  }
  return DQ_OK;
}
