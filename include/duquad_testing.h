/*
 * duquad_testing.h -- test hooks of libduquad.so (not part of the solver API).
 *
 * The paper has no counterpart: these entry points exercise building blocks
 * of the GPU kernels in isolation so that a fault in a tensor-core operand
 * layout shows up as a wrong number in a small test rather than inside a
 * whole solve.
 */
#ifndef DUQUAD_TESTING_H
#define DUQUAD_TESTING_H

#include <stdint.h>

#include "duquad.h"

#ifdef __cplusplus
extern "C" {
#endif

/* D = A * B' on the sm_103a tensor cores (tcgen05.mma, kind::f16, bf16
 * operands, FP32 accumulation in tensor memory), one thread block.
 * A: M x K, B: N x K, D: M x N, all row-major FP32 DEVICE arrays owned by the
 * caller.  split != 0 uses the three-product bf16 hi/lo form
 * hi*hi + hi*lo + lo*hi; split == 0 rounds the operands to bf16 once.
 * bulk != 0 packs B into the operand layout in global memory first and brings
 * it into shared memory with a bulk (TMA-engine) copy; otherwise threads
 * write it.  Limits: M == 128, N a multiple of 16 in [16, 256], K a multiple
 * of 16 in [16, 128]; anything else returns DQ_ERR_INVALID.  A device wait
 * that gives up returns DQ_ERR_TIMEOUT.  stream: cudaStream_t (NULL = legacy
 * default).  Synchronises the stream. */
dq_status dq_test_tc_gemm(const float *A, const float *B, float *D, int32_t M, int32_t N, int32_t K,
                          int32_t split, int32_t bulk, void *stream);

/* The bounded device-side wait the engines use (an mbarrier phase polled
 * against the GPU's global timer, as in the single-pass iteration's bulk-copy
 * ring and the tensor-core batch) in isolation: one thread block waits on an
 * mbarrier that expects one arrival.  complete != 0: the arrival comes first
 * and the call returns DQ_OK.  complete == 0: nothing ever arrives, the wait
 * gives up after limit_ns nanoseconds and the call returns DQ_ERR_TIMEOUT,
 * leaving the CUDA context usable (nothing hangs or traps).  limit_ns in
 * (0, 1e9], else DQ_ERR_INVALID.  stream: cudaStream_t (NULL = legacy
 * default).  Synchronises the stream. */
dq_status dq_test_bounded_wait(uint64_t limit_ns, int32_t complete, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DUQUAD_TESTING_H */
