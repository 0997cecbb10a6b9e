"""The tensor-core building block (tcgen05.mma with TMEM accumulators, bf16 hi/lo operands,
bulk copies into shared memory) against a plain FP64 product of the same FP32 inputs."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(16, 16), (112, 112), (208, 112), (256, 128), (96, 64)])
@pytest.mark.parametrize("bulk", [0, 1])
def test_tc_gemm_split_matches_fp64(N, K, bulk):
    import torch
    from paper_1504_05708_gb300 import duquad as D
    g = torch.Generator(device="cpu").manual_seed(N * 1000 + K)
    A = torch.randn(128, K, generator=g, dtype=torch.float32)
    B = torch.randn(N, K, generator=g, dtype=torch.float32)
    ref = (A.double() @ B.double().T).numpy()
    Ad, Bd = A.cuda(), B.cuda()
    for split, tol in ((1, 4e-5), (0, 2e-2)):
        Dd = torch.full((128, N), float("nan"), device="cuda")
        st = D.lib().dq_test_tc_gemm(Ad.data_ptr(), Bd.data_ptr(), Dd.data_ptr(), 128, N, K, split, bulk,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        D.check(st, (D.OK,))
        out = Dd.cpu().double().numpy()
        scale = np.sqrt(K)  # |entries| ~ sqrt(K) for N(0,1) data
        err = np.abs(out - ref).max() / scale
        assert err <= tol, (split, err)


def test_tc_gemm_rejects_bad_shapes():
    import torch
    from paper_1504_05708_gb300 import duquad as D
    A = torch.zeros(128, 16, device="cuda")
    st = D.lib().dq_test_tc_gemm(A.data_ptr(), A.data_ptr(), A.data_ptr(), 128, 20, 16, 1, 0, None)
    assert st == D.ERR_INVALID
