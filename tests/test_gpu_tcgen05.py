"""The tcgen05 GEMM primitive (cool_debug_gemm_bf16) against a float64 CPU
matmul of the same bf16 values.  FP32 accumulation of K products: the bound
is K 2^-23 sum |a_k b_k| per entry."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 128), (256, 64, 32), (128, 16, 16), (384, 128, 64)])
def test_gemm_bf16_matches_cpu(M, N, K):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08855_b300 import binding as b, build
    build.build()
    L = b.lib()
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    Cd = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.cool_debug_gemm_bf16(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()), C.c_void_p(Cd.data_ptr()),
                                M, N, K, C.c_void_p(err.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    a = A.double().numpy()
    bb = B.double().numpy()
    want = a @ bb.T
    bound = K * 2.0 ** -23 * (np.abs(a) @ np.abs(bb).T) + 1e-30
    got = Cd.cpu().double().numpy()
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)
