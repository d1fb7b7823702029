"""The tcgen05 BF16 GEMM in isolation, against a plain PyTorch FP32 matmul of
the same BF16 values (products of BF16 numbers are exact in FP32, so only the
summation order differs)."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fn():
    from paper_2011_07125_gb300 import binding
    lib = binding.load()
    f = lib.ferminet_diag_bf16_gemm
    vp = C.c_void_p
    f.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("rm", [0, 1])
@pytest.mark.parametrize("M,N,K,tile_n", [(128, 256, 64, 256), (256, 1000, 256, 192), (480, 37, 128, 176),
                                          (256, 4099, 320, 224), (96, 50, 64, 16), (512, 700, 512, 256),
                                          (480, 1500, 256, 240)])
def test_bf16_gemm_matches_torch(M, N, K, tile_n, rm):
    f = _fn()
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    Cm = torch.full((N, M), float("nan"), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = f(A.data_ptr(), B.data_ptr(), Cm.data_ptr(), M, N, K, tile_n, rm,
           C.c_void_p(torch.cuda.current_stream().cuda_stream), st.data_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = B.float() @ A.float().T
    err = (Cm - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * (K ** 0.5), (err, scale)


@pytest.mark.parametrize("M,N,K,tile_n,ks", [(256, 256, 64 * 40, 256, 7), (40, 256, 64 * 9, 256, 9),
                                             (64, 448, 64 * 33, 224, 5), (512, 96, 64 * 3, 96, 3)])
def test_bf16_gemm_splitk_partials(M, N, K, tile_n, ks):
    """Split-K partials (the weight-gradient contractions of the adjoint):
    each range's partial equals the matmul over its own k-blocks."""
    from paper_2011_07125_gb300 import binding
    f = binding.load().ferminet_diag_bf16_gemm_splitk
    vp = C.c_void_p
    f.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp]
    f.restype = C.c_int
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    Cm = torch.full((ks, N, M), float("nan"), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = f(A.data_ptr(), B.data_ptr(), Cm.data_ptr(), M, N, K, tile_n, ks,
           C.c_void_p(torch.cuda.current_stream().cuda_stream), st.data_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    kb = K // 64
    kps = (kb + ks - 1) // ks
    for z in range(ks):
        k0, k1 = 64 * z * kps, 64 * min(kb, (z + 1) * kps)
        ref = B[:, k0:k1].float() @ A[:, k0:k1].float().T
        err = (Cm[z] - ref).abs().max().item()
        assert err <= 1e-5 * max(ref.abs().max().item(), 1.0) * ((k1 - k0) ** 0.5), (z, err)
