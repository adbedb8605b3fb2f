"""The tensor-core GEMM (ncpadj_dense_gemm: tcgen05.mma kind::tf32 into tensor memory) against an
FP64 product of the same FP32 operands: whole tiles, ragged edges in M, N and K, leading dimensions
wider than the rows, alpha and beta, and the two accuracy modes (3xTF32 near FP32, plain TF32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    return pkg.Context(0)


def _err(C, ref, A, B, alpha):
    """max |C - ref| relative to alpha sum_k |a_ik| |b_kj| (the scale of a product's rounding)"""
    scale = abs(alpha) * (A.abs().double() @ B.abs().double()) + 1e-30
    return float(((C.double() - ref) / scale).abs().max())


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 128, 8), (200, 150, 70), (300, 260, 1), (64, 517, 129)])
@pytest.mark.parametrize("split", [True, False])
def test_gemm_matches_fp64(pkg, ctx, M, N, K, split):
    from paper_2603_16478_gb300.binding import dense_gemm
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(K, N, generator=g).cuda()
    C = dense_gemm(ctx, A, B, split=split)
    torch.cuda.synchronize()
    ref = A.double() @ B.double()
    assert _err(C, ref, A, B, 1.0) < (2e-6 if split else 2e-3)


def test_gemm_alpha_beta_and_leading_dimensions(pkg, ctx):
    from paper_2603_16478_gb300.binding import dense_gemm
    g = torch.Generator(device="cpu").manual_seed(5)
    Abig = torch.randn(300, 400, generator=g).cuda()
    Bbig = torch.randn(250, 333, generator=g).cuda()
    Cbig = torch.randn(310, 350, generator=g).cuda()
    A, B = Abig[10:150, 20:250], Bbig[5:235, 3:203]     # 140 x 230 and 230 x 200, row strides 400, 333
    C = Cbig[7:147, 100:300]                             # 140 x 200, row stride 350
    C0 = C.clone()
    outside = Cbig.clone()
    dense_gemm(ctx, A, B, C, alpha=-0.5, beta=2.0)
    torch.cuda.synchronize()
    ref = -0.5 * (A.double() @ B.double()) + 2.0 * C0.double()
    assert _err(C, ref, A, B, 0.5) < 2e-6 + 1e-6 * float(C0.abs().max())
    mask = torch.ones_like(Cbig, dtype=torch.bool)
    mask[7:147, 100:300] = False
    assert torch.equal(Cbig[mask], outside[mask])   # nothing outside C is written


def test_gemm_rejects_bad_arguments(pkg, ctx):
    from paper_2603_16478_gb300.binding import dense_gemm
    A = torch.zeros(4, 3, device="cuda")
    with pytest.raises(ValueError):
        dense_gemm(ctx, A, torch.zeros(4, 5, device="cuda"))
    with pytest.raises(ValueError):
        dense_gemm(ctx, A.double(), torch.zeros(3, 5, device="cuda", dtype=torch.float64))
    lib = ctx.lib
    import ctypes as C
    st = lib.ncpadj_dense_gemm(ctx.handle, 4, 5, 3, 1.0, C.c_void_p(A.data_ptr()), 2, C.c_void_p(A.data_ptr()), 5, 0.0,
                               C.c_void_p(A.data_ptr()), 5, 0, None)
    assert st == 1  # INVALID_ARG: lda < K
