"""The tcgen05 BF16 GEMM of the surrogate (through the C ABI) against plain PyTorch FP32 matmul
of the same BF16-rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_00011_gb300 import build
    build.build()


def _rand(shape, seed, scale=1.0):
    """BF16 CUDA matrix whose row stride is padded to a multiple of 8 elements (TMA rule)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    rows, cols = shape
    ld = (cols + 7) // 8 * 8
    full = torch.zeros((rows, ld), dtype=torch.bfloat16)
    full[:, :cols] = (torch.randn(shape, generator=g) * scale).to(torch.bfloat16)
    return full.cuda()[:, :cols]


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (256, 256, 256), (300, 200, 100), (300, 203, 100),
                                   (37, 1024, 64), (512, 1024, 1024), (512, 10000, 1024),
                                   (129, 136, 1000),
                                   # several tiles per persistent CTA: accumulator reuse, ring wrap
                                   (4096, 4000, 136), (2048, 10000, 64)])
def test_gemm_f32_matches_torch(m, n, k):
    import paper_1904_00011_gb300 as P
    a = _rand((m, k), 1)
    b = _rand((n, k), 2)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    c, _ = P.gemm(a, b, epilogue=P.PCMD_GEMM_F32, err=err)
    ref = a.float() @ b.float().T
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale = ref.abs().max().item()
    assert torch.allclose(c, ref, rtol=1e-4, atol=1e-5 * scale * np.sqrt(k)), \
        (c - ref).abs().max().item()


@pytest.mark.parametrize("epi", ["gelu", "bias_bf16", "bias_f32"])
@pytest.mark.parametrize("m,n,k", [(256, 384, 192), (4096, 2312, 128), (333, 1000, 64),
                                   (100, 203, 64)])
def test_gemm_epilogues(epi, m, n, k):
    import paper_1904_00011_gb300 as P
    a = _rand((m, k), 3, 0.3)
    b = _rand((n, k), 4, 0.3)
    bias = torch.linspace(-1, 1, n, device="cuda", dtype=torch.float32)
    z = a.float() @ b.float().T + bias
    code = {"gelu": P.PCMD_GEMM_BIAS_GELU_BF16, "bias_bf16": P.PCMD_GEMM_BIAS_BF16,
            "bias_f32": P.PCMD_GEMM_BIAS_F32}[epi]
    c, aux = P.gemm(a, b, bias=bias, epilogue=code)
    torch.cuda.synchronize()
    if epi == "gelu":
        ref = torch.nn.functional.gelu(z)
        assert torch.allclose(aux.float(), z, rtol=1e-2, atol=1e-2)
        assert torch.allclose(c.float(), ref, rtol=1e-2, atol=1e-2)
    elif epi == "bias_bf16":
        assert torch.allclose(c.float(), z, rtol=1e-2, atol=1e-2)
    else:
        assert torch.allclose(c, z, rtol=1e-4, atol=1e-4)


def test_gelu_without_preactivation_output():
    import paper_1904_00011_gb300 as P
    m, n, k = 600, 1000, 128
    a = _rand((m, k), 5, 0.3)
    b = _rand((n, k), 6, 0.3)
    bias = torch.linspace(-1, 1, n, device="cuda", dtype=torch.float32)
    c1, aux = P.gemm(a, b, bias=bias, epilogue=P.PCMD_GEMM_BIAS_GELU_BF16)
    c2, none = P.gemm(a, b, bias=bias, epilogue=P.PCMD_GEMM_BIAS_GELU_BF16, want_aux=False)
    torch.cuda.synchronize()
    assert none is None and aux is not None
    assert torch.equal(c1, c2)
