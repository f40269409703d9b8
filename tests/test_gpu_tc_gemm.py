"""The tcgen05 tensor-core GEMM against a float64 matrix product of the same operands.

bf16 operands are exact in float64, so the only error is the FP32 accumulation (relative
~K * 2^-24 of the sum of |terms|). TF32 reads the top 19 bits of each float (the hardware
ignores the rest), so the reference rounds the operands the same way; the remaining error is
again the FP32 accumulation. Shapes cover one tile, ragged M/N/K tails and multi-tile grids.
"""
import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def tf32_trunc(x):
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def run(tf32, M, N, K, epi=0, seed=0):
    rng = np.random.default_rng(seed)
    lda = ((K + 7) // 8) * 8
    A = rng.standard_normal((M, lda)).astype(np.float32)
    B = rng.standard_normal((N, lda)).astype(np.float32)
    dev = torch.device("cuda")
    if tf32:
        Ad, Bd = torch.tensor(A, device=dev), torch.tensor(B, device=dev)
        Aref, Bref = tf32_trunc(A[:, :K]), tf32_trunc(B[:, :K])
    else:
        Ad = torch.tensor(A, device=dev).to(torch.bfloat16)
        Bd = torch.tensor(B, device=dev).to(torch.bfloat16)
        Aref = Ad.float().cpu().numpy()[:, :K]
        Bref = Bd.float().cpu().numpy()[:, :K]
    ref = Aref.astype(np.float64) @ Bref.astype(np.float64).T
    absref = np.abs(Aref.astype(np.float64)) @ np.abs(Bref.astype(np.float64)).T
    C = torch.full((M, N), np.nan, dtype=torch.float32, device=dev)
    bias = torch.tensor(rng.standard_normal(N).astype(np.float32), device=dev)
    if epi == 0:
        fitcore.fit_tc_gemm(tf32, M, N, K, Ad, lda, Bd, lda, 0, C=C, ldc=N)
    else:
        fitcore.fit_tc_gemm(tf32, M, N, K, Ad, lda, Bd, lda, 1, C=C, ldc=N, bias=bias)
        ref = ref + bias.cpu().numpy()[None, :]
    torch.cuda.synchronize()
    assert fitcore.fit_tc_gemm_status() == 0
    got = C.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref) / (absref + 1e-30)
    return err.max()


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 256, 128), (300, 208, 438), (37, 12, 512),
                                   (1024, 512, 448), (129, 400, 200)])
def test_bf16_gemm(M, N, K):
    assert run(False, M, N, K) <= 4e-6 * np.sqrt(K / 64)


@pytest.mark.parametrize("M,N,K", [(128, 48, 400), (256, 400, 2000), (77, 38, 400), (512, 16, 32)])
def test_tf32_gemm(M, N, K):
    assert run(True, M, N, K) <= 4e-6 * np.sqrt(K / 32)


def test_bias_epilogue():
    assert run(False, 200, 120, 96, epi=1) <= 1e-5


@pytest.mark.parametrize("tf32,M,N,K", [(False, 512, 438, 16384), (False, 96, 70, 3000),
                                        (True, 40, 38, 2000), (True, 1, 400, 2000)])
def test_split_k_padded_output(tf32, M, N, K):
    """Small output grids with a long K run split over K with atomic accumulation; the output
    rows are padded (ldc > N) and the padding must stay untouched."""
    rng = np.random.default_rng(11)
    lda = ((K + 7) // 8) * 8
    A = rng.standard_normal((M, lda)).astype(np.float32)
    B = rng.standard_normal((N, lda)).astype(np.float32)
    dev = torch.device("cuda")
    if tf32:
        Ad, Bd = torch.tensor(A, device=dev), torch.tensor(B, device=dev)
        Aref, Bref = tf32_trunc(A[:, :K]), tf32_trunc(B[:, :K])
    else:
        Ad = torch.tensor(A, device=dev).to(torch.bfloat16)
        Bd = torch.tensor(B, device=dev).to(torch.bfloat16)
        Aref, Bref = Ad.float().cpu().numpy()[:, :K], Bd.float().cpu().numpy()[:, :K]
    ref = Aref.astype(np.float64) @ Bref.astype(np.float64).T
    absref = np.abs(Aref.astype(np.float64)) @ np.abs(Bref.astype(np.float64)).T
    ldc = N + 5
    C = torch.full((M, ldc), np.nan, dtype=torch.float32, device=dev)
    fitcore.fit_tc_gemm(tf32, M, N, K, Ad, lda, Bd, lda, 0, C=C, ldc=ldc)
    # accumulate the same product once more (EPI_F32_ADD = 4)
    fitcore.fit_tc_gemm(tf32, M, N, K, Ad, lda, Bd, lda, 4, C=C, ldc=ldc)
    torch.cuda.synchronize()
    assert fitcore.fit_tc_gemm_status() == 0
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isnan(got[:, N:]))
    err = np.abs(got[:, :N] - 2 * ref) / (2 * absref + 1e-30)
    assert err.max() <= 4e-6 * np.sqrt(K / 32)


@pytest.mark.parametrize("M,N,K", [(16384, 512, 512), (5000, 300, 712)])
def test_bf16_gemm_many_tiles_per_cta(M, N, K):
    """More output tiles than SMs: each persistent CTA takes several tiles in turn, alternating
    its two tensor-memory accumulators (one drained by the epilogue while the other fills)."""
    assert run(False, M, N, K) <= 4e-6 * np.sqrt(K / 64)


def _gelu64(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _gelu_grad64(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


@pytest.mark.parametrize("M,N,K", [(300, 208, 438), (4100, 512, 512), (77, 12, 64)])
def test_gelu_epilogues(M, N, K):
    """Epilogue 2 (C = D + bias, Y = bf16(gelu(C))) and epilogue 3 (Y = bf16(D gelu'(aux)))
    against float64: C within the accumulation bound, Y within one bf16 rounding (2^-8
    relative) of the float64 value at the kernel's own C (epilogue 2) or of the float64
    product (epilogue 3), plus the accumulation error carried through."""
    rng = np.random.default_rng(5)
    lda = ((K + 7) // 8) * 8
    dev = torch.device("cuda")
    Ad = torch.tensor(rng.standard_normal((M, lda)).astype(np.float32), device=dev).to(torch.bfloat16)
    Bd = torch.tensor((rng.standard_normal((N, lda)) / np.sqrt(K)).astype(np.float32), device=dev).to(torch.bfloat16)
    Aref = Ad.float().cpu().numpy()[:, :K].astype(np.float64)
    Bref = Bd.float().cpu().numpy()[:, :K].astype(np.float64)
    ref = Aref @ Bref.T
    absref = np.abs(Aref) @ np.abs(Bref).T
    bias = torch.tensor(rng.standard_normal(N).astype(np.float32), device=dev)
    ldy = ((N + 7) // 8) * 8
    C = torch.full((M, N), np.nan, dtype=torch.float32, device=dev)
    Y = torch.zeros((M, ldy), dtype=torch.bfloat16, device=dev)
    fitcore.fit_tc_gemm(False, M, N, K, Ad, lda, Bd, lda, 2, C=C, ldc=N, Y=Y, ldy=ldy, bias=bias)
    aux = torch.tensor(rng.standard_normal((M, N)).astype(np.float32), device=dev)
    Y3 = torch.zeros((M, ldy), dtype=torch.bfloat16, device=dev)
    fitcore.fit_tc_gemm(False, M, N, K, Ad, lda, Bd, lda, 3, Y=Y3, ldy=ldy, aux=aux, ldaux=N)
    torch.cuda.synchronize()
    assert fitcore.fit_tc_gemm_status() == 0
    acc = 4e-6 * np.sqrt(K / 64) * absref
    c = C.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(c - (ref + bias.cpu().numpy()[None, :])) <= acc + 1e-6)
    y = Y.float().cpu().numpy()[:, :N].astype(np.float64)
    g = _gelu64(c)
    assert np.all(np.abs(y - g) <= 2.0 ** -8 * np.abs(g) + 1e-6)
    y3 = Y3.float().cpu().numpy()[:, :N].astype(np.float64)
    gg = _gelu_grad64(aux.cpu().numpy().astype(np.float64))
    want = ref * gg
    assert np.all(np.abs(y3 - want) <= 2.0 ** -8 * np.abs(want) + acc * np.abs(gg) + 1e-6)
