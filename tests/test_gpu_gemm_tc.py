"""The surrogate's tensor-core GEMM (tcgen05 MMAs, FP32 accumulation in
tensor memory), called through mm_gemm_bf16, against the FP64 product of
the same BF16 values.

Tolerance: a product of two BF16 values is exact in FP32, so the only
error is the FP32 summation of K terms (and one more rounding for beta C
or the atomic add): per element |got - ref| <= (K + 4) 2^-23 (sum_k |a_ik
b_kj| + |beta c_ij|), the standard bound for recursive summation with
unit roundoff 2^-24 and a factor 2 of slack for any summation order.
"""
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_7459_gb300 import mm
    mm.lib()


CASES = [
    # name, M, N, K, transposed A, transposed B, batch, shared A, alpha, beta, atomic
    ("x-mode transform shape", 256, 32, 256, False, False, 1, False, 1.0, 0.0, False),
    ("wide N, short K", 256, 256, 32, False, False, 1, False, 1.0, 0.0, False),
    ("ragged, N in one 64 tile", 200, 40, 48, False, False, 1, False, 1.0, 0.0, False),
    ("ragged, wide tiles", 200, 136, 48, False, False, 1, False, 1.0, 0.0, False),
    ("M-major A, K-major B", 384, 32, 64, True, True, 1, False, 1.0, 0.0, False),
    ("M-major A, long ragged K", 256, 32, 200, True, True, 1, False, 1.0, 0.0, False),
    ("batched, shared A, beta", 128, 160, 32, False, False, 3, True, 1.0, 1.0, False),
    ("atomic, odd sizes", 130, 33, 17, False, False, 1, False, 0.5, 0.0, True),
    ("row stride not a multiple of 4", 160, 38, 64, False, False, 1, False, 1.0, 1.0, False),
    ("float4 tail with beta", 130, 36, 64, False, False, 1, False, 1.0, 0.5, False),
    ("few rows, many columns (runs transposed)", 32, 4096, 32, False, False, 2, True, 1.0, 1.0, False),
    ("K = 0", 64, 32, 0, False, False, 1, False, 1.0, 2.0, False),
    # both operands K-contiguous: the whole K resident in shared memory
    ("K-major A and B, all of K resident", 256, 32, 256, False, True, 1, False, 1.0, 0.0, False),
    ("K-major A and B, ragged tiles, beta", 200, 136, 48, False, True, 1, False, 1.0, 0.5, False),
    ("K-major A and B, batched shared A, atomic", 130, 40, 64, False, True, 2, True, 0.5, 0.0, True),
    ("K-major A and B, short K, wide N", 8192, 256, 32, False, True, 1, False, 1.0, 0.0, False),
    ("K-major A and B, K past the resident limit", 128, 64, 288, False, True, 1, False, 1.0, 0.0, False),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gemm_bf16_matches_fp64(case):
    from paper_1406_7459_gb300 import mm
    name, M, N, K, ta, tb, batch, share, alpha, beta, atomic = case
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    Ah = torch.from_numpy(rng.standard_normal((batch, M, K)).astype(np.float32)).to(torch.bfloat16)
    Bh = torch.from_numpy(rng.standard_normal((batch, K, N)).astype(np.float32)).to(torch.bfloat16)
    if share:
        Ah[1:] = Ah[0]
    C0 = torch.from_numpy(rng.standard_normal((batch, M, N)).astype(np.float32))
    Ad = (Ah.transpose(1, 2) if ta else Ah).contiguous().cuda()
    Bd = (Bh.transpose(1, 2) if tb else Bh).contiguous().cuda()
    if K == 0:
        Ad = torch.zeros(1, dtype=torch.bfloat16, device="cuda")
        Bd = torch.zeros(1, dtype=torch.bfloat16, device="cuda")
    Cd = C0.clone().cuda()
    sam, sak = (1, M) if ta else (K, 1)
    sbk, sbn = (1, K) if tb else (N, 1)
    zA = 0 if share else M * K
    mm.mm_gemm_bf16(Ad, Bd, Cd, M, N, K, (sam, sak, sbk, sbn, N, 1), batch=batch,
                    batch_strides=(zA, K * N, M * N), alpha=alpha, beta=beta, atomic=atomic)
    A64, B64, C64 = Ah.double().numpy(), Bh.double().numpy(), C0.double().numpy()
    ref = alpha * np.einsum("zmk,zkn->zmn", A64, B64)
    cterm = C64 if atomic else beta * C64
    ref = ref + cterm
    bound = (K + 4) * 2.0 ** -23 * (abs(alpha) * np.einsum("zmk,zkn->zmn", np.abs(A64), np.abs(B64)) +
                                    np.abs(cterm)) + 1e-30
    got = Cd.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


def test_gemm_bf16_rejects_bad_sizes():
    from paper_1406_7459_gb300 import mm
    A = torch.zeros(16, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(16, dtype=torch.float32, device="cuda")
    for M, N, K, batch in ((0, 4, 4, 1), (4, 0, 4, 1), (4, 4, -1, 1), (4, 4, 4, 0), (4, 4, 4, 70000)):
        with pytest.raises(mm.MMError) as e:
            mm.mm_gemm_bf16(A, A, C, M, N, K, (K, 1, N, 1, N, 1), batch=batch)
        assert e.value.code == -1
