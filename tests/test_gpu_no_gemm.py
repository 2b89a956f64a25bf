"""The tcgen05 BF16 GEMM (lbm_gemm_bf16) against an FP64 product of the same BF16 inputs.

Bound: FP32 accumulation of K exact BF16 products, |C - C_ref| <= 2^-20 * sum_k |a_mk| |b_kn|
(per element), which covers any summation order of the tensor core's FP32 adds.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import _native as nat  # noqa: E402


def _gemm(M, N, K, batch, A, sa, B, sb, C, sc, out_bf16=0, alpha=1.0, beta=0):
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = nat.lib().lbm_gemm_bf16(M, N, K, batch, A.data_ptr(), *sa, B.data_ptr(), *sb, C.data_ptr(), *sc,
                                 out_bf16, ctypes.c_float(alpha), beta, err.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == nat.LBM_OK, nat.status_name(st)
    torch.cuda.synchronize()
    assert int(err.item()) == 0


def _check(Cg, Cr, bound):
    diff = np.abs(Cg - Cr)
    assert (diff <= bound + 1e-30).all(), (diff.max(), bound.max())


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 100, 150), (7, 5, 3), (256, 192, 512)])
def test_gemm_row_major(M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda")
    Ad, Bd = A.cuda(), B.cuda()
    _gemm(M, N, K, 1, Ad, (K, 1, 0), Bd, (N, 1, 0), C, (N, 1, 0))
    a, b = A.float().numpy().astype(np.float64), B.float().numpy().astype(np.float64)
    _check(C.cpu().numpy(), a @ b, 2.0 ** -20 * (np.abs(a) @ np.abs(b)))


def test_gemm_transposed_batched_views():
    """A as an M-contiguous view, B K-contiguous (N x K storage), C column-major, batch 3."""
    M, N, K, nb = 200, 72, 96, 3
    g = torch.Generator().manual_seed(5)
    At = torch.randn(nb, K, M, generator=g).to(torch.bfloat16)  # A[b][m][k] = At[b][k][m]
    Bt = torch.randn(nb, N, K, generator=g).to(torch.bfloat16)  # B[b][k][n] = Bt[b][n][k]
    C = torch.zeros(nb, N, M, device="cuda")                      # C[b][m][n] at (n, m)
    _gemm(M, N, K, nb, At.cuda(), (1, M, K * M), Bt.cuda(), (1, K, N * K), C, (1, M, N * M))
    for i in range(nb):
        a = At[i].float().numpy().astype(np.float64).T
        b = Bt[i].float().numpy().astype(np.float64).T
        _check(C[i].cpu().numpy().T, a @ b, 2.0 ** -20 * (np.abs(a) @ np.abs(b)))


def test_gemm_bf16_output_accumulate_alpha():
    M, N, K = 130, 70, 40
    g = torch.Generator().manual_seed(9)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    C0 = torch.randn(M, N, generator=g).to(torch.bfloat16)
    C = C0.cuda()
    _gemm(M, N, K, 1, A.cuda(), (K, 1, 0), B.cuda(), (N, 1, 0), C, (N, 1, 0), out_bf16=1, alpha=0.5, beta=1)
    a, b = A.float().numpy().astype(np.float64), B.float().numpy().astype(np.float64)
    ref = C0.float().numpy() + 0.5 * (a @ b)
    got = C.float().cpu().numpy()
    # result rounded to BF16 once: half an ulp of 2^-8 relative, plus the accumulation bound
    _check(got, ref, 2.0 ** -8 * np.abs(ref) + 2.0 ** -20 * (np.abs(a) @ np.abs(b)))


@pytest.mark.parametrize("M,N,K,nb", [(64, 24, 64, 1500), (40, 48, 150, 1301), (64, 64, 24, 2000)])
def test_gemm_many_small_products(M, N, K, nb):
    """Batches much larger than the number of CTAs, with B shared by every item (the operator's DFT
    products): items of one or several K slices, through the copy-engine path (K = 64 and 24:
    persistent blocks, two items per tile) and the register-staged one (K = 150, rows not 16-byte
    aligned); every item against its FP64 product at the accumulation bound."""
    g = torch.Generator().manual_seed(M * 31 + nb)
    A = torch.randn(nb, M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(K, N, generator=g).to(torch.bfloat16)
    C = torch.empty(nb, M, N, device="cuda")
    _gemm(M, N, K, nb, A.cuda(), (K, 1, M * K), B.cuda(), (N, 1, 0), C, (N, 1, M * N))
    a = A.float().numpy().astype(np.float64)
    b = B.float().numpy().astype(np.float64)
    ref = np.einsum("imk,kn->imn", a, b)
    bound = 2.0 ** -20 * np.einsum("imk,kn->imn", np.abs(a), np.abs(b))
    _check(C.cpu().numpy(), ref, bound)


def _operand(rng, rows, K, nb, k_major, pad):
    """Rows x K BF16 operand of nb items, stored K-contiguous (k_major) or rows-contiguous, the
    contiguous extent rounded up to a multiple of 8 and padded by `pad` more elements; returns (host array [nb, rows, K], device
    storage, (s_row, s_k, s_batch)); nb = 0 stores one item shared by every batch item."""
    items = max(nb, 1)
    x = torch.from_numpy(rng.normal(size=(items, rows, K)).astype(np.float32)).to(torch.bfloat16)
    if k_major:
        ld = -(-K // 8) * 8 + pad
        store = torch.zeros(items, rows, ld, dtype=torch.bfloat16)
        store[:, :, :K] = x
        strides = (ld, 1, rows * ld if nb else 0)
    else:
        ld = -(-rows // 8) * 8 + pad
        store = torch.zeros(items, K, ld, dtype=torch.bfloat16)
        store[:, :, :rows] = x.transpose(1, 2)
        strides = (1, ld, K * ld if nb else 0)
    return x.float().numpy().astype(np.float64), store.cuda(), strides


@pytest.mark.parametrize("a_k,b_k", [(True, True), (True, False), (False, True), (False, False)])
@pytest.mark.parametrize("M,N,K,nb,b_shared", [(200, 40, 72, 3, False), (130, 120, 200, 2, True),
                                                (300, 264, 136, 1, False), (64, 24, 64, 700, True),
                                                (40, 48, 136, 301, True), (24, 40, 200, 5, False)])
def test_gemm_tma_operand_layouts(a_k, b_k, M, N, K, nb, b_shared):
    """Operands the copy engine can address (16-byte aligned, strides multiples of 8 elements):
    each of A and B K-contiguous or M/N-contiguous, ragged M, N and K (K a multiple of 8 but not
    of 64), batched items or one B shared by all, tiles 64, 128 and 256 columns wide, and items
    of at most 64 rows against a shared B (two items per 128-row tile; an odd count leaves the
    last tile half empty)."""
    rng = np.random.default_rng(M * 13 + N * 7 + K + 2 * a_k + b_k)
    a, Ad, sa = _operand(rng, M, K, nb, a_k, 8)
    b, Bd, sbt = _operand(rng, N, K, 0 if b_shared else nb, b_k, 16)   # stored as N x K
    sb = (sbt[1], sbt[0], sbt[2])                                       # (s_k, s_n, s_batch)
    C = torch.zeros(nb, M, N, device="cuda")
    _gemm(M, N, K, nb, Ad, sa, Bd, sb, C, (N, 1, M * N))
    bt = np.broadcast_to(b, (nb, N, K)) if b_shared else b
    ref = np.einsum("imk,ink->imn", a, bt)
    bound = 2.0 ** -20 * np.einsum("imk,ink->imn", np.abs(a), np.abs(bt))
    _check(C.cpu().numpy(), ref, bound)


@pytest.mark.parametrize("out_bf16", [0, 1])
@pytest.mark.parametrize("c_row_major", [False, True])
@pytest.mark.parametrize("beta", [0, 1])
def test_gemm_tma_alpha_beta_epilogue(out_bf16, c_row_major, beta):
    """The copy-engine path's epilogue, alpha = -0.75, FP32 or BF16 output, C column-major (M
    contiguous) or row-major (N contiguous), ragged rows and a ragged last column box: stored
    through shared memory by the copy engine (beta = 0), added to the previous C by its reduce-add
    (beta, FP32), or stored from registers after loading the previous C (beta, BF16)."""
    M, N, K, nb = 260, 72, 96, 2
    rng = np.random.default_rng(77 + out_bf16 + 2 * c_row_major + 4 * beta)
    a, Ad, sa = _operand(rng, M, K, nb, True, 0)
    b, Bd, sbt = _operand(rng, N, K, nb, False, 8)
    sb = (sbt[1], sbt[0], sbt[2])
    dt = torch.bfloat16 if out_bf16 else torch.float32
    if c_row_major:
        c0 = rng.normal(size=(nb, M, N)).astype(np.float32)            # C[b][m][n] at (b, m, n)
        sc = (N, 1, M * N)
    else:
        c0 = rng.normal(size=(nb, N, M)).astype(np.float32)            # C[b][m][n] at (b, n, m)
        sc = (1, M, N * M)
    C = torch.from_numpy(c0).to(dt).cuda()
    c0 = C.float().cpu().numpy().astype(np.float64)
    _gemm(M, N, K, nb, Ad, sa, Bd, sb, C, sc, out_bf16=out_bf16, alpha=-0.75, beta=beta)
    eq = "imk,ink->imn" if c_row_major else "imk,ink->inm"
    prod = np.einsum(eq, a, b)
    ref = beta * c0 - 0.75 * prod
    bound = 0.75 * 2.0 ** -20 * np.einsum(eq, np.abs(a), np.abs(b))
    if out_bf16:
        bound = bound + 2.0 ** -8 * np.abs(ref)
    _check(C.float().cpu().numpy(), ref, bound)


@pytest.mark.parametrize("beta", [0, 1])
def test_gemm_empty_k_and_thin_shapes(beta):
    """K = 0 is an empty sum: C = 0, or C unchanged with beta.  Then products with one row, one
    column or K = 1 against their FP64 values."""
    M, N = 37, 29
    C0 = torch.randn(M, N, generator=torch.Generator().manual_seed(4))
    C = C0.clone().cuda()
    A = torch.zeros(M, 1, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(1, N, dtype=torch.bfloat16, device="cuda")
    _gemm(M, N, 0, 1, A, (1, 1, 0), B, (N, 1, 0), C, (N, 1, 0), beta=beta)
    assert torch.equal(C.cpu(), C0 if beta else torch.zeros(M, N))
    g = torch.Generator().manual_seed(6)
    for (M, N, K) in [(1, 40, 72), (40, 1, 72), (56, 48, 1), (1, 1, 8)]:
        A = torch.randn(M, K, generator=g).to(torch.bfloat16)
        B = torch.randn(K, N, generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        _gemm(M, N, K, 1, A.cuda(), (K, 1, 0), B.cuda(), (N, 1, 0), C, (N, 1, 0))
        a, b = A.float().numpy().astype(np.float64), B.float().numpy().astype(np.float64)
        _check(C.cpu().numpy(), a @ b, 2.0 ** -20 * (np.abs(a) @ np.abs(b)))
