"""The tcgen05 tensor-core GEMM (TMA + TMEM, BF16 inputs, FP32 accumulation)
against torch's matmul of the same BF16 operands in FP32, through the C ABI,
on ragged shapes (M not a multiple of the 128-row tile, K narrower than one
64-wide k-block, N split over two 192-wide tiles)."""
import ctypes

import pytest
import torch

from paper_2402_17660_gb300 import _lib

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _run(M, N, K, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = _lib.load()
    rc = lib.tnet_debug_tc_gemm(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = A.double() @ B.double().T
    err = (C.double() - ref).abs().max().item()
    scale = ref.abs().max().item()
    return err, scale


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (1, 32, 32), (300, 128, 32), (1000, 256, 128),
                                   (777, 384, 256), (129, 64, 384), (4096, 384, 256), (5000, 32, 128)])
def test_tc_gemm_matches_matmul(M, N, K):
    err, scale = _run(M, N, K)
    # exact BF16 products, FP32 accumulation over K terms
    assert err <= 1e-5 * scale * max(1.0, (K / 64) ** 0.5), (err, scale)


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (1, 32, 32), (300, 128, 128), (777, 384, 256), (129, 64, 384),
                                   (4096, 256, 128), (200, 64, 36), (3000, 32, 384), (20000, 128, 256),
                                   (8192, 384, 384), (5000, 384, 32), (3001, 256, 24), (1500, 384, 100),
                                   (999, 128, 52)])
def test_tc_gemm_3xtf32_matches_fp64(M, N, K):
    """3xTF32 (A B + A_lo B + A B_lo on the tensor cores, A's split formed in
    shared memory, or in tensor memory for the 128- and 192-wide tiles)
    reaches FP32-level accuracy on fp32 inputs, including a ragged last
    k-block and persistent CTAs whose stages wrap many times.
    Each operand is split into its nearest TF32 value and the TF32-rounded
    remainder (below 2^-11 of the value, rounded to within 2^-22 of it), so
    the three products miss the exact one by less than 3 * 2^-22 |a||b| (plus
    FP32 accumulation), elementwise."""
    g = torch.Generator(device="cpu").manual_seed(1)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    Bsplit = torch.empty(2 * N * K, dtype=torch.float32, device="cuda")
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = _lib.load()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.tnet_debug_tc_gemm_f32(M, N, K, p(A), p(B), p(Bsplit), p(C), p(st),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = A.double() @ B.double().T
    scale = A.double().abs() @ B.double().abs().T          # sum_k |a_ik| |b_jk|
    rel = ((C.double() - ref).abs() / scale)
    assert rel.max().item() <= 3 * 2.0 ** -22 + K * 2.0 ** -24, rel.max().item()
    # typical error: at the FP32 accumulation floor (a split that went wrong,
    # e.g. a residual from another tile, shows up near 1e-4)
    assert rel.pow(2).mean().sqrt().item() <= 3e-7, rel.pow(2).mean().sqrt().item()


@pytest.mark.parametrize("cluster", [2, 4])
@pytest.mark.parametrize("x3,M,N,K", [(1, 777, 384, 256), (1, 20000, 128, 256), (1, 4096, 256, 128),
                                      (1, 5000, 384, 32), (1, 129, 64, 384), (1, 1, 32, 32), (1, 1500, 384, 100),
                                      (0, 1000, 256, 128), (0, 777, 384, 256), (0, 300, 128, 64), (0, 1, 32, 32)])
def test_tc_gemm_clusters_match_single_ctas_bitwise(x3, M, N, K, cluster):
    """CTAs in clusters that share each weight stage through TMA multicast
    (each loads 1/cluster of the B rows into every CTA's shared memory, and
    every CTA's MMA issuer releases the stage in all of them) compute exactly
    what lone CTAs do: the same MMAs on the same tiles.  Row counts that leave
    the last cluster with CTAs past the last row tile, a single row, ragged K
    and every column-tile form are included."""
    g = torch.Generator(device="cpu").manual_seed(3)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    if not x3:
        A, B = A.bfloat16(), B.bfloat16()
    Bsplit = torch.empty(2 * N * K, dtype=torch.float32, device="cuda")
    lib = _lib.load()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = []
    for cl in (1, cluster):
        C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert lib.tnet_debug_tc_gemm_cluster(M, N, K, x3, cl, p(A), p(B), p(Bsplit), p(C), p(st), sp) == 0
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        out.append(C)
    assert torch.equal(out[0], out[1])
    ref = A.double() @ B.double().T
    err = (out[1].double() - ref).abs().max().item() / ref.abs().max().item()
    assert err <= (1e-5 if x3 else 2e-2), err


def test_tc_gemm_cluster_rejects_other_sizes():
    lib = _lib.load()
    z = ctypes.c_void_p(0)
    assert lib.tnet_debug_tc_gemm_cluster(128, 128, 64, 1, 3, z, z, z, z, z, z) != 0


def test_bounded_waits_report_timeout_and_leave_the_context_usable():
    """The failure path of the tensor-core kernel, made to happen without a
    fault: the 3xTF32 GEMM runs with its MMA issuer told to issue nothing and
    every mbarrier wait limited to 4096 tries.  The tile loads land and nobody
    consumes them, so the waits run out: the kernel records TIMEOUT (6) in the
    status word, waits for its own copies, frees its tensor memory and
    returns without writing C.  A normal GEMM on the same stream afterwards
    runs and is accurate."""
    M, N, K = 1000, 128, 256
    g = torch.Generator(device="cpu").manual_seed(2)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    Bsplit = torch.empty(2 * N * K, dtype=torch.float32, device="cuda")
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = _lib.load()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.tnet_debug_tc_gemm_timeout(M, N, K, p(A), p(B), p(Bsplit), p(C), 0, p(st), stream) == 1
    rc = lib.tnet_debug_tc_gemm_timeout(M, N, K, p(A), p(B), p(Bsplit), p(C), 4096, p(st), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 6
    assert torch.isnan(C).all()
    st.zero_()
    rc = lib.tnet_debug_tc_gemm_f32(M, N, K, p(A), p(B), p(Bsplit), p(C), p(st), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = A.double() @ B.double().T
    rel = (C.double() - ref).abs() / (A.double().abs() @ B.double().abs().T)
    assert rel.max().item() <= 3 * 2.0 ** -22 + K * 2.0 ** -24
