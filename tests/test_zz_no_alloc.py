"""The allocation-free GEMM entry point (qed_tc_gemm_static), through the C ABI.

It is for callers that cannot allocate device memory (code living inside another
framework's fixed memory pool): its split-K partial sums sit in a static device array.
It must give the same product as qed_tc_gemm (whose partials the caller sums), within the
FP32 accumulation bound of the tensor-core tests, on consecutive calls that reuse the
shared array.  Collected last so a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
qed = pytest.importorskip("paper_2403_07042_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07042_gb300 import build
    build.build()


def _pieces(rng, rows, K, n):
    x = rng.standard_normal((rows, K))
    out = []
    for _ in range(n):
        p = x.astype(np.float16)
        out.append(p)
        x = x - p.astype(np.float64)
    return np.stack(out)


def test_static_scratch_gemm_matches_tc_gemm_twice():
    rng = np.random.default_rng(123)
    cases = [(256, 128, 256, 3, ((0, 0), (0, 1), (1, 0)), 2, 2),
             (384, 256, 512, 4, ((0, 0), (0, 1), (1, 0), (2, 0)), 3, 2)]
    out = None
    for M, N, K, splits, seg, pa, pb in cases:  # two calls in a row on the same scratch
        A = torch.from_numpy(_pieces(rng, M, K, pa)).cuda()
        B = torch.from_numpy(_pieces(rng, N, K, pb)).cuda()
        want = qed.tc_gemm(A, B, segments=seg, splits=splits).double().sum(0).cpu().numpy()
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        got = qed.tc_gemm_static(A, B, segments=seg, splits=splits, out=out).double().cpu().numpy()
        Af, Bf = A.double().cpu().numpy(), B.double().cpu().numpy()
        bound = len(seg) * K * 2.0 ** -23 * (np.abs(Af).sum(0) @ np.abs(Bf).sum(0).T)
        exact = sum(Af[p] @ Bf[q].T for p, q in seg)
        assert np.all(np.abs(got - want) <= bound)
        assert np.all(np.abs(got - exact) <= bound)


def test_static_scratch_allocates_nothing_and_leaves_no_stale_partials():
    """After a first call (which looks up the array's device address), further calls leave
    the device's free memory unchanged; a same-shape call with new inputs returns the new
    product, not partial sums left in the shared array by the previous call."""
    rng = np.random.default_rng(7)
    M, N, K, splits, seg = 256, 256, 256, 4, ((0, 0), (0, 1), (1, 0))
    out = torch.empty((M, N), dtype=torch.float32, device="cuda")
    A0 = torch.from_numpy(_pieces(rng, M, K, 2)).cuda()
    B0 = torch.from_numpy(_pieces(rng, N, K, 2)).cuda()
    qed.tc_gemm_static(A0, B0, segments=seg, splits=splits, out=out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        qed.tc_gemm_static(A0, B0, segments=seg, splits=splits, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    A1 = torch.from_numpy(_pieces(rng, M, K, 2)).cuda()
    B1 = torch.from_numpy(_pieces(rng, N, K, 2)).cuda()
    got = qed.tc_gemm_static(A1, B1, segments=seg, splits=splits, out=out).double().cpu().numpy()
    Af, Bf = A1.double().cpu().numpy(), B1.double().cpu().numpy()
    exact = sum(Af[p] @ Bf[q].T for p, q in seg)
    bound = len(seg) * K * 2.0 ** -23 * (np.abs(Af).sum(0) @ np.abs(Bf).sum(0).T)
    assert np.all(np.abs(got - exact) <= bound)


def test_static_scratch_rejects_bad_out():
    A = torch.zeros((2, 128, 64), dtype=torch.float16, device="cuda")
    B = torch.zeros((2, 128, 64), dtype=torch.float16, device="cuda")
    with pytest.raises(ValueError):
        qed.tc_gemm_static(A, B, out=torch.empty((64, 128), dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        qed.tc_gemm_static(A, B, out=torch.empty((128, 128), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        qed.tc_gemm_static(A, torch.zeros((2, 128, 128), dtype=torch.float16, device="cuda"))


def test_static_scratch_rejects_oversize():
    A = torch.zeros((2, 2048, 64), dtype=torch.float16, device="cuda")
    B = torch.zeros((2, 2048, 64), dtype=torch.float16, device="cuda")
    with pytest.raises(qed.QedError) as ei:
        qed.tc_gemm_static(A, B, splits=2)   # 2 * 2048 * 2048 floats > 4 Mi
    assert ei.value.status == qed.QED_EINVAL
