"""GPU checks of the tcgen05 building blocks on one CTA (w2_debug_umma_gemm):
integer-valued BF16 operands, so every product and sum is exact in the FP32
accumulator and the MMA must reproduce A B bit for bit.  TMEM is prefilled
with a marker word; the dump shows which lanes and columns the MMA wrote.

Order matters: the M = 64 case runs first.  Its A operand's rows 64..127 are
zero in shared memory, so if the hardware read the M field as 128 the lanes
64..127 would hold zero rows and the test fails before any M = 128 MMA is
issued."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MARK = np.uint32(0x7fc0dead)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11354_gb300 import build
    build.build()


def _ints(rng, shape, lim=8):
    return rng.integers(-lim, lim + 1, shape).astype(np.float32)


def _run(M, N, K, a_mn=False, b_mn=False, swap=False, seed=0):
    from paper_2511_11354_gb300 import w2
    rng = np.random.default_rng(seed)
    A, B = _ints(rng, (M, K)), _ints(rng, (K, N))
    dump = w2.umma_gemm(torch.from_numpy(A).cuda().bfloat16(), torch.from_numpy(B).cuda().bfloat16(),
                        a_mn=a_mn, b_mn=b_mn, swap=swap)
    d = dump.cpu().numpy().view(np.uint32)
    return A.astype(np.float64) @ B.astype(np.float64), d


def test_m64_lane_map():
    """M = 64: each of the 64 rows of A B appears exactly once, in full, in
    the first N columns of some lane; columns N..2N keep the marker; every
    lane the MMA touched holds a row."""
    M, N, K = 64, 64, 64
    want, d = _run(M, N, K, seed=1)
    assert np.all(d[:, N:] == MARK), "the MMA wrote beyond N columns"
    vals = d[:, :N].view(np.float32).astype(np.float64)
    touched = [L for L in range(128) if not np.all(d[L, :N] == MARK)]
    lane_of = {}
    for L in touched:
        hits = [m for m in range(M) if np.array_equal(vals[L], want[m])]
        assert len(hits) == 1, f"lane {L} holds no single row of A B (M read as another size?)"
        lane_of[hits[0]] = L
    assert sorted(lane_of) == list(range(M)), "rows missing from TMEM"
    # measured layout: rows 16 q .. 16 q + 15 in lanes 32 q .. 32 q + 15 of each lane quarter
    assert all(lane_of[m] == 32 * (m // 16) + m % 16 for m in range(M)), lane_of


@pytest.mark.parametrize("N,K,b_mn", [(64, 64, False), (64, 64, True), (32, 32, False), (16, 16, True),
                                      (48, 64, True)])
def test_m128_k_major_a(N, K, b_mn):
    """M = 128: lane i holds row i of A B exactly; nothing beyond N columns."""
    want, d = _run(128, N, K, b_mn=b_mn, seed=N + K)
    assert np.all(d[:, N:] == MARK)
    got = d[:, :N].view(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


def test_m64_mn_major_a():
    M, N, K = 64, 32, 64
    want, d = _run(M, N, K, a_mn=True, b_mn=True, seed=9)
    vals = d[:, :N].view(np.float32).astype(np.float64)
    rows = {m for L in range(128) for m in range(M) if np.array_equal(vals[L], want[m])}
    assert rows == set(range(M))


@pytest.mark.parametrize("N,K", [(64, 64), (32, 16)])
def test_m128_mn_major_a(N, K):
    """M = 128 with an MN-major A (the layout of the sheared planes)."""
    want, d = _run(128, N, K, a_mn=True, seed=7 + N)
    assert np.all(d[:, N:] == MARK)
    assert np.array_equal(d[:, :N].view(np.float32).astype(np.float64), want)


def test_stride_convention():
    """The descriptor's two core-matrix strides are not interchangeable: the
    encoding the library uses gives A B, the swapped one does not."""
    want, d = _run(128, 64, 64, b_mn=True, seed=3)
    assert np.array_equal(d[:, :64].view(np.float32).astype(np.float64), want)
    _, ds = _run(128, 64, 64, b_mn=True, swap=True, seed=3)
    assert not np.array_equal(ds[:, :64].view(np.float32).astype(np.float64), want)
