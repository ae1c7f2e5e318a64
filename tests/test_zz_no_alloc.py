"""The allocation-free GEMM entry point, for callers that cannot allocate device memory (a capped or
foreign-owned device allocator, a real-time loop that must not enter the allocator).  It stages
its packed operands in a static device array instead of a workspace.  Its results must match an
FP64 product, and the regular tensor-core entry point rfdd_cgemm, within the tolerance of
tests/test_gpu_gemm.py, on two calls in a row that reuse the same array; padded leading
dimensions and a non-default stream are covered, and a warm call must leave the device's free
memory and torch's allocation count unchanged.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-6  # FP32-level accuracy of the 3xTF32 split, as in tests/test_gpu_gemm.py


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def rnd(shape, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex64)


def padded(torch, X, ld):
    """Device copy of X (rows x cols complex64) in a buffer with leading dimension ld >= cols."""
    rows, cols = X.shape
    buf = np.zeros((rows, ld), dtype=np.complex64)
    buf[:, :cols] = X
    return torch.from_numpy(buf.view(np.float32).copy()).cuda()


def run_noalloc(R, torch, A, B, C0, alpha, beta, pad, stream):
    m, k = A.shape
    n = B.shape[1]
    lda, ldb, ldc = k + pad, n + pad, n + pad
    dA, dB, dC = padded(torch, A, lda), padded(torch, B, ldb), padded(torch, C0, ldc)
    torch.cuda.synchronize()
    R.rfdd_cgemm_noalloc(m, n, k, dA.data_ptr(), lda, dB.data_ptr(), ldb, dC.data_ptr(), ldc, alpha, beta,
                         stream.cuda_stream if stream is not None else 0)
    out = dC.cpu().numpy().view(np.complex64).reshape(m, ldc)
    # the padding columns of C are not touched
    assert np.array_equal(out[:, n:], np.zeros((m, pad), dtype=np.complex64))
    return out[:, :n]


CASES = [(300, 257, 100, 11, -1.0, 1.0, 0), (1024, 65, 128, 12, 1.0, 0.0, 0), (130, 1024, 33, 13, 0.5, -2.0, 3),
         (1, 1, 1, 14, 1.0, 1.0, 5)]


@pytest.mark.parametrize("on_stream", [False, True])
def test_noalloc_matches_fp64_and_cgemm_on_two_calls(R, on_stream):
    import torch
    stream = torch.cuda.Stream() if on_stream else None
    for rep in range(2):  # two calls in a row on the same static array
        for m, n, k, seed, alpha, beta, pad in CASES:
            A, B, C0 = rnd((m, k), seed + rep), rnd((k, n), seed + 1), rnd((m, n), seed + 2)
            got = run_noalloc(R, torch, A, B, C0, alpha, beta, pad, stream)
            exact = beta * C0.astype(np.complex128) + alpha * (A.astype(np.complex128) @ B.astype(np.complex128))
            scale = np.abs(A).max() * np.abs(B).max() * k + np.abs(C0).max()
            assert np.abs(got - exact).max() / scale <= TOL, (m, n, k, rep)
            want = R.rfdd_cgemm(A, B, C0, alpha, beta, 1)
            assert np.abs(got - want).max() / scale <= TOL, (m, n, k, rep)


def test_noalloc_allocates_nothing(R):
    import torch
    m, n, k = 512, 300, 128
    A, B, C0 = rnd((m, k), 21), rnd((k, n), 22), rnd((m, n), 23)
    dA, dB, dC = padded(torch, A, k), padded(torch, B, n), padded(torch, C0, n)
    stream = torch.cuda.Stream()
    args = (m, n, k, dA.data_ptr(), k, dB.data_ptr(), n, dC.data_ptr(), n, 1.0, 0.0, stream.cuda_stream)
    R.rfdd_cgemm_noalloc(*args)  # first call on the device: address look-up, module loading
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        R.rfdd_cgemm_noalloc(*args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    got = dC.cpu().numpy().view(np.complex64).reshape(m, n)
    exact = A.astype(np.complex128) @ B.astype(np.complex128)
    assert np.abs(got - exact).max() / (np.abs(A).max() * np.abs(B).max() * k) <= TOL


def test_noalloc_rejects_sizes_beyond_the_static_array(R):
    with pytest.raises(R.RfddError) as e:
        R.rfdd_cgemm_noalloc(1025, 8, 8, 16, 8, 16, 8, 16, 8)
    assert e.value.code == R.RFDD_EINVAL
    with pytest.raises(R.RfddError) as e:
        R.rfdd_cgemm_noalloc(8, 8, 129, 16, 129, 16, 8, 16, 8)
    assert e.value.code == R.RFDD_EINVAL
    with pytest.raises(R.RfddError) as e:
        R.rfdd_cgemm_noalloc(8, 1025, 8, 16, 8, 16, 1025, 16, 1025)
    assert e.value.code == R.RFDD_EINVAL
