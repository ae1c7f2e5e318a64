"""The allocation-free GEMM entry point, for callers that cannot allocate device memory (a capped or
foreign-owned device allocator, a real-time loop that must not enter the allocator).  It stages
its packed operands in a static device array instead of a workspace; its results must match the
regular tensor-core entry point rfdd_cgemm within the tolerance of tests/test_gpu_gemm.py, on two
calls in a row that reuse the same array.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_cgemm_on_two_calls(R):
    import torch
    cases = [(300, 257, 100, 11, -1.0, 1.0), (1024, 65, 128, 12, 1.0, 0.0)]
    for m, n, k, seed, alpha, beta in cases:
        A, B, C0 = rnd((m, k), seed), rnd((k, n), seed + 1), rnd((m, n), seed + 2)
        want = R.rfdd_cgemm(A, B, C0, alpha, beta, 1)
        dA = torch.from_numpy(A.view(np.float32).copy()).cuda()
        dB = torch.from_numpy(B.view(np.float32).copy()).cuda()
        dC = torch.from_numpy(C0.view(np.float32).copy()).cuda()
        torch.cuda.synchronize()
        R.rfdd_cgemm_noalloc(m, n, k, dA.data_ptr(), k, dB.data_ptr(), n, dC.data_ptr(), n, alpha, beta)
        got = dC.cpu().numpy().view(np.complex64)
        scale = np.abs(A).max() * np.abs(B).max() * k + np.abs(C0).max()
        assert np.abs(got - want).max() / scale <= 2e-6


def test_noalloc_rejects_sizes_beyond_the_static_array(R):
    with pytest.raises(R.RfddError) as e:
        R.rfdd_cgemm_noalloc(1025, 8, 8, 16, 8, 16, 8, 16, 8)
    assert e.value.code == R.RFDD_EINVAL
    with pytest.raises(R.RfddError) as e:
        R.rfdd_cgemm_noalloc(8, 8, 129, 16, 129, 16, 8, 16, 8)
    assert e.value.code == R.RFDD_EINVAL
