"""The complex-FP32 GEMM of the factorisations and solves: the tensor-core GEMM (tcgen05, 3xTF32)
with its automatic kernel choice, its one-CTA and two-CTA kernels forced, and the CUDA-core
kernel, against an FP64 product on ragged shapes that span several tiles (odd and even numbers of
128-row tiles, so the two-CTA kernel meets pairs with a missing second row)."""
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


@pytest.mark.parametrize("engine", [1, 0, 2, 3])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 3, 7), (128, 128, 16), (130, 129, 33), (300, 257, 64),
                                   (1000, 70, 128), (77, 640, 256), (513, 515, 100), (2000, 900, 256),
                                   (1100, 1300, 96)])
def test_cgemm(R, engine, m, n, k):
    A, B, C0 = rnd((m, k), 1), rnd((k, n), 2), rnd((m, n), 3)
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        C = R.rfdd_cgemm(A, B, C0, alpha, beta, engine)
        want = beta * C0.astype(np.complex128) + alpha * (A.astype(np.complex128) @ B.astype(np.complex128))
        scale = np.abs(A).max() * np.abs(B).max() * k + np.abs(C0).max()
        err = np.abs(C - want).max() / scale
        # FP32-level accuracy: the 3xTF32 split keeps about 21 bits per operand
        assert err <= 2e-6, (engine, alpha, beta, err)
