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


def test_autotuner_decides_a_class_and_keeps_results(R):
    """The tile-shape autotuner: repeated launches of one class (complex, K = 256, 2048 x 2048, where
    both kernels can run) alternate between the one-CTA and the two-CTA kernel until each has three
    timings, then one kernel is kept; every result meets the FP32-level bound throughout."""
    R.rfdd_autotune(2)
    was_on = R.rfdd_autotune(1)
    try:
        m = n = 2048
        k = 256
        A, B, C0 = rnd((m, k), 4), rnd((k, n), 5), rnd((m, n), 6)
        want = -(A.astype(np.complex128) @ B.astype(np.complex128)) + C0
        scale = np.abs(A).max() * np.abs(B).max() * k + np.abs(C0).max()
        for _ in range(8):
            C = R.rfdd_cgemm(A, B, C0, -1.0, 1.0, 1)
            assert np.abs(C - want).max() / scale <= 2e-6
        t = R.rfdd_autotune_table()
        cls = [e for e in t if e["complex"] == 1 and e["kbucket"] == 4]
        assert len(cls) == 1, t
        e = cls[0]
        assert e["n"] == [3, 3] and e["winner"] in (0, 1), e
        assert all(v > 0 for v in e["ms_per_gflop"]), e
        # off: no new class is opened
        R.rfdd_autotune(0)
        R.rfdd_cgemm(A[:, :128], B[:128], C0, -1.0, 1.0, 1)
        assert len(R.rfdd_autotune_table()) == len(t)
    finally:
        R.rfdd_autotune(1 if was_on else 0)
