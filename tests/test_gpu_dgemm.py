"""The FP64 products on the eigenvector bases: double-FP32 kernel (engine 1) and FP64 CUDA-core
kernel (engine 0) against numpy's FP64 product, every transpose combination, ragged shapes over
several 64 x 64 tiles, deep K (split over CTAs) and symmetric products (upper tiles mirrored)."""
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
    return np.random.default_rng(seed).standard_normal(shape)


def check(R, m, n, k, ta, tb, engine, alpha, beta, seed=0):
    A = rnd((k, m) if ta else (m, k), seed + 1)
    B = rnd((n, k) if tb else (k, n), seed + 2)
    C0 = rnd((m, n), seed + 3)
    C = R.rfdd_dgemm(A, B, C0, alpha, beta, ta, tb, engine)
    opA = A.T if ta else A
    opB = B.T if tb else B
    want = beta * C0 + alpha * (opA @ opB)
    bound = np.abs(alpha) * (np.abs(opA) @ np.abs(opB)) + np.abs(beta * C0)
    return np.max(np.abs(C - want) / bound)


@pytest.mark.parametrize("engine", [1, 0])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 3, 7), (64, 64, 16), (130, 129, 33), (65, 200, 1000),
                                   (32, 32, 4681), (300, 257, 20000)])
def test_dgemm(R, engine, ta, tb, m, n, k):
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        err = check(R, m, n, k, ta, tb, engine, alpha, beta)
        # engine 1: two floats per operand (2^-48 each) and compensated sums; engine 0: FP64
        tol = 2.0 ** -42 if engine == 1 else 1e-14
        assert err <= tol, (engine, alpha, beta, err)


@pytest.mark.parametrize("engine", [1, 0])
@pytest.mark.parametrize("n,k", [(64, 100), (130, 5000), (257, 64000), (320, 3)])
def test_dgemm_symmetric(R, engine, n, k):
    # A^T (P A) with P symmetric: upper tiles computed, lower mirrored
    Y = rnd((k, n), 7)
    d = np.abs(rnd(k, 8)) + 0.5
    PY = d[:, None] * Y
    C0 = rnd((n, n), 9)
    for alpha, beta in ((1.0, 0.0), (2.0, -0.5)):
        C = R.rfdd_dgemm(Y, PY, C0 if beta else np.zeros((n, n)), alpha, beta, True, False, engine, True)
        want = alpha * (Y.T @ PY) + (beta * C0 if beta else 0.0)
        bound = alpha * (np.abs(Y.T) @ np.abs(PY)) + (np.abs(beta * C0) if beta else 0.0)
        assert np.max(np.abs(C - want) / bound) <= (2.0 ** -42 if engine == 1 else 1e-14)
        if beta == 0.0:
            assert np.array_equal(C, C.T)


def test_dgemm_rejects_bad_sizes(R):
    import paper_1711_09487_gb300 as pkg
    with pytest.raises(pkg.RfddError):
        R.rfdd_dgemm(np.zeros((3, 4)), np.zeros((3, 3)), np.zeros((4, 3)), 1.0, 0.0, True, False, 1, True)
