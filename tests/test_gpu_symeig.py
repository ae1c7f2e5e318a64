"""GPU dense symmetric eigensolver (the projected problem of the Rayleigh-Ritz steps) against
LAPACK: eigenvalues, orthonormal eigenvectors, residuals; clustered and rank-deficient spectra."""
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


def _check(R, H):
    ev, V = R.rfdd_sym_eig(H)
    ref = np.linalg.eigvalsh(H)
    nrm = np.abs(ref).max()
    np.testing.assert_allclose(ev, ref, atol=1e-12 * nrm)
    n = H.shape[0]
    np.testing.assert_allclose(V @ V.T, np.eye(n), atol=1e-12)
    res = np.abs(H @ V.T - V.T * ev).max()
    assert res <= 1e-12 * nrm, res


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 200, 531])
def test_random(R, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    _check(R, A + A.T)


@pytest.mark.parametrize("n", [40, 300])
def test_clustered_and_rank_deficient(R, n):
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.full(6, 3.0), np.full(3, -1.0), np.zeros(n // 2), rng.uniform(5, 9, n - 9 - n // 2)])
    lam[9:9 + n // 2] = 1e-17 * rng.standard_normal(n // 2)
    _check(R, (Q * lam) @ Q.T)
