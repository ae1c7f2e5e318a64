"""C-ABI library checks that need no GPU: it loads, exports every symbol include/rfdd.h declares,
and its host-only paths (options, status strings, quadrature, input validation) behave."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import rfdd_inputs as I
from oracle import rfdd_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as pkg
    pkg.load()
    return pkg


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rfdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rfdd_[a-z_]+)\s*\(", text)))


def test_header_lists_the_boundary():
    syms = declared_symbols()
    for need in ("rfdd_setup", "rfdd_solve", "rfdd_result_get", "rfdd_result_free", "rfdd_destroy",
                 "rfdd_status_string", "rfdd_factor", "rfdd_filter_apply", "rfdd_lanczos"):
        assert need in syms


def test_library_exports_every_declared_symbol(R):
    lib = ctypes.CDLL(R.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(R.SYMBOLS) == declared_symbols()
    out = subprocess.run(["nm", "-D", "--defined-only", R.LIB_PATH], capture_output=True, text=True).stdout
    for s in declared_symbols():
        assert re.search(rf"\bT {s}\b", out), s


def test_options_and_status(R):
    o = R.rfdd_default_options()
    assert o.precision == R.RFDD_MIXED and o.psi == 3 and o.nev_b == 100 and o.block == 32
    assert abs(o.lanczos_tol - 1e-6) < 1e-20 and abs(o.res_tol - 1e-10) < 1e-24 and np.isnan(o.sigma)
    assert R.rfdd_status_string(R.RFDD_ESINGULAR) == "singular factorisation"
    assert R.rfdd_status_string(12345) == "unknown status"


@pytest.mark.parametrize("rule,name", [(0, "midpoint"), (1, "gauss_legendre")])
@pytest.mark.parametrize("nc", [1, 2, 3, 4, 8, 16])
def test_quadrature_matches_oracle(R, rule, name, nc):
    z, w = R.rfdd_quadrature(742.98, 1499.75, nc, rule)
    zo, wo = O.quadrature(742.98, 1499.75, nc, name)
    np.testing.assert_allclose(z, zo, rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(w, wo, rtol=1e-13, atol=1e-13)


def test_quadrature_rejects_bad_interval(R):
    with pytest.raises(R.RfddError) as e:
        R.rfdd_quadrature(2.0, 1.0, 4)
    assert e.value.code == R.RFDD_EINVAL


def _small():
    w = I.workload("q1_2d_24")
    return w.A, w.M, w.part, w.p


def test_setup_rejects_nonsymmetric(R):
    A, M, part, p = _small()
    a = A.to_scipy().tolil()
    a[0, 1] = a[0, 1] + 1.0
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(sp.csr_matrix(a), M, part, p)
    assert e.value.code == R.RFDD_ENOTSYM


def test_setup_rejects_bad_partitions(R):
    A, M, part, p = _small()
    bad = part.copy()
    bad[bad == 1] = 0          # subdomain 1 empty
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(A, M, bad, p)
    assert e.value.code == R.RFDD_EPARTITION
    bad = part.copy()
    bad[bad == -1] = 0         # no interface: subdomains touch
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(A, M, bad, p)
    assert e.value.code == R.RFDD_EPARTITION
    bad = part.copy()
    bad[0] = 7                 # label out of range
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(A, M, bad, p)
    assert e.value.code == R.RFDD_EPARTITION


def test_setup_rejects_indefinite_mass_and_size_mismatch(R):
    A, M, part, p = _small()
    m = M.to_scipy().tolil()
    m[3, 3] = -1.0
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(A, sp.csr_matrix(m), part, p)
    assert e.value.code == R.RFDD_ENOTSPD_M
    A2, M2 = I.q1_pencil(23, 2)
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(A2, M, part, p)
    assert e.value.code == R.RFDD_EINVAL


@pytest.mark.parametrize("which", ["A", "M"])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_setup_rejects_non_finite_values_before_device_work(R, which, bad):
    """A NaN or infinite CSR value is refused by the host validation (RFDD_EINVAL) before any
    kernel launch or device allocation."""
    A, M, part, p = _small()
    c = A if which == "A" else M
    val = c.val.copy()
    val[c.rowptr[5]] = bad          # first stored entry of row 5 (its mirror keeps symmetry out of play)
    bad_csr = I.Csr(c.n, c.rowptr, c.col, val)
    launches = R.rfdd_kernel_launches()
    with pytest.raises(R.RfddError) as e:
        if which == "A":
            R.rfdd_setup(bad_csr, M, part, p)
        else:
            R.rfdd_setup(A, bad_csr, part, p)
    assert e.value.code == R.RFDD_EINVAL
    assert "non-finite" in str(e.value)
    assert R.rfdd_kernel_launches() == launches


def test_setup_rejects_an_unknown_csr_location_before_device_work(R):
    A, M, part, p = _small()
    a, m = R._Csr(A), R._Csr(M)
    a.s.location = 7
    out = R.C.c_void_p()
    pt = np.ascontiguousarray(part, dtype=np.int32)
    launches = R.rfdd_kernel_launches()
    rc = R.load().rfdd_setup(R.C.byref(a.s), R.C.byref(m.s), pt.ctypes.data_as(R.C.POINTER(R.C.c_int32)), p,
                             None, R.C.byref(out))
    assert rc == R.RFDD_EINVAL and "location" in R.load().rfdd_last_error().decode()
    assert R.rfdd_kernel_launches() == launches and not out.value


def _reverse_rows(c):
    """The same matrix with every row's entries stored in decreasing column order."""
    col, val = c.col.copy(), c.val.copy()
    for i in range(c.n):
        a, b = c.rowptr[i], c.rowptr[i + 1]
        col[a:b] = col[a:b][::-1]
        val[a:b] = val[a:b][::-1]
    return I.Csr(c.n, c.rowptr, col, val)


def test_setup_accepts_symmetric_matrices_with_unsorted_rows(R):
    A, M, part, p = _small()
    try:
        R.rfdd_setup(_reverse_rows(A), _reverse_rows(M), part, p)  # succeeds where a GPU is present
    except R.RfddError as e:
        # without a GPU the call gets past validation and fails at the first CUDA call
        assert e.code not in (R.RFDD_ENOTSYM, R.RFDD_EPARTITION, R.RFDD_ENOTSPD_M, R.RFDD_EINVAL), e


def test_setup_rejects_nonsymmetric_with_unsorted_rows(R):
    A, M, part, p = _small()
    Au = _reverse_rows(A)
    Au.val[Au.rowptr[0]] += 1.0  # row 0's largest column, off the diagonal
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(Au, M, part, p)
    assert e.value.code == R.RFDD_ENOTSYM


def test_setup_rejects_one_sided_entry(R):
    A, M, part, p = _small()
    a = A.to_scipy().tolil()
    a[0, 2] = 0.5  # no (2, 0) partner in the pattern of q1_2d_24 (not a stencil neighbour)
    a = sp.csr_matrix(a)
    assert a[2, 0] == 0
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(a, M, part, p)
    assert e.value.code == R.RFDD_ENOTSYM


def test_entry_points_reject_null_arguments_without_touching_the_device(R):
    lib = ctypes.CDLL(R.LIB_PATH)
    lib.rfdd_polish.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.rfdd_inertia.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    lib.rfdd_profile_busy.argtypes = [ctypes.c_int32, ctypes.c_void_p]
    lib.rfdd_profile_get.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.rfdd_polish(None, 1, None, None, None) == R.RFDD_EINVAL
    assert lib.rfdd_inertia(None, 0.5, None) == R.RFDD_EINVAL
    assert lib.rfdd_profile_busy(1, None) == R.RFDD_EINVAL
    assert lib.rfdd_profile_get(1, None, None, None) == R.RFDD_EINVAL


def test_profile_busy_is_zero_without_records(R):
    assert R.rfdd_profile_busy(0) == 0.0 and R.rfdd_profile_busy(1) == 0.0


def test_polish_wrapper_checks_shapes_before_the_call(R):
    class FakeHandle:
        n = 10
        ptr = None
    with pytest.raises(ValueError):
        R.rfdd_polish(FakeHandle(), np.zeros(3), np.zeros((10, 2)))
    with pytest.raises(ValueError):
        R.rfdd_polish(FakeHandle(), np.zeros(2), np.zeros((9, 2)))


def test_setup_rejects_duplicate_entries(R):
    A, M, part, p = _small()
    rp, col, val = A.rowptr.copy(), A.col.copy(), A.val.copy()
    # row 0 stores its diagonal twice (the value split in halves): same matrix, invalid CSR
    a, b = rp[0], rp[1]
    k = a + int(np.flatnonzero(col[a:b] == 0)[0])
    col2 = np.insert(col, k + 1, 0)
    val2 = np.insert(val, k + 1, 0.5 * val[k])
    val2[k] *= 0.5
    rp2 = rp.copy()
    rp2[1:] += 1
    with pytest.raises(R.RfddError) as e:
        R.rfdd_setup(I.Csr(A.n, rp2, col2, val2), M, part, p)
    assert e.value.code == R.RFDD_EINVAL
