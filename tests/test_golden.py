"""Values the paper prints, stored under tests/golden/ with their citations, against the oracle
and against the library's host-side quadrature (no GPU needed)."""
import os

import numpy as np
import pytest

from oracle import rfdd_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [tuple(float(v) for v in line.split()) for line in f if line.strip() and not line.startswith("#")]


def test_golden_midpoint_filter_endpoints_oracle():
    for nc, x, rho in rows("filter_midpoint_endpoints.txt"):
        z, w = O.quadrature(-1.0, 1.0, int(nc), "midpoint")
        assert abs(O.filter_value([x], z, w)[0] - rho) <= 1e-14


def test_golden_midpoint_filter_endpoints_library():
    from paper_1711_09487_gb300 import build
    build.build()
    import paper_1711_09487_gb300 as R
    R.load()
    for nc, x, rho in rows("filter_midpoint_endpoints.txt"):
        z, w = R.rfdd_quadrature(-1.0, 1.0, int(nc), R.RFDD_MIDPOINT)
        val = 2.0 * np.real(np.sum(np.asarray(w) / (x - np.asarray(z))))
        assert abs(val - rho) <= 1e-14, (nc, x, val)
