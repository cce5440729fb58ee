"""The committed phi fits (phi_poly.h) against the closed form, on the CPU.

The decoding kernels evaluate psi(y) = log2(e) phi(y ln 2) as the larger of
two polynomial pieces; this holds only if each piece stays below the other
outside its own range.  Checked here in float64 with the header's float
coefficients, against phi(x) = ln(1 + 2 / (e^x - 1)).
"""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), os.pardir, "paper_1711_01783_gb300", "csrc", "phi_poly.h")


def _coeffs():
    text = open(HDR).read()
    return {m.group(1): float(m.group(2))
            for m in re.finditer(r"#define (MLD_\w+) \(?([-0-9.e+]+)f?\)?", text)}


@pytest.mark.parametrize("pre,tol", [("2", 2e-7), ("2H", 2.1e-4)])
def test_max_of_pieces_is_psi(pre, tol):
    c = _coeffs()
    s = np.array([c[k] for k in sorted(k for k in c if re.fullmatch(f"MLD_PHI{pre}_S\\d", k))])
    l = np.array([c[k] for k in sorted(k for k in c if re.fullmatch(f"MLD_PHI{pre}_L\\d", k))])
    ln2 = np.log(2.0)
    ymin, ymax = np.log1p(2.0 / np.expm1(25.0)) / ln2, 25.0 / ln2
    y = np.geomspace(ymin, ymax, 300001)
    u = y * y
    small = c["MLD_PHI2_C0"] - u * np.polynomial.polynomial.polyval(u, s) - np.log2(y)
    e = 2.0 ** -y
    large = e * np.polynomial.polynomial.polyval(e * e, l)
    ref = np.log1p(2.0 / np.expm1(y * ln2)) / ln2
    rel = np.abs(np.maximum(small, large) / ref - 1.0)
    assert rel.max() < tol, rel.max()
    # each piece is the larger one only where it is accurate
    y0 = c["MLD_PHI2_Y0"]
    assert np.all(small[y > 1.01 * y0] < large[y > 1.01 * y0])
    assert np.all(large[y < 0.99 * y0] < small[y < 0.99 * y0])
