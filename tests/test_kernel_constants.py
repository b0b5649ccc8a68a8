"""Constants written into the CUDA kernels, checked against the mathematics (no GPU).

The fused step forms cos(lat) as the sine of the colatitude with a fitted odd
polynomial of degree 9 (csrc/step.cu, sin_poly).  Its coefficients are read from
the source and checked here against numpy's sine, in float64 and evaluated in
float32 as the kernel does.
"""
import pathlib
import re

import numpy as np

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2211_12616_gb300" / "csrc" / "step.cu"


def _sin_poly_coefficients():
    src = SRC.read_text()
    body = src[src.index("float sin_poly(float x)"):]
    body = body[:body.index("return x * q;")]
    nums = [float(m) for m in re.findall(r"([-+]?\d\.\d+e[-+]\d+|1\.0)f", body)]
    # Horner order: highest coefficient first
    return nums[::-1]


def test_sin_poly_relative_error():
    c = _sin_poly_coefficients()
    assert len(c) == 5 and c[0] == 1.0
    x = np.linspace(1e-7, np.pi / 2, 400_001)
    q = sum(ck * x ** (2 * k) for k, ck in enumerate(c))
    rel = np.abs(x * q - np.sin(x)) / np.sin(x)
    assert rel.max() < 1.5e-8        # the fit, coefficients rounded to float32
    # evaluated in float32 as in the kernel (Horner, fused multiply-adds rounded once)
    xf = x.astype(np.float32)
    x2 = (xf * xf).astype(np.float32)
    qf = np.float32(c[-1])
    for ck in reversed(c[:-1]):
        qf = (qf.astype(np.float64) * x2 + ck).astype(np.float32)
    vf = (xf * qf).astype(np.float64)
    ref = np.sin(xf.astype(np.float64))
    assert (np.abs(vf - ref) / ref).max() < 2e-7


def test_sin_poly_odd_symmetry_and_pole():
    c = _sin_poly_coefficients()
    x = np.array([1e-6, 1.745329e-5, 0.1, 1.0, np.pi / 2])
    v = x * sum(ck * x ** (2 * k) for k, ck in enumerate(c))
    np.testing.assert_allclose(v, np.sin(x), rtol=1e-8)
    np.testing.assert_allclose(-v, (-x) * sum(ck * x ** (2 * k) for k, ck in enumerate(c)))
