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


SURR = pathlib.Path(__file__).resolve().parents[1] / "paper_2211_12616_gb300" / "csrc" / "surrogate.cu"
PHI_T = 4.5


def _phi_coefficients(start, stop):
    src = SURR.read_text()
    body = src[src.index(start):]
    body = body[:body.index(stop)]
    nums = [float(m) for m in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return nums[::-1]          # Horner order in the source: z^12 first; returned as c0 .. c12


def test_gelu_phi_polynomial_against_erf():
    """The GELU of the surrogate kernels forms Phi(x) = 1/2 + x P(x^2 / 10.125 - 1) for |x| <= 4.5
    with a fitted P of degree 12: its error against Phi = (1 + erf(x / sqrt 2)) / 2, exactly and
    evaluated in float32 as the kernels do, and beyond the clamp."""
    from scipy.special import erf
    c = _phi_coefficients("float phi_poly(float x)", "__device__ __forceinline__ float gelu(float x)")
    assert len(c) == 13
    assert c == _phi_coefficients("f2_t gelu2(f2_t x)", "// ---")   # the packed form: same constants
    x = np.linspace(-PHI_T, PHI_T, 400_001)
    phi = 0.5 * (1 + erf(x / np.sqrt(2)))
    z = x * x * (2 / PHI_T ** 2) - 1
    exact = 0.5 + x * sum(ck * z ** k for k, ck in enumerate(c))
    assert np.abs(exact - phi).max() < 4.5e-8     # the fit, coefficients rounded to float32
    xf = x.astype(np.float32)
    zf = (xf.astype(np.float64) * (xf * np.float32(2 / PHI_T ** 2)).astype(np.float64) - 1).astype(np.float32)
    q = np.float32(c[-1])
    for ck in reversed(c[:-1]):
        q = (q.astype(np.float64) * zf + np.float32(ck)).astype(np.float32)
    pf = (xf.astype(np.float64) * q + 0.5).astype(np.float32)
    assert np.abs(pf - phi).max() < 1.1e-7
    # GELU relative error where a bf16 rounding flip could show (|gelu| > 0.04): a few 1e-6
    g = (xf.astype(np.float64) * pf).astype(np.float32)
    big = np.abs(x * phi) > 0.04
    assert (np.abs(g - x * phi)[big] / np.abs(x * phi)[big]).max() < 3e-6
    # beyond the clamp Phi is within 3.4e-6 of 0 or 1
    assert 0.5 * (1 + erf(-PHI_T / np.sqrt(2))) < 3.4e-6
