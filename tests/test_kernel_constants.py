"""Host-side checks of the constants the FP32 kernels hard-code (no GPU needed).

The coefficients are read out of the CUDA header/source text and evaluated
here in float32 the way the kernels evaluate them (Horner with FMA-free
float32 steps, which bounds the FMA form from above).
"""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2104_08309_gb300", "csrc")


def _body(path, name):
    text = open(os.path.join(CSRC, path)).read()
    i = text.index(name)
    return text[i:text.index("\n}\n", i)]


def _floats(body):
    return [float(x) for x in re.findall(r"[-+]?\d\.\d+e[-+]\d+", body)]


def test_sinc_polynomial_accuracy():
    """sinc(u) on |u| <= pi from the degree-6 polynomial in u^2."""
    c = _floats(_body("pft_common.cuh", "float sinc_poly("))
    assert len(c) == 6
    # Horner order in the source: c6, c5, then c4..c1, constant 1
    coef = np.array([1.0] + c[::-1], dtype=np.float32)     # c0..c6
    u = np.linspace(0.0, math.pi, 200001)
    v = (u * u).astype(np.float32)
    acc = np.full_like(v, coef[-1])
    for ck in coef[-2::-1]:
        acc = (acc * v + ck).astype(np.float32)
    ref = np.sinc(u / math.pi)
    assert np.max(np.abs(acc - ref)) < 3e-7


def test_face_series_coefficients_are_inverse_factorials():
    """G = sum_k i^k h_k/(k+2)!: the constants are +-1/(k+2)! and their combinations."""
    c = _floats(_body("pft_pairs.cuh", "void face_series("))
    f = math.factorial
    expected = [1 / f(10), -1 / f(8), 1 / f(6), -1 / f(4),           # Horner in P for the real part
                3 / f(10), -1 / f(8),                                  # T^2 terms
                -1 / 120960, 1 / 2520, -1 / f(5)]                      # imaginary part: -T/5! + PT/2520 - P^2T/120960
    assert len(c) == len(expected)
    for got, want in zip(c, expected):
        assert abs(got - want) <= 1e-6 * abs(want)
    # 2520 = 7!/2 (coefficient 2/7! of P T) and 120960 = 9!/3 (coefficient 3/9! of P^2 T)
    assert f(7) // 2 == 2520 and f(9) // 3 == 120960


def test_long_face_series_coefficients():
    """Long form: A(P) = sum (-1)^j P^j/(2j+2)!, B, D, E from h_9..h_12 (see the kernel comment)."""
    c = _floats(_body("pft_pairs.cuh", "void face_series_long("))
    f = math.factorial
    expected = [1 / f(14), -1 / f(12), 1 / f(10), -1 / f(8), 1 / f(6), -1 / f(4),   # A
                10 / f(14), -6 / f(12), 3 / f(10), -1 / f(8),                       # B (h8, h10, h12 T^2 terms)
                1 / f(14),                                                          # T^4 / 14!
                -5 / f(13), 4 / f(11), -3 / f(9), 2 / f(7), -1 / f(5),              # D
                -4 / f(13), 1 / f(11)]                                              # E
    assert len(c) == len(expected)
    for got, want in zip(c, expected):
        assert abs(got - want) <= 1e-6 * abs(want)
