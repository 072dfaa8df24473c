"""Pins of the Mie series (textbook closed forms and printed sample values)."""
import os

import numpy as np

from oracle import mie

GOLD = os.path.join(os.path.dirname(__file__), "golden", "mie_bohren_huffman_appendixA.txt")


def _golden():
    vals = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_bohren_huffman_sample_output():
    g = _golden()
    x = 2 * np.pi * 0.525 / 0.6328
    assert abs(x - g["x"]) < 5e-4
    a, b = mie.coefficients_homogeneous(x, 1.55 + 0j)
    qext, qsca = mie.efficiencies(a, b, x)
    S1, S2 = mie.amplitudes(a, b, np.array([np.pi]))
    qback = 4 * abs(S1[0]) ** 2 / x ** 2
    assert abs(qext - g["qext"]) < 1e-4 and abs(qsca - g["qsca"]) < 1e-4 and abs(qback - g["qback"]) < 1e-4


def test_rayleigh_limit():
    x, m = 0.01, np.sqrt(4.0 + 0j)
    a, b = mie.coefficients_homogeneous(x, m)
    _, qsca = mie.efficiencies(a, b, x)
    ray = 8.0 / 3.0 * x ** 4 * abs((m * m - 1) / (m * m + 2)) ** 2
    assert abs(qsca / ray - 1) < 1e-3


def test_optical_theorem_and_lossless():
    for eps in (4.0, 4.0 - 0.1j, -2.2319 - 0.1616j):
        m = mie.refractive_index(eps)
        x = 2 * np.pi * 0.5
        a, b = mie.coefficients_homogeneous(x, m)
        qext, qsca = mie.efficiencies(a, b, x)
        S1, S2 = mie.amplitudes(a, b, np.array([0.0]))
        assert abs(S1[0] - S2[0]) < 1e-12 * abs(S1[0])
        assert abs(4 / x ** 2 * S1[0].real - qext) < 1e-10
        if np.imag(eps) == 0:
            assert abs(qext - qsca) < 1e-10
        else:
            assert qext > qsca


def test_coated_reduces_to_homogeneous():
    x = 4.0
    m = 1.8 + 0.05j
    a1, b1 = mie.coefficients_coated(0.6 * x, x, m, m)
    a2, b2 = mie.coefficients_homogeneous(x, m)
    assert np.abs(a1 - a2).max() < 1e-10 and np.abs(b1 - b2).max() < 1e-10
    # vacuum core of vanishing size -> homogeneous sphere of the shell index
    a3, b3 = mie.coefficients_coated(1e-4, x, 1.0 + 0j, m)
    assert np.abs(a3 - a2).max() < 1e-8 and np.abs(b3 - b2).max() < 1e-8


def test_multilayer_reduces_to_homogeneous_and_coated():
    """Equal layers give the homogeneous sphere; two layers give the Aden-Kerker coated sphere
    (an independent formula); a vacuum core gives the shell."""
    m = mie.refractive_index(4.0 - 0.3j)
    a0, b0 = mie.coefficients_homogeneous(3.0, m)
    a1, b1 = mie.coefficients_multilayer([1.0, 2.2, 3.0], [m, m, m], nmax=len(a0))
    assert np.allclose(a1, a0, rtol=1e-9, atol=1e-13) and np.allclose(b1, b0, rtol=1e-9, atol=1e-13)
    for m1, m2 in ((mie.refractive_index(6.0), mie.refractive_index(2.0 - 0.1j)),
                   (1.0 + 0j, mie.refractive_index(-2.2 - 0.16j)),
                   (mie.refractive_index(2.0), mie.refractive_index(5.0))):
        a0, b0 = mie.coefficients_coated(1.4, 2.5, m1, m2)
        a1, b1 = mie.coefficients_multilayer([1.4, 2.5], [m1, m2], nmax=len(a0))
        assert np.allclose(a1, a0, rtol=1e-8, atol=1e-12) and np.allclose(b1, b0, rtol=1e-8, atol=1e-12)


def test_multilayer_lossless_optical_theorem():
    """Five lossless layers (eps 6 .. 2 from the centre out): Q_ext = Q_sca."""
    xs = 2 * np.pi * np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    ms = [mie.refractive_index(e) for e in (6.0, 5.0, 4.0, 3.0, 2.0)]
    a, b = mie.coefficients_multilayer(xs, ms)
    qext, qsca = mie.efficiencies(a, b, xs[-1])
    assert abs(qext - qsca) < 1e-10 * qext
