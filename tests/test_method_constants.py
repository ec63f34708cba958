"""The SDIRK3 tableau compiled into both stiff kernels (no GPU): the constants are read from the
CUDA sources as text and checked against what the method requires (Alexander's L-stable,
stiffly accurate three-stage DIRK of order 3, with an embedded order-2 solution), so that a wrong
digit or a swapped weight fails here before any GPU run."""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2510_23993_gb300", "csrc")
SOURCES = ["stiff_body.cuh", "large.cu"]
NAMES = ["kG", "kB1", "kB2", "kBh1", "kBh2"]


def _constants(fname):
    text = open(os.path.join(CSRC, fname)).read()
    out = {}
    for name in NAMES:
        m = re.search(r"constexpr double " + name + r" = ([-+0-9.eE]+);", text)
        assert m, (fname, name)
        out[name] = float(m.group(1))
    return out


def _tableau(k):
    g = k["kG"]
    c = np.array([g, 0.5 * (1.0 + g), 1.0])
    A = np.array([[g, 0.0, 0.0], [0.5 * (1.0 - g), g, 0.0], [k["kB1"], k["kB2"], g]])
    b = A[2].copy()                      # stiffly accurate: the last stage is the solution
    bh = np.array([k["kBh1"], k["kBh2"], 0.0])
    return A, b, c, bh


@pytest.mark.parametrize("fname", SOURCES)
def test_order_conditions(fname):
    A, b, c, bh = _tableau(_constants(fname))
    assert np.allclose(A.sum(axis=1), c, rtol=0, atol=1e-15)       # row sums are the nodes
    tol = 1e-14
    assert abs(b.sum() - 1.0) < tol                                  # order 1
    assert abs(b @ c - 0.5) < tol                                    # order 2
    assert abs(b @ c**2 - 1.0 / 3.0) < tol                           # order 3, bushy tree
    assert abs(b @ A @ c - 1.0 / 6.0) < tol                          # order 3, tall tree
    # the embedded solution has order 2 and not 3, so b - bh estimates the local error
    assert abs(bh.sum() - 1.0) < tol and abs(bh @ c - 0.5) < tol
    assert abs(bh @ c**2 - 1.0 / 3.0) > 1e-3


@pytest.mark.parametrize("fname", SOURCES)
def test_gamma_is_the_l_stable_root(fname):
    g = _constants(fname)["kG"]
    # with c = (g, (1+g)/2, 1) and a stiffly accurate last row, order 3 fixes g as a root of
    # 6 g^3 - 18 g^2 + 9 g - 1 = 0; the one in (1/3, 1/2) is the one that gives L-stability
    roots = np.roots([6.0, -18.0, 9.0, -1.0])
    real = sorted(r.real for r in roots if abs(r.imag) < 1e-12)
    inside = [r for r in real if 1.0 / 3.0 < r < 0.5]
    assert len(inside) == 1 and abs(inside[0] - g) < 1e-15


@pytest.mark.parametrize("fname", SOURCES)
def test_stability_function(fname):
    A, b, _, _ = _tableau(_constants(fname))
    one = np.ones(3)

    def R(z):
        return 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, one)

    # A-stable: |R| <= 1 on the imaginary axis (the poles 1/g lie in the right half-plane)
    for y in np.concatenate([-np.logspace(-3, 4, 200), np.logspace(-3, 4, 200)]):
        assert abs(R(1j * y)) <= 1.0 + 1e-12
    # L-stable: R vanishes at infinity (stiffly accurate with an invertible A)
    assert abs(R(-1e12)) < 1e-9
    # order 3: R(z) matches exp(z) to O(z^4) near 0
    for z in (1e-2, -1e-2, 1e-2j):
        assert abs(R(z) - np.exp(z)) < 5 * abs(z) ** 4


def test_both_kernels_use_the_same_tableau():
    assert _constants(SOURCES[0]) == _constants(SOURCES[1])
