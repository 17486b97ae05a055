"""Pins for the oracle's Gaussian USFFT against direct nonuniform DFT sums.

The USFFT is an approximation of F(xi) = sum_x f[x] exp(-2 pi i xi x); its
error must fall as the kernel half-width m grows and reach rounding level
at m = 12.  The adjoint (type 1) must be the exact transpose.
"""
import numpy as np
import pytest

from oracle import usfft


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_1d_type2_error_decays_with_m():
    rng = np.random.default_rng(0)
    f = _rand_c(rng, 64)
    xi = rng.uniform(-0.7, 0.7, 200)            # includes |xi| > 1/2 (wrapped taps)
    exact = usfft.nudft1d(f, xi)
    errs = [_rel(usfft.usfft1d_type2(f, xi, m), exact) for m in (2, 4, 6, 8, 12)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[1] < 1e-4          # m = 4
    assert errs[-1] < 1e-11        # m = 12


def test_1d_direct_sum_is_a_plain_dft_on_the_grid():
    # independent check of nudft1d itself: at xi = k/N it is numpy's DFT of the
    # centred sequence
    rng = np.random.default_rng(1)
    N = 32
    f = _rand_c(rng, N)
    k = np.arange(N)
    ref = np.fft.fft(f) * np.exp(2j * np.pi * k * (N // 2) / N)
    assert _rel(usfft.nudft1d(f, k / N), ref) < 1e-13


@pytest.mark.parametrize("shape", [(16, 12), (8, 20)])
def test_2d_type2_matches_direct_sum(shape):
    rng = np.random.default_rng(2)
    f2 = _rand_c(rng, *shape)
    x1 = rng.uniform(-0.7, 0.7, 60)
    x2 = rng.uniform(-0.7, 0.7, 60)
    a = np.arange(shape[0]) - shape[0] // 2
    b = np.arange(shape[1]) - shape[1] // 2
    exact = np.array([np.sum(f2 * np.exp(-2j * np.pi * (p * a[:, None] + q * b[None, :])))
                      for p, q in zip(x1, x2)])
    assert _rel(usfft.usfft2d_type2(f2, x1, x2, 4), exact) < 2.5e-4
    assert _rel(usfft.usfft2d_type2(f2, x1, x2, 12), exact) < 1e-10


def test_type1_is_exact_transpose_1d():
    rng = np.random.default_rng(3)
    N = 48
    f = _rand_c(rng, 5, N)
    xi = rng.uniform(-0.6, 0.6, 70)
    c = _rand_c(rng, 5, 70)
    lhs = np.vdot(usfft.usfft1d_type2(f, xi, 4), c)
    rhs = np.vdot(f, usfft.usfft1d_type1(c, xi, N, 4))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_type1_is_exact_transpose_2d():
    rng = np.random.default_rng(4)
    f2 = _rand_c(rng, 16, 12)
    x1 = rng.uniform(-0.7, 0.7, (7, 9))
    x2 = rng.uniform(-0.7, 0.7, (7, 9))
    c = _rand_c(rng, 7, 9)
    lhs = np.vdot(usfft.usfft2d_type2(f2, x1, x2), c)
    rhs = np.vdot(f2, usfft.usfft2d_type1(c, x1, x2, 16, 12))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_type1_matches_direct_adjoint_sum():
    # the transpose of the exact transform is sum_k c_k exp(+2 pi i xi_k x)
    rng = np.random.default_rng(5)
    N = 32
    xi = rng.uniform(-0.5, 0.5, 40)
    c = _rand_c(rng, 40)
    x = np.arange(N) - N // 2
    exact = np.exp(2j * np.pi * np.outer(x, xi)) @ c
    assert _rel(usfft.usfft1d_type1(c, xi, N, 12), exact) < 1e-10
