"""Gaussian-kernel unequally-spaced FFT (USFFT), FP64, plain NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names the operators F_u1D / F_u2D (Section 2, "Fast Fourier
Transform") and defers their construction to the unequally-spaced FFT of
Dutt and Rokhlin.  The construction written out here is the Gaussian
gridding variant derived from Poisson summation:

For f[x], x in [-N/2, N/2) (centred integer coordinates) and a target
frequency xi, we want F(xi) = sum_x f[x] exp(-2 pi i xi x).  With an
oversampled grid of M = R N points and the Gaussian g(s) = exp(-M^2 s^2 /
(4 beta)), whose Fourier transform is
g^(x) = sqrt(4 pi beta) / M * exp(-4 pi^2 beta x^2 / M^2):

1. deapodise    f'[x] = f[x] * exp(4 pi^2 beta x^2 / M^2) / sqrt(4 pi beta)
                (this is f[x] / (M g^(x)));
2. zero-pad     place f'[x] at index x mod M of a length-M buffer;
3. FFT          P[j] = sum_x f'[x] exp(-2 pi i j x / M);
4. gather       F(xi) ~= sum_{t=0}^{2m-1} exp(-(M xi - j_t)^2 / (4 beta)) P[j_t mod M]
                with j0 = floor(M xi + TAP_SHIFT), j_t = j0 - m + 1 + t.

The paper gives no tap rule.  The window is the 2m grid nodes around M xi;
its switch point is moved TAP_SHIFT = 2^-17 grid units below each node so that
points lying on a node up to rounding (whole slice lines do, at angles that are
multiples of pi/2) are not split between two windows by rounding noise: any
implementation that knows M xi to better than ~1e-6 picks the same window.

beta = m R / (4 pi (R - 1/2)) is the Greengard-Lee choice for a kernel of
half-width m at oversampling R.  Type 1 (the adjoint used by L^H) is the exact
transpose: spread with the same weights, unnormalised inverse DFT
(sign +), crop to [-N/2, N/2), deapodise.

Every function here is parameterised by m so that the error can be driven
to ~1e-12 and compared with a direct sum (``nudft1d``).
"""

from __future__ import annotations

import numpy as np


def gaussian_beta(m: int, R: int = 2) -> float:
    """Gaussian width parameter for half-width m at oversampling R."""
    return m * R / (4.0 * np.pi * (R - 0.5))


def deapod(N: int, M: int, beta: float) -> np.ndarray:
    """Deapodisation factors 1/(M g^(x)) for centred x = -N/2 .. N/2-1."""
    x = np.arange(N, dtype=np.float64) - N // 2
    return np.exp(4.0 * np.pi ** 2 * beta * x ** 2 / M ** 2) / np.sqrt(4.0 * np.pi * beta)


def pad_index(N: int, M: int) -> np.ndarray:
    """Buffer index (x mod M) of each centred coordinate x = -N/2 .. N/2-1."""
    return (np.arange(N) - N // 2) % M


TAP_SHIFT = 2.0 ** -17


def taps(t: np.ndarray, m: int, beta: float):
    """Tap indices (unwrapped) and Gaussian weights for grid positions t = M xi.

    Returns (j, w), each of shape t.shape + (2m,)."""
    t = np.asarray(t, dtype=np.float64)
    j0 = np.floor(t + TAP_SHIFT)
    j = j0[..., None] + (np.arange(2 * m) - m + 1)
    w = np.exp(-((t[..., None] - j) ** 2) / (4.0 * beta))
    return j.astype(np.int64), w


# ----------------------------------------------------------------------------
# direct sums (the plain definition the USFFT approximates)
# ----------------------------------------------------------------------------

def nudft1d(f: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """F(xi) = sum_x f[x] exp(-2 pi i xi x), x centred; f along the last axis."""
    N = f.shape[-1]
    x = np.arange(N) - N // 2
    E = np.exp(-2j * np.pi * np.outer(xi, x))          # [K, N]
    return f @ E.T


# ----------------------------------------------------------------------------
# 1D type 2 (equispaced -> nonuniform) and type 1 (its transpose)
# ----------------------------------------------------------------------------

def usfft1d_type2(f: np.ndarray, xi: np.ndarray, m: int = 4, R: int = 2, axis: int = -1) -> np.ndarray:
    """USFFT of f along ``axis`` at the frequencies xi (cycles per sample).

    The output replaces ``axis`` by len(xi)."""
    f = np.moveaxis(np.asarray(f), axis, -1)
    N = f.shape[-1]
    M = R * N
    beta = gaussian_beta(m, R)
    buf = np.zeros(f.shape[:-1] + (M,), dtype=np.complex128)
    buf[..., pad_index(N, M)] = f * deapod(N, M, beta)
    P = np.fft.fft(buf, axis=-1)                       # sign -
    j, w = taps(M * np.asarray(xi, dtype=np.float64), m, beta)   # [K, 2m]
    out = np.einsum("...kt,kt->...k", P[..., j % M], w)
    return np.moveaxis(out, -1, axis)


def usfft1d_type1(c: np.ndarray, xi: np.ndarray, N: int, m: int = 4, R: int = 2, axis: int = -1) -> np.ndarray:
    """Exact transpose (conjugate adjoint) of ``usfft1d_type2``.

    c holds len(xi) values along ``axis``; the output has N there."""
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, -1)
    M = R * N
    beta = gaussian_beta(m, R)
    j, w = taps(M * np.asarray(xi, dtype=np.float64), m, beta)   # [K, 2m]
    # spread: Q[j mod M] += w c   (one library scatter-add per tap column)
    Q = np.zeros(c.shape[:-1] + (M,), dtype=np.complex128)
    for t in range(2 * m):
        np.add.at(Q, (..., j[:, t] % M), c * w[:, t])
    q = np.fft.ifft(Q, axis=-1) * M                    # sign +, unnormalised
    out = q[..., pad_index(N, M)] * deapod(N, M, beta)
    return np.moveaxis(out, -1, axis)


# ----------------------------------------------------------------------------
# 2D type 2 and type 1 (tensor product of the 1D construction)
# ----------------------------------------------------------------------------

def usfft2d_grid(f2: np.ndarray, m: int = 4, R: int = 2) -> np.ndarray:
    """Steps 1-3 in 2D: deapodise, zero-pad and FFT the last two axes."""
    N1, N2 = f2.shape[-2:]
    M1, M2 = R * N1, R * N2
    beta = gaussian_beta(m, R)
    buf = np.zeros(f2.shape[:-2] + (M1, M2), dtype=np.complex128)
    d = np.outer(deapod(N1, M1, beta), deapod(N2, M2, beta))
    buf[..., pad_index(N1, M1)[:, None], pad_index(N2, M2)[None, :]] = f2 * d
    return np.fft.fft2(buf, axes=(-2, -1))


def usfft2d_gather(P: np.ndarray, xi1: np.ndarray, xi2: np.ndarray, m: int = 4, R: int = 2) -> np.ndarray:
    """Step 4 in 2D: separable Gaussian interpolation of the padded FFT P
    (shape [M1, M2]) at the points (xi1, xi2) (any common shape)."""
    M1, M2 = P.shape
    beta = gaussian_beta(m, R)
    j1, w1 = taps(M1 * xi1, m, beta)                   # [..., 2m]
    j2, w2 = taps(M2 * xi2, m, beta)
    vals = P[(j1 % M1)[..., :, None], (j2 % M2)[..., None, :]]   # [..., 2m, 2m]
    return np.einsum("...ab,...a,...b->...", vals, w1, w2)


def usfft2d_type2(f2: np.ndarray, xi1: np.ndarray, xi2: np.ndarray, m: int = 4, R: int = 2) -> np.ndarray:
    """2D USFFT of f2 [N1, N2] at (xi1, xi2): sum f2[x1,x2] exp(-2 pi i (xi1 x1 + xi2 x2))."""
    return usfft2d_gather(usfft2d_grid(f2, m, R), xi1, xi2, m, R)


def usfft2d_type1(c: np.ndarray, xi1: np.ndarray, xi2: np.ndarray, N1: int, N2: int,
                  m: int = 4, R: int = 2) -> np.ndarray:
    """Exact transpose of ``usfft2d_type2``: values c at (xi1, xi2) -> [N1, N2]."""
    M1, M2 = R * N1, R * N2
    beta = gaussian_beta(m, R)
    j1, w1 = taps(M1 * np.asarray(xi1), m, beta)
    j2, w2 = taps(M2 * np.asarray(xi2), m, beta)
    c = np.asarray(c, dtype=np.complex128)
    flat = ((j1 % M1)[..., :, None] * M2 + (j2 % M2)[..., None, :]).reshape(-1)
    val = (c[..., None, None] * w1[..., :, None] * w2[..., None, :]).reshape(-1)
    Q = (np.bincount(flat, weights=val.real, minlength=M1 * M2)
         + 1j * np.bincount(flat, weights=val.imag, minlength=M1 * M2)).reshape(M1, M2)
    q = np.fft.ifft2(Q) * (M1 * M2)                    # sign +, unnormalised
    d = np.outer(deapod(N1, M1, beta), deapod(N2, M2, beta))
    return q[pad_index(N1, M1)[:, None], pad_index(N2, M2)[None, :]] * d
