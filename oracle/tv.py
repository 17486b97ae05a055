"""Total-variation pieces of ADMM-TV, FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper writes the regulariser as alpha ||u||_TV (Eq. 1) and uses a
gradient operator (the nabla of Algorithms 1 and 2) without giving its
discretisation.  Readings taken here:

* grad: forward differences along each axis of u[n1, n0, n2] (component 0
  along x = axis 0, 1 along z = axis 1, 2 along y = axis 2) with a zero
  difference at the last index (Neumann boundary).  Output [3, n1, n0, n2].
* div = -grad^T, the exact negative transpose (a backward difference with
  matching ends), so <grad u, p> = -<u, div p>.
* TV(u) = sum over voxels of the Euclidean norm of the 3-vector grad u.
* shrink_iso(z, k) = max(0, 1 - k / |z|) z per voxel (|z| the 3-vector
  norm, 0 maps to 0): the proximal map of k * sum |z|.
"""

from __future__ import annotations

import numpy as np


def grad(u: np.ndarray) -> np.ndarray:
    g = np.zeros((3,) + u.shape, dtype=u.dtype)
    for a in range(3):
        d = np.diff(u, axis=a)                        # u[i+1] - u[i], length N-1
        sl = [slice(None)] * 3
        sl[a] = slice(0, u.shape[a] - 1)
        g[(a,) + tuple(sl)] = d
    return g


def div(p: np.ndarray) -> np.ndarray:
    """-grad^T p: for each axis, p[i] (i <= N-2) minus p[i-1] (i >= 1)."""
    out = np.zeros(p.shape[1:], dtype=p.dtype)
    for a in range(3):
        N = p.shape[1 + a]
        pa = p[a]
        head = [slice(None)] * 3
        head[a] = slice(0, N - 1)
        out[tuple(head)] += pa[tuple(head)]
        tail_dst = [slice(None)] * 3
        tail_dst[a] = slice(1, N)
        out[tuple(tail_dst)] -= pa[tuple(head)]
    return out


def tv(u: np.ndarray) -> float:
    g = grad(u)
    return float(np.sum(np.sqrt(np.sum(g * g, axis=0))))


def shrink_iso(z: np.ndarray, k: float) -> np.ndarray:
    mag = np.sqrt(np.sum(z * z, axis=0))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(mag > 0, np.maximum(0.0, 1.0 - k / np.where(mag > 0, mag, 1.0)), 0.0)
    return z * f
