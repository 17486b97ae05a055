"""Seeded synthetic inputs for laminography reconstruction.

This module holds none of the method's arithmetic: it draws phantoms, angles
and noise only.  Both the CUDA path's tests/benchmarks and the FP64 oracle
use it, so the two see identical inputs.

The paper reconstructs real laminography scans (a mouse brain and other
samples at 1K^3 .. 2K^3, Section 6.1) that are not available here; these
generators stand in for them:

* ``ellipsoid_phantom``: additive random ellipsoids (centres within radius
  0.35 n laterally and |z| < 0.3 nz, semi-axes U(0.05, 0.25) n (x, y) and
  U(0.05, 0.25) nz (z), rotation from three uniform Euler angles, density
  U(0.1, 1)), evaluated at voxel centres.
* ``circuit_phantom``: a thin-layer integrated-circuit-like pattern (the IC
  use case the paper's introduction names): 4 layers of thickness 3 voxels,
  each with 40 axis-aligned traces of width 2-6 voxels and 20 vias (radius 2
  cylinders joining adjacent layers), density 1.
* ``angles``: n_theta rotation angles uniform on [0, 2 pi).
* ``noise``: seeded standard-normal array; the caller scales it to
  sigma = 1 % of max |Re L u|.

Arrays are float64 torch tensors laid out u[x, z, y] (n1, n0, n2), on any
torch device (GPU evaluation keeps the 1024^3 phantom fast).
"""

from __future__ import annotations

import math

import numpy as np
import torch


def angles(n_theta: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(n_theta, dtype=np.float64) / n_theta


def _euler(a: float, b: float, c: float) -> np.ndarray:
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    rz1 = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    rz2 = np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1]])
    return rz1 @ ry @ rz2


def ellipsoid_params(n: int, nz: int, count: int, seed: int):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        rad = 0.35 * n * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        c = np.array([rad * math.cos(ang), rad * math.sin(ang), rng.uniform(-0.3, 0.3) * nz])
        ax = np.array([rng.uniform(0.05, 0.25) * n, rng.uniform(0.05, 0.25) * n,
                       rng.uniform(0.05, 0.25) * nz])
        R = _euler(*rng.uniform(0, 2 * np.pi, 3))
        rho = rng.uniform(0.1, 1.0)
        out.append((c, ax, R, rho))
    return out


def _coords(n: int, nz: int, device, dtype):
    x = torch.arange(n, device=device, dtype=dtype) - n // 2
    z = torch.arange(nz, device=device, dtype=dtype) - nz // 2
    return x, z


def ellipsoid_phantom(n: int, nz: int, count: int = 12, seed: int = 1234,
                      device="cpu", dtype=torch.float64, chunk: int = 64) -> torch.Tensor:
    """u[x, z, y] = sum of ellipsoid densities at the voxel centres."""
    params = ellipsoid_params(n, nz, count, seed)
    x, z = _coords(n, nz, device, dtype)
    y = x
    u = torch.zeros((n, nz, n), device=device, dtype=dtype)
    for x0 in range(0, n, chunk):
        xs = x[x0:x0 + chunk][:, None, None]
        zs = z[None, :, None]
        ys = y[None, None, :]
        acc = torch.zeros((xs.shape[0], nz, n), device=device, dtype=dtype)
        for c, ax, R, rho in params:
            # body coordinates q = R^T (r - c); inside if sum (q_k / a_k)^2 <= 1
            dx, dy, dz = xs - c[0], ys - c[1], zs - c[2]
            s = 0
            for k in range(3):
                qk = R[0, k] * dx + R[1, k] * dy + R[2, k] * dz
                s = s + (qk / ax[k]) ** 2
            acc += rho * (s <= 1.0).to(dtype)
        u[x0:x0 + chunk] = acc
    return u


def circuit_phantom(n: int, nz: int, seed: int = 1238, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Binary thin-layer circuit mask (1 inside traces and vias), u[x, z, y]."""
    rng = np.random.default_rng(seed)
    mask = torch.zeros((n, nz, n), device=device, dtype=torch.bool)
    layers = [int(round(nz / 2 + f * nz)) for f in (-0.2, -0.07, 0.07, 0.2)]
    lo, hi = int(0.15 * n), int(0.85 * n)
    for zc in layers:
        z0, z1 = max(zc - 1, 0), min(zc + 2, nz)
        for _ in range(40):
            width = int(rng.integers(2, 7))
            length = int(rng.uniform(0.1, 0.5) * n)
            a = int(rng.integers(lo, max(lo + 1, hi - length)))
            b = int(rng.integers(lo, hi - width))
            if rng.uniform() < 0.5:
                mask[a:a + length, z0:z1, b:b + width] = True
            else:
                mask[b:b + width, z0:z1, a:a + length] = True
    r = torch.arange(n, device=device, dtype=dtype)
    for i in range(len(layers) - 1):
        for _ in range(20):
            cx, cy = rng.uniform(lo, hi, 2)
            disk = ((r[:, None] - cx) ** 2 + (r[None, :] - cy) ** 2) <= 4.0
            mask[:, layers[i]:layers[i + 1] + 1, :] |= disk[:, None, :]
    return mask.to(dtype)


def ellipsoid_circuit_phantom(n: int, nz: int, seed: int = 1238, device="cpu",
                              dtype=torch.float64) -> torch.Tensor:
    u = ellipsoid_phantom(n, nz, 12, seed, device, dtype)
    c = circuit_phantom(n, nz, seed + 1, device, dtype)
    return torch.where(c > 0, torch.ones_like(u), u)


def noise(shape, seed: int, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Standard-normal array drawn with a seeded torch generator on the CPU."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(shape, generator=gen, dtype=torch.float32).to(device=device, dtype=dtype)


def gaussian_blob(n: int, nz: int, centre, sigma: float, dtype=torch.float64) -> torch.Tensor:
    """exp(-|r - c|^2 / (2 sigma^2)) at centred voxel coordinates, u[x, z, y]."""
    x, z = _coords(n, nz, "cpu", dtype)
    cx, cy, cz = centre
    return torch.exp(-((x[:, None, None] - cx) ** 2 + (x[None, None, :] - cy) ** 2
                       + (z[None, :, None] - cz) ** 2) / (2 * sigma * sigma))
