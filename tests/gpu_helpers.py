"""Shared helpers for the GPU parity tests (oracle on the CPU, CUDA path via the C ABI)."""
from __future__ import annotations

import numpy as np
import torch

from oracle import lamino as olam
from paper_2511_01893_b300 import inputs
from paper_2511_01893_b300 import lamino as glam

# Tolerances (relative L2 against the FP64 oracle).  FP32: 1e-5 per operator
# application, 1e-4 on the volume after ADMM iterations.  FP64: rounding only.
TOL_F32_OP = 1e-5
TOL_F32_ADMM = 1e-4
TOL_F64_OP = 1e-12


def rel(a, b) -> float:
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    b = b.detach().cpu().numpy() if isinstance(b, torch.Tensor) else np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_geom(n, nz, h, w, theta, phi, m=4):
    return olam.Geometry(n1=n, n0=nz, n2=n, h=h, w=w, theta=np.asarray(theta), phi=phi, m=m)


def plan_and_geom(n, nz, h, w, T, phi, prec, m=4, theta=None):
    theta = inputs.angles(T) if theta is None else np.asarray(theta)
    return glam.Plan(n, nz, h, w, theta, phi, m=m, prec=prec), oracle_geom(n, nz, h, w, theta, phi, m)


def rand_vol(n, nz, seed):
    return np.random.default_rng(seed).standard_normal((n, nz, n))


def rand_data(T, h, w, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((T, h, w)) + 1j * rng.standard_normal((T, h, w))


def tol(prec):
    return TOL_F32_OP if prec == "f32" else TOL_F64_OP
