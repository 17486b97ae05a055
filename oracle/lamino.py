"""Laminographic forward operator L, its adjoint, and the exact projection.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Shapes follow Section 2 of the paper: u[n1, n0, n2] (x, z, y; z = n0 is the
rotation axis), u1[n1, h, n2] after F_u1D, u2[n_theta, h, w] after F_u2D,
d[n_theta, h, w] after F*_2D.

Geometry (the paper does not print it; this is the reading used throughout).
Centred coordinates: voxel r = (ix - n1/2, iy - n2/2, iz - n0/2); detector
s = iu - w/2, t = iv - h/2; frequencies ku in [-w/2, w/2), kv in [-h/2, h/2).
The detector plane of angle theta at tilt phi is spanned by

    e_u = (cos th, sin th, 0),   e_v = (sin ph sin th, -sin ph cos th, cos ph),

so phi is the beam's elevation out of the sample (x, y) plane and phi = 0 is
ordinary tomography about z.  The Fourier slice of angle theta holds

    xi(theta, kv, ku) = (ku / w) e_u + (kv / h) e_v,

and xi_z = (kv / h) cos phi does not depend on theta, which is what lets L
factor into a 1D transform along n0 -> h followed by one 2D transform per kv
plane (F_u1D then F_u2D).  The band-limited projection is

    (L u)[theta, iv, iu] = 1/(h w) sum_{kv, ku} u^(xi) exp(+2 pi i (ku s / w + kv t / h)),
    u^(xi) = sum_r u(r) exp(-2 pi i xi . r).

L-hat (``lhat``) is L without the last step (the frequency-domain form that
Algorithm 2 works in).  u is real; L u is complex-valued and is not
truncated to its real part.  Adjoints are taken under Re <a, b>; for a real
u the adjoint of L is Re(L^H .).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import usfft


@dataclass(frozen=True)
class Geometry:
    n1: int            # x
    n0: int            # z (rotation axis)
    n2: int            # y
    h: int             # detector rows (v)
    w: int             # detector columns (u)
    theta: np.ndarray  # [n_theta] rotation angles, rad
    phi: float         # tilt, rad
    m: int = 4         # Gaussian half-width
    R: int = 2         # oversampling

    @property
    def n_theta(self) -> int:
        return len(self.theta)


def centred(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) - n // 2


def _xi(th, kv, ku, phi):
    """xi = ku e_u + kv e_v for kv, ku already divided by h, w (broadcasting)."""
    sp, cp = np.sin(phi), np.cos(phi)
    xi_x = ku * np.cos(th) + kv * sp * np.sin(th)
    xi_y = ku * np.sin(th) - kv * sp * np.cos(th)
    xi_z = kv * cp
    return xi_x, xi_y, xi_z


def slice_frequencies(g: Geometry):
    """(xi_x, xi_y) of shape [n_theta, h, w] and xi_z of shape [h]."""
    th = np.asarray(g.theta, dtype=np.float64)[:, None, None]
    kv = centred(g.h)[None, :, None] / g.h
    ku = centred(g.w)[None, None, :] / g.w
    xi_x, xi_y, _ = _xi(th, kv, ku, g.phi)
    _, _, xi_z = _xi(0.0, centred(g.h) / g.h, 0.0, g.phi)
    return xi_x, xi_y, xi_z


def slice_frequency_points(g: Geometry, t, kv, ku):
    """(xi_x, xi_y, xi_z) of the slice points (theta index t, row kv in [0, h),
    column ku in [0, w)), given as equal-length index arrays."""
    th = np.asarray(g.theta, dtype=np.float64)[np.asarray(t)]
    kvr = (np.asarray(kv, dtype=np.float64) - g.h // 2) / g.h
    kur = (np.asarray(ku, dtype=np.float64) - g.w // 2) / g.w
    return _xi(th, kvr, kur, g.phi)


# ----------------------------------------------------------------------------
# the three stages and their transposes
# ----------------------------------------------------------------------------

def f_u1d(u: np.ndarray, g: Geometry) -> np.ndarray:
    """F_u1D: u[n1, n0, n2] -> u1[n1, h, n2], USFFT along z at xi_z."""
    _, _, xi_z = slice_frequencies(g)
    return usfft.usfft1d_type2(u, xi_z, g.m, g.R, axis=1)


def f_u1d_adj(u1: np.ndarray, g: Geometry) -> np.ndarray:
    """F*_u1D: transpose of f_u1d, u1[n1, h, n2] -> complex [n1, n0, n2]."""
    _, _, xi_z = slice_frequencies(g)
    return usfft.usfft1d_type1(u1, xi_z, g.n0, g.m, g.R, axis=1)


def f_u2d(u1: np.ndarray, g: Geometry) -> np.ndarray:
    """F_u2D: u1[n1, h, n2] -> u2[n_theta, h, w], one 2D USFFT per kv plane."""
    xi_x, xi_y, _ = slice_frequencies(g)
    out = np.empty((g.n_theta, g.h, g.w), dtype=np.complex128)
    for kv in range(g.h):
        P = usfft.usfft2d_grid(u1[:, kv, :], g.m, g.R)
        out[:, kv, :] = usfft.usfft2d_gather(P, xi_x[:, kv, :], xi_y[:, kv, :], g.m, g.R)
    return out


def f_u2d_adj(u2: np.ndarray, g: Geometry) -> np.ndarray:
    """F*_u2D: transpose of f_u2d, u2[n_theta, h, w] -> u1[n1, h, n2]."""
    xi_x, xi_y, _ = slice_frequencies(g)
    out = np.empty((g.n1, g.h, g.n2), dtype=np.complex128)
    for kv in range(g.h):
        out[:, kv, :] = usfft.usfft2d_type1(u2[:, kv, :], xi_x[:, kv, :], xi_y[:, kv, :],
                                            g.n1, g.n2, g.m, g.R)
    return out


def _centred_dft_matrix(n: int, sign: int) -> np.ndarray:
    k = centred(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


def f_2d_inv(u2: np.ndarray) -> np.ndarray:
    """F*_2D: d[th, iv, iu] = 1/(h w) sum_{kv,ku} u2 exp(+2 pi i (ku s/w + kv t/h))."""
    _, h, w = u2.shape
    Eh = _centred_dft_matrix(h, +1)
    Ew = _centred_dft_matrix(w, +1)
    return Eh @ u2 @ Ew.T / (h * w)


def f_2d(d: np.ndarray) -> np.ndarray:
    """F_2D: the unnormalised centred forward DFT, exact inverse of f_2d_inv."""
    _, h, w = d.shape
    Eh = _centred_dft_matrix(h, -1)
    Ew = _centred_dft_matrix(w, -1)
    return Eh @ d @ Ew.T


def f_2d_inv_adj(d: np.ndarray) -> np.ndarray:
    """Transpose of F*_2D, i.e. F_2D / (h w)."""
    _, h, w = d.shape
    return f_2d(d) / (h * w)


# ----------------------------------------------------------------------------
# L-hat, L and adjoints
# ----------------------------------------------------------------------------

def lhat(u: np.ndarray, g: Geometry) -> np.ndarray:
    """L-hat u = F_u2D F_u1D u (Algorithm 2, forward pass)."""
    return f_u2d(f_u1d(u, g), g)


def lhat_adj(r: np.ndarray, g: Geometry, real: bool = True) -> np.ndarray:
    """L-hat^H r = F*_u1D F*_u2D r (Algorithm 2, adjoint pass); Re for a real u."""
    v = f_u1d_adj(f_u2d_adj(r, g), g)
    return v.real if real else v


def lam_forward(u: np.ndarray, g: Geometry) -> np.ndarray:
    """L u = F*_2D F_u2D F_u1D u (Algorithm 1, forward pass)."""
    return f_2d_inv(lhat(u, g))


def lam_adjoint(d: np.ndarray, g: Geometry, real: bool = True) -> np.ndarray:
    """L^H d = F*_u1D F*_u2D (F_2D d / (h w)); Re for a real u."""
    return lhat_adj(f_2d_inv_adj(d), g, real)


# ----------------------------------------------------------------------------
# exact (direct-sum) versions: the definition the USFFT approximates
# ----------------------------------------------------------------------------

def lhat_exact(u: np.ndarray, g: Geometry) -> np.ndarray:
    """u^(xi) by direct summation over all voxels at every slice frequency."""
    xi_x, xi_y, xi_z = slice_frequencies(g)
    rx = centred(g.n1)
    rz = centred(g.n0)
    ry = centred(g.n2)
    out = np.empty((g.n_theta, g.h, g.w), dtype=np.complex128)
    for kv in range(g.h):
        ex = np.exp(-2j * np.pi * xi_x[:, kv, :, None] * rx)          # [T, w, n1]
        ey = np.exp(-2j * np.pi * xi_y[:, kv, :, None] * ry)          # [T, w, n2]
        ez = np.exp(-2j * np.pi * xi_z[kv] * rz)                      # [n0]
        uz = np.tensordot(u, ez, axes=([1], [0]))                    # [n1, n2]
        out[:, kv, :] = np.einsum("twa,ab,twb->tw", ex, uz, ey)
    return out


def lhat_exact_points(voxels, values, g: Geometry, t, kv, ku) -> np.ndarray:
    """u^(xi) at the slice points (t[i], kv[i], ku[i]) for a volume that is zero
    except u[ix, iz, iy] = values[k] at voxels[k] = (ix, iz, iy): the direct sum
    of the definition, at any size (cost: points x voxels)."""
    xi_x, xi_y, xi_z = slice_frequency_points(g, t, kv, ku)
    vox = np.asarray(voxels, dtype=np.float64)
    rx = vox[:, 0] - g.n1 // 2
    rz = vox[:, 1] - g.n0 // 2
    ry = vox[:, 2] - g.n2 // 2
    phase = np.outer(xi_x, rx) + np.outer(xi_y, ry) + np.outer(xi_z, rz)
    return np.exp(-2j * np.pi * phase) @ np.asarray(values, dtype=np.complex128)


def lhat_adj_exact_points(t, kv, ku, values, g: Geometry, voxels, real: bool = True) -> np.ndarray:
    """(L-hat^H r)[ix, iz, iy] at voxels[k] = (ix, iz, iy) for data that is zero
    except r[t[i], kv[i], ku[i]] = values[i]: sum_i r_i exp(+2 pi i xi_i . r),
    the transpose of lhat_exact under Re <a, b> (Re for a real u)."""
    xi_x, xi_y, xi_z = slice_frequency_points(g, t, kv, ku)
    vox = np.asarray(voxels, dtype=np.float64)
    rx = vox[:, 0] - g.n1 // 2
    rz = vox[:, 1] - g.n0 // 2
    ry = vox[:, 2] - g.n2 // 2
    phase = np.outer(rx, xi_x) + np.outer(ry, xi_y) + np.outer(rz, xi_z)
    v = np.exp(2j * np.pi * phase) @ np.asarray(values, dtype=np.complex128)
    return v.real if real else v


def _xi_z(g: Geometry) -> np.ndarray:
    return _xi(0.0, centred(g.h) / g.h, 0.0, g.phi)[2]


def lhat_sparse_points(voxels, values, g: Geometry, t, kv, ku) -> np.ndarray:
    """lhat(u, g)[t, kv, ku] for a volume that is zero except
    u[ix, iz, iy] = values[k] at voxels[k] = (ix, iz, iy) (distinct voxels),
    by the steps of lhat restricted to what those outputs need: F_u1D of the
    occupied (x, y) columns, then for each sampled kv the F_u2D grid of that
    plane gathered at its sampled points.  Equal to lhat up to rounding order;
    its cost does not grow with n_theta, h or w, so it reaches full sizes."""
    vox = np.asarray(voxels)
    t, kv, ku = np.asarray(t), np.asarray(kv), np.asarray(ku)
    cols, inv = np.unique(vox[:, [0, 2]], axis=0, return_inverse=True)
    ucols = np.zeros((len(cols), g.n0))
    np.add.at(ucols, (inv.ravel(), vox[:, 1]), np.asarray(values, dtype=np.float64))
    u1c = usfft.usfft1d_type2(ucols, _xi_z(g), g.m, g.R, axis=-1)      # [columns, h]
    xi_x, xi_y, _ = slice_frequency_points(g, t, kv, ku)
    out = np.empty(len(t), dtype=np.complex128)
    for k in np.unique(kv):
        plane = np.zeros((g.n1, g.n2), dtype=np.complex128)
        plane[cols[:, 0], cols[:, 1]] = u1c[:, k]
        P = usfft.usfft2d_grid(plane, g.m, g.R)
        sel = kv == k
        out[sel] = usfft.usfft2d_gather(P, xi_x[sel], xi_y[sel], g.m, g.R)
    return out


def lhat_adj_sparse_points(t, kv, ku, values, g: Geometry, voxels, real: bool = True) -> np.ndarray:
    """lhat_adj(r, g)[ix, iz, iy] at voxels[k] = (ix, iz, iy) for data that is
    zero except r[t[i], kv[i], ku[i]] = values[i] (distinct points): F*_u2D of
    each occupied kv plane from its non-zero points (zero points add nothing
    to the spread), then F*_u1D of the sampled (x, y) columns."""
    t, kv, ku = np.asarray(t), np.asarray(kv), np.asarray(ku)
    values = np.asarray(values, dtype=np.complex128)
    vox = np.asarray(voxels)
    xi_x, xi_y, _ = slice_frequency_points(g, t, kv, ku)
    col = np.zeros((len(vox), g.h), dtype=np.complex128)
    for k in np.unique(kv):
        sel = kv == k
        a = usfft.usfft2d_type1(values[sel], xi_x[sel], xi_y[sel], g.n1, g.n2, g.m, g.R)
        col[:, k] = a[vox[:, 0], vox[:, 2]]
    v = usfft.usfft1d_type1(col, _xi_z(g), g.n0, g.m, g.R, axis=-1)    # [voxels, n0]
    out = v[np.arange(len(vox)), vox[:, 1]]
    return out.real if real else out


def lam_forward_exact(u: np.ndarray, g: Geometry) -> np.ndarray:
    return f_2d_inv(lhat_exact(u, g))


# ----------------------------------------------------------------------------
# FBP-style single pass (a one-pass baseline next to the iterative method)
# ----------------------------------------------------------------------------

def fbp_weights(g: Geometry) -> np.ndarray:
    """Inverse density of the slice points per unit volume of frequency space,
    as a function of ku alone: pi cos(phi) |ku| / (T w^2 h), |ku| read as 1/4 at
    ku = 0 (the mean of |t| over the centre cell, t in units of 1/w).

    Derivation (the paper gives no filter; this is the density compensation of
    the geometry above).  Plane kv lies at xi_z = (kv/h) cos(phi); in it, the
    T lines xi_xy(ku) = (ku/w)(cos th, sin th) + (kv/h) sin(phi) (sin th, -cos th)
    are tangent to the circle of radius rho0 = |kv| sin(phi)/h and carry w
    points per unit length.  At radius rho each line crosses the ring twice, so
    the in-plane density is T w / (pi sqrt(rho^2 - rho0^2)), and
    sqrt(rho^2 - rho0^2) = |ku|/w.  The planes are cos(phi)/h apart."""
    ku = np.abs(centred(g.w))
    ku[g.w // 2] = 0.25
    return np.pi * np.cos(g.phi) * ku / (g.n_theta * g.w ** 2 * g.h)


def fbp(d: np.ndarray, g: Geometry) -> np.ndarray:
    """u = Re L_hat^H (W . F_2D d): since F_2D d = L_hat u for d = L u, this is
    the quadrature of the inverse Fourier integral over the sampled slices."""
    return lhat_adj(f_2d(d) * fbp_weights(g)[None, None, :], g)


def accuracy_error(r_comp: np.ndarray, r: np.ndarray) -> float:
    """E of Section 6.1 (Eq. 4): ||R_comp - R||_F / ||R_comp||_F."""
    return float(np.linalg.norm((r_comp - r).ravel()) / np.linalg.norm(np.ravel(r_comp)))
