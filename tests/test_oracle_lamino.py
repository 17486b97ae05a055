"""Pins for the oracle's laminographic operator L (and L-hat, adjoints).

* P1: L-hat against the direct-sum definition sum_r u(r) exp(-2 pi i xi.r)
  on small volumes; error falls with m and reaches rounding at m = 12.
* P2: adjoint identities for L and for every stage.
* P3: a Gaussian blob, whose projection has a closed form (Fourier slice
  theorem), pins phi, theta, signs and the 1/(h w) normalisation.
* P4: phi = 0 reduces to tomography about z (sums along y at theta = 0 and
  along x at theta = pi/2).
* FBP (the one-pass baseline): FBP(L u) recovers blobs whose spectra the
  slices cover; the missing cone is not recovered.
"""
import numpy as np
import pytest

from oracle import lamino
from oracle.lamino import Geometry, centred
from oracle import lamino as olam
from oracle import usfft
from paper_2511_01893_b300 import inputs


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.ravel(b))


def _geom(n1=16, n0=16, n2=16, h=16, w=16, T=16, phi=0.5, m=4, seed=0):
    rng = np.random.default_rng(seed)
    return Geometry(n1=n1, n0=n0, n2=n2, h=h, w=w, theta=rng.uniform(0, 2 * np.pi, T), phi=phi, m=m)


@pytest.mark.parametrize("dims", [(16, 16, 16, 16, 16, 16), (12, 8, 12, 10, 14, 5)])
def test_lhat_matches_direct_nudft(dims):
    n1, n0, n2, h, w, T = dims
    rng = np.random.default_rng(10)
    u = rng.standard_normal((n1, n0, n2))
    errs = []
    for m in (2, 4, 6, 8, 12):
        g = _geom(n1, n0, n2, h, w, T, phi=0.61, m=m)
        errs.append(_rel(lamino.lhat(u, g), lamino.lhat_exact(u, g)))
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[1] < 2e-4
    assert errs[-1] < 1e-10


def test_lhat_direct_sum_rotation_and_tilt_conventions():
    # at phi = 0 the exact slice at theta = 0 is the DFT of the sum over y in
    # (x, z): independent of the operator code
    rng = np.random.default_rng(11)
    n = 8
    u = rng.standard_normal((n, n, n))
    g = Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=np.array([0.0]), phi=0.0)
    s = u.sum(axis=2)                                     # [x, z]
    k = np.arange(n)
    ph = np.exp(2j * np.pi * k * (n // 2) / n)            # centring phase
    ref = (np.fft.fft2(s) * ph[:, None] * ph[None, :]).T   # [kz, kx]
    ref = np.roll(np.roll(ref, n // 2, 0), n // 2, 1)      # frequency order -n/2..n/2-1
    assert _rel(lamino.lhat_exact(u, g)[0], ref) < 1e-12


def test_adjoint_identity_full_operator():
    g = _geom(n1=12, n0=8, n2=12, h=10, w=14, T=7, phi=0.4)
    rng = np.random.default_rng(12)
    u = rng.standard_normal((12, 8, 12))
    v = rng.standard_normal((7, 10, 14)) + 1j * rng.standard_normal((7, 10, 14))
    Lu = lamino.lam_forward(u, g)
    lhs = np.vdot(Lu, v).real
    rhs = np.vdot(u, lamino.lam_adjoint(v, g))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Lu) * np.linalg.norm(v)
    Lh = lamino.lhat(u, g)
    lhs = np.vdot(Lh, v).real
    rhs = np.vdot(u, lamino.lhat_adj(v, g))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Lh) * np.linalg.norm(v)


def test_adjoint_identity_per_stage():
    g = _geom(n1=12, n0=8, n2=12, h=10, w=14, T=7, phi=0.4)
    rng = np.random.default_rng(13)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    a, b = c(12, 8, 12), c(12, 10, 12)
    assert abs(np.vdot(lamino.f_u1d(a, g), b) - np.vdot(a, lamino.f_u1d_adj(b, g))) < 1e-12 * 1e3
    a, b = c(12, 10, 12), c(7, 10, 14)
    assert abs(np.vdot(lamino.f_u2d(a, g), b) - np.vdot(a, lamino.f_u2d_adj(b, g))) < 1e-12 * 1e4
    a, b = c(7, 10, 14), c(7, 10, 14)
    assert abs(np.vdot(lamino.f_2d_inv(a), b) - np.vdot(a, lamino.f_2d_inv_adj(b))) < 1e-12 * 1e2


def test_f2d_cancels_f2d_inverse():
    rng = np.random.default_rng(14)
    x = rng.standard_normal((3, 10, 14)) + 1j * rng.standard_normal((3, 10, 14))
    assert _rel(lamino.f_2d(lamino.f_2d_inv(x)), x) < 1e-13
    assert _rel(lamino.f_2d_inv(lamino.f_2d(x)), x) < 1e-13


def _blob_case(m):
    n, nz, h, w, T = 48, 48, 48, 48, 6
    phi = np.deg2rad(30.0)
    th = np.linspace(0, 2 * np.pi, T, endpoint=False) + 0.3
    c = np.array([3.3, -2.1, 1.7])
    s = 2.5
    rx = centred(n)[:, None, None]
    rz = centred(nz)[None, :, None]
    ry = centred(n)[None, None, :]
    u = np.exp(-((rx - c[0]) ** 2 + (ry - c[1]) ** 2 + (rz - c[2]) ** 2) / (2 * s * s))
    g = Geometry(n1=n, n0=nz, n2=n, h=h, w=w, theta=th, phi=phi, m=m)
    # closed form: the line integral of the blob along the beam b = e_u x e_v
    # is sqrt(2 pi) s exp(-((s_det - c.e_u)^2 + (t_det - c.e_v)^2) / (2 s^2))
    thc = th[:, None, None]
    cu = c[0] * np.cos(thc) + c[1] * np.sin(thc)
    cv = c[0] * np.sin(phi) * np.sin(thc) - c[1] * np.sin(phi) * np.cos(thc) + c[2] * np.cos(phi)
    S = centred(w)[None, None, :]
    Tt = centred(h)[None, :, None]
    proj = np.sqrt(2 * np.pi) * s * np.exp(-((S - cu) ** 2 + (Tt - cv) ** 2) / (2 * s * s))
    return lamino.lam_forward(u, g), proj


def test_gaussian_blob_projection_closed_form():
    d4, proj = _blob_case(4)
    assert _rel(d4, proj) < 1e-4
    d10, proj = _blob_case(10)
    assert _rel(d10, proj) < 1e-10


def test_phi_zero_is_tomography():
    n = 16
    u = np.zeros((n, n, n))
    u[3:9, 5:12, 2:13] = 1.0                      # axis-aligned box [x, z, y]
    u[10:14, 2:6, 4:7] = 0.5
    th = np.array([0.0, np.pi / 2])
    g = Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=th, phi=0.0, m=12)
    d = lamino.lam_forward(u, g)
    # theta = 0: beam along -y, detector u <-> x, v <-> z
    assert _rel(d[0], u.sum(axis=2).T) < 1e-10
    # theta = pi/2: beam along +x, detector u <-> y, v <-> z
    assert _rel(d[1], u.sum(axis=0)) < 1e-10


def test_accuracy_metric():
    a = np.array([3.0, 4.0])
    assert lamino.accuracy_error(a, a * 0.9) == pytest.approx(0.1)


def _sparse_case(n1, n0, n2, h, w, T, K, S, seed):
    rng = np.random.default_rng(seed)
    g = _geom(n1, n0, n2, h, w, T, phi=0.52, seed=seed)
    flat = rng.choice(n1 * n0 * n2, K, replace=False)
    vox = np.stack(np.unravel_index(flat, (n1, n0, n2)), axis=1)
    vals = rng.standard_normal(K)
    u = np.zeros((n1, n0, n2))
    u[vox[:, 0], vox[:, 1], vox[:, 2]] = vals
    flat = rng.choice(T * h * w, S, replace=False)
    t, kv, ku = np.unravel_index(flat, (T, h, w))
    return g, vox, vals, u, t, kv, ku


@pytest.mark.parametrize("dims", [(16, 12, 16, 10, 14, 9), (24, 16, 20, 16, 12, 7)])
def test_point_sampled_forms_match_the_full_operators(dims):
    # the point-sampled direct sum and the point-sampled USFFT steps against
    # the full-array functions they restrict (lhat_exact pinned by the closed
    # forms above, lhat by the direct sum)
    g, vox, vals, u, t, kv, ku = _sparse_case(*dims, K=30, S=200, seed=11)
    full = lamino.lhat(u, g)
    assert _rel(lamino.lhat_sparse_points(vox, vals, g, t, kv, ku), full[t, kv, ku]) < 1e-12
    assert _rel(lamino.lhat_exact_points(vox, vals, g, t, kv, ku), lamino.lhat_exact(u, g)[t, kv, ku]) < 1e-12
    rng = np.random.default_rng(12)
    rv = rng.standard_normal(len(t)) + 1j * rng.standard_normal(len(t))
    r = np.zeros((g.n_theta, g.h, g.w), dtype=np.complex128)
    r[t, kv, ku] = rv
    adj = lamino.lhat_adj(r, g)
    got = lamino.lhat_adj_sparse_points(t, kv, ku, rv, g, vox)
    assert _rel(got, adj[vox[:, 0], vox[:, 1], vox[:, 2]]) < 1e-12
    # the exact adjoint sum is the transpose of the exact forward sum
    lhs = np.vdot(rv, lamino.lhat_exact_points(vox, vals, g, t, kv, ku)).real
    rhs = np.dot(vals, lamino.lhat_adj_exact_points(t, kv, ku, rv, g, vox))
    assert abs(lhs - rhs) < 1e-10 * np.linalg.norm(rv) * np.linalg.norm(vals) * len(t)


# ---- FBP-style single pass (oracle.lamino.fbp) --------------------------------
# Pin: FBP(L u) recovers a band-limited volume whose spectrum the slices cover.
# Laminography misses the cone of frequencies within phi of the z axis, so the
# laminographic pins use blobs elongated along z (spectra near xi_z = 0); the
# phi = 0 (tomography) pin uses a round blob.  A wrong constant (a missing
# cos(phi), pi or 1/T), the ramp on the wrong axis or a missing 1/4 at ku = 0
# moves the scale or the error far outside these bounds.

def _blob(n, sxy, sz, c=(1.3, -0.7, 2.1)):
    x = np.arange(n) - n // 2
    X, Z, Y = np.meshgrid(x, x, x, indexing="ij")
    return np.exp(-((X - c[0]) ** 2 + (Y - c[2]) ** 2) / (2 * sxy ** 2) - (Z - c[1]) ** 2 / (2 * sz ** 2))


@pytest.mark.parametrize("phi_deg,sxy,sz,tol", [(0.0, 2.5, 2.5, 0.06), (30.0, 2.5, 8.0, 0.09), (20.0, 2.5, 8.0, 0.07)])
def test_fbp_recovers_blob(phi_deg, sxy, sz, tol):
    n, T = 32, 64
    g = olam.Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=inputs.angles(T), phi=np.deg2rad(phi_deg))
    u = _blob(n, sxy, sz)
    r = olam.fbp(olam.lam_forward(u, g), g)
    assert np.linalg.norm(r - u) / np.linalg.norm(u) < tol
    assert abs(np.vdot(r, u).real / np.vdot(u, u).real - 1) < 0.025


def test_fbp_missing_cone_is_not_recovered():
    # a round blob at phi = 30 deg loses its missing-cone content: scale < 0.95
    n, T = 32, 64
    g = olam.Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=inputs.angles(T), phi=np.deg2rad(30.0))
    u = _blob(n, 2.5, 2.5)
    r = olam.fbp(olam.lam_forward(u, g), g)
    assert np.vdot(r, u).real / np.vdot(u, u).real < 0.95


def test_tap_rule_on_grid_nodes_matches_direct_nudft():
    # theta at multiples of pi/2 and phi = 30 deg put every in-plane slice point
    # exactly on a node of the padded grid (M xi = (2 ku, -kv) up to sign and
    # order): the tap window's switch point (2^-17 below each node) decides
    # which 2m nodes serve it.  At m = 12 the USFFT is exact to ~1e-12, so a
    # window shifted by one node, or taps read from the wrong side, shows here.
    n, nz, T = 16, 8, 4
    g = Geometry(n1=n, n0=nz, n2=n, h=n, w=n, theta=np.arange(T) * np.pi / 2, phi=np.pi / 6, m=12)
    xi_x, xi_y, _ = lamino.slice_frequencies(g)
    M = 2 * n
    for a in (M * xi_x, M * xi_y):
        assert np.abs(a - np.round(a)).max() < 1e-12
    rng = np.random.default_rng(3)
    u = rng.standard_normal((n, nz, n))
    assert _rel(lamino.lhat(u, g), lamino.lhat_exact(u, g)) < 1e-10
    r = rng.standard_normal((T, n, n)) + 1j * rng.standard_normal((T, n, n))
    # the transpose at the same nodes, against the transpose of the direct sum
    lhs = np.vdot(lamino.lhat_exact(u, g), r).real
    rhs = np.vdot(u, lamino.lhat_adj(r, g)).real
    assert abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(r)) < 1e-10


def test_hermitian_pairs_of_slice_points():
    """P5: for a real volume the slice point (theta, -ku, -kv) sits at the
    negated position of (theta, ku, kv), so where all three tap windows mirror
    (j0(-t) = -j0(t) - 1 for the z, x and y grid positions t) the value there
    is the conjugate of its partner's value, to rounding.  Where a position
    lies within the tap shift of a grid node (whole lines at theta in
    (pi/2)Z; at phi = 30 deg also x at theta = pi/2) the windows differ by a
    cell, and so do the two values, by no more than the truncation error.
    The oracle computes every plane from its own padded FFT, so this checks
    the identity the paired GPU gather and spread are built on."""
    n, T = 16, 16
    g = Geometry(n1=n, n0=n, n2=n, h=n, w=n, theta=2 * np.pi * np.arange(T) / T, phi=np.deg2rad(30.0))
    u = np.random.default_rng(21).standard_normal((n, n, n))
    L = lamino.lhat(u, g)
    xi_x, xi_y, xi_z = lamino.slice_frequencies(g)
    kv = np.arange(1, g.h)[None, :, None]  # partner row h - kv: centred -kv
    ku = np.arange(1, g.w)[None, None, :]  # partner column w - ku: centred -ku
    t_idx = np.arange(T)[:, None, None]
    p, q = L[t_idx, kv, ku], L[t_idx, g.h - kv, g.w - ku]
    # the partner positions are the exact negatives
    assert np.array_equal(xi_x[t_idx, g.h - kv, g.w - ku], -xi_x[t_idx, kv, ku])
    assert np.array_equal(xi_y[t_idx, g.h - kv, g.w - ku], -xi_y[t_idx, kv, ku])
    assert np.array_equal(xi_z[g.h - kv[0, :, 0]], -xi_z[kv[0, :, 0]])

    def mirrors(t):
        return np.floor(-t + usfft.TAP_SHIFT) == -np.floor(t + usfft.TAP_SHIFT) - 1

    mir = (mirrors(2 * g.n1 * xi_x[t_idx, kv, ku]) & mirrors(2 * g.n2 * xi_y[t_idx, kv, ku])
           & mirrors(2 * g.n0 * xi_z[kv[0, :, 0]])[None, :, None])
    scale = np.abs(L).max()
    d = np.abs(q - np.conj(p))
    assert 0.5 < mir.mean() < 1.0
    assert d[mir].max() < 1e-12 * scale
    assert 1e-9 * scale < d[~mir].max() < 1e-2 * scale
