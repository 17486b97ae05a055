"""GPU parity of L, L^H, their stages, F_2D and TV against the FP64 oracle.

Every comparison calls the CUDA path through the C ABI (liblamino.so) and the
oracle on the same seeded inputs.  Sizes span several tiles and batches and
include non-cubic shapes, phi = 0 (tomography) and a large tilt.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL_F32_OP, TOL_F64_OP, plan_and_geom, rand_data, rand_vol, rel, tol
from oracle import lamino as olam
from oracle import tv as otv
from oracle import usfft as ousfft
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

GEOMS = [
    # n, nz, h, w, T, phi
    (16, 16, 16, 16, 16, np.deg2rad(30.0)),
    (32, 16, 8, 64, 12, np.deg2rad(30.0)),
    (64, 32, 64, 32, 40, np.deg2rad(20.0)),
    (32, 32, 32, 32, 24, 0.0),
    (16, 8, 16, 16, 9, np.deg2rad(70.0)),
    # sizes with factors 3 and 5 (mixed-radix FFTs, 32 x 32 plane tiles)
    (48, 24, 40, 48, 30, np.deg2rad(25.0)),
    (80, 40, 60, 80, 18, np.deg2rad(35.0)),
]
IDS = ["cube16", "flat32", "mixed64", "phi0", "steep", "radix3", "radix5"]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("geom", GEOMS, ids=IDS)
def test_u1d_forward_and_adjoint(geom, prec):
    n, nz, h, w, T, phi = geom
    plan, g = plan_and_geom(n, nz, h, w, T, phi, prec)
    u = rand_vol(n, nz, 1)
    ref = olam.f_u1d(u, g)                          # [n1, h, n2]
    got = plan.u1d_fwd(torch.from_numpy(u)).cpu().numpy().transpose(1, 0, 2)
    assert rel(got, ref) < tol(prec)
    c = np.random.default_rng(2).standard_normal((n, h, n)) + 1j * np.random.default_rng(3).standard_normal((n, h, n))
    ref = olam.f_u1d_adj(c, g).real
    got = plan.u1d_adj(torch.from_numpy(np.ascontiguousarray(c.transpose(1, 0, 2)))).cpu().numpy()
    assert rel(got, ref) < tol(prec)


@pytest.mark.parametrize("spread", ["tiles", "halo", "atomic", "exact", "tiles_exact", "tiles2", "sweep"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("geom", GEOMS, ids=IDS)
def test_u2d_forward_and_adjoint(geom, prec, spread):
    n, nz, h, w, T, phi = geom
    plan, g = plan_and_geom(n, nz, h, w, T, phi, prec)
    plan = glam.Plan(n, nz, h, w, g.theta, phi, prec=prec, spread=spread)
    rng = np.random.default_rng(4)
    u1 = rng.standard_normal((n, h, n)) + 1j * rng.standard_normal((n, h, n))
    ref = olam.f_u2d(u1, g)
    got = plan.u2d_fwd(torch.from_numpy(np.ascontiguousarray(u1.transpose(1, 0, 2)))).cpu().numpy()
    assert rel(got, ref) < tol(prec)
    d = rand_data(T, h, w, 5)
    ref = olam.f_u2d_adj(d, g)
    got = plan.u2d_adj(torch.from_numpy(d)).cpu().numpy().transpose(1, 0, 2)
    assert rel(got, ref) < tol(prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("geom", GEOMS, ids=IDS)
def test_lam_forward_adjoint(geom, prec):
    n, nz, h, w, T, phi = geom
    plan, g = plan_and_geom(n, nz, h, w, T, phi, prec)
    u = rand_vol(n, nz, 6)
    assert rel(plan.forward(torch.from_numpy(u)), olam.lam_forward(u, g)) < tol(prec)
    assert rel(plan.forward_hat(torch.from_numpy(u)), olam.lhat(u, g)) < tol(prec)
    d = rand_data(T, h, w, 7)
    assert rel(plan.adjoint(torch.from_numpy(d)), olam.lam_adjoint(d, g)) < tol(prec)
    assert rel(plan.adjoint_hat(torch.from_numpy(d)), olam.lhat_adj(d, g)) < tol(prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_forward_hermitian_pairs(prec):
    """For a real volume the paired gather sums each pair of mirror slice
    points (theta, ku, kv) / (theta, -ku, -kv) once: where the z, x and y tap
    windows mirror, L-hat u at the mirror point is bitwise the conjugate of its
    partner's value.  Where a position lies within the tap shift of a grid
    node the mirror window is a cell lower and the value is summed on its own,
    so it differs, as the oracle's does (test_oracle_lamino P5); both kinds
    match the oracle (test_lam_forward_adjoint)."""
    n, T = 32, 24
    plan, g = plan_and_geom(n, n, n, n, T, np.deg2rad(30.0), prec)
    L = plan.forward_hat(torch.from_numpy(rand_vol(n, n, 8))).cpu().numpy()
    xi_x, xi_y, xi_z = olam.slice_frequencies(g)
    kv = np.arange(1, n // 2)[None, :, None]   # the paired planes and their mirrors h - kv
    ku = np.arange(1, n)[None, None, :]        # partner column w - ku
    t = np.arange(T)[:, None, None]

    def mirrors(x):
        return np.floor(-x + ousfft.TAP_SHIFT) == -np.floor(x + ousfft.TAP_SHIFT) - 1

    mir = (mirrors(2 * n * xi_x[t, kv, ku]) & mirrors(2 * n * xi_y[t, kv, ku])
           & mirrors(2 * n * xi_z[kv[0, :, 0]])[None, :, None])
    p, q = L[t, kv, ku], L[t, n - kv, n - ku]
    assert 0.5 < mir.mean() < 1.0
    assert np.array_equal(q[mir].real, p[mir].real) and np.array_equal(q[mir].imag, -p[mir].imag)
    assert np.abs(q[~mir] - np.conj(p[~mir])).max() > 1e-9 * np.abs(L).max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_fused_subtraction(prec):
    n, nz, h, w, T, phi = 32, 32, 32, 32, 16, np.deg2rad(30.0)
    plan, g = plan_and_geom(n, nz, h, w, T, phi, prec)
    u = rand_vol(n, nz, 8)
    sub = rand_data(T, h, w, 9)
    ref = olam.lhat(u, g) - sub
    got = plan.forward_hat(torch.from_numpy(u), sub=torch.from_numpy(sub))
    assert rel(got, ref) < tol(prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_fft2d_both_directions(prec):
    plan, g = plan_and_geom(16, 16, 32, 64, 5, 0.3, prec)
    x = rand_data(5, 32, 64, 10)
    assert rel(plan.fft2d(torch.from_numpy(x), inverse=True), olam.f_2d_inv(x)) < tol(prec)
    assert rel(plan.fft2d(torch.from_numpy(x), inverse=False), olam.f_2d(x)) < tol(prec)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_tv_grad_div(prec):
    plan, _ = plan_and_geom(16, 32, 16, 16, 4, 0.3, prec)
    u = rand_vol(16, 32, 11)
    assert rel(plan.tv_grad(torch.from_numpy(u)), otv.grad(u)) < tol(prec)
    p = np.random.default_rng(12).standard_normal((3, 16, 32, 16))
    assert rel(plan.tv_div(torch.from_numpy(p)), otv.div(p)) < tol(prec)


def test_adjoint_identity_on_gpu_f64():
    n, nz, h, w, T = 32, 16, 32, 32, 20
    plan, _ = plan_and_geom(n, nz, h, w, T, 0.4, "f64")
    u = torch.from_numpy(rand_vol(n, nz, 13)).cuda()
    v = torch.from_numpy(rand_data(T, h, w, 14)).cuda()
    Lu = plan.forward(u)
    lhs = torch.vdot(Lu.flatten(), v.flatten()).real.item()
    rhs = torch.dot(u.flatten(), plan.adjoint(v).flatten()).item()
    assert abs(lhs - rhs) <= 1e-12 * Lu.norm().item() * v.norm().item()


def test_tiny_and_ragged_batches(monkeypatch):
    # a single angle, and h = 16 planes in batches of 3 (ragged last batch)
    n, nz, h, w, T = 8, 8, 16, 8, 1
    monkeypatch.setenv("LAMINO_PLANES_PER_BATCH", "3")
    plan, g = plan_and_geom(n, nz, h, w, T, 0.5, "f64")
    assert plan.info()["planes_per_batch"] == 3
    u = rand_vol(n, nz, 15)
    assert rel(plan.forward(torch.from_numpy(u)), olam.lam_forward(u, g)) < 1e-12
    d = rand_data(T, h, w, 17)
    assert rel(plan.adjoint(torch.from_numpy(d)), olam.lam_adjoint(d, g)) < 1e-12


@pytest.mark.parametrize("m", [2, 3, 4, 8])
def test_adjoint_spread_variants_other_widths(m):
    # every spread variant at other kernel half-widths (window 2m x 2m)
    n, nz, h, w, T = 32, 16, 32, 32, 12
    plan, g = plan_and_geom(n, nz, h, w, T, 0.5, "f32", m=m)
    d = rand_data(T, h, w, 18)
    ref = olam.f_u2d_adj(d, g)
    for spread in ("tiles", "halo", "atomic", "exact", "tiles_exact", "tiles2", "sweep"):
        p = glam.Plan(n, nz, h, w, plan.theta, 0.5, m=m, prec="f32", spread=spread)
        got = p.u2d_adj(torch.from_numpy(d)).cpu().numpy().transpose(1, 0, 2)
        assert rel(got, ref) < tol("f32"), spread


def test_adjoint_spreads_are_bitwise_reproducible():
    # the default (per-warp tiles summed in a fixed order) and the exact
    # fixed-point spread give the same bits on every run
    n, nz, h, w, T = 64, 32, 64, 64, 48
    plan, g = plan_and_geom(n, nz, h, w, T, 0.5, "f32")
    d = torch.from_numpy(rand_data(T, h, w, 16)).cuda()
    a, b = plan.adjoint(d), plan.adjoint(d)
    assert torch.equal(a, b)
    exact = glam.Plan(n, nz, h, w, plan.theta, 0.5, prec="f32", spread="exact")
    e1, e2 = exact.adjoint(d), exact.adjoint(d)
    assert torch.equal(e1, e2)
    tx = glam.Plan(n, nz, h, w, plan.theta, 0.5, prec="f32", spread="tiles_exact")
    t1, t2 = tx.adjoint(d), tx.adjoint(d)
    assert torch.equal(t1, t2)
    h2 = glam.Plan(n, nz, h, w, plan.theta, 0.5, prec="f32", spread="tiles2")
    s1, s2 = h2.adjoint(d), h2.adjoint(d)
    assert torch.equal(s1, s2)
    assert rel(s1, e1) < 2e-6
    sw = glam.Plan(n, nz, h, w, plan.theta, 0.5, prec="f32", spread="sweep")
    w1, w2 = sw.adjoint(d), sw.adjoint(d)
    assert torch.equal(w1, w2)
    assert rel(w1, e1) < 2e-6
    # the same products formed in another order (wx (wy v) against wy (wx v)): ~1 ulp apart
    assert rel(t1, e1) < 3e-7
    fast = glam.Plan(n, nz, h, w, plan.theta, 0.5, prec="f32", fast_adjoint=True)
    assert rel(fast.adjoint(d), e1) < 2e-6
    assert rel(a, e1) < 2e-6
    ref = olam.lam_adjoint(d.cpu().numpy(), g)
    assert rel(a, ref) < 1e-5
    assert rel(e1, ref) < 1e-5


@pytest.mark.parametrize("prec,m", [("f32", 4), ("f32", 8), ("f64", 4), ("f64", 8)])
def test_sweep_spread_on_dense_planes_matches_exact_sums(prec, m):
    # 360 lines through the middle of the centre planes: thousands of records
    # per warp band there, so the row sweep fills and sorts its record buffer
    # many times; the exact centre jobs are off, so every plane job sweeps.
    # Reference (oracle-pinned in the tests above): in FP32 the tile spread
    # with exact fixed-point sums; in FP64 the plain tile spread, since the
    # fixed-point grid (step ~ 2^-61 x a bound on the cell sums, per product,
    # growing with the window) is coarser than FP64 rounding for small cells.
    n, nz, h, w, T = 128, 32, 128, 128, 360
    plan, g = plan_and_geom(n, nz, h, w, T, 0.5, prec, m=m)
    d = torch.from_numpy(rand_data(T, h, w, 21)).cuda()
    ex = glam.Plan(n, nz, h, w, plan.theta, 0.5, m=m, prec=prec, spread="tiles_exact" if prec == "f32" else "tiles")
    sw = glam.Plan(n, nz, h, w, plan.theta, 0.5, m=m, prec=prec, spread="sweep").set_exact_centre_jobs(0)
    a, b = sw.u2d_adj(d), ex.u2d_adj(d)
    assert torch.equal(a, sw.u2d_adj(d))
    assert rel(a, b) < (2e-6 if prec == "f32" else TOL_F64_OP)
    # the centre plane alone (every line passes its origin) against the oracle
    xi_x, xi_y, _ = olam.slice_frequencies(g)
    c = h // 2
    ref = ousfft.usfft2d_type1(d.cpu().numpy()[:, c, :], xi_x[:, c, :], xi_y[:, c, :], n, n, g.m, g.R)
    assert rel(a[c].cpu().numpy(), ref) < tol(prec)


@pytest.mark.parametrize("n", [48, 64])
def test_autotune_keeps_results_bitwise(n):
    # launch shapes change only how lines and points are grouped into blocks
    plan, g = plan_and_geom(n, n // 2, n, n, n, 0.4, "f32")
    u = torch.from_numpy(rand_vol(n, n // 2, 19)).cuda().float()
    d = torch.from_numpy(rand_data(n, n, n, 20)).cuda().to(torch.complex64)
    f0, a0 = plan.forward(u), plan.adjoint(d)
    t = plan.autotune(reps=1)
    assert t > 0
    info = plan.info()
    assert info["gather_tile"] in (16, 32, 64) and (2 * n) % info["gather_tile"] == 0
    assert torch.equal(plan.forward(u), f0)
    assert torch.equal(plan.adjoint(d), a0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_threads_per_block_keep_results_bitwise(prec):
    # 256 or 512 threads per z-stage / plane-FFT block: the lines per block
    # change, the arithmetic of every line does not
    n = 256
    plan, g = plan_and_geom(n, n // 4, n // 4, n, 8, 0.4, prec)
    u = torch.from_numpy(rand_vol(n, n // 4, 23)).cuda().to(plan.rdtype)
    d = torch.from_numpy(rand_data(8, n // 4, n, 24)).cuda().to(plan.cdtype)
    f0, a0 = plan.forward(u), plan.adjoint(d)
    for z, f in [(256, 512), (512, 256), (256, 256)]:
        plan.set_threads(z=z, fft=f)
        info = plan.info()
        assert (info["z_threads"], info["fft_threads"]) == (z, f)
        assert torch.equal(plan.forward(u), f0)
        assert torch.equal(plan.adjoint(d), a0)
    with pytest.raises(glam.LaminoError):
        plan.set_threads(z=384)


def test_spread_stage_entry_point(monkeypatch):
    # the spread alone (timed by bench.py as the dominant kernel): one batch
    # of plane jobs into the workspace planes, arguments checked on the host;
    # 4 planes per batch, fewer than the 33 plane jobs
    monkeypatch.setenv("LAMINO_PLANES_PER_BATCH", "4")
    n, nz, h, w, T = 64, 16, 64, 64, 24
    plan, g = plan_and_geom(n, nz, h, w, T, 0.4, "f32")
    assert plan.info()["planes_per_batch"] == 4
    d = torch.from_numpy(rand_data(T, h, w, 25)).cuda().to(torch.complex64)
    nb = plan.spread(d)
    assert 1 <= nb <= plan.info()["planes_per_batch"]
    assert nb <= plan.job_planes(0, nb) <= 2 * nb
    assert plan.job_planes(0, plan.info()["plane_jobs"]) == h
    assert plan.job_planes(0, plan.info()["plane_jobs"] + 1) == -1
    with pytest.raises(glam.LaminoError, match="outside"):
        plan.spread(d, plan.info()["plane_jobs"], 1)
    with pytest.raises(glam.LaminoError, match="workspace holds"):
        plan.spread(d, 0, plan.info()["planes_per_batch"] + 1)
    torch.cuda.synchronize()
    # the full adjoint after the standalone spread is unchanged
    assert rel(plan.adjoint_hat(d), olam.lhat_adj(rand_data(T, h, w, 25), g)) < TOL_F32_OP


def test_hat_workspace_serves_the_hat_operators():
    n, nz, h, w, T = 32, 16, 32, 32, 12
    full, g = plan_and_geom(n, nz, h, w, T, 0.4, "f32")
    hat = glam.Plan(n, nz, h, w, full.theta, 0.4, prec="f32", workspace="hat")
    assert hat.ws.numel() < full.ws.numel()
    u = torch.from_numpy(rand_vol(n, nz, 21)).cuda().float()
    d = torch.from_numpy(rand_data(T, h, w, 22)).cuda().to(torch.complex64)
    assert torch.equal(hat.forward_hat(u), full.forward_hat(u))
    assert torch.equal(hat.adjoint_hat(d), full.adjoint_hat(d))
    assert torch.equal(hat.forward(u), full.forward(u))
    with pytest.raises(glam.LaminoError, match="full workspace"):
        hat.adjoint(d)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("geom", [GEOMS[0], GEOMS[2], GEOMS[3], GEOMS[5]], ids=["cube16", "mixed64", "phi0", "radix3"])
def test_fbp_single_pass(geom, prec):
    # the one-pass baseline lam_fbp against the oracle's FBP on random data
    n, nz, h, w, T, phi = geom
    plan, g = plan_and_geom(n, nz, h, w, T, phi, prec)
    d = rand_data(T, h, w, 7)
    ref = olam.fbp(d, g)
    got = plan.fbp(torch.from_numpy(d)).cpu().numpy()
    assert rel(got, ref) < tol(prec)


def test_fbp_of_the_forward_recovers_a_z_elongated_blob():
    # GPU end to end: FP32 L then FBP at 32^3, phi = 30 deg (the oracle pin's case)
    n, T = 32, 64
    plan, g = plan_and_geom(n, n, n, n, T, np.deg2rad(30.0), "f32")
    x = np.arange(n) - n // 2
    X, Z, Y = np.meshgrid(x, x, x, indexing="ij")
    u = np.exp(-((X - 1.3) ** 2 + (Y - 2.1) ** 2) / (2 * 2.5 ** 2) - (Z + 0.7) ** 2 / (2 * 8.0 ** 2))
    r = plan.fbp(plan.forward(torch.from_numpy(u))).cpu().numpy()
    ref = olam.fbp(olam.lam_forward(u, g), g)
    assert rel(r, ref) < TOL_F32_OP
    assert rel(r, u) < 0.09
