"""Parity at full size, on sampled outputs, in the launch configuration the
benchmark times.

Workloads: n = nz = h = w = n_theta = 1024 (the large ADMM-TV workload) and
2048 (the stress size), 30 degree tilt, angles on [0, 2 pi), FP32 plans with
their default launch shapes and the L_hat-only workspace.

The FP64 oracle cannot run the full operators at these sizes.  It can
evaluate them at sampled points when the input is sparse (its point-sampled
forms restrict the same USFFT steps to what the sampled outputs need):

* L_hat of a volume with K point sources, at S random slice points, spread
  over a few kv planes;
* Re L_hat^H of data with K non-zero slice points (a few kv planes), at S
  random voxels.

Every sampled output depends on every source, so an indexing, window or
sign error anywhere in the path shows.  The bound is the FP32 per-operator
tolerance (relative L2 over the samples).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import TOL_F32_OP, oracle_geom, rel
from oracle import lamino as olam
from paper_2511_01893_b300 import inputs
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

PHI = np.deg2rad(30.0)
K_SOURCES, N_PLANES, S_PER_PLANE, S_VOXELS = 64, 3, 400, 1500


@pytest.fixture(scope="module", params=[1024, 2048], ids=["n1024", "n2048"])
def full(request):
    n = request.param
    theta = inputs.angles(n)
    plan = glam.Plan(n, n, n, n, theta, PHI, prec="f32", workspace="hat")
    g = oracle_geom(n, n, n, n, theta, PHI)
    yield n, plan, g
    del plan
    torch.cuda.empty_cache()


def test_forward_hat_at_sampled_points(full):
    n, plan, g = full
    rng = np.random.default_rng(n + 1)
    flat = rng.choice(n ** 3, K_SOURCES, replace=False)
    vox = np.stack(np.unravel_index(flat, (n, n, n)), axis=1)
    vals = rng.standard_normal(K_SOURCES)
    u = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    idx = torch.from_numpy(vox.T.copy()).cuda()
    u[idx[0], idx[1], idx[2]] = torch.from_numpy(vals).float().cuda()
    d = plan.forward_hat(u)
    del u
    planes = rng.choice(n, N_PLANES, replace=False)
    kv = np.repeat(planes, S_PER_PLANE)
    t = rng.integers(0, n, kv.size)
    ku = rng.integers(0, n, kv.size)
    got = d[torch.from_numpy(t).cuda(), torch.from_numpy(kv).cuda(), torch.from_numpy(ku).cuda()]
    del d
    # the oracle sees the FP32 source values the GPU holds
    ref = olam.lhat_sparse_points(vox, vals.astype(np.float32).astype(np.float64), g, t, kv, ku)
    assert rel(got, ref) < TOL_F32_OP


def test_adjoint_hat_at_sampled_voxels(full):
    n, plan, g = full
    rng = np.random.default_rng(n + 2)
    planes = rng.choice(n, N_PLANES, replace=False)
    kv = np.repeat(planes, K_SOURCES // N_PLANES)
    pos = rng.choice(n * n, kv.size, replace=False)  # distinct (theta, ku) per point
    t, ku = np.unravel_index(pos, (n, n))
    vals = (rng.standard_normal(kv.size) + 1j * rng.standard_normal(kv.size)).astype(np.complex64)
    r = torch.zeros((n, n, n), dtype=torch.complex64, device="cuda")
    r[torch.from_numpy(t).cuda(), torch.from_numpy(kv).cuda(), torch.from_numpy(ku).cuda()] = \
        torch.from_numpy(vals).cuda()
    v = plan.adjoint_hat(r)
    del r
    flat = rng.choice(n ** 3, S_VOXELS, replace=False)
    vox = np.stack(np.unravel_index(flat, (n, n, n)), axis=1)
    got = v[torch.from_numpy(vox[:, 0]).cuda(), torch.from_numpy(vox[:, 1]).cuda(),
            torch.from_numpy(vox[:, 2]).cuda()]
    del v
    ref = olam.lhat_adj_sparse_points(t, kv, ku, vals.astype(np.complex128), g, vox)
    assert rel(got, ref) < TOL_F32_OP
