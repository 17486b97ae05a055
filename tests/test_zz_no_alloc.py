"""lamx_u2d_fwd_static (F_u2D through the library's static plane scratch, no
workspace) against lamx_u2d_fwd (workspace planes), called twice in a row.

Collected last on purpose: it must pass in a fresh process and after every
other test has used the library.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import rel, tol
from paper_2511_01893_b300 import inputs
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

CASES = [
    # n, nz, h, w, T, prec, with sub.  Planes per batch = 8 MiB / (2n)^2 values:
    (512, 16, 16, 64, 6, "f32", False),  # 1 per batch, 16 batches
    (256, 8, 8, 32, 5, "f64", True),  # 2 per batch, 4 batches
    (64, 32, 64, 64, 20, "f64", True),  # 32 per batch, 2 batches
    (32, 16, 16, 32, 7, "f32", True),  # one batch
]


def _rand_c(shape, seed, dtype):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.from_numpy(x).to(device="cuda", dtype=dtype).contiguous()


@pytest.mark.parametrize("case", CASES, ids=["f32_n512", "f64_n256_sub", "f64_n64_sub", "f32_n32_sub"])
def test_static_scratch_forward_matches_workspace_forward(case):
    n, nz, h, w, T, prec, with_sub = case
    plan = glam.Plan(n, nz, h, w, inputs.angles(T), np.deg2rad(30.0), prec=prec)
    u1 = _rand_c((h, n, n), 21, plan.cdtype)
    sub = _rand_c((T, h, w), 22, plan.cdtype) if with_sub else None
    ref = plan.u2d_fwd(u1, sub=sub)
    outs = []
    for _ in range(2):
        out = torch.full((T, h, w), float("nan"), dtype=plan.cdtype, device="cuda")
        plan.u2d_fwd_static(u1, out, sub=sub)
        outs.append(out)
    torch.cuda.synchronize()
    for out in outs:
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert rel(out, ref) < tol(prec)


def test_static_scratch_rejects_planes_beyond_its_size():
    # n = 1024 in FP32: one padded 2048^2 plane is 32 MiB > 8 MiB
    n, nz, h, w, T = 1024, 8, 8, 8, 2
    plan = glam.Plan(n, nz, h, w, inputs.angles(T), 0.5, prec="f32")
    u1 = torch.zeros((h, n, n), dtype=plan.cdtype, device="cuda")
    out = torch.zeros((T, h, w), dtype=plan.cdtype, device="cuda")
    with pytest.raises(glam.LaminoError, match="static scratch"):
        plan.u2d_fwd_static(u1, out)
    torch.cuda.synchronize()
    assert not out.any()
