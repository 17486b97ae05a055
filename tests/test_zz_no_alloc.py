"""lamx_u2d_fwd_static (F_u2D through the library's static plane scratch, no
workspace) against lamx_u2d_fwd (workspace planes), called twice in a row.

Collected last on purpose: it must pass in a fresh process and after every
other test has used the library.
"""
import ctypes

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
    outs = [torch.full((T, h, w), float("nan"), dtype=plan.cdtype, device="cuda") for _ in range(2)]
    # the first call on the device looks up the scratch array's address; the
    # second must leave the device's free memory and torch's allocator as they were
    plan.u2d_fwd_static(u1, outs[0], sub=sub)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    plan.u2d_fwd_static(u1, outs[1], sub=sub)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for out in outs:
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert rel(out, ref) < tol(prec)


def test_static_scratch_rejects_arrays_off_the_plans_device():
    n, nz, h, w, T = 32, 16, 16, 32, 7
    plan = glam.Plan(n, nz, h, w, inputs.angles(T), np.deg2rad(30.0), prec="f32")
    u1 = _rand_c((h, n, n), 21, plan.cdtype)
    out = torch.zeros((T, h, w), dtype=plan.cdtype, device="cuda")
    # host memory handed straight to the C ABI is refused before any launch
    host = np.zeros((T, h, w), dtype=np.complex64)
    st = glam.lib().lamx_u2d_fwd_static(plan._h, ctypes.c_void_p(u1.data_ptr()), ctypes.c_void_p(host.ctypes.data),
                                        None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1 and b"not device memory" in glam.lib().lam_last_error()
    with pytest.raises(glam.LaminoError):
        plan.u2d_fwd_static(u1.cpu(), out)
    torch.cuda.synchronize()
    assert not out.any()


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
