"""L and TV as torch.autograd functions whose backward passes are the
hand-written adjoint / -div kernels.

Differentiation workload: volume 128^3, 128 angles, detector 128 x 128,
tilt 20 degrees.  The gradient of 1/2 ||L u - d||^2 + alpha TV_eps(u) is
checked against central finite differences (FP64 path) and against the FP64
oracle's gradient (FP32 path)."""
import numpy as np
import pytest
import torch

from gpu_helpers import oracle_geom, rel
from oracle import lamino as olam
from oracle import tv as otv
from paper_2511_01893_b300 import inputs
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

N, T, PHI = 128, 128, np.deg2rad(20.0)
ALPHA, EPS = 1e-2, 0.1


@pytest.fixture(scope="module")
def case():
    theta = inputs.angles(T)
    u0 = inputs.ellipsoid_phantom(N, N, 12, seed=1236)
    u = 0.5 * u0 + 0.1 * torch.from_numpy(np.random.default_rng(1).standard_normal(u0.shape))
    return theta, u0, u


def _objective(plan, u, d):
    r = glam.lam(u, plan) - d
    return 0.5 * (r.abs() ** 2).sum().to(torch.float64) + ALPHA * glam.tv(u, plan, EPS)


def test_f64_gradient_matches_finite_differences(case):
    theta, u0, u = case
    plan = glam.Plan(N, N, N, N, theta, PHI, prec="f64")
    d = plan.forward(u0)
    x = u.cuda().requires_grad_()
    _objective(plan, x, d).backward()
    v = torch.from_numpy(np.random.default_rng(2).standard_normal(u.shape)).cuda()
    h = 1e-4
    with torch.no_grad():
        fp = _objective(plan, u.cuda() + h * v, d).item()
        fm = _objective(plan, u.cuda() - h * v, d).item()
    fd = (fp - fm) / (2 * h)
    an = torch.dot(x.grad.flatten(), v.flatten()).item()
    assert abs(fd - an) <= 1e-9 * x.grad.norm().item() * v.norm().item()


def test_f32_gradient_matches_oracle(case):
    theta, u0, u = case
    g = oracle_geom(N, N, N, N, theta, PHI)
    un, u0n = u.numpy(), u0.numpy()
    d = olam.lam_forward(u0n, g)
    r = olam.lam_forward(un, g) - d
    gg = otv.grad(un)
    ref = olam.lam_adjoint(r, g) + ALPHA * (-otv.div(gg / np.sqrt((gg * gg).sum(0) + EPS * EPS)))
    plan = glam.Plan(N, N, N, N, theta, PHI, prec="f32")
    x = u.float().cuda().requires_grad_()
    _objective(plan, x, torch.from_numpy(d.astype(np.complex64)).cuda()).backward()
    assert rel(x.grad, ref) < 1e-5


def test_tv_value_matches_oracle(case):
    theta, _, u = case
    plan = glam.Plan(N, N, N, N, theta, PHI, prec="f64")
    val, grad = plan.tv_smooth(u.cuda(), EPS)
    gg = otv.grad(u.numpy())
    m = np.sqrt((gg * gg).sum(0) + EPS * EPS)
    assert val == pytest.approx(m.sum(), rel=1e-12)
    assert rel(grad, -otv.div(gg / m)) < 1e-12
