"""Memoization of F*_u2D per plane job inside ADMM-TV (LAM_OPT_MEMO_TAU).

Each plane job keeps one (key, value) item; a call whose key has cosine
similarity above tau with the item's reuses the stored plane (times the
least-squares factor) instead of spreading and transforming.  Checked on
the plain workload (64^3, 64 angles, phi = 30 deg):

* a threshold no key reaches serves nothing from the cache: bitwise the
  result without memoization, every job looked up;
* a threshold every key passes serves every call after the first from the
  cache (the first fills the items): the counts follow, the run stays finite;
* the approximation error against the run without memoization (the paper's
  accuracy metric E, Section 6.1) and the number of reused jobs both fall as
  tau rises.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import rel
from oracle import lamino as olam
from paper_2511_01893_b300 import inputs
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

N, T = 64, 64
PHI = np.deg2rad(30.0)


@pytest.fixture(scope="module")
def data():
    theta = inputs.angles(T)
    g = olam.Geometry(n1=N, n0=N, n2=N, h=N, w=N, theta=theta, phi=PHI)
    u = inputs.ellipsoid_phantom(N, N, 12, seed=1234).numpy()
    clean = olam.lam_forward(u, g)
    return theta, torch.from_numpy(clean + 0.01 * np.abs(clean.real).max() * inputs.noise((T, N, N), seed=99).numpy())


def _run(theta, d, tau, iters):
    plan = glam.Plan(N, N, N, N, theta, PHI, prec="f32").set_memo(tau)
    a = glam.Admm(plan).init(d, 1e-3, 0.5, 4)
    a.run(iters)
    assert a.status() == 0
    return a.u.clone(), a.scalars(), plan.info()["plane_jobs"]


def test_memo_that_never_hits_is_bitwise_plain(data):
    theta, d = data
    ref, _, _ = _run(theta, d, 0.0, 2)
    got, sc, njobs = _run(theta, d, 0.9999, 2)
    assert sc["memo_hits"] == 0
    assert sc["memo_lookups"] == 2 * 4 * njobs
    assert torch.equal(got, ref)


def test_memo_that_always_hits_serves_every_later_call(data):
    theta, d = data
    got, sc, njobs = _run(theta, d, 0.0001, 2)
    assert sc["memo_lookups"] == 2 * 4 * njobs
    # the first call fills every item; later calls hit unless a key turned
    # against its item (cosine similarity below 1e-4: early residual planes can
    # flip sign), and such a miss refills the item
    assert 0.9 * (sc["memo_lookups"] - njobs) <= sc["memo_hits"] <= sc["memo_lookups"] - njobs
    assert torch.isfinite(got).all()


def test_memo_error_and_reuse_fall_as_tau_rises(data):
    theta, d = data
    ref, _, _ = _run(theta, d, 0.0, 8)
    res = []
    for tau in (0.5, 0.9, 0.99):
        u, sc, _ = _run(theta, d, tau, 8)
        res.append((rel(u, ref), sc["memo_hits"]))
    assert res[0][1] >= res[1][1] >= res[2][1]
    assert res[0][1] > 0
    assert res[2][0] <= res[0][0] + 1e-6
