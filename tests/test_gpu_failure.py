"""Failure detection without a GPU fault: the host makes the failure (a NaN in
the data, an index the kernel's own check refuses) and the library reports it
as a status, with the CUDA context still usable afterwards.

* A NaN in the data reaches the FP64 reductions of the first CG step; the
  state's status word turns LAM_ENAN (-5), admm_status reports it and the
  one-call reconstruct() returns it.
* The LAM_BOUNDS_CHECK build (liblamino_checked.so) runs the operators with
  index checks at the table- and geometry-derived accesses: on valid inputs it
  reports no failure and computes bitwise what the plain build computes; its
  self-test entry point writes at an index outside its scratch, which the
  check refuses (the site is recorded, nothing is written) and
  lam_plan_status reports as LAM_EBOUNDS (-7).  It runs in a child process
  that loads the checked library through LAMINO_LIB.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2511_01893_b300 import build, inputs
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, NZ, H, W, T = 32, 32, 32, 32, 24
PHI = np.deg2rad(30.0)


def _data(seed=3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((T, H, W)) + 1j * rng.standard_normal((T, H, W))).astype(np.complex64)


def test_nan_in_data_sets_admm_status():
    plan = glam.Plan(N, NZ, H, W, inputs.angles(T), PHI, prec="f32")
    d = _data()
    d[5, 7, 9] = np.nan
    a = glam.Admm(plan).init(torch.from_numpy(d), 1e-3, 0.5, 4)
    assert a.status() == 0  # nothing reduced yet
    a.step()
    assert a.status() == -5
    assert "non-finite" in glam.lib().lam_last_error().decode()
    # the context is still usable: a clean state on the same plan runs normally
    b = glam.Admm(plan).init(torch.from_numpy(_data()), 1e-3, 0.5, 4)
    b.step()
    assert b.status() == 0
    assert torch.isfinite(b.u).all()


def test_nan_in_data_fails_reconstruct():
    d = _data().real.copy()
    d[2, 3, 4] = np.nan
    with pytest.raises(glam.LaminoError, match="status -5"):
        glam.reconstruct(d, inputs.angles(T), PHI, N, NZ, 2, 1e-3, 0.5)


_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2511_01893_b300 import inputs, lamino as glam
out = {"checked": glam.lib().lam_bounds_checked()}
rng = np.random.default_rng(11)
u = torch.from_numpy(rng.standard_normal((32, 32, 32)).astype(np.float32)).cuda()
res = {}
for spread in ("tiles", "halo", "atomic"):
    plan = glam.Plan(32, 32, 32, 32, inputs.angles(24), np.deg2rad(30.0), prec="f32", spread=spread)
    d = plan.forward_hat(u)
    v = plan.adjoint_hat(d)
    res[spread] = (d, v)
    out["status_" + spread] = plan.status()
torch.save({k: (d.cpu(), v.cpu()) for k, (d, v) in res.items()}, sys.argv[2])
plan = glam.Plan(32, 32, 32, 32, inputs.angles(24), np.deg2rad(30.0), prec="f32")
s = torch.cuda.current_stream().cuda_stream
out["selftest_in_range"] = glam.lib().lamx_bounds_selftest(plan._h, 63, s)
out["status_after_in_range"] = plan.status()
out["selftest_out_of_range"] = glam.lib().lamx_bounds_selftest(plan._h, 64, s)
out["status_after_out_of_range"] = plan.status()
out["message"] = glam.lib().lam_last_error().decode()
out["status_cleared"] = plan.status()
torch.cuda.synchronize()
print(json.dumps(out))
"""


def test_bounds_checked_build(tmp_path):
    lib = build.build(checked=True)
    dump = str(tmp_path / "checked.pt")
    env = dict(os.environ, LAMINO_LIB=lib)
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, dump], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] == 1
    assert out["status_tiles"] == out["status_halo"] == out["status_atomic"] == 0
    assert out["selftest_in_range"] == 0 and out["status_after_in_range"] == 0
    assert out["selftest_out_of_range"] == 0  # the launch itself is fine
    assert out["status_after_out_of_range"] == -7
    assert "self-test" in out["message"]
    assert out["status_cleared"] == 0
    # the checks change no result: bitwise the plain build's (deterministic spreads)
    got = torch.load(dump)
    rng = np.random.default_rng(11)
    u = torch.from_numpy(rng.standard_normal((32, 32, 32)).astype(np.float32)).cuda()
    for spread in ("tiles", "halo"):
        plan = glam.Plan(32, 32, 32, 32, inputs.angles(24), PHI, prec="f32", spread=spread)
        d = plan.forward_hat(u)
        v = plan.adjoint_hat(d)
        assert torch.equal(d.cpu(), got[spread][0])
        assert torch.equal(v.cpu(), got[spread][1])
        assert plan.status() == 0
