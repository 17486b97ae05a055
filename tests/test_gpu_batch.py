"""Batched operators and batched ADMM-TV (several problems of uneven sizes in
one persistent launch per stage) against the single-plan calls.

The batched path runs the same kernel bodies on the same arguments, so every
result must be bitwise equal to the per-plan result; one problem is also
checked against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import oracle_geom, rand_data, rand_vol, rel
from oracle import lamino as olam
from paper_2511_01893_b300 import inputs
from paper_2511_01893_b300 import lamino as glam

pytestmark = pytest.mark.gpu

# uneven sizes (n multiple of 16; nz = n / 2; T = n angles; detector n x n),
# tilts spread over [20, 40] degrees
SIZES = [32, 48, 64, 80]


def _plans(prec="f32", sizes=SIZES):
    out = []
    for i, n in enumerate(sizes):
        phi = np.deg2rad(20.0 + 20.0 * i / max(len(sizes) - 1, 1))
        out.append(glam.Plan(n, n // 2, n, n, inputs.angles(n), phi, prec=prec))
    return out


def test_batched_equals_single_for_autotuned_power_of_two_among_mixed_radix():
    # the batch runs every problem through the mixed-radix kernel variant when
    # any problem needs it; a power-of-two problem's single-plan calls run the
    # power-of-two variant (and, at 2n >= 512, the compile-time-length one),
    # with launch shapes from the autotuner: the results must not depend on it
    plans = _plans("f32", [96, 128, 160, 256])
    for p in plans:
        p.autotune(reps=1)
    batch = glam.Batch(plans)
    us = [torch.from_numpy(rand_vol(p.n, p.nz, 40 + i)).cuda().float() for i, p in enumerate(plans)]
    ds = [torch.from_numpy(rand_data(p.T, p.h, p.w, 50 + i)).cuda().to(torch.complex64) for i, p in enumerate(plans)]
    fb, ab = batch.forward_hat(us), batch.adjoint_hat(ds)
    for k, p in enumerate(plans):
        assert torch.equal(fb[k], p.forward_hat(us[k]))
        assert torch.equal(ab[k], p.adjoint_hat(ds[k]))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batched_operators_equal_single_plan_calls(prec):
    plans = _plans(prec)
    batch = glam.Batch(plans)
    us = [torch.from_numpy(rand_vol(p.n, p.nz, 40 + i)).cuda().to(p.rdtype) for i, p in enumerate(plans)]
    ds = [torch.from_numpy(rand_data(p.T, p.h, p.w, 50 + i)).cuda().to(p.cdtype) for i, p in enumerate(plans)]
    for got, p, u in zip(batch.forward_hat(us), plans, us):
        assert torch.equal(got, p.forward_hat(u))
    for got, p, d in zip(batch.adjoint_hat(ds), plans, ds):
        assert torch.equal(got, p.adjoint_hat(d))
    for got, p, u in zip(batch.forward(us), plans, us):
        assert torch.equal(got, p.forward(u))
    for got, p, d in zip(batch.adjoint(ds), plans, ds):
        assert torch.equal(got, p.adjoint(d))
    info = batch.info()
    assert all(info[st]["work"] > 0 and 0 < info[st]["grid"] <= info[st]["work"] for st in glam.Batch.STAGES)


def test_batched_forward_matches_oracle():
    plans = _plans("f32", [48, 32])
    batch = glam.Batch(plans)
    p = plans[0]
    g = oracle_geom(p.n, p.nz, p.h, p.w, p.theta, p.phi)
    u = rand_vol(p.n, p.nz, 60)
    u2 = rand_vol(plans[1].n, plans[1].nz, 61)
    got = batch.forward([torch.from_numpy(u), torch.from_numpy(u2)])[0]
    assert rel(got, olam.lam_forward(u, g)) < 1e-5


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_batched_admm_equals_single_plan_admm(graph):
    plans = _plans("f32")
    batch = glam.Batch(plans)
    datas = []
    for i, p in enumerate(plans):
        u = inputs.ellipsoid_phantom(p.n, p.nz, 8, seed=70 + i, device="cuda")
        d = p.forward(u)
        gen = torch.Generator(device="cuda").manual_seed(80 + i)
        d.real.add_(torch.randn(d.shape, generator=gen, device="cuda"), alpha=0.01 * d.real.abs().max().item())
        datas.append(d)
    single = [glam.Admm(p).init(d, 1e-3, 0.5, 3) for p, d in zip(plans, datas)]
    for a in single:
        a.run(3)
    batched = [glam.Admm(p).init(d, 1e-3, 0.5, 3) for p, d in zip(plans, datas)]
    batch.set_streams(0)  # the persistent batched stages (the default is concurrent)
    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            batch.admm_run(batched, 3, graph=True)
        s.synchronize()
        assert batch.info()["graph_kernels"] > 0
    else:
        batch.admm_run(batched, 3)
    for a, b in zip(single, batched):
        assert b.status() == 0
        assert torch.equal(a.u, b.u)
        assert np.array_equal(a.history(), b.history())


@pytest.mark.parametrize("streams,graph,prec", [(2, False, "f32"), (4, True, "f32"), (3, True, "f64")],
                         ids=["2eager", "4graph", "3graph-f64"])
def test_concurrent_batch_admm_equals_single_plan_admm(streams, graph, prec):
    # concurrent mode: each problem's own outer iteration on side stream i mod
    # streams, forked from and joined to the caller's stream; the states must
    # evolve bitwise as under single-plan runs, whatever the interleaving
    plans = _plans(prec)
    batch = glam.Batch(plans).set_streams(streams)
    datas = []
    for i, p in enumerate(plans):
        u = inputs.ellipsoid_phantom(p.n, p.nz, 8, seed=90 + i, device="cuda").to(p.rdtype)
        datas.append(p.forward(u))
    single = [glam.Admm(p).init(d, 1e-3, 0.5, 3) for p, d in zip(plans, datas)]
    for a in single:
        a.run(3)
    conc = [glam.Admm(p).init(d, 1e-3, 0.5, 3) for p, d in zip(plans, datas)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.admm_run(conc, 2, graph=graph)
        batch.admm_run(conc, 1, graph=graph)
    s.synchronize()
    for a, b in zip(single, conc):
        assert b.status() == 0
        assert torch.equal(a.u, b.u)
        assert np.array_equal(a.history(), b.history())


def test_concurrent_batch_runs_memoized_and_plain_states_together():
    # the concurrent mode runs admm_step per problem, so options the
    # persistent batch refuses (memoization) work, bitwise as single runs
    plans = _plans("f32", [32, 48])
    plans[1].set_memo(0.92)
    datas = [p.forward(inputs.ellipsoid_phantom(p.n, p.nz, 8, seed=95 + i, device="cuda"))
             for i, p in enumerate(plans)]
    single = [glam.Admm(p).init(d, 1e-3, 0.5, 2) for p, d in zip(plans, datas)]
    for a in single:
        a.run(3)
    batch = glam.Batch(plans).set_streams(0)
    conc = [glam.Admm(p).init(d, 1e-3, 0.5, 2) for p, d in zip(plans, datas)]
    with pytest.raises(glam.LaminoError, match="memoize"):
        batch.admm_run(conc, 1)
    conc = [glam.Admm(p).init(d, 1e-3, 0.5, 2) for p, d in zip(plans, datas)]
    batch.set_streams(2).admm_run(conc, 3)
    torch.cuda.synchronize()
    for a, b in zip(single, conc):
        assert torch.equal(a.u, b.u)


def test_concurrent_batch_refuses_a_shared_workspace():
    p = _plans("f32", [32])[0]
    with pytest.raises(glam.LaminoError, match="share a workspace"):
        glam.Batch([p, p]).set_streams(2)


def test_batch_rejects_mixed_precision_and_bad_counts():
    p32 = _plans("f32", [32])[0]
    p64 = _plans("f64", [32])[0]
    with pytest.raises(glam.LaminoError, match="same precision"):
        glam.Batch([p32, p64])
    with pytest.raises(glam.LaminoError, match="count"):
        glam.Batch([p32] * 33)
